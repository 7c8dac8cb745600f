// Learned rank predictor: a 16-64-1 tanh MLP in fp32 with hand-written
// forward, gradient and Adam kernels, trained on (features of a gate update
// -> log2 of the rank a sketch must capture: singular values above
// max(cutoff/100, Mw eps) ||sigma||) pairs. Its prediction sizes the
// randomized range-finder sketch of the SVD (sketch.cu); the full Jacobi SVD
// is the fallback, and the sketch's explicit residual decides between them.
//
// Parameter layout (kMlpParams floats): W1[64][16] (row = hidden unit),
// b1[64], w2[64], b2.   y = b2 + sum_h w2[h] tanh(b1[h] + sum_i W1[h][i] x_i)
// Loss: mean squared error over the batch.
//
// Features of a two-site gate on bond s (16, fixed affine scaling):
//   log2(chi_{s-1})/10, log2(chi_{s+1})/10, log2(chi_s)/10, 4.5 e_p(U),
//   ln of the 6 largest Lambda_{s-1} / 25, ln of the 6 largest Lambda_{s+1} / 25
// (missing values padded with ln(max(cutoff, 1e-13)) / 25). e_p is the
// entangling power of U (Zanardi, Zalka, Faoro, PRA 62, 030301, 2000).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <numeric>
#include <random>
#include <vector>

#include "../../include/mps.h"
#include "engine.cuh"
#include "kernels.cuh"
#include "mlp.cuh"

namespace mpsgb {

constexpr float kB1 = 0.9f, kB2 = 0.999f, kAdamEps = 1e-8f;

// One block of 64 threads per sample: hidden unit h = threadIdx.x.
__device__ __forceinline__ float mlp_sample(const float* P, const float* x, float* a_out) {
  __shared__ float red[64];
  const int h = threadIdx.x;
  float z = P[kMlpB1 + h];
#pragma unroll
  for (int i = 0; i < kMlpIn; ++i) z = fmaf(P[kMlpW1 + h * kMlpIn + i], x[i], z);
  const float a = tanhf(z);
  *a_out = a;
  red[h] = P[kMlpW2 + h] * a;
  __syncthreads();
  for (int o = 32; o > 0; o >>= 1) {
    if (h < o) red[h] += red[h + o];
    __syncthreads();
  }
  const float y = red[0] + P[kMlpB2];
  __syncthreads();
  return y;
}

__global__ void __launch_bounds__(64) k_mlp_fwd(const float* P, const float* X, int B, float* Y) {
  const int b = blockIdx.x;
  if (b >= B) return;
  float a;
  const float y = mlp_sample(P, X + (size_t)b * kMlpIn, &a);
  if (threadIdx.x == 0) Y[b] = y;
}

// Gradient of the mean squared error over the batch samples idx[0..B),
// accumulated into G (zeroed by the caller); loss accumulated into *loss.
__global__ void __launch_bounds__(64) k_mlp_grad(const float* P, const float* X, const float* T, const int* idx,
                                                 int B, float* G, float* loss) {
  const int b = blockIdx.x;
  if (b >= B) return;
  const int sidx = idx ? idx[b] : b;
  const float* x = X + (size_t)sidx * kMlpIn;
  float a;
  const float y = mlp_sample(P, x, &a);
  const float r = y - T[sidx];
  const float dy = 2.f * r / (float)B;
  const int h = threadIdx.x;
  if (h == 0) {
    atomicAdd(loss, r * r / (float)B);
    atomicAdd(&G[kMlpB2], dy);
  }
  atomicAdd(&G[kMlpW2 + h], dy * a);
  const float dz = dy * P[kMlpW2 + h] * (1.f - a * a);
  atomicAdd(&G[kMlpB1 + h], dz);
#pragma unroll
  for (int i = 0; i < kMlpIn; ++i) atomicAdd(&G[kMlpW1 + h * kMlpIn + i], dz * x[i]);
}

// Adam (Kingma & Ba 2015) with bias correction, step t >= 1.
__global__ void k_adam(float* P, const float* G, float* M, float* V, int n, float lr, int t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = G[i];
  const float m = kB1 * M[i] + (1.f - kB1) * g;
  const float v = kB2 * V[i] + (1.f - kB2) * g * g;
  M[i] = m;
  V[i] = v;
  const float mh = m / (1.f - powf(kB1, (float)t));
  const float vh = v / (1.f - powf(kB2, (float)t));
  P[i] -= lr * mh / (sqrtf(vh) + kAdamEps);
}

// Features of gate tasks (one thread per task).
__global__ void k_features(const FeatureTask* ft, int n, float* X) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const FeatureTask& f = ft[t];
  float* x = X + (size_t)t * kMlpIn;
  const int xl = f.chi[f.site], x0 = f.chi[f.site + 1], xr = f.chi[f.site + f.k];
  x[0] = log2f((float)xl) / 10.f;
  x[1] = log2f((float)xr) / 10.f;
  x[2] = log2f((float)x0) / 10.f;
  x[3] = 4.5f * f.ep;
  const float pad = logf(fmaxf((float)f.cutoff, 1e-13f)) / 25.f;
  for (int i = 0; i < 6; ++i) {
    x[4 + i] = i < xl ? logf(fmaxf((float)f.lamL[i], 1e-30f)) / 25.f : pad;
    x[10 + i] = i < xr ? logf(fmaxf((float)f.lamR[i], 1e-30f)) / 25.f : pad;
  }
}

void launch_mlp_fwd(const float* P, const float* X, int B, float* Y, cudaStream_t st) {
  if (B > 0) k_mlp_fwd<<<B, 64, 0, st>>>(P, X, B, Y);
}
void launch_features(const FeatureTask* ft, int n, float* X, cudaStream_t st) {
  if (n > 0) k_features<<<(n + 127) / 128, 128, 0, st>>>(ft, n, X);
}

// Entangling power of a two-qubit gate: e_p(U) = (4/9) [E(U) + E(U S) - E(S)],
// E(V) = 1 - Tr((R R^H)^2)/16 with R the realignment R[(i,k),(j,l)] = V[(i,j),(k,l)]
// (the sum of the fourth powers of V's operator-Schmidt coefficients), S = SWAP.
double entangling_power(const double* U) {
  typedef std::complex<double> cd;
  auto opE = [](const cd* V) {
    cd R[16];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j)
        for (int k = 0; k < 2; ++k)
          for (int l = 0; l < 2; ++l) R[(i * 2 + k) * 4 + (j * 2 + l)] = V[(i * 2 + j) * 4 + (k * 2 + l)];
    cd RR[16];
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        cd s = 0;
        for (int c = 0; c < 4; ++c) s += R[a * 4 + c] * std::conj(R[b * 4 + c]);
        RR[a * 4 + b] = s;
      }
    double tr = 0;
    for (int a = 0; a < 16; ++a) tr += std::norm(RR[a]);
    return 1.0 - tr / 16.0;
  };
  cd V[16], VS[16];
  for (int e = 0; e < 16; ++e) V[e] = cd(U[2 * e], U[2 * e + 1]);
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      const int cs = (c & 1) * 2 + (c >> 1);  // SWAP permutes the column index bits
      VS[r * 4 + c] = V[r * 4 + cs];
    }
  return (4.0 / 9.0) * (opE(V) + opE(VS) - 0.75);
}

}  // namespace mpsgb

// ------------------------------------------------------------------ C ABI ---

using namespace mpsgb;

struct mps_mlp {
  float* P = nullptr;   // parameters (device)
  float* G = nullptr;   // gradient
  float* M = nullptr;   // Adam moments
  float* V = nullptr;
  float* d_loss = nullptr;
  int t = 0;            // Adam step
};

namespace {
int mfail(int code, const char* msg) {
  set_error_message(msg);
  return code;
}
#define MCK(call)                                                  \
  do {                                                             \
    if ((call) != cudaSuccess) return mfail(MPS_ERR_CUDA, #call);  \
  } while (0)
}  // namespace

extern "C" {

int mps_mlp_create(unsigned long long seed, mps_mlp_handle* out) {
  if (!out) return mfail(MPS_ERR_ARG, "out is NULL");
  *out = nullptr;
  mps_mlp* m = new mps_mlp();
  const size_t bytes = sizeof(float) * kMlpParams;
  if (dev_alloc((void**)&m->P, bytes) != cudaSuccess || dev_alloc((void**)&m->G, bytes) != cudaSuccess ||
      dev_alloc((void**)&m->M, bytes) != cudaSuccess || dev_alloc((void**)&m->V, bytes) != cudaSuccess ||
      dev_alloc((void**)&m->d_loss, sizeof(float)) != cudaSuccess) {
    mps_mlp_destroy(m);
    return mfail(MPS_ERR_NOMEM, "MLP buffers");
  }
  // Glorot-uniform weights, zero biases
  std::mt19937_64 rng(seed);
  std::vector<float> p(kMlpParams, 0.f);
  const float a1 = std::sqrt(6.f / (kMlpIn + kMlpHid)), a2 = std::sqrt(6.f / (kMlpHid + 1));
  std::uniform_real_distribution<float> u1(-a1, a1), u2(-a2, a2);
  for (int i = 0; i < kMlpHid * kMlpIn; ++i) p[kMlpW1 + i] = u1(rng);
  for (int h = 0; h < kMlpHid; ++h) p[kMlpW2 + h] = u2(rng);
  if (cudaMemcpy(m->P, p.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(m->M, 0, bytes) != cudaSuccess || cudaMemset(m->V, 0, bytes) != cudaSuccess) {
    mps_mlp_destroy(m);
    return mfail(MPS_ERR_CUDA, "MLP init");
  }
  *out = m;
  return MPS_OK;
}

int mps_mlp_destroy(mps_mlp_handle m) {
  if (!m) return MPS_OK;
  cudaFree(m->P);
  cudaFree(m->G);
  cudaFree(m->M);
  cudaFree(m->V);
  cudaFree(m->d_loss);
  delete m;
  return MPS_OK;
}

int mps_mlp_params(mps_mlp_handle m, float* get, const float* set) {
  if (!m) return mfail(MPS_ERR_ARG, "NULL MLP");
  if (set) {
    MCK(cudaMemcpy(m->P, set, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice));
    MCK(cudaMemset(m->M, 0, sizeof(float) * kMlpParams));
    MCK(cudaMemset(m->V, 0, sizeof(float) * kMlpParams));
    m->t = 0;
  }
  if (get) MCK(cudaMemcpy(get, m->P, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost));
  return MPS_OK;
}

int mps_mlp_forward(mps_mlp_handle m, int B, const float* X, float* Y) {
  if (!m || B < 0 || (B > 0 && (!X || !Y))) return mfail(MPS_ERR_ARG, "bad arguments");
  if (B == 0) return MPS_OK;
  float *dX = nullptr, *dY = nullptr;
  if (dev_alloc((void**)&dX, sizeof(float) * kMlpIn * B) != cudaSuccess || dev_alloc((void**)&dY, sizeof(float) * B) != cudaSuccess) {
    cudaFree(dX);
    return mfail(MPS_ERR_NOMEM, "MLP batch");
  }
  cudaError_t e = cudaMemcpy(dX, X, sizeof(float) * kMlpIn * B, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    launch_mlp_fwd(m->P, dX, B, dY, nullptr);
    e = cudaMemcpy(Y, dY, sizeof(float) * B, cudaMemcpyDeviceToHost);
  }
  cudaFree(dX);
  cudaFree(dY);
  return e == cudaSuccess ? MPS_OK : mfail(MPS_ERR_CUDA, "MLP forward");
}

int mps_mlp_loss_grad(mps_mlp_handle m, int B, const float* X, const float* T, float* loss, float* grad) {
  if (!m || B < 1 || !X || !T) return mfail(MPS_ERR_ARG, "bad arguments");
  float *dX = nullptr, *dT = nullptr;
  if (dev_alloc((void**)&dX, sizeof(float) * kMlpIn * B) != cudaSuccess || dev_alloc((void**)&dT, sizeof(float) * B) != cudaSuccess) {
    cudaFree(dX);
    return mfail(MPS_ERR_NOMEM, "MLP batch");
  }
  cudaError_t e = cudaMemcpy(dX, X, sizeof(float) * kMlpIn * B, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dT, T, sizeof(float) * B, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->G, 0, sizeof(float) * kMlpParams);
  if (e == cudaSuccess) e = cudaMemset(m->d_loss, 0, sizeof(float));
  if (e == cudaSuccess) {
    k_mlp_grad<<<B, 64>>>(m->P, dX, dT, nullptr, B, m->G, m->d_loss);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && loss) e = cudaMemcpy(loss, m->d_loss, sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && grad) e = cudaMemcpy(grad, m->G, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost);
  cudaFree(dX);
  cudaFree(dT);
  return e == cudaSuccess ? MPS_OK : mfail(MPS_ERR_CUDA, "MLP gradient");
}

int mps_mlp_train(mps_mlp_handle m, int N, const float* X, const float* T, int epochs, int batch, float lr,
                  unsigned long long seed, float* loss_out) {
  if (!m || N < 1 || !X || !T || epochs < 1 || batch < 1 || !(lr > 0.f)) return mfail(MPS_ERR_ARG, "bad arguments");
  float *dX = nullptr, *dT = nullptr;
  int* dI = nullptr;
  if (dev_alloc((void**)&dX, sizeof(float) * kMlpIn * N) != cudaSuccess || dev_alloc((void**)&dT, sizeof(float) * N) != cudaSuccess ||
      dev_alloc((void**)&dI, sizeof(int) * N) != cudaSuccess) {
    cudaFree(dX);
    cudaFree(dT);
    return mfail(MPS_ERR_NOMEM, "training set");
  }
  cudaError_t e = cudaMemcpy(dX, X, sizeof(float) * kMlpIn * N, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dT, T, sizeof(float) * N, cudaMemcpyHostToDevice);
  std::mt19937_64 rng(seed);
  std::vector<int> perm(N);
  std::iota(perm.begin(), perm.end(), 0);
  float last = 0.f;
  for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
    std::shuffle(perm.begin(), perm.end(), rng);
    e = cudaMemcpy(dI, perm.data(), sizeof(int) * N, cudaMemcpyHostToDevice);
    float sum = 0.f;
    int nb = 0;
    for (int b0 = 0; b0 < N && e == cudaSuccess; b0 += batch, ++nb) {
      const int B = std::min(batch, N - b0);
      cudaMemset(m->G, 0, sizeof(float) * kMlpParams);
      cudaMemset(m->d_loss, 0, sizeof(float));
      k_mlp_grad<<<B, 64>>>(m->P, dX, dT, dI + b0, B, m->G, m->d_loss);
      m->t += 1;
      k_adam<<<(kMlpParams + 255) / 256, 256>>>(m->P, m->G, m->M, m->V, kMlpParams, lr, m->t);
      float l = 0.f;
      e = cudaMemcpy(&l, m->d_loss, sizeof(float), cudaMemcpyDeviceToHost);
      sum += l;
    }
    last = nb ? sum / nb : 0.f;
  }
  cudaFree(dX);
  cudaFree(dT);
  cudaFree(dI);
  if (e != cudaSuccess) return mfail(MPS_ERR_CUDA, "training");
  if (loss_out) *loss_out = last;
  return MPS_OK;
}

}  // extern "C"

namespace mpsgb {
const float* mlp_params(const mps_mlp* m) { return m ? m->P : nullptr; }
}  // namespace mpsgb

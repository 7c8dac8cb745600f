// Readout kernels: amplitudes (Eq. 1 at one basis state) and the small
// complex binary64 GEMM used to contract transfer matrices for reduced
// density operators and expectation values (Sec. 3.2, "RDO": the
// tracing-out operation). Not on the gate-update hot path.
#include "engine.cuh"
#include "kernels.cuh"

namespace mpsgb {

__device__ __forceinline__ double2 rfma(double2 a, double2 b, double2 acc) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
  return acc;
}

// One CTA per bit string: v <- v Gamma_s[b_s] Lambda_s for s = 0..n-1.
__global__ void __launch_bounds__(256) k_amplitudes(const double2* gamma, const double* lambda, const int* chi,
                                                    int n, int cap, const unsigned char* bits, double2* out) {
  extern __shared__ double2 sh[];
  double2* v = sh;
  double2* w = sh + cap;
  const unsigned char* b = bits + (size_t)blockIdx.x * n;
  if (threadIdx.x == 0) v[0] = make_double2(1.0, 0.0);
  __syncthreads();
  for (int s = 0; s < n; ++s) {
    const int xl = chi[s], xr = chi[s + 1];
    const double2* g = gamma + ((size_t)s * 2 + (b[s] & 1)) * cap * cap;
    const double* lam = lambda + (size_t)(s + 1) * cap;
    for (int c = threadIdx.x; c < xr; c += blockDim.x) {
      double2 acc = make_double2(0.0, 0.0);
      for (int a = 0; a < xl; ++a) acc = rfma(v[a], g[(size_t)a * cap + c], acc);
      w[c] = make_double2(lam[c] * acc.x, lam[c] * acc.y);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < xr; c += blockDim.x) v[c] = w[c];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = v[0];
}

// As[i][a][c] = Gamma_s[i][a][c] * Lambda_s[c], dense [2][xl][xr]
__global__ void k_scale_site(const double2* g, const double* lam, int xl, int xr, int cap, double2* out) {
  const int total = 2 * xl * xr;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int i = e / (xl * xr), rem = e % (xl * xr);
    const int a = rem / xr, c = rem % xr;
    const double2 v = g[((size_t)i * cap + a) * cap + c];
    out[e] = make_double2(v.x * lam[c], v.y * lam[c]);
  }
}

// C_z (+)= op(A_z) op(B_z), 16x16 tiles, row-major operands. opA: A^T if
// transA; opB: B^T if transB, then conjugated if conjB.
__global__ void __launch_bounds__(256) k_zgemm(int M, int N, int K, const double2* A, int lda, long long sA,
                                               int transA, const double2* B, int ldb, long long sB, int conjB,
                                               int transB, double2* C, int ldc, long long sC, int accumulate) {
  __shared__ double2 As[16][17], Bs[16][17];
  A += sA * blockIdx.z;
  B += sB * blockIdx.z;
  C += sC * blockIdx.z;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m = blockIdx.y * 16 + ty, n = blockIdx.x * 16 + tx;
  double2 acc = make_double2(0.0, 0.0);
  for (int k0 = 0; k0 < K; k0 += 16) {
    {  // As[ty][tx] = opA[m][k0+tx]
      const int kk = k0 + tx;
      double2 v = make_double2(0.0, 0.0);
      if (m < M && kk < K) v = transA ? A[(size_t)kk * lda + m] : A[(size_t)m * lda + kk];
      As[ty][tx] = v;
    }
    {  // Bs[ty][tx] = opB[k0+ty][n]
      const int kk = k0 + ty;
      double2 v = make_double2(0.0, 0.0);
      if (kk < K && n < N) {
        v = transB ? B[(size_t)n * ldb + kk] : B[(size_t)kk * ldb + n];
        if (conjB) v.y = -v.y;
      }
      Bs[ty][tx] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) acc = rfma(As[ty][k], Bs[k][tx], acc);
    __syncthreads();
  }
  if (m < M && n < N) {
    double2* c = C + (size_t)m * ldc + n;
    if (accumulate) {
      const double2 o = *c;
      acc.x += o.x;
      acc.y += o.y;
    }
    *c = acc;
  }
}

// Sequential sampling, one step (one warp per sample m): the weights of
// b_s = 0 and 1, p_i = <W_i R W_i^H> with W_i = V A_i (row m of W_i, T_i =
// W_i R), b = 0 when u < p_0 / (p_0 + p_1), then V <- W_b / sqrt(p_b).
__global__ void k_sample_step(int S, int xr, const double2* W0, const double2* W1, const double2* T0,
                              const double2* T1, const double* u, int ustride, unsigned char* bits, double2* V) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= S) return;
  const size_t row = (size_t)warp * xr;
  double p0 = 0.0, p1 = 0.0;
  for (int c = lane; c < xr; c += 32) {
    const double2 w0 = W0[row + c], t0 = T0[row + c], w1 = W1[row + c], t1 = T1[row + c];
    p0 = fma(t0.x, w0.x, fma(t0.y, w0.y, p0));  // Re(t conj(w))
    p1 = fma(t1.x, w1.x, fma(t1.y, w1.y, p1));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    p0 += __shfl_xor_sync(0xffffffffu, p0, o);
    p1 += __shfl_xor_sync(0xffffffffu, p1, o);
  }
  const int b = u[(size_t)warp * ustride] < p0 / (p0 + p1) ? 0 : 1;
  if (lane == 0) bits[(size_t)warp * ustride] = (unsigned char)b;
  const double pb = b ? p1 : p0;
  const double inv = pb > 0.0 ? 1.0 / sqrt(pb) : 0.0;
  const double2* Wb = b ? W1 : W0;
  for (int c = lane; c < xr; c += 32) {
    const double2 w = Wb[row + c];
    V[row + c] = make_double2(inv * w.x, inv * w.y);
  }
}

// out = a0 X0 + a1 X1 (complex coefficients), element-wise
__global__ void k_combine2(long long n, double2 a0, const double2* X0, double2 a1, const double2* X1, double2* out) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const double2 x = X0[e], y = X1[e];
    out[e] = make_double2(a0.x * x.x - a0.y * x.y + a1.x * y.x - a1.y * y.y,
                          a0.x * x.y + a0.y * x.x + a1.x * y.y + a1.y * y.x);
  }
}

__global__ void k_fill_one(double2* v, int count) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) v[e] = make_double2(1.0, 0.0);
}

void launch_sample_step(int S, int xr, const double2* W0, const double2* W1, const double2* T0, const double2* T1,
                        const double* u, int ustride, unsigned char* bits, double2* V, cudaStream_t st) {
  k_sample_step<<<(S * 32 + 255) / 256, 256, 0, st>>>(S, xr, W0, W1, T0, T1, u, ustride, bits, V);
}

void launch_combine2(long long n, double2 a0, const double2* X0, double2 a1, const double2* X1, double2* out,
                     cudaStream_t st) {
  long long b = (n + 255) / 256;
  if (b > 4096) b = 4096;
  k_combine2<<<(int)(b < 1 ? 1 : b), 256, 0, st>>>(n, a0, X0, a1, X1, out);
}

void launch_fill_one(double2* v, int count, cudaStream_t st) {
  k_fill_one<<<(count + 255) / 256, 256, 0, st>>>(v, count);
}

void launch_amplitudes(const double2* gamma, const double* lambda, const int* chi, int n, int cap,
                       const unsigned char* bits, int count, double2* out, cudaStream_t st) {
  k_amplitudes<<<count, 256, 2 * cap * sizeof(double2), st>>>(gamma, lambda, chi, n, cap, bits, out);
}

void launch_scale_site(const double2* g, const double* lam, int xl, int xr, int cap, double2* out, cudaStream_t st) {
  int el = 2 * xl * xr;
  int bx = (el + 255) / 256;
  if (bx > 1024) bx = 1024;
  k_scale_site<<<bx, 256, 0, st>>>(g, lam, xl, xr, cap, out);
}

void launch_zgemm(int M, int N, int K, const double2* A, int lda, long long sA, int transA, const double2* B,
                  int ldb, long long sB, int conjB, int transB, double2* C, int ldc, long long sC, int accumulate,
                  long long batch, cudaStream_t st) {
  // the batch runs in grid.z chunks of at most 65535
  for (long long b0 = 0; b0 < batch; b0 += 65535) {
    const int nb = (int)(batch - b0 < 65535 ? batch - b0 : 65535);
    dim3 g((N + 15) / 16, (M + 15) / 16, nb);
    k_zgemm<<<g, 256, 0, st>>>(M, N, K, A + sA * b0, lda, sA, transA, B + sB * b0, ldb, sB, conjB, transB,
                               C + sC * b0, ldc, sC, accumulate);
  }
}

}  // namespace mpsgb

// The second workload of the paper's matrix library (Sec. 2 and its NMR
// example): diagonalisation of Hermitian matrices, functions of them (exp_H,
// the thermal state exp(-beta H) / Tr), the free-induction-decay record of an
// observable under H, and the modulus of its zero-padded discrete Fourier
// transform, batched over many independent problems.
//
//   k_heev      - cyclic two-sided Jacobi on one D x D Hermitian matrix per
//                 CTA (D <= 64), H and the accumulated eigenvectors V in
//                 shared memory; each round rotates the D/2 disjoint pairs of
//                 a round-robin ordering: all row rotations, then all column
//                 rotations, then the pair's diagonal entries set and its
//                 off-diagonal entries zeroed (the same 2 x 2 Hermitian Schur
//                 rotation as the inner solve of the blocked Jacobi SVD)
//   k_hfun      - V diag(f(lambda)) V^H for f = exp(a x) or the Boltzmann weights
//   k_fid_prep  - rho' = P rho P^H, then rho~ = V^H rho' V and O~ = V^H O V
//   k_fid       - s(t_m) = sum_jk rho~_jk O~_kj exp(-i (lambda_j - lambda_k) m dt)
//   k_fft_*     - radix-2 decimation-in-time FFT of the zero-padded record
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mps.h"
#include "kernels.cuh"

using namespace mpsgb;

namespace {

constexpr int kHMaxD = 64;
constexpr int kHThreads = 256;
constexpr double kHEps = 1.1102230246251565e-16;  // 2^-53
constexpr int kHMaxSweeps = 60;

__device__ __forceinline__ double2 cmulh(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 conjh(double2 a) { return make_double2(a.x, -a.y); }

__device__ __forceinline__ void h_pair(int nbe, int r, int p, int& I, int& J) {
  if (p == 0) {
    I = nbe - 1;
    J = r;
  } else {
    I = (r + p) % (nbe - 1);
    J = (r - p + nbe - 1) % (nbe - 1);
  }
}

// Dynamic shared memory: Hs[D][D+1], Vs[D][D+1] (double2), then per pair of a
// round: c, t|g|, h_pp, h_qq (double), s e^{i phi} (double2), on (int).
size_t heev_smem(int D) {
  const int nbe = D + (D & 1);
  return 2 * (size_t)D * (D + 1) * sizeof(double2) + (size_t)(nbe / 2) * (4 * sizeof(double) + sizeof(double2)) +
         (size_t)(nbe / 2) * sizeof(int) + 64;
}

__global__ void __launch_bounds__(kHThreads) k_heev(int D, const double2* __restrict__ Hg, double* __restrict__ wg,
                                                    double2* __restrict__ Vg, int* __restrict__ status,
                                                    int max_sweeps, int* __restrict__ sweeps_out,
                                                    unsigned long long* __restrict__ rotations) {
  extern __shared__ __align__(16) unsigned char hsm[];
  const int b = blockIdx.x, tid = threadIdx.x;
  const int ld = D + 1, nbe = D + (D & 1), np = nbe / 2;
  double2* Hs = (double2*)hsm;
  double2* Vs = Hs + (size_t)D * ld;
  double* rc_c = (double*)(Vs + (size_t)D * ld);
  double* rc_tg = rc_c + np;
  double* rc_a = rc_tg + np;
  double* rc_b = rc_a + np;
  double2* rc_se = (double2*)(rc_b + np);
  int* rc_on = (int*)(rc_se + np);
  __shared__ double red[kHThreads / 32];
  __shared__ int any;
  __shared__ unsigned int nrot;
  if (tid == 0) nrot = 0;
  const double2* H = Hg + (size_t)b * D * D;
  double f = 0.0;
  for (int e = tid; e < D * D; e += kHThreads) {
    const int r = e / D, c = e % D;
    const double2 h = H[e];
    Hs[r * ld + c] = h;
    Vs[r * ld + c] = make_double2(r == c ? 1.0 : 0.0, 0.0);
    f += h.x * h.x + h.y * h.y;
  }
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) f += __shfl_xor_sync(0xffffffffu, f, m);
  if ((tid & 31) == 0) red[tid >> 5] = f;
  __syncthreads();
  double frob2 = 0.0;
  for (int w = 0; w < kHThreads / 32; ++w) frob2 += red[w];
  const double tol = (double)D * kHEps * sqrt(frob2);
  int sweep = 0;
  bool conv = false;
  while (sweep < max_sweeps) {
    __syncthreads();
    if (tid == 0) any = 0;
    __syncthreads();
    for (int r = 0; r < nbe - 1; ++r) {
      if (tid < np) {
        int p, q;
        h_pair(nbe, r, tid, p, q);
        int on = 0;
        if (p < D && q < D) {
          const double al = Hs[p * ld + p].x, be = Hs[q * ld + q].x;
          const double2 g = Hs[p * ld + q];
          const double g2 = g.x * g.x + g.y * g.y;
          if (sqrt(g2) > tol) {
            // [al g; conj(g) be] = D [al |g|; |g| be] D^H, D = diag(e^{i phi}, 1):
            // the real symmetric Schur rotation of the middle matrix with
            // t e^{i phi} = 2 sign(d) g / (|d| + sqrt(d^2 + 4|g|^2)), d = be - al
            const double d = be - al;
            const double sg = (d < 0.0 ? -2.0 : 2.0) / (fabs(d) + sqrt(d * d + 4.0 * g2));
            const double tx = sg * g.x, ty = sg * g.y;
            const double c = 1.0 / sqrt(1.0 + tx * tx + ty * ty);
            rc_c[tid] = c;
            rc_tg[tid] = sg * g2;
            rc_a[tid] = al;
            rc_b[tid] = be;
            rc_se[tid] = make_double2(c * tx, c * ty);
            on = 1;
            any = 1;
            atomicAdd(&nrot, 1u);
          }
        }
        rc_on[tid] = on;
      }
      __syncthreads();
      // rows: H <- J^H H (row p: c H_p - s e^{i phi} H_q ; row q: s e^{-i phi} H_p + c H_q)
      for (int e = tid; e < np * D; e += kHThreads) {
        const int pr = e / D, col = e % D;
        if (!rc_on[pr]) continue;
        int p, q;
        h_pair(nbe, r, pr, p, q);
        const double c = rc_c[pr];
        const double2 se = rc_se[pr];
        const double2 x = Hs[p * ld + col], y = Hs[q * ld + col];
        const double2 sy = cmulh(se, y), cx = cmulh(conjh(se), x);
        Hs[p * ld + col] = make_double2(c * x.x - sy.x, c * x.y - sy.y);
        Hs[q * ld + col] = make_double2(cx.x + c * y.x, cx.y + c * y.y);
      }
      __syncthreads();
      // columns: H <- H J and V <- V J (col p: c a_p - s e^{-i phi} a_q ; col q: s e^{i phi} a_p + c a_q)
      for (int e = tid; e < 2 * np * D; e += kHThreads) {
        const int which = e / (np * D), rem = e % (np * D);
        const int pr = rem / D, row = rem % D;
        if (!rc_on[pr]) continue;
        int p, q;
        h_pair(nbe, r, pr, p, q);
        double2* M = which ? Vs : Hs;
        const double c = rc_c[pr];
        const double2 se = rc_se[pr];
        const double2 x = M[row * ld + p], y = M[row * ld + q];
        const double2 sy = cmulh(conjh(se), y), sx = cmulh(se, x);
        M[row * ld + p] = make_double2(c * x.x - sy.x, c * x.y - sy.y);
        M[row * ld + q] = make_double2(sx.x + c * y.x, sx.y + c * y.y);
      }
      __syncthreads();
      if (tid < np && rc_on[tid]) {
        int p, q;
        h_pair(nbe, r, tid, p, q);
        Hs[p * ld + p] = make_double2(rc_a[tid] - rc_tg[tid], 0.0);
        Hs[q * ld + q] = make_double2(rc_b[tid] + rc_tg[tid], 0.0);
        Hs[p * ld + q] = make_double2(0.0, 0.0);
        Hs[q * ld + p] = make_double2(0.0, 0.0);
      }
      __syncthreads();
    }
    ++sweep;
    __syncthreads();
    if (!any) {
      conv = true;
      break;
    }
  }
  // ascending eigenvalues (ties by index), eigenvectors as the columns of V
  for (int j = tid; j < D; j += kHThreads) {
    const double lj = Hs[j * ld + j].x;
    int rank = 0;
    for (int i = 0; i < D; ++i) {
      const double li = Hs[i * ld + i].x;
      rank += (li < lj) || (li == lj && i < j);
    }
    wg[(size_t)b * D + rank] = lj;
    for (int r = 0; r < D; ++r) Vg[(size_t)b * D * D + (size_t)r * D + rank] = Vs[r * ld + j];
  }
  if (tid == 0) {
    if (!conv) atomicCAS(status, 0, MPS_ERR_NOCONVERGE);
    atomicMax(sweeps_out, sweep);
    atomicAdd(rotations, (unsigned long long)nrot);
  }
}

// out = V diag(f) V^H with f_k = exp(a lambda_k) (kind 0, a complex), the
// Boltzmann weights exp(-beta (lambda_k - lambda_0)) / Z (kind 1, beta = a.x),
// or those weights minus 1/D (kind 2, the thermal state minus I/D).
__global__ void k_hfun(int D, const double* __restrict__ w, const double2* __restrict__ V, int kind, double2 a,
                       double2* __restrict__ out) {
  __shared__ double2 fk[kHMaxD];
  __shared__ double Z;
  const int b = blockIdx.x, tid = threadIdx.x;
  const double* wb = w + (size_t)b * D;
  const double2* Vb = V + (size_t)b * D * D;
  if (tid < D) {
    if (kind == 0) {
      const double mag = exp(a.x * wb[tid]);
      double sn, cs;
      sincos(a.y * wb[tid], &sn, &cs);
      fk[tid] = make_double2(mag * cs, mag * sn);
    } else {
      const double ref = a.x >= 0.0 ? wb[0] : wb[D - 1];  // the largest weight is 1
      // kind 1: e^{-beta (lambda_k - ref)}; kind 2: expm1 of the same exponent
      fk[tid] = make_double2(kind == 1 ? exp(-a.x * (wb[tid] - ref)) : expm1(-a.x * (wb[tid] - ref)), 0.0);
    }
  }
  __syncthreads();
  if (tid == 0) {
    double z = 0.0;
    for (int k = 0; k < D; ++k) z += fk[k].x;
    if (kind == 2) {
      // p_k - 1/D = (e_k - mean e) / (D (1 + mean e)) with e_k = expm1(...):
      // no cancellation against 1/D when beta (lambda - ref) is small
      const double mean = z / D;
      for (int k = 0; k < D; ++k) fk[k].x -= mean;
      z = D * (1.0 + mean);
    }
    Z = kind == 0 ? 1.0 : z;
  }
  __syncthreads();
  const double iz = 1.0 / Z;
  for (int e = tid; e < D * D; e += blockDim.x) {
    const int r = e / D, c = e % D;
    double2 acc = make_double2(0.0, 0.0);
    for (int k = 0; k < D; ++k) {
      const double2 t = cmulh(cmulh(Vb[(size_t)r * D + k], fk[k]), conjh(Vb[(size_t)c * D + k]));
      acc.x += t.x;
      acc.y += t.y;
    }
    out[(size_t)b * D * D + e] = make_double2(acc.x * iz, acc.y * iz);
  }
}

// rho' = P rho P^H (P may be null), rho~ = V^H rho' V, O~ = V^H O V;
// A[j,k] = rho~_jk O~_kj. Shared: three D x D tiles.
__global__ void k_fid_prep(int D, const double2* __restrict__ rho, const double2* __restrict__ O,
                           const double2* __restrict__ P, const double2* __restrict__ V, double2* __restrict__ A) {
  extern __shared__ __align__(16) unsigned char fsm[];
  double2* T0 = (double2*)fsm;
  double2* T1 = T0 + D * D;
  double2* T2 = T1 + D * D;
  const int b = blockIdx.x, tid = threadIdx.x;
  const double2* Vb = V + (size_t)b * D * D;
  const double2* rb = rho + (size_t)b * D * D;
  const double2* Ob = O + (size_t)b * D * D;
  const double2* Pb = P ? P + (size_t)b * D * D : nullptr;
  const double2 z = make_double2(0.0, 0.0);
  // T0 = P rho (or rho)
  for (int e = tid; e < D * D; e += blockDim.x) {
    const int r = e / D, c = e % D;
    if (!Pb) {
      T0[e] = rb[e];
      continue;
    }
    double2 acc = z;
    for (int k = 0; k < D; ++k) {
      const double2 t = cmulh(Pb[(size_t)r * D + k], rb[(size_t)k * D + c]);
      acc.x += t.x;
      acc.y += t.y;
    }
    T0[e] = acc;
  }
  __syncthreads();
  // T1 = T0 P^H (or T0)
  for (int e = tid; e < D * D; e += blockDim.x) {
    const int r = e / D, c = e % D;
    if (!Pb) {
      T1[e] = T0[e];
      continue;
    }
    double2 acc = z;
    for (int k = 0; k < D; ++k) {
      const double2 t = cmulh(T0[r * D + k], conjh(Pb[(size_t)c * D + k]));
      acc.x += t.x;
      acc.y += t.y;
    }
    T1[e] = acc;
  }
  __syncthreads();
  // T2 = V^H T1
  for (int e = tid; e < D * D; e += blockDim.x) {
    const int r = e / D, c = e % D;
    double2 acc = z;
    for (int k = 0; k < D; ++k) {
      const double2 t = cmulh(conjh(Vb[(size_t)k * D + r]), T1[k * D + c]);
      acc.x += t.x;
      acc.y += t.y;
    }
    T2[e] = acc;
  }
  __syncthreads();
  // T0 = rho~ = T2 V
  for (int e = tid; e < D * D; e += blockDim.x) {
    const int r = e / D, c = e % D;
    double2 acc = z;
    for (int k = 0; k < D; ++k) {
      const double2 t = cmulh(T2[r * D + k], Vb[(size_t)k * D + c]);
      acc.x += t.x;
      acc.y += t.y;
    }
    T0[e] = acc;
  }
  __syncthreads();
  // T2 = V^H O
  for (int e = tid; e < D * D; e += blockDim.x) {
    const int r = e / D, c = e % D;
    double2 acc = z;
    for (int k = 0; k < D; ++k) {
      const double2 t = cmulh(conjh(Vb[(size_t)k * D + r]), Ob[(size_t)k * D + c]);
      acc.x += t.x;
      acc.y += t.y;
    }
    T2[e] = acc;
  }
  __syncthreads();
  // T1 = O~ = T2 V ; A[j,k] = rho~_jk O~_kj
  for (int e = tid; e < D * D; e += blockDim.x) {
    const int r = e / D, c = e % D;
    double2 acc = z;
    for (int k = 0; k < D; ++k) {
      const double2 t = cmulh(T2[r * D + k], Vb[(size_t)k * D + c]);
      acc.x += t.x;
      acc.y += t.y;
    }
    T1[e] = acc;
  }
  __syncthreads();
  for (int e = tid; e < D * D; e += blockDim.x) {
    const int j = e / D, k = e % D;
    A[(size_t)b * D * D + e] = cmulh(T0[j * D + k], T1[k * D + j]);
  }
}

// s[b][m] = sum_jk A[j,k] exp(-i (lambda_j - lambda_k) m dt), one thread per
// sample; A and the frequency differences staged in shared memory.
__global__ void k_fid(int D, const double2* __restrict__ A, const double* __restrict__ w, double dt, int N,
                      double2* __restrict__ sig) {
  extern __shared__ __align__(16) unsigned char ssm[];
  double2* As = (double2*)ssm;
  double* Ws = (double*)(As + D * D);
  const int b = blockIdx.y, tid = threadIdx.x;
  for (int e = tid; e < D * D; e += blockDim.x) As[e] = A[(size_t)b * D * D + e];
  for (int e = tid; e < D; e += blockDim.x) Ws[e] = w[(size_t)b * D + e];
  __syncthreads();
  const int m = blockIdx.x * blockDim.x + tid;
  if (m >= N) return;
  const double t = (double)m * dt;
  double sx = 0.0, sy = 0.0;
  for (int j = 0; j < D; ++j)
    for (int k = 0; k < D; ++k) {
      double sn, cs;
      sincos(-(Ws[j] - Ws[k]) * t, &sn, &cs);
      const double2 a = As[j * D + k];
      sx += a.x * cs - a.y * sn;
      sy += a.x * sn + a.y * cs;
    }
  sig[(size_t)b * N + m] = make_double2(sx, sy);
}

// bit-reversed copy of x (n_in values, zero-padded to L = 2^p)
__global__ void k_fft_load(int n_in, int p, const double2* __restrict__ x, double2* __restrict__ y) {
  const int b = blockIdx.y;
  const int L = 1 << p;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L; i += gridDim.x * blockDim.x) {
    const int j = (int)(__brev((unsigned)i) >> (32 - p));
    y[(size_t)b * L + j] = i < n_in ? x[(size_t)b * n_in + i] : make_double2(0.0, 0.0);
  }
}

// one butterfly stage of half-size h: x_i, x_j <- x_i + w x_j, x_i - w x_j,
// w = exp(-2 pi i pos / (2h))
__global__ void k_fft_stage(int p, int h, double2* __restrict__ y) {
  const int b = blockIdx.y;
  const int L = 1 << p;
  double2* yb = y + (size_t)b * L;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < L / 2; t += gridDim.x * blockDim.x) {
    const int grp = t / h, pos = t % h;
    const int i = grp * 2 * h + pos, j = i + h;
    double sn, cs;
    sincospi(-(double)pos / (double)h, &sn, &cs);
    const double2 xi = yb[i], xj = yb[j];
    const double2 wx = make_double2(cs * xj.x - sn * xj.y, cs * xj.y + sn * xj.x);
    yb[i] = make_double2(xi.x + wx.x, xi.y + wx.y);
    yb[j] = make_double2(xi.x - wx.x, xi.y - wx.y);
  }
}

__global__ void k_fft_abs(long long total, const double2* __restrict__ y, double* __restrict__ out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = hypot(y[e].x, y[e].y);
}

int h_fail(int code, const std::string& msg) {
  set_error_message(msg.c_str());
  return code;
}

#define HCK(call)                                                                             \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return h_fail(e_ == cudaErrorMemoryAllocation ? MPS_ERR_NOMEM : MPS_ERR_CUDA,           \
                    std::string(#call) + ": " + cudaGetErrorString(e_));                      \
  } while (0)

// scratch freed on every return path
struct Scratch {
  std::vector<void*> p;
  ~Scratch() {
    for (void* q : p) cudaFree(q);
  }
  cudaError_t get(void** out, size_t bytes) {
    cudaError_t e = dev_alloc(out, bytes);
    if (e == cudaSuccess) p.push_back(*out);
    return e;
  }
};

thread_local long long g_last_sweeps = 0, g_last_rotations = 0;

int heev_run(int count, int D, const double2* H, double* w, double2* V, cudaStream_t st, Scratch& sc) {
  int* d_st = nullptr;
  HCK(sc.get((void**)&d_st, 4 * sizeof(int)));  // status, sweeps, rotations (64-bit, 8-aligned)
  HCK(cudaMemsetAsync(d_st, 0, 4 * sizeof(int), st));
  const size_t smem = heev_smem(D);
  HCK(cudaFuncSetAttribute(k_heev, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_heev<<<count, kHThreads, smem, st>>>(D, H, w, V, d_st, kHMaxSweeps, d_st + 1,
                                         (unsigned long long*)(d_st + 2));
  HCK(cudaGetLastError());
  int hs[4] = {0, 0, 0, 0};
  HCK(cudaMemcpyAsync(hs, d_st, sizeof(hs), cudaMemcpyDeviceToHost, st));
  HCK(cudaStreamSynchronize(st));
  unsigned long long rot = 0;
  std::memcpy(&rot, hs + 2, sizeof(rot));
  g_last_sweeps = hs[1];
  g_last_rotations = (long long)rot;
  if (hs[0] != 0) return h_fail(hs[0], "Hermitian Jacobi hit its sweep limit");
  return MPS_OK;
}

int check_dims(int count, int D) {
  if (count < 1 || D < 1) return h_fail(MPS_ERR_ARG, "need count >= 1 and D >= 1");
  if (D > kHMaxD) return h_fail(MPS_ERR_TOO_LARGE, "matrix dimension above 64");
  return MPS_OK;
}

}  // namespace

extern "C" {

int mps_heev_batched(int count, int D, const double* d_H, double* d_w, double* d_V, void* stream) {
  int rc = check_dims(count, D);
  if (rc != MPS_OK) return rc;
  if (!d_H || !d_w || !d_V) return h_fail(MPS_ERR_ARG, "null pointer");
  Scratch sc;
  return heev_run(count, D, (const double2*)d_H, d_w, (double2*)d_V, (cudaStream_t)stream, sc);
}

int mps_hermitian_function_batched(int count, int D, const double* d_H, int kind, double a_re, double a_im,
                                   double* d_out, void* stream) {
  int rc = check_dims(count, D);
  if (rc != MPS_OK) return rc;
  if (!d_H || !d_out || kind < 0 || kind > 2) return h_fail(MPS_ERR_ARG, "bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  Scratch sc;
  double* w = nullptr;
  double2* V = nullptr;
  HCK(sc.get((void**)&w, (size_t)count * D * sizeof(double)));
  HCK(sc.get((void**)&V, (size_t)count * D * D * sizeof(double2)));
  rc = heev_run(count, D, (const double2*)d_H, w, V, st, sc);
  if (rc != MPS_OK) return rc;
  k_hfun<<<count, 128, 0, st>>>(D, w, V, kind, make_double2(a_re, a_im), (double2*)d_out);
  HCK(cudaGetLastError());
  HCK(cudaStreamSynchronize(st));
  return MPS_OK;
}

int mps_fid_batched(int count, int D, const double* d_rho, const double* d_H, const double* d_O, const double* d_P,
                    double dt, int N, double* d_signal, void* stream) {
  int rc = check_dims(count, D);
  if (rc != MPS_OK) return rc;
  if (!d_rho || !d_H || !d_O || !d_signal || N < 1 || !(dt == dt)) return h_fail(MPS_ERR_ARG, "bad argument");
  if (count > 65535) return h_fail(MPS_ERR_TOO_LARGE, "count above 65535");
  cudaStream_t st = (cudaStream_t)stream;
  Scratch sc;
  double* w = nullptr;
  double2 *V = nullptr, *A = nullptr;
  HCK(sc.get((void**)&w, (size_t)count * D * sizeof(double)));
  HCK(sc.get((void**)&V, (size_t)count * D * D * sizeof(double2)));
  HCK(sc.get((void**)&A, (size_t)count * D * D * sizeof(double2)));
  rc = heev_run(count, D, (const double2*)d_H, w, V, st, sc);
  if (rc != MPS_OK) return rc;
  const size_t s1 = 3 * (size_t)D * D * sizeof(double2);
  HCK(cudaFuncSetAttribute(k_fid_prep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s1));
  k_fid_prep<<<count, 256, s1, st>>>(D, (const double2*)d_rho, (const double2*)d_O, (const double2*)d_P, V, A);
  HCK(cudaGetLastError());
  const size_t s2 = (size_t)D * D * sizeof(double2) + (size_t)D * sizeof(double);
  HCK(cudaFuncSetAttribute(k_fid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s2));
  dim3 grid((N + 127) / 128, count);
  k_fid<<<grid, 128, s2, st>>>(D, A, w, dt, N, (double2*)d_signal);
  HCK(cudaGetLastError());
  HCK(cudaStreamSynchronize(st));
  return MPS_OK;
}

int mps_hermitian_last_stats(long long* max_sweeps, long long* rotations) {
  if (max_sweeps) *max_sweeps = g_last_sweeps;
  if (rotations) *rotations = g_last_rotations;
  return MPS_OK;
}

int mps_dft_abs_batched(int count, int n_in, const double* d_x, int n_out, double* d_abs, void* stream) {
  if (count < 1 || count > 65535 || n_in < 1 || n_out < n_in || !d_x || !d_abs)
    return h_fail(MPS_ERR_ARG, "bad argument");
  int p = 0;
  while ((1 << p) < n_out) ++p;
  if ((1 << p) != n_out || p < 1 || p > 26) return h_fail(MPS_ERR_ARG, "n_out must be a power of two in [2, 2^26]");
  cudaStream_t st = (cudaStream_t)stream;
  Scratch sc;
  double2* y = nullptr;
  HCK(sc.get((void**)&y, (size_t)count * n_out * sizeof(double2)));
  const int blocks = std::min(1024, (n_out + 255) / 256);
  k_fft_load<<<dim3(blocks, count), 256, 0, st>>>(n_in, p, (const double2*)d_x, y);
  HCK(cudaGetLastError());
  for (int h = 1; h < n_out; h <<= 1) {
    k_fft_stage<<<dim3(std::max(1, std::min(1024, (n_out / 2 + 255) / 256)), count), 256, 0, st>>>(p, h, y);
    HCK(cudaGetLastError());
  }
  const long long total = (long long)count * n_out;
  k_fft_abs<<<(int)std::min<long long>(4096, (total + 255) / 256), 256, 0, st>>>(total, y, d_abs);
  HCK(cudaGetLastError());
  HCK(cudaStreamSynchronize(st));
  return MPS_OK;
}

}  // extern "C"

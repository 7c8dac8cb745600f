// Randomized range-finder SVD of a gate update's working matrix A (Mw x Nw),
// sized by the rank predictor (Halko, Martinsson & Tropp, SIAM Review 53,
// 2011): Omega Gaussian (Nw x r), Y = A Omega, Q = orth(Y) by the one-sided
// Jacobi kernels, B^H = A^H Q, residual ||A - Q B||_F; when the
// residual is within the truncation threshold, the SVD of B gives A's
// leading singular triplets, otherwise the full Jacobi SVD runs.
//
// Omega: Philox4x32-10 counter-based generator (Salmon, Moraes, Dror & Shaw,
// SC 2011) keyed by a seed, counter (row, column, task), Box-Muller normals.
#include <cuda_runtime.h>

#include <cstdint>

#include "engine.cuh"
#include "kernels.cuh"
#include "sketch.cuh"

namespace mpsgb {

// ---------------------------------------------------------------- Philox ---

__device__ __forceinline__ void philox_round(uint32_t c[4], uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
  const uint32_t hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
  const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
  c[0] = n0;
  c[1] = lo1;
  c[2] = n2;
  c[3] = lo0;
}

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    philox_round(c, k0, k1);
    k0 += W0;
    k1 += W1;
  }
}

// Complex standard normal entries (E|z|^2 = 1) of Omega for every sketch task.
__global__ void k_omega(const SketchTask* st, unsigned long long seed) {
  const SketchTask& s = st[blockIdx.y];
  const size_t total = (size_t)s.Nw * s.r;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const uint32_t i = (uint32_t)(e % s.Nw), j = (uint32_t)(e / s.Nw);
    uint32_t c[4] = {i, j, (uint32_t)s.id, 0x5eed5u};
    philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    const double u1 = ((double)c[0] + 0.5) * 2.3283064365386963e-10;  // (0, 1)
    const double u2 = ((double)c[1] + 0.5) * 2.3283064365386963e-10;
    const double rad = sqrt(-log(u1));  // Box-Muller with variance 1/2 per component
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    s.Om[(size_t)i + (size_t)j * s.Nw] = make_double2(rad * cs, rad * sn);
  }
}

// Q = Y / sigma_y column by column. The Jacobi leaves columns with
// ||y|| <= Mw eps ||Y||_F unrotated (numerically zero), so they are not
// orthogonal to the others: Q drops every column up to twice that bound.
__global__ void k_scale_q(const SketchTask* st, const double* sig, const TaskMeta* mety) {
  const SketchTask& s = st[blockIdx.y];
  const double* sg = sig + (size_t)blockIdx.y * s.rcap;
  const double tiny = 2.0 * (double)s.Mw * 1.1102230246251565e-16 * sqrt(mety[blockIdx.y].frob2);
  const size_t total = (size_t)s.Mw * s.r;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / s.Mw);
    const double f = sg[j] > tiny ? 1.0 / sg[j] : 0.0;
    const double2 v = s.Y[e];
    s.Y[e] = make_double2(v.x * f, v.y * f);
  }
}

// res[t] += sum |A - T2|^2 over the task's Mw x Nw entries
__global__ void k_residual(const SketchTask* st, double* res) {
  const SketchTask& s = st[blockIdx.y];
  const size_t total = (size_t)s.Mw * s.Nw;
  double acc = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const double2 a = s.A[e], t = s.T2[e];
    const double dx = a.x - t.x, dy = a.y - t.y;
    acc = fma(dx, dx, fma(dy, dy, acc));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(&res[blockIdx.y], acc);
}

// Accepted sketch: V[:, j] = (B^H Wb)[:, j] / sigma'_j for j < r, zero for
// j >= r; A[:, j >= r] = 0 (A[:, j < r] was written by the product Q Wb diag(sigma')).
__global__ void k_sketch_finish(const SketchTask* st, const double* sigb, const int* accept) {
  const SketchTask& s = st[blockIdx.y];
  if (!accept[blockIdx.y]) return;
  const double* sg = sigb + (size_t)blockIdx.y * s.rcap;
  const size_t nv = (size_t)s.Nw * s.Nw, na = (size_t)s.Mw * s.Nw;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nv + na; e += (size_t)gridDim.x * blockDim.x) {
    if (e < nv) {
      const int j = (int)(e / s.Nw), i = (int)(e % s.Nw);
      double2 v = make_double2(0.0, 0.0);
      if (j < s.r && sg[j] > 0.0) {
        const double2 b = s.Bh[(size_t)i + (size_t)j * s.Nw];
        v = make_double2(b.x / sg[j], b.y / sg[j]);
      }
      s.V[e] = v;
    } else {
      const size_t f = e - nv;
      if ((int)(f / s.Mw) >= s.r) s.A[f] = make_double2(0.0, 0.0);
    }
  }
}

// Marks accepted tasks done (no full SVD) and adds the sketch residual to the
// discarded weight; rejected tasks stay active for the full Jacobi SVD.
// Acceptance: ||A - Q Q^H A||_F <= delta ||A||_F with delta = max(cutoff / 100,
// Mw eps). A projection moves a singular value sigma_i by at most
// delta^2 ||A||^2 / sigma_i, so every value the cutoff keeps
// (sigma_i > cutoff ||A||) moves by less than 1e-4 cutoff ||A||.
__global__ void k_sketch_mark(const SketchTask* st, int n, const double* res, int* accept, TaskMeta* meta) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const SketchTask& s = st[t];
  TaskMeta& m = meta[s.task];
  const double thr = fmax(0.01 * s.cutoff, (double)s.Mw * 1.1102230246251565e-16);
  const int ok = m.status == 0 && res[t] <= thr * thr * m.frob2;
  accept[t] = ok;
  if (ok) {
    m.active = 0;
    m.disc += m.frob2 > 0.0 ? res[t] / m.frob2 : 0.0;
  }
}

static inline int gridn(long long el) {
  long long b = (el + 255) / 256;
  if (b > 512) b = 512;
  if (b < 1) b = 1;
  return (int)b;
}

void launch_omega(const SketchTask* st, int n, long long el_ub, unsigned long long seed, cudaStream_t s) {
  k_omega<<<dim3(gridn(el_ub), n), 256, 0, s>>>(st, seed);
}
void launch_scale_q(const SketchTask* st, int n, long long el_ub, const double* sig, const TaskMeta* mety,
                    cudaStream_t s) {
  k_scale_q<<<dim3(gridn(el_ub), n), 256, 0, s>>>(st, sig, mety);
}
void launch_residual(const SketchTask* st, int n, long long el_ub, double* res, cudaStream_t s) {
  k_residual<<<dim3(gridn(el_ub), n), 256, 0, s>>>(st, res);
}
void launch_sketch_mark(const SketchTask* st, int n, const double* res, int* accept, TaskMeta* meta, cudaStream_t s) {
  k_sketch_mark<<<(n + 127) / 128, 128, 0, s>>>(st, n, res, accept, meta);
}
void launch_sketch_finish(const SketchTask* st, int n, long long el_ub, const double* sigb, const int* accept,
                          cudaStream_t s) {
  k_sketch_finish<<<dim3(gridn(el_ub), n), 256, 0, s>>>(st, sigb, accept);
}

}  // namespace mpsgb

// Beyond binary64: the gate update of Sec. 3.1 in double-double arithmetic
// (about 106 significant bits) for small bond dimensions (chi_max <= 32).
//
// The paper's library runs the whole simulation in MPFR multiprecision
// (Sec. 1, Sec. 3.2 sets 256 bits) because the truncated Schmidt spectra of
// Eq. (2) span many orders of magnitude. This path keeps the state of Eq. (1)
// (Gamma and Lambda) as double-words and runs every step of the update in
// double-word arithmetic (dd.cuh): theta formation with the gate, the
// one-sided Jacobi SVD (rotation angles, the orthogonality test and the
// column updates), truncation and renormalisation, and the Lambda^-1 rewrite.
//
// Kernels (one CTA per gate of a layer of disjoint gates):
//   k_dd_theta  - theta of (s, s+1) with the Lambda weights and the gate, into
//                 the Jacobi working matrix (theta, or theta^H when wide)
//   k_dd_precondition - binary64 sweeps on the high parts, then A <- A V1
//                 with V1 the binary64 right factor made unitary in
//                 double-word (the double-word sweeps start nearly converged)
//   k_dd_jacobi - cyclic one-sided Jacobi in round-robin order: each warp
//                 takes one column pair of a round, lanes stride the rows,
//                 the three inner products are reduced across the warp by
//                 shuffles; sweeps run until no pair needs a rotation
//   k_dd_finish - order, truncation, renormalisation, rewrite of Gamma_s,
//                 Lambda_s, Gamma_{s+1} and the new bond dimension
// The bond dimensions stay on the device; every kernel reads them there, and
// the grids are sized by chi_max, so a layer needs no host round trip.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mps.h"
#include "dd.cuh"
#include "kernels.cuh"

using namespace mpsgb;

namespace {

constexpr int kDdMaxCap = 32;
constexpr int kDdW = 2 * kDdMaxCap;              // largest working-matrix dimension
constexpr double kEpsDd = 4.930380657631324e-32;  // 2^-104: resolution of the double-word Jacobi
constexpr int kDdThreads = 512;
constexpr int kDdWarps = kDdThreads / 32;
constexpr int kDdStages = 4;  // pinned staging slots for host gates

// executed binary64 operations of the Jacobi kernel, per row and per pair
constexpr long long kDdDotFlopsPerRow = 2 * (2 * 8 + kFlopsDdAdd + kFlopsDdAdd) + kFlopsCddMul + 2 * kFlopsDdAdd;
constexpr long long kDdRotFlopsPerRow = 2 * (2 * kFlopsDdMul + kFlopsCddMul + 2 * kFlopsDdAdd);

struct DdMeta {
  int mw, nw, tall, status, sweeps, site;
};

__device__ __forceinline__ cdd load_gate(const double* hi, const double* lo, int e) {
  const dd re = lo ? two_sum(hi[2 * e], lo[2 * e]) : dd_make(hi[2 * e]);
  const dd im = lo ? two_sum(hi[2 * e + 1], lo[2 * e + 1]) : dd_make(hi[2 * e + 1]);
  return cdd{re, im};
}

__device__ __forceinline__ void dd_pair(int nbe, int r, int p, int& I, int& J) {
  if (p == 0) {
    I = nbe - 1;
    J = r;
  } else {
    I = (r + p) % (nbe - 1);
    J = (r - p + nbe - 1) % (nbe - 1);
  }
}

__global__ void k_dd_reset(cdd* G, dd* L, int* chi, int n, int cap) {
  const long long gsz = (long long)n * 2 * cap * cap;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < gsz; e += (long long)gridDim.x * blockDim.x) {
    const long long site_off = e % (2LL * cap * cap);
    G[e] = cdd_make(site_off == 0 ? 1.0 : 0.0, 0.0);
  }
  const long long lsz = (long long)(n + 1) * cap;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < lsz; e += (long long)gridDim.x * blockDim.x)
    L[e] = dd_make(e % cap == 0 ? 1.0 : 0.0);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e <= n; e += (long long)gridDim.x * blockDim.x)
    chi[e] = 1;
}

// Gamma_s[i] <- sum_k u[i,k] Gamma_s[k]
__global__ void k_dd_apply1(cdd* G, const int* chi, int cap, const int* sites, const double* Uhi, const double* Ulo) {
  const int g = blockIdx.x, s = sites[g];
  const cdd u00 = load_gate(Uhi + 8 * g, Ulo ? Ulo + 8 * g : nullptr, 0);
  const cdd u01 = load_gate(Uhi + 8 * g, Ulo ? Ulo + 8 * g : nullptr, 1);
  const cdd u10 = load_gate(Uhi + 8 * g, Ulo ? Ulo + 8 * g : nullptr, 2);
  const cdd u11 = load_gate(Uhi + 8 * g, Ulo ? Ulo + 8 * g : nullptr, 3);
  const int xl = chi[s], xr = chi[s + 1];
  cdd* G0 = G + (size_t)s * 2 * cap * cap;
  cdd* G1 = G0 + (size_t)cap * cap;
  for (int e = threadIdx.x; e < xl * xr; e += blockDim.x) {
    const int a = e / xr, c = e % xr;
    const cdd x0 = G0[(size_t)a * cap + c], x1 = G1[(size_t)a * cap + c];
    G0[(size_t)a * cap + c] = cdd_add(cdd_mul(u00, x0), cdd_mul(u01, x1));
    G1[(size_t)a * cap + c] = cdd_add(cdd_mul(u10, x0), cdd_mul(u11, x1));
  }
}

// theta[(i,a),(j,c)] = sum_{kl} U[(ij),(kl)] T_kl[a,c],
// T_kl[a,c] = Lambda_{s-1}[a] Lambda_{s+1}[c] sum_b Gamma_s[k,a,b] Lambda_s[b] Gamma_{s+1}[l,b,c];
// rows i*xl + a, columns j*xr + c. The working matrix A (column-major, mw x
// nw) is theta when theta is tall or square, else theta^H.
__global__ void k_dd_theta(const cdd* __restrict__ G, const dd* __restrict__ L, const int* __restrict__ chi, int cap,
                           const int* __restrict__ sites, const double* __restrict__ Uhi,
                           const double* __restrict__ Ulo, cdd* __restrict__ Aw, DdMeta* __restrict__ meta,
                           unsigned long long* __restrict__ flops) {
  const int g = blockIdx.x, s = sites[g];
  __shared__ cdd U[16];
  if (threadIdx.x < 16) U[threadIdx.x] = load_gate(Uhi + 32 * g, Ulo ? Ulo + 32 * g : nullptr, threadIdx.x);
  __syncthreads();
  const int xl = chi[s], xm = chi[s + 1], xr = chi[s + 2];
  const dd* ll = L + (size_t)s * cap;
  const dd* lm = L + (size_t)(s + 1) * cap;
  const dd* lr = L + (size_t)(s + 2) * cap;
  const cdd* G0 = G + (size_t)s * 2 * cap * cap;
  const cdd* G1 = G + (size_t)(s + 1) * 2 * cap * cap;
  const int M = 2 * xl, N = 2 * xr;
  const bool tall = M >= N;
  const int mw = tall ? M : N, nw = tall ? N : M;
  if (threadIdx.x == 0) {
    meta[g] = DdMeta{mw, nw, tall ? 1 : 0, 0, 0, s};
    atomicAdd(flops, (unsigned long long)xl * xr *
                         ((unsigned long long)xm * (4 * kFlopsDdMul + 4 * (kFlopsCddMul + 2 * kFlopsDdAdd)) +
                          kFlopsDdMul + 4 * 2 * kFlopsDdMul + 16 * (kFlopsCddMul + 2 * kFlopsDdAdd)));
  }
  cdd* A = Aw + (size_t)g * kDdW * kDdW;
  const cdd zero = cdd_make(0.0, 0.0);
  for (int e = threadIdx.x; e < xl * xr; e += blockDim.x) {
    const int a = e / xr, c = e % xr;
    cdd T[4] = {zero, zero, zero, zero};
    for (int b = 0; b < xm; ++b) {
      const cdd p0 = cdd_scale(lm[b], G0[(size_t)a * cap + b]);
      const cdd p1 = cdd_scale(lm[b], G0[(size_t)(cap + a) * cap + b]);
      const cdd q0 = G1[(size_t)b * cap + c];
      const cdd q1 = G1[(size_t)(cap + b) * cap + c];
      T[0] = cdd_add(T[0], cdd_mul(p0, q0));
      T[1] = cdd_add(T[1], cdd_mul(p0, q1));
      T[2] = cdd_add(T[2], cdd_mul(p1, q0));
      T[3] = cdd_add(T[3], cdd_mul(p1, q1));
    }
    const dd w = dd_mul(ll[a], lr[c]);
#pragma unroll
    for (int kl = 0; kl < 4; ++kl) T[kl] = cdd_scale(w, T[kl]);
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        cdd acc = zero;
#pragma unroll
        for (int kl = 0; kl < 4; ++kl) acc = cdd_add(acc, cdd_mul(U[(i * 2 + j) * 4 + kl], T[kl]));
        const int r = i * xl + a, col = j * xr + c;
        if (tall) A[(size_t)col * mw + r] = acc;
        else A[(size_t)r * mw + col] = cdd_conj(acc);
      }
  }
}

__device__ __forceinline__ void warp_sum_dd(dd& v) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) v = dd_add(v, shfl_xor_dd(v, m));
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}

constexpr double kEps64 = 1.1102230246251565e-16;  // 2^-53
constexpr int kDdPreSweeps = 40;                   // binary64 sweep limit of the preconditioner
constexpr size_t kDdPreSmem = 2 * (size_t)kDdW * kDdW * sizeof(double2);

// Preconditioner of the double-word Jacobi (one CTA per gate). The binary64
// sweeps do most of the orthogonalisation at a fraction of the double-word
// cost; the double-word sweeps that follow only have to remove what binary64
// cannot resolve (off-diagonals ~1e-15 -> ~1e-30: quadratic convergence).
//   1. Binary64 cyclic one-sided Jacobi on the high parts of A (shared
//      memory), accumulating V64 (unitary to ~1e-15).
//   2. V64 made unitary to double-word accuracy: with E = V64^H V64 - I
//      (products of doubles summed exactly enough in double-word),
//      V1 = V64 (I + E)^{-1/2} = V64 (I - E/2 + 3 E^2 / 8) + O(E^3); E^2 is
//      ~1e-30 and needs only binary64.
//   3. A <- A V1 and V <- V1 in double-word arithmetic.
// Only the high parts steer step 1, so its rounding never reaches the
// result: the double-word sweeps decide convergence on A V1 itself.
__global__ void __launch_bounds__(kDdThreads, 1)
    k_dd_precondition(cdd* __restrict__ Aw, cdd* __restrict__ Vw, cdd* __restrict__ Sw,
                      const DdMeta* __restrict__ meta, unsigned long long* __restrict__ flops) {
  extern __shared__ __align__(16) unsigned char psm[];
  double2* A64 = (double2*)psm;
  double2* V64 = A64 + (size_t)kDdW * kDdW;
  const int g = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int mw = meta[g].mw, nw = meta[g].nw;
  cdd* A = Aw + (size_t)g * kDdW * kDdW;
  cdd* V = Vw + (size_t)g * kDdW * kDdW;
  cdd* S = Sw + (size_t)g * kDdW * kDdW;
  __shared__ double red[kDdWarps];
  __shared__ int rotated;
  __shared__ unsigned long long fl;
  double f = 0.0;
  for (int e = tid; e < mw * nw; e += kDdThreads) {
    const double2 a = make_double2(A[e].re.hi, A[e].im.hi);
    A64[e] = a;
    f += a.x * a.x + a.y * a.y;
  }
  for (int e = tid; e < nw * nw; e += kDdThreads) V64[e] = make_double2(e / nw == e % nw ? 1.0 : 0.0, 0.0);
  f = warp_sum_d(f);
  if (lane == 0) red[warp] = f;
  if (tid == 0) fl = 0;
  __syncthreads();
  double frob = 0.0;
  for (int w = 0; w < kDdWarps; ++w) frob += red[w];
  const double tol = (double)mw * kEps64;
  const double tiny = tol * tol * frob;
  unsigned long long myfl = 0;
  // ---- 1. binary64 sweeps
  for (int sweep = 0; sweep < kDdPreSweeps; ++sweep) {
    __syncthreads();
    if (tid == 0) rotated = 0;
    __syncthreads();
    for (int r = 0; r < nw - 1; ++r) {
      for (int p = warp; p < nw / 2; p += kDdWarps) {
        int I, J;
        dd_pair(nw, r, p, I, J);
        double2* ap = A64 + (size_t)I * mw;
        double2* aq = A64 + (size_t)J * mw;
        double app = 0.0, aqq = 0.0, gx = 0.0, gy = 0.0;
        for (int row = lane; row < mw; row += 32) {
          const double2 x = ap[row], y = aq[row];
          app = fma(x.x, x.x, fma(x.y, x.y, app));
          aqq = fma(y.x, y.x, fma(y.y, y.y, aqq));
          gx = fma(x.x, y.x, fma(x.y, y.y, gx));
          gy = fma(x.x, y.y, fma(-x.y, y.x, gy));
        }
        app = warp_sum_d(app);
        aqq = warp_sum_d(aqq);
        gx = warp_sum_d(gx);
        gy = warp_sum_d(gy);
        if (lane == 0) myfl += 8ull * mw + 20;
        if (!(app > tiny) || !(aqq > tiny)) continue;
        const double g2 = gx * gx + gy * gy;
        if (!(sqrt(g2) > tol * sqrt(app) * sqrt(aqq))) continue;
        const double d = aqq - app;
        const double sg = (d < 0.0 ? -2.0 : 2.0) / (fabs(d) + sqrt(d * d + 4.0 * g2));
        const double tx = sg * gx, ty = sg * gy;
        const double c = 1.0 / sqrt(1.0 + tx * tx + ty * ty);
        const double sx = c * tx, sy = c * ty;  // s e^{i phi}
        for (int row = lane; row < mw + nw; row += 32) {
          double2* cp = row < mw ? ap + row : V64 + (size_t)I * nw + (row - mw);
          double2* cq = row < mw ? aq + row : V64 + (size_t)J * nw + (row - mw);
          const double2 x = *cp, y = *cq;
          // x' = c x - conj(se) y ; y' = se x + c y
          *cp = make_double2(c * x.x - (sx * y.x + sy * y.y), c * x.y - (sx * y.y - sy * y.x));
          *cq = make_double2(fma(sx, x.x, -sy * x.y) + c * y.x, fma(sx, x.y, sy * x.x) + c * y.y);
        }
        if (lane == 0) {
          rotated = 1;
          myfl += 12ull * (mw + nw) + 20;
        }
      }
      __syncthreads();
    }
    __syncthreads();
    if (!rotated) break;
  }
  // ---- 2. E = V64^H V64 - I in double-word, into S (column-major, S[j nw + i] = E_ij)
  for (int e = tid; e < nw * nw; e += kDdThreads) {
    const int i = e % nw, j = e / nw;
    dd re = dd_make(0.0), im = dd_make(0.0);
    for (int k = 0; k < nw; ++k) {
      const double2 a = V64[(size_t)i * nw + k], b = V64[(size_t)j * nw + k];
      re = dd_add(re, dd_add(two_prod(a.x, b.x), two_prod(a.y, b.y)));
      im = dd_add(im, dd_sub(two_prod(a.x, b.y), two_prod(a.y, b.x)));
    }
    if (i == j) re = dd_add_d(re, -1.0);
    S[e] = cdd{re, im};
  }
  __syncthreads();
  // E^2 (binary64, from the high parts) into the A64 area (no longer needed)
  double2* E2 = A64;
  for (int e = tid; e < nw * nw; e += kDdThreads) {
    const int i = e % nw, j = e / nw;
    double x = 0.0, y = 0.0;
    for (int k = 0; k < nw; ++k) {
      const cdd a = S[(size_t)k * nw + i], b = S[(size_t)j * nw + k];
      x = fma(a.re.hi, b.re.hi, fma(-a.im.hi, b.im.hi, x));
      y = fma(a.re.hi, b.im.hi, fma(a.im.hi, b.re.hi, y));
    }
    E2[e] = make_double2(x, y);
  }
  __syncthreads();
  // M = I - E/2 + 3 E^2 / 8, in S
  for (int e = tid; e < nw * nw; e += kDdThreads) {
    const cdd s = S[e];
    const double2 q = E2[e];
    dd re = dd_add_d(dd{-0.5 * s.re.hi, -0.5 * s.re.lo}, 0.375 * q.x);
    const dd im = dd_add_d(dd{-0.5 * s.im.hi, -0.5 * s.im.lo}, 0.375 * q.y);
    if (e % nw == e / nw) re = dd_add_d(re, 1.0);
    S[e] = cdd{re, im};
  }
  __syncthreads();
  // V1 = V64 M into V
  for (int e = tid; e < nw * nw; e += kDdThreads) {
    const int i = e % nw, j = e / nw;
    cdd acc = cdd_make(0.0, 0.0);
    for (int k = 0; k < nw; ++k) {
      const double2 a = V64[(size_t)k * nw + i];
      const cdd m = S[(size_t)j * nw + k];
      const dd re = dd_sub(dd_mul_d(m.re, a.x), dd_mul_d(m.im, a.y));
      const dd im = dd_add(dd_mul_d(m.im, a.x), dd_mul_d(m.re, a.y));
      acc = cdd_add(acc, cdd{re, im});
    }
    V[e] = acc;
  }
  __syncthreads();
  // B = A V1 into S, then A <- B
  for (int e = tid; e < mw * nw; e += kDdThreads) {
    const int r = e % mw, j = e / mw;
    cdd acc = cdd_make(0.0, 0.0);
    for (int k = 0; k < nw; ++k) acc = cdd_add(acc, cdd_mul(A[(size_t)k * mw + r], V[(size_t)j * nw + k]));
    S[e] = acc;
  }
  __syncthreads();
  for (int e = tid; e < mw * nw; e += kDdThreads) A[e] = S[e];
  if (lane == 0 && myfl) atomicAdd(&fl, myfl);
  __syncthreads();
  if (tid == 0) {
    const unsigned long long n3 = (unsigned long long)nw * nw * nw;
    atomicAdd(flops, fl + n3 * (4 * 2 + 4 * kFlopsDdAdd) + n3 * 8 +
                         n3 * (4 * 6 + 4 * kFlopsDdAdd) + (unsigned long long)mw * nw * nw *
                         (kFlopsCddMul + 2 * kFlopsDdAdd));
  }
}

// One-sided Jacobi on the columns of A (mw x nw, column-major) with V
// accumulated (nw x nw): the pair (p, q) is rotated while
// |a_p^H a_q| > mw eps_dd ||a_p|| ||a_q||; columns with
// ||a_j|| <= mw eps_dd ||A||_F are numerically zero and are not rotated.
// The rotation is the real symmetric Schur rotation of
// [app |g|; |g| aqq] conjugated by the phase of g = a_p^H a_q:
// t e^{i phi} = 2 sign(d) g / (|d| + sqrt(d^2 + 4|g|^2)), d = aqq - app,
// c = 1/sqrt(1 + t^2), a_p <- c a_p - conj(s e^{i phi}) a_q,
// a_q <- s e^{i phi} a_p + c a_q.
__global__ void __launch_bounds__(kDdThreads, 1)
    k_dd_jacobi(cdd* __restrict__ Aw, cdd* __restrict__ Vw, dd* __restrict__ sig, DdMeta* __restrict__ meta,
                int max_sweeps, unsigned long long* __restrict__ flops) {
  const int g = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int mw = meta[g].mw, nw = meta[g].nw;
  cdd* A = Aw + (size_t)g * kDdW * kDdW;
  cdd* V = Vw + (size_t)g * kDdW * kDdW;  // holds V1 from k_dd_precondition
  __shared__ double red[kDdWarps];
  __shared__ int rotated;
  __shared__ unsigned long long fl;
  double f = 0.0;
  for (int e = tid; e < mw * nw; e += kDdThreads) f += A[e].re.hi * A[e].re.hi + A[e].im.hi * A[e].im.hi;
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) f += __shfl_xor_sync(0xffffffffu, f, m);
  if (lane == 0) red[warp] = f;
  if (tid == 0) fl = 0;
  __syncthreads();
  double frob = 0.0;
  for (int w = 0; w < kDdWarps; ++w) frob += red[w];
  const double tol = (double)mw * kEpsDd;
  const double tiny = tol * tol * frob;
  unsigned long long myfl = 0;
  int sweep = 0;
  bool conv = false;
  while (sweep < max_sweeps) {
    __syncthreads();
    if (tid == 0) rotated = 0;
    __syncthreads();
    for (int r = 0; r < nw - 1; ++r) {
      for (int p = warp; p < nw / 2; p += kDdWarps) {
        int I, J;
        dd_pair(nw, r, p, I, J);
        cdd* ap = A + (size_t)I * mw;
        cdd* aq = A + (size_t)J * mw;
        dd app = dd_make(0.0), aqq = dd_make(0.0);
        cdd gq = cdd_make(0.0, 0.0);
        for (int row = lane; row < mw; row += 32) {
          const cdd x = ap[row], y = aq[row];
          app = dd_add(app, cdd_abs2(x));
          aqq = dd_add(aqq, cdd_abs2(y));
          gq = cdd_add(gq, cdd_cmul(x, y));
        }
        warp_sum_dd(app);
        warp_sum_dd(aqq);
        warp_sum_dd(gq.re);
        warp_sum_dd(gq.im);
        if (lane == 0) myfl += (unsigned long long)mw * kDdDotFlopsPerRow + 4 * 5 * kFlopsDdAdd;
        if (!(app.hi > tiny) || !(aqq.hi > tiny)) continue;
        const double gabs = sqrt(gq.re.hi * gq.re.hi + gq.im.hi * gq.im.hi);
        if (!(gabs > tol * sqrt(app.hi) * sqrt(aqq.hi))) continue;
        const dd d = dd_sub(aqq, app);
        const dd g2 = cdd_abs2(gq);
        const dd root = dd_sqrt(dd_add(dd_sqr(d), dd_mul_d(g2, 4.0)));
        const dd den = dd_add(d.hi < 0.0 ? dd_neg(d) : d, root);
        dd sg = dd_div(dd_make(2.0), den);
        if (d.hi < 0.0) sg = dd_neg(sg);
        const cdd te = cdd_scale(sg, gq);
        const dd c = dd_div(dd_make(1.0), dd_sqrt(dd_add(dd_make(1.0), cdd_abs2(te))));
        const cdd se = cdd_scale(c, te);
        for (int row = lane; row < mw; row += 32) {
          const cdd x = ap[row], y = aq[row];
          ap[row] = cdd_sub(cdd_scale(c, x), cdd_cmul(se, y));
          aq[row] = cdd_add(cdd_mul(se, x), cdd_scale(c, y));
        }
        cdd* vp = V + (size_t)I * nw;
        cdd* vq = V + (size_t)J * nw;
        for (int row = lane; row < nw; row += 32) {
          const cdd x = vp[row], y = vq[row];
          vp[row] = cdd_sub(cdd_scale(c, x), cdd_cmul(se, y));
          vq[row] = cdd_add(cdd_mul(se, x), cdd_scale(c, y));
        }
        if (lane == 0) {
          rotated = 1;
          myfl += (unsigned long long)(mw + nw) * kDdRotFlopsPerRow + 12 * kFlopsDdAdd + 12 * kFlopsDdMul;
        }
      }
      __syncthreads();
    }
    ++sweep;
    __syncthreads();
    if (!rotated) {
      conv = true;
      break;
    }
  }
  // sigma_j = ||a_j||
  for (int j = warp; j < nw; j += kDdWarps) {
    dd acc = dd_make(0.0);
    for (int row = lane; row < mw; row += 32) acc = dd_add(acc, cdd_abs2(A[(size_t)j * mw + row]));
    warp_sum_dd(acc);
    if (lane == 0) sig[(size_t)g * kDdW + j] = dd_sqrt(acc);
  }
  if (lane == 0 && myfl) atomicAdd(&fl, myfl);
  __syncthreads();
  if (tid == 0) {
    meta[g].sweeps = sweep;
    meta[g].status = conv ? 0 : MPS_ERR_NOCONVERGE;
    atomicAdd(flops, fl);
  }
}

// Order (descending, ties by index), truncation, renormalisation and the
// rewrite Gamma'_s = X / Lambda_{s-1}, Lambda'_s, Gamma'_{s+1} = Y^H / Lambda_{s+1}.
__global__ void k_dd_finish(cdd* __restrict__ G, dd* __restrict__ L, int* __restrict__ chi, int cap, int chi_max,
                            double cutoff, const cdd* __restrict__ Aw, const cdd* __restrict__ Vw,
                            const dd* __restrict__ sig, const DdMeta* __restrict__ meta, int* __restrict__ status,
                            unsigned long long* __restrict__ counters) {
  const int g = blockIdx.x, tid = threadIdx.x;
  const DdMeta mt = meta[g];
  if (mt.status != 0) {  // the gate is left unapplied
    if (tid == 0) atomicCAS(status, 0, mt.status);
    return;
  }
  const int s = mt.site, mw = mt.mw, nw = mt.nw;
  const dd* sg = sig + (size_t)g * kDdW;
  __shared__ int ord[kDdW];
  __shared__ dd inv_sig[kDdW];
  __shared__ dd lam[kDdW];
  __shared__ int kk;
  for (int j = tid; j < nw; j += blockDim.x) {
    int rank = 0;
    for (int i = 0; i < nw; ++i) rank += (dd_gt(sg[i], sg[j]) || (i < j && sg[i].hi == sg[j].hi && sg[i].lo == sg[j].lo));
    ord[rank] = j;
    inv_sig[j] = sg[j].hi > 0.0 ? dd_div(dd_make(1.0), sg[j]) : dd_make(0.0);
  }
  __syncthreads();
  if (tid == 0) {
    dd total = dd_make(0.0);
    for (int j = 0; j < nw; ++j) total = dd_add(total, dd_sqr(sg[j]));
    const double rel = fmax(cutoff, (double)mw * kEpsDd);
    const dd thr = dd_mul_d(dd_sqrt(total), rel);
    int k = 0;
    for (int j = 0; j < nw; ++j) k += dd_gt(sg[j], thr);
    k = min(max(k, 1), chi_max);
    dd kept = dd_make(0.0);
    for (int c = 0; c < k; ++c) kept = dd_add(kept, dd_sqr(sg[ord[c]]));
    const dd nk = dd_sqrt(kept);
    for (int c = 0; c < k; ++c)
      lam[c] = nk.hi > 0.0 ? dd_div(sg[ord[c]], nk) : dd_make(c == 0 ? 1.0 : 0.0);
    kk = k;
    atomicAdd(&counters[0], (unsigned long long)mt.sweeps);
  }
  __syncthreads();
  const int k = kk;
  const int xl = chi[s], xr = chi[s + 2];
  const cdd* A = Aw + (size_t)g * kDdW * kDdW;
  const cdd* V = Vw + (size_t)g * kDdW * kDdW;
  const dd* ll = L + (size_t)s * cap;
  const dd* lr = L + (size_t)(s + 2) * cap;
  cdd* G0 = G + (size_t)s * 2 * cap * cap;
  cdd* G1 = G + (size_t)(s + 1) * 2 * cap * cap;
  // X[(i,a), j] and Y[(j,b), j'] of theta = X Sigma Y^H: tall: X = A / sigma,
  // Y = V; wide (A = theta^H): X = V, Y = A / sigma.
  for (int e = tid; e < 2 * xl * k; e += blockDim.x) {
    const int c = e % k, ia = e / k, i = ia / xl, a = ia % xl;
    const int j = ord[c];
    cdd x = mt.tall ? cdd_scale(inv_sig[j], A[(size_t)j * mw + ia]) : V[(size_t)j * nw + ia];
    const dd il = ll[a].hi > 0.0 ? dd_div(dd_make(1.0), ll[a]) : dd_make(0.0);
    G0[((size_t)i * cap + a) * cap + c] = cdd_scale(il, x);
  }
  for (int e = tid; e < 2 * k * xr; e += blockDim.x) {
    const int b = e % xr, jc = e / xr, jj = jc / k, c = jc % k;
    const int j = ord[c];
    const int row = jj * xr + b;
    cdd y = mt.tall ? V[(size_t)j * nw + row] : cdd_scale(inv_sig[j], A[(size_t)j * mw + row]);
    const dd il = lr[b].hi > 0.0 ? dd_div(dd_make(1.0), lr[b]) : dd_make(0.0);
    G1[((size_t)jj * cap + c) * cap + b] = cdd_scale(il, cdd_conj(y));
  }
  for (int c = tid; c < cap; c += blockDim.x) L[(size_t)(s + 1) * cap + c] = c < k ? lam[c] : dd_make(0.0);
  __syncthreads();
  if (tid == 0) chi[s + 1] = k;
}

// <bits|psi> = Gamma_0[b_0] Lambda_0 Gamma_1[b_1] ... Gamma_{n-1}[b_{n-1}], one CTA per string
__global__ void k_dd_amp(const cdd* __restrict__ G, const dd* __restrict__ L, const int* __restrict__ chi, int n,
                         int cap, const unsigned char* __restrict__ bits, double* __restrict__ out) {
  __shared__ cdd v[kDdMaxCap], w[kDdMaxCap];
  const unsigned char* b = bits + (size_t)blockIdx.x * n;
  const int t = threadIdx.x;
  if (t < kDdMaxCap) v[t] = cdd_make(t == 0 ? 1.0 : 0.0, 0.0);
  __syncthreads();
  for (int s = 0; s < n; ++s) {
    const int an = chi[s], cn = chi[s + 1], i = b[s] & 1;
    if (t < cn) {
      cdd acc = cdd_make(0.0, 0.0);
      for (int a = 0; a < an; ++a) acc = cdd_add(acc, cdd_mul(v[a], G[((size_t)(s * 2 + i) * cap + a) * cap + t]));
      w[t] = cdd_scale(L[(size_t)(s + 1) * cap + t], acc);
    }
    __syncthreads();
    if (t < cn) v[t] = w[t];
    __syncthreads();
  }
  if (t == 0) {
    double* o = out + 4 * (size_t)blockIdx.x;
    o[0] = v[0].re.hi;
    o[1] = v[0].re.lo;
    o[2] = v[0].im.hi;
    o[3] = v[0].im.lo;
  }
}

int dd_fail(int code, const std::string& msg) {
  set_error_message(msg.c_str());
  return code;
}

#define DCK(call)                                                                             \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return dd_fail(e_ == cudaErrorMemoryAllocation ? MPS_ERR_NOMEM : MPS_ERR_CUDA,          \
                     std::string(#call) + ": " + cudaGetErrorString(e_));                     \
  } while (0)

}  // namespace

struct mps_dd_state {
  int n = 0, cap = 0, max_sweeps = kMaxSweeps;
  double cutoff = 0.0;
  cudaStream_t st = nullptr;
  cdd* G = nullptr;
  dd* L = nullptr;
  int* chi = nullptr;
  cdd* A = nullptr;
  cdd* V = nullptr;
  cdd* S = nullptr;  // scratch of the preconditioner, one working matrix per gate
  dd* sig = nullptr;
  DdMeta* meta = nullptr;
  int* status = nullptr;
  unsigned long long* counters = nullptr;  // [0] sweeps, [1] executed binary64 operations
  // gate staging: device copies of one layer (sites, U hi, U lo), and
  // kDdStages pinned host slots, each reused after its event
  int* d_sites[kDdStages] = {};
  double* d_U[kDdStages] = {};
  char* h_stage[kDdStages] = {};
  cudaEvent_t ev[kDdStages] = {};
  int slot = 0;
  size_t stage_bytes = 0;
  long long updates = 0;
};

namespace {

void dd_free(mps_dd_state* h) {
  if (!h) return;
  cudaFree(h->G);
  cudaFree(h->L);
  cudaFree(h->chi);
  cudaFree(h->A);
  cudaFree(h->V);
  cudaFree(h->S);
  cudaFree(h->sig);
  cudaFree(h->meta);
  cudaFree(h->status);
  cudaFree(h->counters);
  for (int i = 0; i < kDdStages; ++i) {
    cudaFree(h->d_sites[i]);
    cudaFree(h->d_U[i]);
    if (h->h_stage[i]) cudaFreeHost(h->h_stage[i]);
    if (h->ev[i]) cudaEventDestroy(h->ev[i]);
  }
  delete h;
}

int dd_reset(mps_dd_state* h) {
  k_dd_reset<<<64, 256, 0, h->st>>>(h->G, h->L, h->chi, h->n, h->cap);
  DCK(cudaGetLastError());
  DCK(cudaMemsetAsync(h->status, 0, sizeof(int), h->st));
  DCK(cudaMemsetAsync(h->counters, 0, 2 * sizeof(unsigned long long), h->st));
  h->updates = 0;
  return MPS_OK;
}

int dd_collect(mps_dd_state* h) {
  DCK(cudaStreamSynchronize(h->st));
  int st = 0;
  DCK(cudaMemcpy(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st != 0) {
    DCK(cudaMemset(h->status, 0, sizeof(int)));
    return dd_fail(st, "double-word Jacobi SVD hit its sweep limit (the gate was left unapplied)");
  }
  return MPS_OK;
}

// byte offset of the gate matrices in a staging slot (after the sites)
size_t dd_stage_ofs(int n) { return ((size_t)n * sizeof(int) + 15) & ~(size_t)15; }

int dd_check_sites(const mps_dd_state* h, int k, int ng, const int* sites) {
  std::vector<int> s(sites, sites + ng);
  std::sort(s.begin(), s.end());
  for (int i = 0; i < ng; ++i) {
    if (s[i] < 0 || s[i] + k > h->n) return dd_fail(MPS_ERR_ARG, "gate site out of range");
    if (i > 0 && s[i] < s[i - 1] + k) return dd_fail(MPS_ERR_ARG, "gates of a layer must act on disjoint qubits");
  }
  return MPS_OK;
}

// d_sites, d_Uhi, d_Ulo: device arrays of the layer (d_Ulo may be null)
int dd_launch_layer(mps_dd_state* h, int k, int ng, const int* d_sites, const double* d_Uhi, const double* d_Ulo) {
  if (k == 1) {
    k_dd_apply1<<<ng, 128, 0, h->st>>>(h->G, h->chi, h->cap, d_sites, d_Uhi, d_Ulo);
    DCK(cudaGetLastError());
    return MPS_OK;
  }
  k_dd_theta<<<ng, 256, 0, h->st>>>(h->G, h->L, h->chi, h->cap, d_sites, d_Uhi, d_Ulo, h->A, h->meta,
                                      h->counters + 1);
  DCK(cudaGetLastError());
  k_dd_precondition<<<ng, kDdThreads, kDdPreSmem, h->st>>>(h->A, h->V, h->S, h->meta, h->counters + 1);
  DCK(cudaGetLastError());
  k_dd_jacobi<<<ng, kDdThreads, 0, h->st>>>(h->A, h->V, h->sig, h->meta, h->max_sweeps, h->counters + 1);
  DCK(cudaGetLastError());
  k_dd_finish<<<ng, 256, 0, h->st>>>(h->G, h->L, h->chi, h->cap, h->cap, h->cutoff, h->A, h->V, h->sig, h->meta,
                                       h->status, h->counters);
  DCK(cudaGetLastError());
  h->updates += ng;
  return MPS_OK;
}

}  // namespace

extern "C" {

int mps_dd_create(int n, int chi_max, double cutoff, mps_dd_handle* out) {
  if (!out) return dd_fail(MPS_ERR_ARG, "null output handle");
  *out = nullptr;
  if (n < 2 || chi_max < 1 || !(cutoff >= 0.0) || !(cutoff < 1.0))
    return dd_fail(MPS_ERR_ARG, "mps_dd_create: need n >= 2, chi_max >= 1, 0 <= cutoff < 1");
  if (chi_max > kDdMaxCap) return dd_fail(MPS_ERR_TOO_LARGE, "mps_dd_create: chi_max above 32");
  mps_dd_state* h = new mps_dd_state();
  h->n = n;
  h->cap = chi_max;
  h->cutoff = cutoff;
  const int slots = n;  // at most n gates in one layer
  h->stage_bytes = dd_stage_ofs(n) + 2 * (size_t)slots * 32 * sizeof(double);
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = dev_alloc(p, bytes);
  };
  A((void**)&h->G, (size_t)n * 2 * chi_max * chi_max * sizeof(cdd));
  A((void**)&h->L, (size_t)(n + 1) * chi_max * sizeof(dd));
  A((void**)&h->chi, (size_t)(n + 1) * sizeof(int));
  const int gmax = std::max(1, n / 2);
  A((void**)&h->A, (size_t)gmax * kDdW * kDdW * sizeof(cdd));
  A((void**)&h->V, (size_t)gmax * kDdW * kDdW * sizeof(cdd));
  A((void**)&h->S, (size_t)gmax * kDdW * kDdW * sizeof(cdd));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_dd_precondition, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDdPreSmem);
  A((void**)&h->sig, (size_t)gmax * kDdW * sizeof(dd));
  A((void**)&h->meta, (size_t)gmax * sizeof(DdMeta));
  A((void**)&h->status, sizeof(int));
  A((void**)&h->counters, 2 * sizeof(unsigned long long));
  for (int i = 0; i < kDdStages; ++i) {
    A((void**)&h->d_sites[i], (size_t)slots * sizeof(int));
    A((void**)&h->d_U[i], 2 * (size_t)slots * 32 * sizeof(double));
    if (e == cudaSuccess) e = host_alloc((void**)&h->h_stage[i], h->stage_bytes);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev[i], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    dd_free(h);
    return dd_fail(e == cudaErrorMemoryAllocation ? MPS_ERR_NOMEM : MPS_ERR_CUDA,
                   std::string("mps_dd_create: ") + cudaGetErrorString(e));
  }
  int rc = dd_reset(h);
  if (rc == MPS_OK) rc = dd_collect(h);
  if (rc != MPS_OK) {
    dd_free(h);
    return rc;
  }
  *out = h;
  return MPS_OK;
}

int mps_dd_destroy(mps_dd_handle h) {
  if (!h) return dd_fail(MPS_ERR_ARG, "null handle");
  cudaStreamSynchronize(h->st);
  dd_free(h);
  return MPS_OK;
}

int mps_dd_set_stream(mps_dd_handle h, void* stream) {
  if (!h) return dd_fail(MPS_ERR_ARG, "null handle");
  DCK(cudaStreamSynchronize(h->st));
  h->st = (cudaStream_t)stream;
  return MPS_OK;
}

int mps_dd_reset(mps_dd_handle h) {
  if (!h) return dd_fail(MPS_ERR_ARG, "null handle");
  return dd_reset(h);
}

int mps_dd_apply_layer(mps_dd_handle h, int k, int n_gates, const int* sites, const double* U_hi, const double* U_lo) {
  if (!h || (n_gates > 0 && (!sites || !U_hi))) return dd_fail(MPS_ERR_ARG, "null argument");
  if (k != 1 && k != 2) return dd_fail(MPS_ERR_ARG, "mps_dd_apply_layer: k must be 1 or 2");
  if (n_gates < 0 || n_gates > h->n) return dd_fail(MPS_ERR_ARG, "mps_dd_apply_layer: bad gate count");
  if (n_gates == 0) return MPS_OK;
  int rc = dd_check_sites(h, k, n_gates, sites);
  if (rc != MPS_OK) return rc;
  const int d = 1 << k;
  const size_t ue = (size_t)n_gates * d * d * 2;  // doubles of one part
  const int sl = h->slot;
  h->slot = (h->slot + 1) % kDdStages;
  DCK(cudaEventSynchronize(h->ev[sl]));  // the slot's previous copies have finished
  char* hs = h->h_stage[sl];
  std::memcpy(hs, sites, (size_t)n_gates * sizeof(int));
  double* hu = (double*)(hs + dd_stage_ofs(h->n));
  std::memcpy(hu, U_hi, ue * sizeof(double));
  if (U_lo) std::memcpy(hu + ue, U_lo, ue * sizeof(double));
  DCK(cudaMemcpyAsync(h->d_sites[sl], hs, (size_t)n_gates * sizeof(int), cudaMemcpyHostToDevice, h->st));
  DCK(cudaMemcpyAsync(h->d_U[sl], hu, (U_lo ? 2 : 1) * ue * sizeof(double), cudaMemcpyHostToDevice, h->st));
  DCK(cudaEventRecord(h->ev[sl], h->st));
  return dd_launch_layer(h, k, n_gates, h->d_sites[sl], h->d_U[sl], U_lo ? h->d_U[sl] + ue : nullptr);
}

int mps_dd_apply_layer_device(mps_dd_handle h, int k, int n_gates, const int* sites, const int* d_sites,
                              const double* d_U_hi, const double* d_U_lo) {
  if (!h || (n_gates > 0 && (!sites || !d_sites || !d_U_hi))) return dd_fail(MPS_ERR_ARG, "null argument");
  if (k != 1 && k != 2) return dd_fail(MPS_ERR_ARG, "mps_dd_apply_layer_device: k must be 1 or 2");
  if (n_gates < 0 || n_gates > h->n) return dd_fail(MPS_ERR_ARG, "mps_dd_apply_layer_device: bad gate count");
  if (n_gates == 0) return MPS_OK;
  int rc = dd_check_sites(h, k, n_gates, sites);
  if (rc != MPS_OK) return rc;
  return dd_launch_layer(h, k, n_gates, d_sites, d_U_hi, d_U_lo);
}

int mps_dd_sync(mps_dd_handle h) {
  if (!h) return dd_fail(MPS_ERR_ARG, "null handle");
  return dd_collect(h);
}

int mps_dd_bond_dims(mps_dd_handle h, int* chi) {
  if (!h || !chi) return dd_fail(MPS_ERR_ARG, "null argument");
  int rc = dd_collect(h);
  if (rc != MPS_OK) return rc;
  DCK(cudaMemcpy(chi, h->chi, (size_t)(h->n + 1) * sizeof(int), cudaMemcpyDeviceToHost));
  return MPS_OK;
}

int mps_dd_get_schmidt(mps_dd_handle h, int bond, double* hi, double* lo, int* len) {
  if (!h || !len) return dd_fail(MPS_ERR_ARG, "null argument");
  if (bond < 0 || bond > h->n - 2) return dd_fail(MPS_ERR_ARG, "bond out of range");
  int rc = dd_collect(h);
  if (rc != MPS_OK) return rc;
  int k = 0;
  DCK(cudaMemcpy(&k, h->chi + bond + 1, sizeof(int), cudaMemcpyDeviceToHost));
  std::vector<dd> v(k);
  DCK(cudaMemcpy(v.data(), h->L + (size_t)(bond + 1) * h->cap, k * sizeof(dd), cudaMemcpyDeviceToHost));
  for (int c = 0; c < k; ++c) {
    if (hi) hi[c] = v[c].hi;
    if (lo) lo[c] = v[c].lo;
  }
  *len = k;
  return MPS_OK;
}

int mps_dd_amplitudes(mps_dd_handle h, int count, const unsigned char* bits, double* out) {
  if (!h || (count > 0 && (!bits || !out)) || count < 0) return dd_fail(MPS_ERR_ARG, "bad argument");
  if (count == 0) return MPS_OK;
  int rc = dd_collect(h);
  if (rc != MPS_OK) return rc;
  unsigned char* db = nullptr;
  double* dout = nullptr;
  cudaError_t e = dev_alloc((void**)&db, (size_t)count * h->n);
  if (e == cudaSuccess) e = dev_alloc((void**)&dout, (size_t)count * 4 * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpyAsync(db, bits, (size_t)count * h->n, cudaMemcpyHostToDevice, h->st);
  if (e == cudaSuccess) {
    k_dd_amp<<<count, 32, 0, h->st>>>(h->G, h->L, h->chi, h->n, h->cap, db, dout);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, dout, (size_t)count * 4 * sizeof(double), cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  cudaFree(db);
  cudaFree(dout);
  if (e != cudaSuccess)
    return dd_fail(e == cudaErrorMemoryAllocation ? MPS_ERR_NOMEM : MPS_ERR_CUDA,
                   std::string("mps_dd_amplitudes: ") + cudaGetErrorString(e));
  return MPS_OK;
}

int mps_dd_stats(mps_dd_handle h, long long* updates, long long* sweeps, double* flops) {
  if (!h) return dd_fail(MPS_ERR_ARG, "null handle");
  int rc = dd_collect(h);
  if (rc != MPS_OK) return rc;
  unsigned long long c[2] = {0, 0};
  DCK(cudaMemcpy(c, h->counters, sizeof(c), cudaMemcpyDeviceToHost));
  if (updates) *updates = h->updates;
  if (sweeps) *sweeps = (long long)c[0];
  if (flops) *flops = (double)c[1];
  return MPS_OK;
}

int mps_dd_set_limits(mps_dd_handle h, int max_sweeps) {
  if (!h || max_sweeps < 1 || max_sweeps > kMaxSweeps) return dd_fail(MPS_ERR_ARG, "max_sweeps out of range");
  h->max_sweeps = max_sweeps;
  return MPS_OK;
}

}  // extern "C"

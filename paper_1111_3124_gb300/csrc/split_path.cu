// Split-precision form of the two-site update (MPS_PREC_SPLIT).
//
//   1. theta: T = X Y with X[(k,a),c] = Lambda_{s-1}[a] Gamma_s[k,a,c] Lambda_s[c]
//      and Y[c,(l,b)] = Gamma_{s+1}[l,c,b] Lambda_{s+1}[b] by the split-precision
//      GEMM (ozaki_tc.cu); the gate mixes the four (k,l) blocks (k_gate_mix2).
//   2. fp32 blocked one-sided Jacobi on a copy of the working matrix
//      (rotation angles in binary64): an approximate right factor V32.
//   3. V = V32 in binary64, re-orthonormalised by two Newton-Schulz steps
//      V <- V (3 I - V^H V) / 2, products by the split-precision GEMM.
//   4. B = A V (split-precision GEMM): columns orthogonal to ~5e-6.
//   5. Gram polish: G = B^H B by the split-precision GEMM (its error is
//      ~2^-56 sqrt(Mw) |b_p||b_q|, far below the Mw eps |b_p||b_q| that the
//      test resolves); the binary64 test |g_pq| <= Mw eps sqrt(g_pp g_qq) on
//      G; from such a start all pair rotations are small and nearly commute,
//      so one simultaneous step takes the skew-Hermitian X whose (p,q) entry
//      is the Jacobi angle of the pair's 2 x 2 problem with g_pq's phase
//      (x_pq ~ g_pq / (g_qq - g_pp)), W = exp(X) to fourth order,
//      B <- B W (columns balanced by their norms), V <- V W; a
//      near-degenerate pair (|x_pq| > 1e-3) is left out of X and rotated by
//      its exact Jacobi rotation. Three steps, then a last Gram test; a task
//      still above the tolerance goes on to
//   6. binary64 blocked Jacobi sweeps on B, which keep the column norms, the
//      orthogonality test and the rotation angles in binary64.
// A three-site update forms theta in binary64 (two contraction steps) and
// runs steps 2-6 on each of its two splits (the second one's working matrix
// is copied from T to A and back).
// Truncation and the Lambda^-1 rewrite are those of the binary64 path.
#include "engine.cuh"
#include "kernels.cuh"
#include "ozaki.cuh"

namespace mpsgb {

// Fills one OzJob per task for the product `kind`.
__global__ void k_oz_jobs(const GateTask* tasks, const TaskMeta* meta, OzJob* jobs, int ntask, int kind, int s,
                          unsigned long long* flops) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntask) return;
  const GateTask& tk = tasks[t];
  const TaskMeta& mt = meta[t];
  OzJob j = {};
  j.alpha = 1.0;
  const long long cap = tk.cap;
  if (mt.status) {
    jobs[t] = j;  // M = N = K = 0: nothing to do
    return;
  }
  if (kind >= kOzAhA && kind <= kOzVW && (!mt.active || mt.hard)) {
    jobs[t] = j;  // converged, or left to the blocked sweeps
    return;
  }
  const int nw = mt.Nw;
  switch (kind) {
    case kOzAhA:  // P = A^H A (Nw x Nw, inner Mw)
      j.a.p = tk.A;
      j.a.s_r = mt.Mw;
      j.a.s_k = 1;
      j.a.conj = 1;
      j.b.p = tk.A;
      j.b.s_r = mt.Mw;
      j.b.s_k = 1;
      j.M = j.N = nw;
      j.K = mt.Mw;
      j.C = tk.P;
      j.ldc = nw;
      j.herm = 1;
      break;
    case kOzXX:  // Q = P P
    case kOzX3:  // V2 = P Q
      j.a.p = tk.P;
      j.a.s_r = 1;
      j.a.s_k = nw;
      j.b.p = kind == kOzXX ? tk.P : tk.Q;
      j.b.s_r = nw;
      j.b.s_k = 1;
      j.M = j.N = j.K = nw;
      j.C = kind == kOzXX ? tk.Q : tk.V2;
      j.ldc = nw;
      j.herm = kind == kOzXX;  // X X, X skew-Hermitian (X^3 = X Q is skew only up to rounding: X Q != Q X)
      break;
    case kOzX4:  // T = Q Q
      j.a.p = tk.Q;
      j.a.s_r = 1;
      j.a.s_k = nw;
      j.b.p = tk.Q;
      j.b.s_r = nw;
      j.b.s_k = 1;
      j.M = j.N = j.K = nw;
      j.C = tk.T;
      j.ldc = nw;
      j.herm = 1;
      break;
    case kOzAW:  // T = (A D^-1)(D P), D = diag(||a_k||) (k_gram_scales): each
                 // column of the product keeps its rounding relative to its own norm
      j.a.p = tk.A;
      j.a.s_r = 1;
      j.a.s_k = mt.Mw;
      j.a.kscale = reinterpret_cast<const double*>(tk.V2);
      j.b.p = tk.P;
      j.b.s_r = nw;
      j.b.s_k = 1;
      j.b.kscale = reinterpret_cast<const double*>(tk.V2) + nw;
      j.M = mt.Mw;
      j.N = j.K = nw;
      j.C = tk.T;
      j.ldc = mt.Mw;
      break;
    case kOzVW:  // Q = V P
      j.a.p = tk.V;
      j.a.s_r = 1;
      j.a.s_k = nw;
      j.b.p = tk.P;
      j.b.s_r = nw;
      j.b.s_k = 1;
      j.M = j.N = j.K = nw;
      j.C = tk.Q;
      j.ldc = nw;
      break;
    case kOzTheta:  // T = X Y, 2 chi_L x 2 chi_R, inner chi_s
      j.a.p = tk.g0;
      j.a.rb = mt.xl;
      j.a.s_rb = cap * cap;
      j.a.s_r = cap;
      j.a.s_k = 1;
      j.a.rscale = tk.lamL;
      j.a.kscale = tk.lam0;
      j.b.p = tk.g1;
      j.b.rb = mt.xr;
      j.b.s_rb = cap * cap;
      j.b.s_r = 1;
      j.b.s_k = cap;
      j.b.rscale = tk.lamR;
      j.M = 2 * mt.xl;
      j.N = 2 * mt.xr;
      j.K = mt.x0;
      j.C = tk.T;
      j.ldc = 2 * mt.xl;
      break;
    case kOzVhV:  // P = V^H V
      j.a.p = tk.V;
      j.a.s_r = mt.Nw;
      j.a.s_k = 1;
      j.a.conj = 1;
      j.b.p = tk.V;
      j.b.s_r = mt.Nw;
      j.b.s_k = 1;
      j.M = j.N = j.K = mt.Nw;
      j.C = tk.P;
      j.ldc = mt.Nw;
      j.herm = 1;
      break;
    case kOzVP:  // Q = V P
      j.a.p = tk.V;
      j.a.s_r = 1;
      j.a.s_k = mt.Nw;
      j.b.p = tk.P;
      j.b.s_r = mt.Nw;
      j.b.s_k = 1;
      j.M = j.N = j.K = mt.Nw;
      j.C = tk.Q;
      j.ldc = mt.Nw;
      break;
    default:  // kOzAV: T = A V
      j.a.p = tk.A;
      j.a.s_r = 1;
      j.a.s_k = mt.Mw;
      j.b.p = tk.V;
      j.b.s_r = mt.Nw;
      j.b.s_k = 1;
      j.M = mt.Mw;
      j.N = mt.Nw;
      j.K = mt.Nw;
      j.C = tk.T;
      j.ldc = mt.Mw;
      break;
  }
  jobs[t] = j;
  if (flops) {  // tensor-core flops of the s(s+1)/2 slice pairs of this job (8 per complex multiply-add)
    unsigned long long f = (unsigned long long)(s * (s + 1) / 2) * 8ull * (unsigned long long)j.M *
                           (unsigned long long)j.N * (unsigned long long)j.K;
    if (j.herm) {  // the tiles on and above the diagonal only
      const unsigned long long nt = (unsigned long long)(j.N + 63) / 64;
      f = f / (nt * nt) * (nt * (nt + 1) / 2);
    }
    atomicAdd(flops, f);
  }
}

// theta[(i,a),(j,b)] = sum_{kl} U[(ij),(kl)] T[(k,a),(l,b)], written as the
// working matrix (theta, or theta^H when theta is wide), column-major.
__global__ void __launch_bounds__(256) k_gate_mix2(const GateTask* tasks, const TaskMeta* meta) {
  const GateTask& tk = tasks[blockIdx.y];
  const TaskMeta& mt = meta[blockIdx.y];
  if (mt.status) return;
  const int xl = mt.xl, xr = mt.xr, M = 2 * xl;
  double2 u[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) u[e] = tk.U[e];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < xl * xr; e += gridDim.x * blockDim.x) {
    const int a = e % xl, b = e / xl;
    double2 t[4];
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
      for (int l = 0; l < 2; ++l) t[k * 2 + l] = tk.T[(size_t)(k * xl + a) + (size_t)(l * xr + b) * M];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        double2 th = make_double2(0.0, 0.0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const double2 w = u[(i * 2 + j) * 4 + q];
          th.x = fma(w.x, t[q].x, fma(-w.y, t[q].y, th.x));
          th.y = fma(w.x, t[q].y, fma(w.y, t[q].x, th.y));
        }
        const int row = i * xl + a, col = j * xr + b;
        if (mt.tall) tk.A[(size_t)row + (size_t)col * mt.Mw] = th;
        else tk.A[(size_t)col + (size_t)row * mt.Mw] = make_double2(th.x, -th.y);
      }
  }
}

// The working matrix's columns ranked by decreasing norm (ties by index),
// into perm: the fp32 sweeps start on A P, so that columns of similar size
// share a block and their coupling is taken by the inner solves. One CTA per
// task; a warp per column for the norms.
__global__ void __launch_bounds__(256) k_sort_cols(const GateTask* tasks, const TaskMeta* meta) {
  extern __shared__ double cn[];
  const GateTask& tk = tasks[blockIdx.x];
  const TaskMeta& mt = meta[blockIdx.x];
  if (mt.status) return;
  const int Mw = mt.Mw, Nw = mt.Nw, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = warp; j < Nw; j += 8) {
    double acc = 0.0;
    for (int r = lane; r < Mw; r += 32) {
      const double2 v = tk.A[(size_t)r + (size_t)j * Mw];
      acc = fma(v.x, v.x, fma(v.y, v.y, acc));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) cn[j] = acc;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < Nw; j += blockDim.x) {
    const double nj = cn[j];
    int rank = 0;
    for (int i = 0; i < Nw; ++i) rank += cn[i] > nj || (cn[i] == nj && i < j);
    tk.perm[rank] = j;
  }
}

// A32 = fp32(A P), V32 = P (P the permutation of k_sort_cols: column j is
// column perm[j] of A)
__global__ void k_to_f32(const GateTask* tasks, const TaskMeta* meta) {
  const GateTask& tk = tasks[blockIdx.y];
  const TaskMeta& mt = meta[blockIdx.y];
  if (mt.status) return;
  const size_t na = (size_t)mt.Mw * mt.Nw, nv = (size_t)mt.Nw * mt.Nw;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < na + nv; e += (size_t)gridDim.x * blockDim.x) {
    if (e < na) {
      const size_t j = e / mt.Mw, r = e % mt.Mw;
      const double2 v = tk.A[r + (size_t)tk.perm[j] * mt.Mw];
      tk.A32[e] = make_float2((float)v.x, (float)v.y);
    } else {
      const size_t f = e - na;
      tk.V32[f] = make_float2((int)(f % mt.Nw) == tk.perm[f / mt.Nw] ? 1.f : 0.f, 0.f);
    }
  }
}

// V = binary64(V32)
__global__ void k_v_to_f64(const GateTask* tasks, const TaskMeta* meta) {
  const GateTask& tk = tasks[blockIdx.y];
  const TaskMeta& mt = meta[blockIdx.y];
  if (mt.status) return;
  const size_t nv = (size_t)mt.Nw * mt.Nw;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nv; e += (size_t)gridDim.x * blockDim.x) {
    const float2 v = tk.V32[e];
    tk.V[e] = make_double2((double)v.x, (double)v.y);
  }
}

// Newton-Schulz step V <- (3 V - V (V^H V)) / 2 = 1.5 V - 0.5 Q
__global__ void k_ns_update(const GateTask* tasks, const TaskMeta* meta) {
  const GateTask& tk = tasks[blockIdx.y];
  const TaskMeta& mt = meta[blockIdx.y];
  if (mt.status) return;
  const size_t nv = (size_t)mt.Nw * mt.Nw;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nv; e += (size_t)gridDim.x * blockDim.x) {
    const double2 v = tk.V[e], q = tk.Q[e];
    tk.V[e] = make_double2(fma(1.5, v.x, -0.5 * q.x), fma(1.5, v.y, -0.5 * q.y));
  }
}

// A = T (Mw x Nw) and re-arm the task for binary64 sweeps
__global__ void k_take_product(const GateTask* tasks, TaskMeta* meta) {
  const GateTask& tk = tasks[blockIdx.y];
  TaskMeta& mt = meta[blockIdx.y];
  if (mt.status) return;
  const size_t na = (size_t)mt.Mw * mt.Nw;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < na; e += (size_t)gridDim.x * blockDim.x)
    tk.A[e] = tk.T[e];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    mt.active = 1;
    mt.rotated = 0;
    mt.sweeps = 0;
    mt.maxoff = 0u;
    mt.hard = 0;
  }
}

// ---------------------------------------------------------- Gram polish ---

constexpr double kEps64 = 1.1102230246251565e-16;  // 2^-53
constexpr double kGramXMax = 1e-3;  // larger first-order rotations: left to the blocked sweeps

__device__ __forceinline__ bool polishing(const TaskMeta& mt) { return !mt.status && mt.active && !mt.hard; }

// sigma[p] = g_pp (the diagonal, kept while P is overwritten by X), and its
// square root in V2 (free until X^3 is formed)
__global__ void k_gram_diag(const GateTask* tasks, TaskMeta* meta) {
  const GateTask& tk = tasks[blockIdx.y];
  TaskMeta& mt = meta[blockIdx.y];
  if (!polishing(mt)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) mt.nhard = 0;
  double* sq = reinterpret_cast<double*>(tk.V2);  // free until X^3: the square roots k_gram_x needs per pair
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < mt.Nw; p += gridDim.x * blockDim.x) {
    const double g = tk.P[(size_t)p + (size_t)p * mt.Nw].x;
    tk.sigma[p] = g;
    sq[p] = sqrt(g);
  }
}

// The binary64 orthogonality test of every pair on G (numerically zero
// columns, g_jj <= (Mw eps)^2 ||A||_F^2, excluded, as in the blocked sweeps):
// mt.rotated <- a pair above Mw eps; with form_x, P <- X in place.
__global__ void k_gram_x(const GateTask* tasks, TaskMeta* meta, int form_x) {
  const GateTask& tk = tasks[blockIdx.y];
  TaskMeta& mt = meta[blockIdx.y];
  if (!polishing(mt)) return;
  const int nw = mt.Nw;
  const double tol = (double)mt.Mw * kEps64;
  const double tiny = tol * tol * mt.frob2;
  const double* sq = reinterpret_cast<const double*>(tk.V2);
  int above = 0, hard = 0;
  float mx = 0.f;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)nw * nw;
       e += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(e % nw), q = (int)(e / nw);
    double2 x = make_double2(0.0, 0.0);
    if (p != q) {
      const double app = tk.sigma[p], aqq = tk.sigma[q];
      const double2 g = tk.P[e];
      if (app > tiny && aqq > tiny) {
        const double gabs = hypot(g.x, g.y);
        const double ratio = gabs / (sq[p] * sq[q]);  // sq = sqrt(sigma), from k_gram_diag
        above |= ratio > tol;
        mx = fmaxf(mx, (float)ratio);
        // the exact Jacobi angle of the pair's 2 x 2 problem, tan 2t =
        // 2 |g_pq| / (g_qq - g_pp), with g_pq's phase: exp of the resulting
        // generator is that pair's rotation (first order in the others)
        // (the small solution |t| <= pi/4 taken directly, so that an angle
        // below pi's last bit is not lost to cancellation). x = g t / |g|;
        // for z = 2|g| / |d| < 1e-2, t / |g| = (1 - z^2/3 + z^4/5 - z^6/7) / |d|
        // (the arctangent series, relative error below z^8 / 9 < 2e-17)
        double xa = 0.0;  // |x_pq|
        if (gabs > 0.0) {
          const double dd = aqq - app, ad = fabs(dd);
          double f;
          if (2.0 * gabs < 1e-2 * ad) {
            const double inv = 1.0 / ad;
            const double z = 2.0 * gabs * inv, z2 = z * z;
            f = inv * fma(-z2, fma(-z2, fma(-z2, 1.0 / 7.0, 1.0 / 5.0), 1.0 / 3.0), 1.0);
          } else {
            f = 0.5 * atan2(2.0 * gabs, ad) / gabs;
          }
          if (dd < 0.0) f = -f;
          x = make_double2(g.x * f, g.y * f);
          xa = fabs(f) * gabs;
        }
        if (xa > kGramXMax) {
          // near-degenerate pair: left out of X and rotated exactly by
          // k_givens (up to kMaxGivens per task, else the blocked sweeps)
          if (ratio > tol && p < q) {
            const int slot = atomicAdd(&mt.nhard, 1);
            if (slot < kMaxGivens) {
              const double t = xa;
              const double sn = sin(t) / t;
              mt.hp[slot] = p;
              mt.hq[slot] = q;
              mt.hc[slot] = cos(t);
              mt.hs[slot] = make_double2(x.x * sn, x.y * sn);
            } else {
              hard = 1;
            }
          }
          x = make_double2(0.0, 0.0);
        }
      }
    }
    if (form_x) tk.P[e] = x;
  }
  if (__syncthreads_or(above) && threadIdx.x == 0) mt.rotated = 1;
  if (__syncthreads_or(hard) && threadIdx.x == 0) mt.hard = 1;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0.f) atomicMax(&mt.maxoff, __float_as_uint(mx));
}

// After a Gram test: a task with no pair above the tolerance is done; on the
// last test every other task is re-armed for the blocked binary64 sweeps and
// counted in active_count.
__global__ void k_gram_end(TaskMeta* meta, int ntask, int final_step, int* active_count) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntask) return;
  TaskMeta& mt = meta[t];
  if (mt.status || !mt.active) return;
  if (!mt.hard && !mt.rotated) {
    mt.active = 0;  // every pair within the tolerance
  } else if (final_step) {
    mt.hard = 0;
    mt.sweeps = 0;
    atomicAdd(active_count, 1);
  }
  mt.rotated = 0;
  mt.maxoff = 0u;
}

// P <- exp(X) to fourth order: I + X + X^2/2 + X^3/6 + X^4/24 (X in P, X^2 in
// Q, X^3 in V2, X^4 in T). Unitary up to |X|^5/120 (< 1e-17 for |X| <= 1e-3)
// with every entry's rounding relative to its own size: a Newton-Schulz
// correction through W^H W = I + O(eps) would put an absolute eps on each
// entry, which the small columns of B W feel relative to their norms.
__global__ void k_form_w(const GateTask* tasks, const TaskMeta* meta) {
  const GateTask& tk = tasks[blockIdx.y];
  const TaskMeta& mt = meta[blockIdx.y];
  if (!polishing(mt)) return;
  const int nw = mt.Nw;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)nw * nw;
       e += (size_t)gridDim.x * blockDim.x) {
    const double2 x = tk.P[e], x2 = tk.Q[e], x3 = tk.V2[e], x4 = tk.T[e];
    const double d = (e % nw) == (e / nw) ? 1.0 : 0.0;
    const double hx = fma(x4.x, 1.0 / 24.0, fma(x3.x, 1.0 / 6.0, 0.5 * x2.x));
    const double hy = fma(x4.y, 1.0 / 24.0, fma(x3.y, 1.0 / 6.0, 0.5 * x2.y));
    tk.P[e] = make_double2(d + (x.x + hx), x.y + hy);
  }
}

// Column scales of the product A W, in V2 (free after k_form_w): 1/||a_k||
// then ||a_k|| (1 for numerically zero columns), from the Gram diagonal.
__global__ void k_gram_scales(const GateTask* tasks, const TaskMeta* meta) {
  const GateTask& tk = tasks[blockIdx.y];
  const TaskMeta& mt = meta[blockIdx.y];
  if (!polishing(mt)) return;
  const double tol = (double)mt.Mw * kEps64, tiny = tol * tol * mt.frob2;
  double* sc = reinterpret_cast<double*>(tk.V2);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < mt.Nw; k += gridDim.x * blockDim.x) {
    const double g = tk.sigma[k];
    const double d = g > tiny ? sqrt(g) : 1.0;
    sc[k] = 1.0 / d;
    sc[mt.Nw + k] = d;
  }
}

// The exact Jacobi rotations of the near-degenerate pairs, applied in turn to
// every row of A and V: columns (p, q) <- (c a_p - conj(s) a_q, s a_p + c a_q)
// with s = sin t e^{i phi} (the pair's block of exp(X) with its exact angle).
__global__ void k_givens(const GateTask* tasks, const TaskMeta* meta) {
  const GateTask& tk = tasks[blockIdx.y];
  const TaskMeta& mt = meta[blockIdx.y];
  if (!polishing(mt) || mt.nhard <= 0) return;
  const int nh = mt.nhard < kMaxGivens ? mt.nhard : kMaxGivens;
  const int rows = mt.Mw + mt.Nw;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
    double2* M = r < mt.Mw ? tk.A : tk.V;
    const int ld = r < mt.Mw ? mt.Mw : mt.Nw;
    const int row = r < mt.Mw ? r : r - mt.Mw;
    for (int i = 0; i < nh; ++i) {
      const size_t ip = (size_t)row + (size_t)mt.hp[i] * ld, iq = (size_t)row + (size_t)mt.hq[i] * ld;
      const double2 a = M[ip], b = M[iq], s = mt.hs[i];
      const double c = mt.hc[i];
      M[ip] = make_double2(c * a.x - (s.x * b.x + s.y * b.y), c * a.y - (s.x * b.y - s.y * b.x));
      M[iq] = make_double2(fma(s.x, a.x, -s.y * a.y) + c * b.x, fma(s.x, a.y, s.y * a.x) + c * b.y);
    }
  }
}

// A <- T and V <- Q after the rotation products
__global__ void k_take_t(const GateTask* tasks, const TaskMeta* meta) {
  const GateTask& tk = tasks[blockIdx.y];
  const TaskMeta& mt = meta[blockIdx.y];
  if (!polishing(mt)) return;
  const size_t na = (size_t)mt.Mw * mt.Nw, nv = (size_t)mt.Nw * mt.Nw;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < na + nv; e += (size_t)gridDim.x * blockDim.x) {
    if (e < na) tk.A[e] = tk.T[e];
    else tk.V[e - na] = tk.Q[e - na];
  }
}

// Three-site second split: the working matrix (Mw x Nw, column-major) from T
// to A before the split SVD (to_t = 0) and back after it (to_t = 1).
__global__ void k_copy_work(const GateTask* tasks, const TaskMeta* meta, int to_t) {
  const GateTask& tk = tasks[blockIdx.y];
  const TaskMeta& mt = meta[blockIdx.y];
  if (mt.status) return;
  const size_t na = (size_t)mt.Mw * mt.Nw;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < na; e += (size_t)gridDim.x * blockDim.x) {
    if (to_t) tk.T[e] = tk.A[e];
    else tk.A[e] = tk.T[e];
  }
}

static inline int grid_for(long long el) {
  long long b = (el + 255) / 256;
  if (b > 1024) b = 1024;
  if (b < 1) b = 1;
  return (int)b;
}

void launch_oz_jobs(const GateTask* t, const TaskMeta* m, OzJob* jobs, int ntask, int kind, int s,
                    unsigned long long* flops, cudaStream_t st) {
  k_oz_jobs<<<(ntask + 127) / 128, 128, 0, st>>>(t, m, jobs, ntask, kind, s, flops);
}
void launch_gate_mix2(const GateTask* t, const TaskMeta* m, int ntask, int xl_ub, int xr_ub, cudaStream_t st) {
  k_gate_mix2<<<dim3(grid_for((long long)xl_ub * xr_ub), ntask), 256, 0, st>>>(t, m);
}
void launch_to_f32(const GateTask* t, const TaskMeta* m, int ntask, int nw_ub, long long el_ub, cudaStream_t st) {
  k_sort_cols<<<ntask, 256, (size_t)nw_ub * sizeof(double), st>>>(t, m);
  k_to_f32<<<dim3(grid_for(el_ub), ntask), 256, 0, st>>>(t, m);
}
void launch_v_to_f64(const GateTask* t, const TaskMeta* m, int ntask, long long el_ub, cudaStream_t st) {
  k_v_to_f64<<<dim3(grid_for(el_ub), ntask), 256, 0, st>>>(t, m);
}
void launch_ns_update(const GateTask* t, const TaskMeta* m, int ntask, long long el_ub, cudaStream_t st) {
  k_ns_update<<<dim3(grid_for(el_ub), ntask), 256, 0, st>>>(t, m);
}
void launch_take_product(const GateTask* t, TaskMeta* m, int ntask, long long el_ub, cudaStream_t st) {
  k_take_product<<<dim3(grid_for(el_ub), ntask), 256, 0, st>>>(t, m);
}
void launch_copy_work(const GateTask* t, const TaskMeta* m, int ntask, long long el_ub, int to_t, cudaStream_t st) {
  k_copy_work<<<dim3(grid_for(el_ub), ntask), 256, 0, st>>>(t, m, to_t);
}
void launch_givens(const GateTask* t, const TaskMeta* m, int ntask, int rows_ub, cudaStream_t st) {
  k_givens<<<dim3((rows_ub + 255) / 256, ntask), 256, 0, st>>>(t, m);
}
void launch_gram_diag(const GateTask* t, TaskMeta* m, int ntask, int nw_ub, cudaStream_t st) {
  k_gram_diag<<<dim3((nw_ub + 255) / 256, ntask), 256, 0, st>>>(t, m);
}
void launch_gram_x(const GateTask* t, TaskMeta* m, int ntask, long long el_ub, int form_x, cudaStream_t st) {
  k_gram_x<<<dim3(grid_for(el_ub), ntask), 256, 0, st>>>(t, m, form_x);
}
void launch_gram_end(TaskMeta* m, int ntask, int final_step, int* active_count, cudaStream_t st) {
  k_gram_end<<<(ntask + 127) / 128, 128, 0, st>>>(m, ntask, final_step, active_count);
}
void launch_form_w(const GateTask* t, const TaskMeta* m, int ntask, long long el_ub, cudaStream_t st) {
  k_form_w<<<dim3(grid_for(el_ub), ntask), 256, 0, st>>>(t, m);
}
void launch_gram_scales(const GateTask* t, const TaskMeta* m, int ntask, int nw_ub, cudaStream_t st) {
  k_gram_scales<<<dim3((nw_ub + 255) / 256, ntask), 256, 0, st>>>(t, m);
}
void launch_take_t(const GateTask* t, const TaskMeta* m, int ntask, long long el_ub, cudaStream_t st) {
  k_take_t<<<dim3(grid_for(el_ub), ntask), 256, 0, st>>>(t, m);
}

}  // namespace mpsgb

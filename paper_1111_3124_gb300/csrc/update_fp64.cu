// Gate-update kernels of the native binary64 path, and the blocked Jacobi's
// fp32 variant that the split-precision path (split_path.cu) preconditions
// with.
//
// Steps of one two-site update (Sec. 3.1: a U(4) gate on qubits s, s+1
// rewrites only Gamma_s, Lambda_s, Gamma_{s+1}; the update follows Vidal,
// PRL 91, 147902 (2003), to which the paper defers):
//   k_contract    theta[(i,a),(j,b)] = Lambda_{s-1}[a] Lambda_{s+1}[b]
//                   sum_{kl} U[(ij),(kl)] sum_c Gamma_s[k,a,c] Lambda_s[c] Gamma_{s+1}[l,c,b]
//                 written as the SVD working matrix (theta, or theta^H when
//                 theta is wide), column-major;
//   k_jacobi_pair blocked one-sided Jacobi: one CTA per block pair of a
//                 round-robin round, Gram of the 2b columns, Hermitian Jacobi
//                 of the Gram in shared memory, rotation of the columns of A
//                 and of the accumulated V;
//   k_colnorms    singular values = column norms of the converged A;
//   k_truncate    descending order (ties by index), kept rank, discarded
//                 weight, renormalised Lambda_s ("very small coefficients ...
//                 are truncated out", Sec. 3.1);
//   k_emit_left / k_emit_right
//                 Gamma'_s = X / Lambda_{s-1}, Gamma'_{s+1} = Y^H / Lambda_{s+1}
//                 (binary64 division), coalesced stores.
// A three-site update (U(8), Sec. 1 / Sec. 3.1) contracts two steps of
// k_contract, splits once, forms the second matrix diag(lambda_1) Y_1^H with
// k_form_second and splits again.
#include "engine.cuh"
#include "kernels.cuh"

namespace mpsgb {

// ---------------------------------------------------------------- helpers ---

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// acc + a*b
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 acc) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
  return acc;
}
// acc + conj(a)*b
__device__ __forceinline__ double2 cfma_cj(double2 a, double2 b, double2 acc) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
  return acc;
}
__device__ __forceinline__ double2 cscale(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

constexpr double kEps = 1.1102230246251565e-16;  // 2^-53

// --------------------------------------------------------------- set-up ---

// stage 0: first (or only) split of a k-site update; stage 1: second split of
// a three-site update (rows (j,c) of diag(lambda_1) Y_1^H, columns (l,b)).
__global__ void k_setup(const GateTask* tasks, TaskMeta* meta, int ntask, int stage) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntask) return;
  const GateTask& tk = tasks[t];
  TaskMeta& m = meta[t];
  if (stage == 0) {
    m.xl = tk.chi[tk.site];
    m.x0 = tk.chi[tk.site + 1];
    m.x1 = tk.k == 3 ? tk.chi[tk.site + 2] : m.x0;
    m.xr = tk.chi[tk.site + tk.k];
    m.M = 2 * m.xl;
    m.N = (tk.k == 3 ? 4 : 2) * m.xr;
    m.status = 0;
    m.disc = 0.0;
    m.sweeps_total = 0;
    m.k1 = 0;
  } else {
    m.M = 2 * m.k1;
    m.N = 2 * m.xr;
  }
  m.tall = m.M >= m.N;
  m.Mw = m.tall ? m.M : m.N;
  m.Nw = m.tall ? m.N : m.M;
  m.active = m.status == 0;
  m.rotated = 0;
  m.sweeps = 0;
  m.frob2 = 0.0;
  m.maxoff = 0u;
}

// ||A||_F^2 of every task's working matrix (invariant under the rotations).
// Columns with ||a_j|| <= Mw eps ||A||_F are numerically zero: the Jacobi
// leaves them alone and the truncation drops them.
__global__ void k_frob(const GateTask* tasks, TaskMeta* meta, int second) {
  const GateTask& tk = tasks[blockIdx.y];
  TaskMeta& mt = meta[blockIdx.y];
  if (mt.status) return;
  const double2* A = second ? tk.T : tk.A;
  const size_t total = (size_t)mt.Mw * mt.Nw;
  double s = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const double2 v = A[e];
    s = fma(v.x, v.x, fma(v.y, v.y, s));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(&mt.frob2, s);
}

// ------------------------------------------------------------ contraction ---

constexpr int kTile = 32;
constexpr int kKc = 8;

// out_{k l}[a,b] = dl[a] dr[b] sum_c X_k[a,c] dm[c] Y_l[c,b]   (k < NK, l < NL)
// MODE 0: raw blocks into T as [k*NL+l][a][b] with capacity strides.
// MODE 1: gate mix into the working matrix:
//   theta[(i,a),(J,b)] = sum_{K} U[(i*NL+J), K] out_K[a,b], K = k*NL + l.
template <int NK, int NL, int MODE>
__global__ void __launch_bounds__(256) k_contract(const GateTask* tasks, const TaskMeta* meta) {
  const GateTask& tk = tasks[blockIdx.z];
  const TaskMeta& mt = meta[blockIdx.z];
  if (mt.status) return;
  const int cap = tk.cap;
  int R, Kd, Cn;
  const double2 *X, *Y;
  const double *dl, *dm, *dr;
  if (MODE == 0) {  // B_{mn} = Gamma_{s+1}[m] Lambda_{s+1} Gamma_{s+2}[n] Lambda_{s+2}
    X = tk.g1; Y = tk.g2; R = mt.x0; Kd = mt.x1; Cn = mt.xr;
    dl = nullptr; dm = tk.lam1; dr = tk.lamR;
  } else if (NL == 2) {  // two-site theta
    X = tk.g0; Y = tk.g1; R = mt.xl; Kd = mt.x0; Cn = mt.xr;
    dl = tk.lamL; dm = tk.lam0; dr = tk.lamR;
  } else {  // three-site theta from Gamma_s and B (in T)
    X = tk.g0; Y = tk.T; R = mt.xl; Kd = mt.x0; Cn = mt.xr;
    dl = tk.lamL; dm = tk.lam0; dr = nullptr;
  }
  const int a_base = blockIdx.y * kTile, b_base = blockIdx.x * kTile;
  if (a_base >= R || b_base >= Cn) return;

  __shared__ double2 Xs[NK][kTile][kKc + 1];
  __shared__ double2 Ys[NL][kKc][kTile + 1];
  const int tid = threadIdx.x;
  const int ta = tid >> 4, tb = tid & 15;
  double2 acc[NK * NL][2][2];
#pragma unroll
  for (int q = 0; q < NK * NL; ++q)
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int u = 0; u < 2; ++u) acc[q][r][u] = make_double2(0.0, 0.0);

  for (int c0 = 0; c0 < Kd; c0 += kKc) {
    for (int e = tid; e < NK * kTile * kKc; e += 256) {
      const int k = e / (kTile * kKc), rem = e % (kTile * kKc);
      const int a = rem / kKc, c = rem % kKc;
      const int ga = a_base + a, gc = c0 + c;
      double2 v = make_double2(0.0, 0.0);
      if (ga < R && gc < Kd) v = cscale(dm[gc], X[((size_t)k * cap + ga) * cap + gc]);
      Xs[k][a][c] = v;
    }
    for (int e = tid; e < NL * kKc * kTile; e += 256) {
      const int l = e / (kKc * kTile), rem = e % (kKc * kTile);
      const int c = rem / kTile, b = rem % kTile;
      const int gc = c0 + c, gb = b_base + b;
      double2 v = make_double2(0.0, 0.0);
      if (gc < Kd && gb < Cn) v = Y[((size_t)l * cap + gc) * cap + gb];
      Ys[l][c][b] = v;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < kKc; ++c) {
      double2 xv[NK][2], yv[NL][2];
#pragma unroll
      for (int k = 0; k < NK; ++k) {
        xv[k][0] = Xs[k][2 * ta][c];
        xv[k][1] = Xs[k][2 * ta + 1][c];
      }
#pragma unroll
      for (int l = 0; l < NL; ++l) {
        yv[l][0] = Ys[l][c][2 * tb];
        yv[l][1] = Ys[l][c][2 * tb + 1];
      }
#pragma unroll
      for (int k = 0; k < NK; ++k)
#pragma unroll
        for (int l = 0; l < NL; ++l)
#pragma unroll
          for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int u = 0; u < 2; ++u) acc[k * NL + l][r][u] = cfma(xv[k][r], yv[l][u], acc[k * NL + l][r][u]);
    }
    __syncthreads();
  }

#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int a = a_base + 2 * ta + r, b = b_base + 2 * tb + u;
      if (a >= R || b >= Cn) continue;
      const double sl = dl ? dl[a] : 1.0, sr = dr ? dr[b] : 1.0;
      const double s = sl * sr;
      if (MODE == 0) {
#pragma unroll
        for (int q = 0; q < NK * NL; ++q) tk.T[((size_t)q * cap + a) * cap + b] = cscale(s, acc[q][r][u]);
      } else {
        constexpr int D = NK * NL;
        for (int i = 0; i < 2; ++i)
          for (int J = 0; J < NL; ++J) {
            double2 th = make_double2(0.0, 0.0);
#pragma unroll
            for (int q = 0; q < D; ++q) th = cfma(tk.U[(i * NL + J) * D + q], acc[q][r][u], th);
            th = cscale(s, th);
            const int row = i * R + a, col = J * Cn + b;
            if (mt.tall) tk.A[(size_t)row + (size_t)col * mt.Mw] = th;
            else tk.A[(size_t)col + (size_t)row * mt.Mw] = cconj(th);
          }
      }
    }
}

// ------------------------------------------------------------------ Jacobi ---

__device__ __forceinline__ double2* work_A(const GateTask& tk, int second) { return second ? tk.T : tk.A; }

__global__ void k_init_V(const GateTask* tasks, const TaskMeta* meta) {
  const GateTask& tk = tasks[blockIdx.y];
  const TaskMeta& mt = meta[blockIdx.y];
  if (!mt.active) return;
  const size_t nw = (size_t)mt.Nw;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nw * nw; e += (size_t)gridDim.x * blockDim.x) {
    const size_t r = e % nw, c = e / nw;
    tk.V[e] = make_double2(r == c ? 1.0 : 0.0, 0.0);
  }
}

// Circle-method (round-robin) pairing of nbe players (nbe even), round r,
// pair p: player nbe-1 meets r; the others meet (r+p, r-p) mod (nbe-1).
__device__ __forceinline__ void rr_pair(int nbe, int r, int p, int& I, int& J) {
  if (p == 0) { I = nbe - 1; J = r; }
  else {
    I = (r + p) % (nbe - 1);
    J = (r - p + nbe - 1) % (nbe - 1);
  }
}

// Complex type and unit roundoff of the arithmetic a Jacobi sweep runs in.
template <typename R> struct Cx;
template <> struct Cx<double> {
  typedef double2 T;
  static constexpr double eps = 1.1102230246251565e-16;  // 2^-53
};
template <> struct Cx<float> {
  typedef float2 T;
  static constexpr double eps = 5.9604644775390625e-08;  // 2^-24
};
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 acc) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
  return acc;
}
__device__ __forceinline__ float2 cfma_cj(float2 a, float2 b, float2 acc) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
  return acc;
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
template <typename C, typename R> __device__ __forceinline__ C mkc(R x, R y);
template <> __device__ __forceinline__ double2 mkc<double2, double>(double x, double y) { return make_double2(x, y); }
template <> __device__ __forceinline__ float2 mkc<float2, float>(float x, float y) { return make_float2(x, y); }

// One block pair (I, J) of a round: Gram of the 2b columns, Hermitian Jacobi
// of the Gram, rotation of A's and V's columns. R = double: the binary64
// sweep on (A, V) or (T, V); R = float: the fp32 preconditioning sweep on
// (A32, V32). Rotation angles are computed in binary64 in both cases.
template <int BW, typename R>
__global__ void __launch_bounds__(256) k_jacobi_pair(const GateTask* tasks, TaskMeta* meta, int round, int second,
                                                     unsigned long long* flops) {
  typedef typename Cx<R>::T C;
  constexpr double EPS = Cx<R>::eps;
  constexpr int C2 = 2 * BW;
  constexpr int NE = C2 * (C2 + 1) / 2;        // Gram entries (p <= q)
  constexpr int RCH = 64;                      // rows per staged chunk
  constexpr int CPT = RCH * C2 / 256;          // rotated outputs per thread (one row, CPT columns)
  static_assert(RCH * C2 == 256 * CPT, "rotation tiling");
  TaskMeta& mt = meta[blockIdx.y];
  if (!mt.active) return;
  const GateTask& tk = tasks[blockIdx.y];
  const int Mw = mt.Mw, Nw = mt.Nw;
  const int nb = (Nw + BW - 1) / BW;
  const int nbe = nb + (nb & 1);
  if (round >= nbe - 1) return;
  const int p = blockIdx.x;
  if (p >= nbe / 2) return;
  int I, J;
  rr_pair(nbe, round, p, I, J);
  C* A;
  C* Vm;
  if constexpr (sizeof(R) == 8) {
    A = work_A(tk, second);
    Vm = tk.V;
  } else {
    A = tk.A32;
    Vm = tk.V32;
  }
  const C zero = mkc<C, R>((R)0, (R)0);

  __shared__ int cols[C2];
  __shared__ C chunk[RCH][C2 + 1];
  __shared__ C G[C2][C2 + 1];
  __shared__ C W[C2][C2 + 1];
  __shared__ double rc_tg[C2 / 2], rc_a[C2 / 2], rc_b[C2 / 2];
  __shared__ R rc_c[C2 / 2];   // cos of the binary64 angle, rounded once to the working type
  __shared__ C rc_se[C2 / 2];  // s e^{i phi}, likewise
  __shared__ int rc_on[C2 / 2];
  __shared__ int need, any, nrot;
  const int tid = threadIdx.x;
  if (tid < C2) {
    const int blk = tid < BW ? I : J;
    const int j = blk * BW + (tid % BW);
    cols[tid] = (blk < nb && j < Nw) ? j : -1;
  }
  if (tid == 0) {
    need = 0;
    nrot = 0;
  }
  __syncthreads();

  // ---- Gram G = [A_I A_J]^H [A_I A_J]
  if constexpr (sizeof(R) == 4) {
    // fp32: 2 x 2 tiles of the upper block triangle, four independent
    // accumulators per thread
    constexpr int H = C2 / 2, NT = H * (H + 1) / 2;
    static_assert(NT <= 256, "block too wide");
    int ti = 0, tj = 0;
    if (tid < NT) {
      int rem = tid;
      while (rem >= H - ti) { rem -= H - ti; ++ti; }
      tj = ti + rem;
    }
    C a00 = zero, a01 = zero, a10 = zero, a11 = zero;
    for (int r0 = 0; r0 < Mw; r0 += RCH) {
      for (int e = tid; e < RCH * C2; e += 256) {
        const int col = e / RCH, row = e % RCH;
        const int gc = cols[col];
        chunk[row][col] = (gc >= 0 && r0 + row < Mw) ? A[(size_t)(r0 + row) + (size_t)gc * Mw] : zero;
      }
      __syncthreads();
      if (tid < NT) {
#pragma unroll 8
        for (int row = 0; row < RCH; ++row) {
          const C x0 = chunk[row][2 * ti], x1 = chunk[row][2 * ti + 1];
          const C y0 = chunk[row][2 * tj], y1 = chunk[row][2 * tj + 1];
          a00 = cfma_cj(x0, y0, a00);
          a01 = cfma_cj(x0, y1, a01);
          a10 = cfma_cj(x1, y0, a10);
          a11 = cfma_cj(x1, y1, a11);
        }
      }
      __syncthreads();
    }
    if (tid < NT) {
      const int p0 = 2 * ti, q0 = 2 * tj;
      G[p0][q0] = a00;
      G[p0][q0 + 1] = a01;
      G[p0 + 1][q0] = a10;
      G[p0 + 1][q0 + 1] = a11;
      if (ti != tj) {
        G[q0][p0] = cconj(a00);
        G[q0 + 1][p0] = cconj(a01);
        G[q0][p0 + 1] = cconj(a10);
        G[q0 + 1][p0 + 1] = cconj(a11);
      }
    }
  } else {
    // binary64 (FP64-pipe bound): one upper-triangle entry per thread
    static_assert(NE <= 256, "block too wide");
    int gp = 0, gq = 0;
    if (tid < NE) {
      int rem = tid;
      while (rem >= C2 - gp) { rem -= C2 - gp; ++gp; }
      gq = gp + rem;
    }
    C g = zero;
    for (int r0 = 0; r0 < Mw; r0 += RCH) {
      for (int e = tid; e < RCH * C2; e += 256) {
        const int col = e / RCH, row = e % RCH;
        const int gc = cols[col];
        chunk[row][col] = (gc >= 0 && r0 + row < Mw) ? A[(size_t)(r0 + row) + (size_t)gc * Mw] : zero;
      }
      __syncthreads();
      if (tid < NE) {
#pragma unroll 8
        for (int row = 0; row < RCH; ++row) g = cfma_cj(chunk[row][gp], chunk[row][gq], g);
      }
      __syncthreads();
    }
    if (tid < NE) {
      G[gp][gq] = g;
      G[gq][gp] = cconj(g);
    }
  }
  __syncthreads();
  // ---- convergence test on the actual columns: |g_pq| <= Mw eps sqrt(g_pp g_qq),
  // numerically zero columns (g_jj <= (Mw eps)^2 ||A||_F^2) excluded
  // binary64: Mw eps, the test of the oracle; fp32 preconditioning: the noise
  // floor of an fp32 Gram, 4 sqrt(Mw) eps_32
  const double tolc = sizeof(R) == 8 ? (double)Mw * EPS : 4.0 * sqrt((double)Mw) * EPS;
  // numerically zero columns: at binary64 resolution in both precisions, so the
  // fp32 passes still orthogonalise small (but nonzero) columns
  const double tiny = (double)Mw * kEps * (double)Mw * kEps * mt.frob2;
  const float tinyf = (float)tiny;  // a value that rounds to it compares the same way up to one ulp
  __shared__ unsigned int smax;
  if (tid == 0) smax = 0u;
  __syncthreads();
  for (int e = tid; e < C2 * C2; e += 256) {
    const int pp = e / C2, qq = e % C2;
    if (pp >= qq) continue;
    if constexpr (sizeof(R) == 8) {
      const double app = G[pp][pp].x, aqq = G[qq][qq].x;
      const double gabs = hypot(G[pp][qq].x, G[pp][qq].y);
      if (app > tiny && aqq > tiny) {
        const double ratio = gabs / (sqrt(app) * sqrt(aqq));
        if (ratio > tolc) need = 1;
        atomicMax(&smax, __float_as_uint((float)ratio));
      }
    } else {
      // the fp32 preconditioner's own stopping test, at fp32 resolution (the
      // binary64 sweeps that follow make the binary64 test)
      const float app = G[pp][pp].x, aqq = G[qq][qq].x;
      if (app > tinyf && aqq > tinyf) {
        const float ratio = hypotf(G[pp][qq].x, G[pp][qq].y) * (rsqrtf(app) * rsqrtf(aqq));
        if (ratio > (float)tolc) need = 1;
        atomicMax(&smax, __float_as_uint(ratio));
      }
    }
  }
  __syncthreads();
  if (tid == 0 && smax) atomicMax(&mt.maxoff, smax);
  int nv = 0;  // valid columns of this pair
  for (int c = 0; c < C2; ++c) nv += cols[c] >= 0;
  if (!need) {
    if (flops && tid == 0) atomicAdd(flops, 4ull * nv * (nv + 1) * (unsigned long long)Mw);
    return;
  }

  // ---- Hermitian Jacobi on G (two-sided, cyclic by circle-method rounds)
  for (int e = tid; e < C2 * C2; e += 256) W[e / C2][e % C2] = mkc<C, R>((e / C2) == (e % C2) ? (R)1 : (R)0, (R)0);
  __syncthreads();
  // Far from convergence, in the first sweeps, one inner sweep per pairing
  // (block Jacobi with an approximate inner solve: every rotation still lowers
  // off(A^H A), and the outer test above uses the fresh Gram); near
  // convergence, or once a hard matrix has used those sweeps, the inner solve
  // runs to convergence (the quadratic stop relies on it).
  const int inner_max = __uint_as_float(smax) > kQuadStop && mt.sweeps < kInnerFarSweeps ? kInnerSweepsFar : 24;
  for (int isw = 0; isw < inner_max; ++isw) {
    if (tid == 0) any = 0;
    __syncthreads();
    for (int ir = 0; ir < C2 - 1; ++ir) {
      if (tid < C2 / 2) {
        int pp, qq;
        rr_pair(C2, ir, tid, pp, qq);
        const double al = (double)G[pp][pp].x, be = (double)G[qq][qq].x;
        const double gx = (double)G[pp][qq].x, gy = (double)G[pp][qq].y;
        const double g2 = gx * gx + gy * gy;
        int on = al > tiny && be > tiny && g2 > 0.0 && g2 > EPS * EPS * al * be;
        rc_on[tid] = on;
        if (on) {
          // [al g; conj(g) be] = D [al |g|; |g| be] D^H, D = diag(e^{i phi}, 1):
          // the real symmetric Schur rotation of the middle matrix (Golub & Van
          // Loan, sym.schur2) in binary64, written with one square root:
          // t = tan = 2 sign(d) |g| / (|d| + sqrt(d^2 + 4|g|^2)), d = be - al,
          // so t e^{i phi} = 2 sign(d) g / (|d| + sqrt(...)) and t |g| likewise
          const double d = be - al;
          const double rD = 1.0 / (fabs(d) + sqrt(fma(d, d, 4.0 * g2)));
          const double sg = d < 0.0 ? -2.0 * rD : 2.0 * rD;
          const double tx = sg * gx, ty = sg * gy;
          const double c = rsqrt(1.0 + (tx * tx + ty * ty));
          rc_c[tid] = (R)c;
          rc_tg[tid] = sg * g2;  // t |g|
          rc_a[tid] = al;
          rc_b[tid] = be;
          rc_se[tid] = mkc<C, R>((R)(c * tx), (R)(c * ty));  // s e^{i phi}
          any = 1;
          atomicAdd(&nrot, 1);
        }
      }
      __syncthreads();
      // rows: G <- J^H G  (row p: c G_p - s e^{i phi} G_q ; row q: s e^{-i phi} G_p + c G_q)
      for (int e = tid; e < (C2 / 2) * C2; e += 256) {
        const int pr = e / C2, col = e % C2;
        if (!rc_on[pr]) continue;
        int pp, qq;
        rr_pair(C2, ir, pr, pp, qq);
        const R c = rc_c[pr];
        const C se = rc_se[pr];
        const C x = G[pp][col], y = G[qq][col];
        const C sy = cmul(se, y), cx = cmul(cconj(se), x);
        G[pp][col] = mkc<C, R>(c * x.x - sy.x, c * x.y - sy.y);
        G[qq][col] = mkc<C, R>(cx.x + c * y.x, cx.y + c * y.y);
      }
      __syncthreads();
      // columns: G <- G J and W <- W J (col p: c a_p - s e^{-i phi} a_q ; col q: s e^{i phi} a_p + c a_q)
      for (int e = tid; e < 2 * (C2 / 2) * C2; e += 256) {
        const int which = e / ((C2 / 2) * C2);
        const int rem = e % ((C2 / 2) * C2);
        const int pr = rem / C2, row = rem % C2;
        if (!rc_on[pr]) continue;
        int pp, qq;
        rr_pair(C2, ir, pr, pp, qq);
        C(*Mx)[C2 + 1] = which ? W : G;
        const R c = rc_c[pr];
        const C se = rc_se[pr];
        const C x = Mx[row][pp], y = Mx[row][qq];
        const C sy = cmul(cconj(se), y), sx = cmul(se, x);
        Mx[row][pp] = mkc<C, R>(c * x.x - sy.x, c * x.y - sy.y);
        Mx[row][qq] = mkc<C, R>(sx.x + c * y.x, sx.y + c * y.y);
      }
      __syncthreads();
      if (tid < C2 / 2 && rc_on[tid]) {
        int pp, qq;
        rr_pair(C2, ir, tid, pp, qq);
        G[pp][qq] = zero;
        G[qq][pp] = zero;
        G[pp][pp] = mkc<C, R>((R)(rc_a[tid] - rc_tg[tid]), (R)0);
        G[qq][qq] = mkc<C, R>((R)(rc_b[tid] + rc_tg[tid]), (R)0);
      }
      __syncthreads();
    }
    const int any_r = any;
    __syncthreads();
    if (!any_r) break;
  }

  // ---- rotate the columns of A (Mw rows) and of V (Nw rows) by W: each
  // thread one row of the staged chunk and CPT consecutive output columns
  // (independent accumulators; W's row k is a broadcast across the warp)
  const int rrow = tid % RCH, c0 = (tid / RCH) * CPT;
  for (int pass = 0; pass < 2; ++pass) {
    C* Mx = pass == 0 ? A : Vm;
    const int rows = pass == 0 ? Mw : Nw;
    for (int r0 = 0; r0 < rows; r0 += RCH) {
      for (int e = tid; e < RCH * C2; e += 256) {
        const int col = e / RCH, row = e % RCH;
        const int gc = cols[col];
        chunk[row][col] = (gc >= 0 && r0 + row < rows) ? Mx[(size_t)(r0 + row) + (size_t)gc * rows] : zero;
      }
      __syncthreads();
      if (r0 + rrow < rows) {
        C o[CPT];
#pragma unroll
        for (int c = 0; c < CPT; ++c) o[c] = zero;
#pragma unroll
        for (int k = 0; k < C2; ++k) {
          const C x = chunk[rrow][k];
#pragma unroll
          for (int c = 0; c < CPT; ++c) o[c] = cfma(x, W[k][c0 + c], o[c]);
        }
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
          const int gc = cols[c0 + c];
          if (gc >= 0) Mx[(size_t)(r0 + rrow) + (size_t)gc * rows] = o[c];
        }
      }
      __syncthreads();
    }
  }
  if (tid == 0) {
    mt.rotated = 1;
    // executed flops: Gram, inner rotations (rows/cols of G, cols of W), column rotations
    if (flops)
      atomicAdd(flops, 4ull * nv * (nv + 1) * (unsigned long long)Mw + 60ull * C2 * (unsigned long long)nrot +
                           8ull * nv * C2 * (unsigned long long)(Mw + Nw));
  }
}

// End of a sweep: converged when no pair rotated, or (qstop > 0) when the
// largest scaled off-diagonal met before rotation was below qstop: cyclic
// Jacobi converges quadratically, so what remains after such a sweep is
// O(n qstop^2), under the rotation threshold.
__global__ void k_sweep_end(TaskMeta* meta, int ntask, int max_sweeps, int* active_count, int fail_at_limit,
                            float qstop) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntask) return;
  TaskMeta& m = meta[t];
  if (!m.active) return;
  m.sweeps += 1;
  m.sweeps_total += 1;
  const float maxoff = __uint_as_float(m.maxoff);
  m.maxoff = 0u;
  if (!m.rotated || (qstop > 0.f && maxoff < qstop)) {
    m.active = 0;
  } else if (m.sweeps >= max_sweeps) {
    m.active = 0;
    if (fail_at_limit) {
      m.status = -4;                     // MPS_ERR_NOCONVERGE
      atomicExch(active_count + 1, -4);  // sticky per-handle status word
    }
  } else {
    atomicAdd(active_count, 1);
  }
  m.rotated = 0;
}

// sigma_j = ||A_j||_2, one warp per column
__global__ void k_colnorms(const GateTask* tasks, const TaskMeta* meta, int second) {
  const GateTask& tk = tasks[blockIdx.y];
  const TaskMeta& mt = meta[blockIdx.y];
  if (mt.status) return;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + w;
  if (j >= mt.Nw) return;
  const double2* A = work_A(tk, second) + (size_t)j * mt.Mw;
  double s = 0.0;
  for (int r = lane; r < mt.Mw; r += 32) {
    const double2 v = A[r];
    s = fma(v.x, v.x, fma(v.y, v.y, s));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) tk.sigma[j] = sqrt(s);
}

// Block-wide sum over 1024 threads (fixed reduction order).
__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    if (lane == 0) red[32] = r;
  }
  __syncthreads();
  r = red[32];
  __syncthreads();
  return r;
}

// Truncation (one CTA of 1024 threads per task): order, rank, weights, Lambda.
// stage 0 writes bond s (lam0, chi[site+1]); stage 1 writes bond s+1.
__global__ void __launch_bounds__(1024) k_truncate(const GateTask* tasks, TaskMeta* meta, int stage, int chi_cap) {
  const GateTask& tk = tasks[blockIdx.x];
  TaskMeta& mt = meta[blockIdx.x];
  if (mt.status) return;
  __shared__ double sg[2 * kMaxCap];
  __shared__ double red[33];
  const int nw = mt.Nw;
  for (int j = threadIdx.x; j < nw; j += blockDim.x) sg[j] = tk.sigma[j];
  __syncthreads();
  double part = 0.0;
  for (int j = threadIdx.x; j < nw; j += blockDim.x) part += sg[j] * sg[j];
  const double total = block_sum(part, red);
  const double rel = fmax(tk.cutoff, (double)mt.Mw * kEps);  // values at the SVD's resolution count as zero
  const double thr = rel * sqrt(total);
  // rank_j = #{i: s_i > s_j} + #{i < j: s_i == s_j}
  const double thr_sk = fmax(0.01 * tk.cutoff, (double)mt.Mw * kEps) * sqrt(total);
  int cntp = 0, cskp = 0;
  for (int j = threadIdx.x; j < nw; j += blockDim.x) {
    const double sj = sg[j];
    int rank = 0;
    for (int i = 0; i < nw; ++i) {
      const double si = sg[i];
      rank += (si > sj) || (si == sj && i < j);
    }
    tk.perm[rank] = j;
    cntp += sj > thr;
    cskp += sj > thr_sk;
  }
  const int cnt = (int)block_sum((double)cntp, red);
  const int csk = (int)block_sum((double)cskp, red);
  const int cap_k = chi_cap < tk.cap ? chi_cap : tk.cap;
  int k = cnt < cap_k ? cnt : cap_k;
  if (k < 1) k = 1;
  __syncthreads();
  double kp = 0.0, dp = 0.0;
  for (int c = threadIdx.x; c < nw; c += blockDim.x) {
    const double v = sg[tk.perm[c]];
    if (c < k) kp += v * v; else dp += v * v;
  }
  const double kept = block_sum(kp, red);
  const double dropped = block_sum(dp, red);
  const double nk = sqrt(kept);
  double* lam = stage == 0 ? tk.lam0 : tk.lam1;
  for (int c = threadIdx.x; c < k; c += blockDim.x)
    lam[c] = nk > 0.0 ? sg[tk.perm[c]] / nk : (c == 0 ? 1.0 : 0.0);
  if (threadIdx.x == 0) {
    tk.chi[tk.site + 1 + stage] = k;
    mt.knew = k;
    mt.ksk = csk;
    if (stage == 0) mt.k1 = k;
    mt.disc += total > 0.0 ? dropped / total : 0.0;
    mt.kept_norm = nk;
  }
}

// Column scale of the left/right factor: the working matrix A holds X sigma,
// so its columns are divided by sigma (0 where sigma = 0); V is unitary.
__device__ __forceinline__ double col_scale(const double* sigma, int j, bool fromA) {
  if (!fromA) return 1.0;
  const double s = sigma[j];
  return s > 0.0 ? 1.0 / s : 0.0;
}

// Gamma_out[i][a][c] = Lmat[(i*R + a), perm c] / div[a]  (i < 2, a < R, c < k)
// stage 0: Gamma'_s  (R = chi_{s-1}, div = Lambda_{s-1}); stage 1: Gamma'_{s+1}
// (R = k1, div = the new Lambda_s). 32 x 32 tiles transposed through shared memory.
__global__ void __launch_bounds__(256) k_emit_left(const GateTask* tasks, const TaskMeta* meta, int stage) {
  const int t = blockIdx.z >> 1, i = blockIdx.z & 1;
  const GateTask& tk = tasks[t];
  const TaskMeta& mt = meta[t];
  if (mt.status) return;
  const int R = stage == 0 ? mt.xl : mt.k1;
  const int kk = mt.knew;
  const int a0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  if (a0 >= R || c0 >= kk) return;
  const bool fromA = mt.tall;  // left factor: A/sigma if tall, else V
  const double2* L = fromA ? work_A(tk, stage) : tk.V;
  const int ld = fromA ? mt.Mw : mt.Nw;
  const double* div = stage == 0 ? tk.lamL : tk.lam0;
  double2* out = stage == 0 ? tk.g0 : tk.g1;
  const int cap = tk.cap;
  __shared__ double2 tile[32][33];
  for (int e = threadIdx.x; e < 1024; e += 256) {
    const int cl = e >> 5, al = e & 31;
    const int a = a0 + al, c = c0 + cl;
    double2 v = make_double2(0.0, 0.0);
    if (a < R && c < kk) {
      const int j = tk.perm[c];
      v = cscale(col_scale(tk.sigma, j, fromA) / div[a], L[(size_t)(i * R + a) + (size_t)j * ld]);
    }
    tile[al][cl] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 1024; e += 256) {
    const int al = e >> 5, cl = e & 31;
    const int a = a0 + al, c = c0 + cl;
    if (a < R && c < kk) out[((size_t)i * cap + a) * cap + c] = tile[al][cl];
  }
}

// Gamma_out[j][c][b] = conj(Rmat[(j*Cn + b), perm c]) / Lambda_out[b]  (j < 2, c < k, b < Cn)
// stage 0: Gamma'_{s+1} of a two-site update (or, for k = 3, nothing);
// stage 1: Gamma'_{s+2} of a three-site update.
__global__ void __launch_bounds__(256) k_emit_right(const GateTask* tasks, const TaskMeta* meta, int stage) {
  const int t = blockIdx.z >> 1, jj = blockIdx.z & 1;
  const GateTask& tk = tasks[t];
  const TaskMeta& mt = meta[t];
  if (mt.status) return;
  const int c = blockIdx.y;
  const int kk = mt.knew;
  if (c >= kk) return;
  const int Cn = mt.xr;
  const bool fromA = !mt.tall;  // right factor: V if tall, else A/sigma
  const double2* Rm = fromA ? work_A(tk, stage) : tk.V;
  const int ld = fromA ? mt.Mw : mt.Nw;
  double2* out = stage == 0 ? tk.g1 : tk.g2;
  const int cap = tk.cap;
  const int j = tk.perm[c];
  const double cs = col_scale(tk.sigma, j, fromA);
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < Cn; b += gridDim.x * blockDim.x) {
    const double2 v = Rm[(size_t)(jj * Cn + b) + (size_t)j * ld];
    out[((size_t)jj * cap + c) * cap + b] = cscale(cs / tk.lamR[b], cconj(v));
  }
}

// Three-site update, second matrix: M2[(j,c),(l,b)] = lambda_1[c] conj(Y1[((j*2+l)*xr + b), perm c]),
// rows j*k1 + c, columns l*xr + b; written into T as the second working matrix.
// Runs after k_truncate(stage 0) and before k_setup(stage 1) changes Mw/Nw/tall.
__global__ void __launch_bounds__(256) k_form_second(const GateTask* tasks, const TaskMeta* meta) {
  const int t = blockIdx.z;
  const GateTask& tk = tasks[t];
  const TaskMeta& mt = meta[t];
  if (mt.status) return;
  const int k1 = mt.k1, xr = mt.xr;
  const int c = blockIdx.y;
  if (c >= k1) return;
  const bool fromA = !mt.tall;  // first split's right factor
  const double2* Rm = fromA ? tk.A : tk.V;
  const int ld = fromA ? mt.Mw : mt.Nw;
  const int j1 = tk.perm[c];
  const double sc = col_scale(tk.sigma, j1, fromA) * tk.lam0[c];
  const int M2 = 2 * k1, N2 = 2 * xr;
  const bool tall2 = M2 >= N2;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 4 * xr; e += gridDim.x * blockDim.x) {
    const int jl = e / xr, b = e % xr;
    const int j = jl >> 1, l = jl & 1;
    const double2 v = cscale(sc, cconj(Rm[(size_t)(jl * xr + b) + (size_t)j1 * ld]));
    const int row = j * k1 + c, col = l * xr + b;
    if (tall2) tk.T[(size_t)row + (size_t)col * M2] = v;
    else tk.T[(size_t)col + (size_t)row * N2] = cconj(v);
  }
}

// Single-site gate: Gamma_s[i] <- sum_k u[i,k] Gamma_s[k]
__global__ void k_apply1(const SiteTask* tasks) {
  const SiteTask& tk = tasks[blockIdx.y];
  const int xl = tk.chi[tk.site], xr = tk.chi[tk.site + 1];
  const int cap = tk.cap;
  const double2 u00 = tk.U[0], u01 = tk.U[1], u10 = tk.U[2], u11 = tk.U[3];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < xl * xr; e += gridDim.x * blockDim.x) {
    const int a = e / xr, c = e % xr;
    double2* p0 = tk.g + (size_t)a * cap + c;
    double2* p1 = tk.g + ((size_t)cap + a) * cap + c;
    const double2 x0 = *p0, x1 = *p1;
    *p0 = cfma(u01, x1, cmul(u00, x0));
    *p1 = cfma(u11, x1, cmul(u10, x0));
  }
}

// ------------------------------------------------------------ host wrappers ---

static inline int cdiv(int a, int b) { return (a + b - 1) / b; }

void launch_setup(const GateTask* t, TaskMeta* m, int ntask, int stage, cudaStream_t st) {
  k_setup<<<cdiv(ntask, 128), 128, 0, st>>>(t, m, ntask, stage);
}

void launch_frob(const GateTask* t, TaskMeta* m, int ntask, long long el_ub, int second, cudaStream_t st) {
  long long bx = (el_ub + 255) / 256;
  if (bx > 256) bx = 256;
  if (bx < 1) bx = 1;
  k_frob<<<dim3((int)bx, ntask), 256, 0, st>>>(t, m, second);
}

void launch_contract2(const GateTask* t, const TaskMeta* m, int ntask, int a_ub, int b_ub, cudaStream_t st) {
  dim3 g(cdiv(b_ub, kTile), cdiv(a_ub, kTile), ntask);
  k_contract<2, 2, 1><<<g, 256, 0, st>>>(t, m);
}

void launch_contract3(const GateTask* t, const TaskMeta* m, int ntask, int x0_ub, int xl_ub, int xr_ub,
                      cudaStream_t st) {
  dim3 g1(cdiv(xr_ub, kTile), cdiv(x0_ub, kTile), ntask);
  k_contract<2, 2, 0><<<g1, 256, 0, st>>>(t, m);
  dim3 g2(cdiv(xr_ub, kTile), cdiv(xl_ub, kTile), ntask);
  k_contract<2, 4, 1><<<g2, 256, 0, st>>>(t, m);
}

void launch_init_V(const GateTask* t, const TaskMeta* m, int ntask, int nw_ub, cudaStream_t st) {
  long long el = (long long)nw_ub * nw_ub;
  int bx = (int)((el + 255) / 256);
  if (bx > 1024) bx = 1024;
  if (bx < 1) bx = 1;
  k_init_V<<<dim3(bx, ntask), 256, 0, st>>>(t, m);
}

void launch_jacobi_round(const GateTask* t, TaskMeta* m, int ntask, int round, int pairs_ub, int second,
                         unsigned long long* flops, cudaStream_t st) {
  k_jacobi_pair<kBlockW, double><<<dim3(pairs_ub, ntask), 256, 0, st>>>(t, m, round, second, flops);
}

void launch_sweep_end(TaskMeta* m, int ntask, int max_sweeps, int* active_count, cudaStream_t st) {
  k_sweep_end<<<cdiv(ntask, 128), 128, 0, st>>>(m, ntask, max_sweeps, active_count, 1, kQuadStop);
}

void launch_sweep_end_nofail(TaskMeta* m, int ntask, int max_sweeps, int* active_count, cudaStream_t st) {
  k_sweep_end<<<cdiv(ntask, 128), 128, 0, st>>>(m, ntask, max_sweeps, active_count, 0, 0.f);
}


void launch_colnorms(const GateTask* t, const TaskMeta* m, int ntask, int nw_ub, int second, cudaStream_t st) {
  k_colnorms<<<dim3(cdiv(nw_ub, 8), ntask), 256, 0, st>>>(t, m, second);
}

void launch_truncate(const GateTask* t, TaskMeta* m, int ntask, int stage, int chi_cap, cudaStream_t st) {
  k_truncate<<<ntask, 1024, 0, st>>>(t, m, stage, chi_cap);
}

void launch_emit_left(const GateTask* t, const TaskMeta* m, int ntask, int r_ub, int k_ub, int stage,
                      cudaStream_t st) {
  k_emit_left<<<dim3(cdiv(k_ub, 32), cdiv(r_ub, 32), 2 * ntask), 256, 0, st>>>(t, m, stage);
}

void launch_emit_right(const GateTask* t, const TaskMeta* m, int ntask, int cn_ub, int k_ub, int stage,
                       cudaStream_t st) {
  k_emit_right<<<dim3(cdiv(cn_ub, 256), k_ub, 2 * ntask), 256, 0, st>>>(t, m, stage);
}

void launch_form_second(const GateTask* t, const TaskMeta* m, int ntask, int k1_ub, int xr_ub, cudaStream_t st) {
  k_form_second<<<dim3(cdiv(4 * xr_ub, 256), k1_ub, ntask), 256, 0, st>>>(t, m);
}

void launch_apply1(const SiteTask* t, int ntask, int el_ub, cudaStream_t st) {
  int bx = cdiv(el_ub, 256);
  if (bx > 512) bx = 512;
  if (bx < 1) bx = 1;
  k_apply1<<<dim3(bx, ntask), 256, 0, st>>>(t);
}

}  // namespace mpsgb

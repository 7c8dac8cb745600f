// The fp32 preconditioning sweep of the split-precision SVD: one launch per
// round-robin round of the blocked one-sided Jacobi method, one CTA per block
// pair (I, J) of every task, on the fp32 copies (A32, V32) of the working
// matrix and of the accumulated right rotations.
//
// Per CTA (2b columns, b = BW):
//   1. Gram G = [A_I A_J]^H [A_I A_J] from 64-row chunks staged in shared
//      memory (the next chunk is loaded into registers while the current one
//      is multiplied; one barrier per chunk); 4 x 4 tiles of the upper
//      triangle, the rows of a chunk split over several threads per tile and
//      the partial tiles summed in a fixed order.
//   2. The fp32 test |g_pq| <= 4 sqrt(Mw) eps_32 sqrt(g_pp g_qq) (numerically
//      zero columns excluded at binary64 resolution); a pair that passes is
//      left alone.
//   3. One cyclic sweep of the two-sided Hermitian Jacobi method on G
//      (circle-method rounds of 2b/2 disjoint rotations); after a sweep's
//      first round of block pairs, only the b rounds of pairs across the two
//      blocks (the test of step 2 likewise). An inner round is one
//      barrier: in every warp, lane l forms the rotation of pair l and the
//      threads take those of their row pair and column pair by shuffle, read
//      the 2 x 2 block of G those rotations touch, then write J_i^H G_blk J_j
//      into the other of two copies of G (every block is written, changed or
//      not); the product W of the rotations is accumulated in the same pass.
//      The rotation of a 2 x 2 Hermitian problem [a g; conj(g) b] is the real
//      symmetric Schur rotation (Golub & Van Loan) conjugated by
//      diag(e^{i phi}, 1): t e^{i phi} = 2 sign(d) g / (|d| + sqrt(d^2 + 4|g|^2)),
//      d = b - a, c = 1 / sqrt(1 + |t|^2), new diagonal a - t|g|, b + t|g|,
//      formed on the problem scaled by a power of two (see make_rot).
//   4. [A_I A_J] <- [A_I A_J] W and [V_I V_J] <- [V_I V_J] W, chunk by chunk,
//      2 x 4 register tiles (W read as 16-byte broadcasts), stores of 32
//      consecutive rows per warp.
// The binary64 sweeps that follow (Gram polish, blocked binary64 Jacobi) make
// the binary64 orthogonality test, so this stage only has to bring the
// columns close to orthogonal.
#include <algorithm>

#include "engine.cuh"
#include "kernels.cuh"

namespace mpsgb {

namespace {

__device__ __forceinline__ float2 f_fma(float2 a, float2 b, float2 acc) {  // acc + a b
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
  return acc;
}
__device__ __forceinline__ float2 f_fma_cj(float2 a, float2 b, float2 acc) {  // acc + conj(a) b
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
  return acc;
}
__device__ __forceinline__ float2 f_mul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 f_conj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 f_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 f_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 f_scale(float s, float2 a) { return make_float2(s * a.x, s * a.y); }

// Circle-method pairing of n players (n even), round r, pair p.
__device__ __forceinline__ void rr_pair_f(int n, int r, int p, int& I, int& J) {
  if (p == 0) {
    I = n - 1;
    J = r;
  } else {
    I = (r + p) % (n - 1);
    J = (r - p + n - 1) % (n - 1);
  }
}

// Jacobi rotation of columns (p, q) for the 2 x 2 Hermitian [al g; conj(g) be]:
// col p' = c col_p - conj(se) col_q, col q' = se col_p + c col_q.
struct Rot {
  float c;
  float2 se;  // s e^{i phi}
  float tg;   // t |g|: the diagonal moves by -tg (p) and +tg (q)
  bool on;
};

// The 2 x 2 problem is first scaled by a power of two to O(1), so that no
// square of an entry underflows, then the rotation is formed as
// t e^{i phi} = sg g with sg = 2 sign(d) / (|d| + sqrt(d^2 + 4|g|^2)) and
// c = 1 / sqrt(1 + |t|^2), with correctly rounded square roots and divisions.
// This keeps c^2 + |s|^2 - 1 an unbiased rounding error: an approximate
// reciprocal square root or hypotenuse with a one-sided error would shrink
// or grow every rotation the same way, and over a sweep the accumulated V
// would drift from unitary, which the preconditioned columns then inherit.
__device__ __forceinline__ Rot make_rot(float al, float be, float2 g, float tinyf) {
  Rot r;
  r.c = 1.f;
  r.se = make_float2(0.f, 0.f);
  r.tg = 0.f;
  r.on = false;
  if (!(al > tinyf && be > tinyf)) return r;
  // e with max(al, be) = m 2^e, m in [0.5, 1), and sc = 2^-e: from the bits
  // for a normal maximum below 2^126 (the same values frexpf and ldexpf give,
  // in fewer dependent steps), by the library otherwise
  const float mab = fmaxf(al, be);
  const bool bits = mab >= 1.17549435e-38f && mab < 8.50705917e+37f;
  int e;
  float sc;
  if (bits) {
    e = ((__float_as_int(mab) >> 23) & 0xff) - 126;
    sc = __int_as_float((127 - e) << 23);  // exact
  } else {
    frexpf(mab, &e);
    sc = ldexpf(1.f, -e);  // exact
  }
  const float a = al * sc, b = be * sc, gx = g.x * sc, gy = g.y * sc;
  const float g2 = fmaf(gx, gx, gy * gy);
  // |g| > eps_32 sqrt(a b)
  if (!(g2 > 0.f && g2 > (3.5527137e-15f * a) * b)) return r;
  r.on = true;
  const float d = b - a;
  const float sg = (d < 0.f ? -2.f : 2.f) / (fabsf(d) + sqrtf(fmaf(d, d, 4.f * g2)));
  const float tx = sg * gx, ty = sg * gy;
  r.c = 1.f / sqrtf(1.f + fmaf(tx, tx, ty * ty));
  r.se = make_float2(r.c * tx, r.c * ty);
  // t |g| in the original scale (times 2^e: one rounding, as ldexpf)
  r.tg = bits ? (sg * g2) * __int_as_float((127 + e) << 23) : ldexpf(sg * g2, e);
  return r;
}

__device__ __forceinline__ Rot shfl_rot(const Rot& r, int src) {
  Rot o;
  o.c = __shfl_sync(0xffffffffu, r.c, src);
  o.se.x = __shfl_sync(0xffffffffu, r.se.x, src);
  o.se.y = __shfl_sync(0xffffffffu, r.se.y, src);
  o.tg = __shfl_sync(0xffffffffu, r.tg, src);
  o.on = __shfl_sync(0xffffffffu, (int)r.on, src) != 0;
  return o;
}

constexpr int kRch = 64;  // rows per staged chunk

// Shared memory of one CTA (dynamic: above the 48 KB static limit).
template <int BW, int RCH = kRch>
struct JacobiSmem {
  static constexpr int C2 = 2 * BW, NP = BW, LD = C2 + 1;
  float2 buf[2][RCH][LD];           // staged chunks; the Gram's partial tiles
  float2 G[2][C2][LD];              // Gram of the block pair; the inner sweep alternates the two copies
  float2 W[C2][C2 + 2];             // accumulated rotation (16-byte aligned rows, padded against bank conflicts)
  unsigned char prs[C2 - 1][NP][2];  // inner circle-method pairs
  int cols[C2];
  int need;  // 0: the pair is left alone; 1: it rotates (2 after the V wait of a scheduled launch, 3 if it ran out)
  int nrot;
  unsigned int smax;
};

}  // namespace

// ---- Ordering between the CTAs of the scheduled launch (see below)

constexpr unsigned long long kSchedWaitNs = 2000000000ull;
// q_sweep of a task that no longer sweeps: above every sweep number, so that
// a wait on any later sweep of that task ends at once (the item is then skipped)
constexpr int kSweepStopped = 1 << 30;

namespace {

__device__ __forceinline__ unsigned long long sched_clock_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int add_acq_rel_gpu(int* p, int v) {
  int old;
  asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// Thread 0 of a CTA: waits until *p >= v. false: the error word is set (this
// wait ran out, or another CTA's did).
__device__ bool wait_at_least(const int* p, int v, int* err) {
  if (ld_acquire_gpu(p) >= v) return true;
  const unsigned long long t0 = sched_clock_ns();
  for (;;) {
    __nanosleep(256);
    if (ld_acquire_gpu(p) >= v) return true;
    if (*(volatile int*)err) return false;
    if (sched_clock_ns() - t0 > kSchedWaitNs) {
      atomicExch(err, 1);
      return false;
    }
  }
}

}  // namespace

// The scheduled launch releases a pair's A columns as soon as they are
// rotated and rotates its V columns once the previous round has finished
// with them: aver / vver are the task's per-block counters of rounds done on
// A and on V, step the item's round number (sweeps included).
struct PairRelease {
  int* aver;
  int* vver;
  int step;
  int* err;
};

// Columns of A32 and V32 are read at L2 (ld.global.cg): under the scheduled
// launch below, other CTAs of the same launch wrote them.
__device__ __forceinline__ float2 ld_col(const float2* p) { return __ldcg(p); }

// One block pair (I, J) of task `task` in round `round`: steps 1-4 above.
// FUSED: the CTA rotates the columns of A32 and V32 itself (step 4 below).
// Otherwise it writes W (and whether the pair rotated) to the task's Wp /
// Wneed, and k_rot_tc applies W on the tensor cores. Every early return is
// taken by the whole CTA. make_prs: fill the inner pairing table (it depends
// only on BW, so a CTA that runs several pairs fills it once).
template <int BW, bool FUSED, int NTHR = 256>
__device__ __forceinline__ void pair_f32(const GateTask* tasks, TaskMeta* meta, int task, int round, int pair,
                                         unsigned long long* flops, unsigned char* jsm_raw, bool make_prs,
                                         const PairRelease* rel = nullptr) {
  constexpr int C2 = 2 * BW;                // columns of a block pair
  constexpr int NP = C2 / 2;                // disjoint rotations per inner round
  constexpr int RCH = NTHR / 4;             // rows per staged chunk (kRch at 256 threads)
  constexpr int LD = C2 + 1;                // padded chunk row, in float2
  constexpr int PER = RCH * C2 / NTHR;       // staged elements per thread
  constexpr int TB = C2 / 4;                // 4 x 4 Gram tiles per dimension
  constexpr int NT = TB * (TB + 1) / 2;     // upper-triangle tiles
  constexpr int RED = 2 * RCH * LD / 16;    // partial tiles the chunk buffers hold
  constexpr int NPART0 = NTHR / NT;
  constexpr int NPART = NPART0 * NT <= RED ? NPART0 : RED / NT;  // threads per tile
  constexpr int NCG = C2 / 4;               // rotation: column groups of 4
  constexpr int SLOTS = NTHR / NCG;          // rotation: row slots
  constexpr int TR = RCH / SLOTS;           // rotation: rows per thread and chunk
  static_assert(NP * NP <= NTHR && RCH * C2 % NTHR == 0 && RCH % SLOTS == 0, "tiling");
  static_assert(NPART >= 1, "Gram tiling");
  static_assert(NP * NP % 32 == 0 && NP <= 32, "2 x 2 blocks fill whole warps");

  TaskMeta& mt = meta[task];
  if (!mt.active) return;
  const GateTask& tk = tasks[task];
  const int Mw = mt.Mw, Nw = mt.Nw;
  const int nb = (Nw + BW - 1) / BW;
  const int nbe = nb + (nb & 1);
  if (round >= nbe - 1 || pair >= nbe / 2) return;
  int I, J;
  rr_pair_f(nbe, round, pair, I, J);
  float2* const A = tk.A32;
  float2* const Vm = tk.V32;
  const float2 zero = make_float2(0.f, 0.f);

  JacobiSmem<BW, RCH>& S = *reinterpret_cast<JacobiSmem<BW, RCH>*>(jsm_raw);
  int* const cols = S.cols;
  auto& buf = S.buf;
  auto& G = S.G[0];  // the Gram and the test; the inner sweep reads S.G[it & 1] and writes the other
  auto& W = S.W;
  auto& prs = S.prs;
  int& need = S.need;
  int& nrot = S.nrot;
  unsigned int& smax = S.smax;
  const int tid = threadIdx.x;
  if (tid < C2) {
    const int blk = tid < BW ? I : J;
    const int j = blk * BW + (tid % BW);
    cols[tid] = (blk < nb && j < Nw) ? j : -1;
  }
  for (int e = tid; make_prs && e < (C2 - 1) * NP; e += NTHR) {
    int p, q;
    rr_pair_f(C2, e / NP, e % NP, p, q);
    prs[e / NP][e % NP][0] = (unsigned char)p;
    prs[e / NP][e % NP][1] = (unsigned char)q;
  }
  if (tid == 0) {
    need = 0;
    nrot = 0;
    smax = 0u;
  }
  __syncthreads();

  // ---- 1. Gram of the 2b columns
  float2 pf[PER];
  auto fetch = [&](const float2* M, int rows, int r0) {
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int e = tid + NTHR * j, col = e / RCH, row = e % RCH;
      const int gc = cols[col];
      pf[j] = (gc >= 0 && r0 + row < rows) ? ld_col(&M[(size_t)(r0 + row) + (size_t)gc * rows]) : zero;
    }
  };
  auto stash = [&](int b) {
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int e = tid + NTHR * j;
      buf[b][e % RCH][e / RCH] = pf[j];
    }
  };
  const int gtile = tid / NPART, gpart = tid % NPART;
  int ti = 0, tj = 0;
  if (gtile < NT) {
    int rem = gtile;
    while (rem >= TB - ti) {
      rem -= TB - ti;
      ++ti;
    }
    tj = ti + rem;
  }
  float2 acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = zero;
  const int nch_a = (Mw + RCH - 1) / RCH;
  fetch(A, Mw, 0);
  stash(0);
  __syncthreads();
  for (int ch = 0; ch < nch_a; ++ch) {
    if (ch + 1 < nch_a) fetch(A, Mw, (ch + 1) * RCH);
    if (gtile < NT) {
      const int rmax = min(RCH, Mw - ch * RCH);
      for (int row = gpart; row < rmax; row += NPART) {
        float2 x[4], y[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          x[a] = buf[ch & 1][row][4 * ti + a];
          y[a] = buf[ch & 1][row][4 * tj + a];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = f_fma_cj(x[a], y[b], acc[a][b]);
      }
    }
    if (ch + 1 < nch_a) stash((ch + 1) & 1);
    __syncthreads();
  }
  // partial tiles -> G (fixed summation order over the parts); entry-major,
  // so that a warp's stores and a warp's loads touch consecutive words
  constexpr int NSLOT = NT * NPART;
  float2* red = &buf[0][0][0];
  if (gtile < NT) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) red[(a * 4 + b) * NSLOT + gtile * NPART + gpart] = acc[a][b];
  }
  __syncthreads();
  for (int e = tid; e < NT * 16; e += NTHR) {
    const int tile = e % NT, ent = e / NT;
    int ri = 0, rem = tile;
    while (rem >= TB - ri) {
      rem -= TB - ri;
      ++ri;
    }
    const int rj = ri + rem;
    float2 s = zero;
    for (int part = 0; part < NPART; ++part) s = f_add(s, red[ent * NSLOT + tile * NPART + part]);
    const int p = 4 * ri + ent / 4, q = 4 * rj + ent % 4;
    if (p < q) {
      G[p][q] = s;
      G[q][p] = f_conj(s);
    } else if (p == q) {
      G[p][p] = make_float2(s.x, 0.f);
    }
  }
  for (int e = tid; e < C2 * C2; e += NTHR) W[e / C2][e % C2] = make_float2((e / C2) == (e % C2) ? 1.f : 0.f, 0.f);
  __syncthreads();

  // ---- 2. test (binary64 zero threshold, fp32 resolution)
  // The first round of a sweep treats every pair of the block pair's columns;
  // the later rounds only the pairs across the two blocks (each block's own
  // pairs were treated at the sweep's first round, where every block takes
  // part once). Every column pair is still tested and rotated at least once a
  // sweep, so a sweep without a rotation still means every pair passed.
  const bool cross = round > 0;
  const float tolc = (float)(4.0 * sqrt((double)Mw) * 5.9604644775390625e-08);
  const float tinyf = (float)((double)Mw * 1.1102230246251565e-16 * (double)Mw * 1.1102230246251565e-16 * mt.frob2);
  {
    float mx = 0.f;
    int nd = 0;
    for (int e = tid; e < C2 * C2; e += NTHR) {
      const int p = e / C2, q = e % C2;
      if (p >= q || (cross && (p >= BW || q < BW))) continue;
      const float al = G[p][p].x, be = G[q][q].x;
      if (al > tinyf && be > tinyf) {
        const float ratio = hypotf(G[p][q].x, G[p][q].y) * (rsqrtf(al) * rsqrtf(be));
        nd |= ratio > tolc;
        mx = fmaxf(mx, ratio);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((tid & 31) == 0 && mx > 0.f) atomicMax(&smax, __float_as_uint(mx));
    if (__syncthreads_or(nd) && tid == 0) need = 1;
  }
  __syncthreads();
  if (tid == 0 && smax) atomicMax(&mt.maxoff, smax);
  int nv = 0;
  for (int c = 0; c < C2; ++c) nv += cols[c] >= 0;
  if (!need) {
    if (tid == 0) {
      if (flops) atomicAdd(flops, 4ull * nv * (nv + 1) * (unsigned long long)Mw);
      if (!FUSED) tk.Wneed[pair] = 0;
    }
    return;
  }

  // ---- 3. one cyclic sweep of the Hermitian Jacobi method on G, W = product of the rotations
  const int bi = tid / NP, bj = tid % NP;  // row pair, column pair of this thread's 2 x 2 block
  const int lane = tid & 31;
  const bool blk_warp = (tid & ~31) < NP * NP;  // warps holding 2 x 2 blocks (NP * NP is a multiple of 32)
  // the pairs of inner round ir: the circle method over the 2b columns, or
  // (cross) column l of block I with column (l + ir) mod b of block J
  const int nround = cross ? BW : C2 - 1;
  auto inner_pair = [&](int ir, int l, int& P, int& Q) {
    if (cross) {
      P = l;
      Q = BW + (l + ir) % BW;
    } else {
      P = prs[ir][l][0];
      Q = prs[ir][l][1];
    }
  };
  for (int it = 0; it < kF32InnerSweeps * nround; ++it) {
    const int ir = it % nround;
    auto& Gc = S.G[it & 1];        // this round reads one copy of G ...
    auto& Gn = S.G[(it & 1) ^ 1];  // ... and writes all of the other: one barrier per round
    Rot ri = {1.f, zero, 0.f, false}, rj = ri;
    int Pi = 0, Qi = 0, Pj = 0, Qj = 0;
    float2 x00 = zero, x01 = zero, x10 = zero, x11 = zero;
    float2 w[2][2] = {{zero, zero}, {zero, zero}};
    if (blk_warp) {  // warp-uniform
      // lane l forms the rotation of pair l mod NP (every block warp forms all
      // of them): that is this thread's column pair bj, and its row pair's
      // comes from lane bi by shuffle
      Rot mine;
      {
        int Pl, Ql;
        inner_pair(ir, lane % NP, Pl, Ql);
        mine = make_rot(Gc[Pl][Pl].x, Gc[Ql][Ql].x, Gc[Pl][Ql], tinyf);
      }
      ri = shfl_rot(mine, bi % 32);
      rj = mine;
      inner_pair(ir, bi % NP, Pi, Qi);
      inner_pair(ir, bj, Pj, Qj);
      if (tid < NP * NP) {
        x00 = Gc[Pi][Pj];
        x01 = Gc[Pi][Qj];
        x10 = Gc[Qi][Pj];
        x11 = Gc[Qi][Qj];
#pragma unroll
        for (int m = 0; m < 2; ++m) {
          w[m][0] = W[bi + NP * m][Pj];
          w[m][1] = W[bi + NP * m][Qj];
        }
      }
    }
    if (tid < NP * NP) {
      if (bi == bj) {
        if (ri.on) {
          Gn[Pi][Pi] = make_float2(x00.x - ri.tg, 0.f);
          Gn[Qi][Qi] = make_float2(x11.x + ri.tg, 0.f);
          Gn[Pi][Qi] = zero;
          Gn[Qi][Pi] = zero;
          atomicAdd(&nrot, 1);
        } else {
          Gn[Pi][Pi] = x00;
          Gn[Pi][Qi] = x01;
          Gn[Qi][Pi] = x10;
          Gn[Qi][Qi] = x11;
        }
      } else if (ri.on || rj.on) {
        // rows: Y = J_i^H X (row P' = c X_P - se X_Q, row Q' = conj(se) X_P + c X_Q)
        const float2 y00 = f_sub(f_scale(ri.c, x00), f_mul(ri.se, x10));
        const float2 y01 = f_sub(f_scale(ri.c, x01), f_mul(ri.se, x11));
        const float2 y10 = f_add(f_mul(f_conj(ri.se), x00), f_scale(ri.c, x10));
        const float2 y11 = f_add(f_mul(f_conj(ri.se), x01), f_scale(ri.c, x11));
        // columns: Z = Y J_j (col P' = c Y_P - conj(se) Y_Q, col Q' = se Y_P + c Y_Q)
        Gn[Pi][Pj] = f_sub(f_scale(rj.c, y00), f_mul(f_conj(rj.se), y01));
        Gn[Qi][Pj] = f_sub(f_scale(rj.c, y10), f_mul(f_conj(rj.se), y11));
        Gn[Pi][Qj] = f_add(f_mul(rj.se, y00), f_scale(rj.c, y01));
        Gn[Qi][Qj] = f_add(f_mul(rj.se, y10), f_scale(rj.c, y11));
      } else {
        Gn[Pi][Pj] = x00;
        Gn[Pi][Qj] = x01;
        Gn[Qi][Pj] = x10;
        Gn[Qi][Qj] = x11;
      }
      if (rj.on) {
#pragma unroll
        for (int m = 0; m < 2; ++m) {
          W[bi + NP * m][Pj] = f_sub(f_scale(rj.c, w[m][0]), f_mul(f_conj(rj.se), w[m][1]));
          W[bi + NP * m][Qj] = f_add(f_mul(rj.se, w[m][0]), f_scale(rj.c, w[m][1]));
        }
      }
    }
    __syncthreads();
  }

  if (!FUSED) {  // hand W to the tensor-core rotation
    float2* Wo = tk.Wp + (size_t)pair * C2 * C2;
    for (int e = tid; e < C2 * C2; e += NTHR) Wo[e] = W[e / C2][e % C2];
    if (tid == 0) {
      tk.Wneed[pair] = 1;
      mt.rotated = 1;
      if (flops)
        atomicAdd(flops, 4ull * nv * (nv + 1) * (unsigned long long)Mw + 60ull * C2 * (unsigned long long)nrot +
                             8ull * nv * C2 * (unsigned long long)(Mw + Nw));
    }
    return;
  }

  // ---- 4. [A_I A_J] W and [V_I V_J] W
  const int slot = tid % SLOTS, cg = tid / SLOTS;
  const int nch_v = (Nw + RCH - 1) / RCH;
  const int nch = nch_a + nch_v;
  fetch(A, Mw, 0);
  stash(0);
  __syncthreads();
  for (int ch = 0; ch < nch; ++ch) {
    const bool isA = ch < nch_a;
    float2* const M = isA ? A : Vm;
    const int rows = isA ? Mw : Nw;
    const int r0 = (isA ? ch : ch - nch_a) * RCH;
    const bool at_v = rel && ch + 1 == nch_a;  // V is fetched only after its wait below
    if (ch + 1 < nch && !at_v) {
      const bool nA = ch + 1 < nch_a;
      fetch(nA ? A : Vm, nA ? Mw : Nw, (nA ? ch + 1 : ch + 1 - nch_a) * RCH);
    }
    float2 o[TR][4];
#pragma unroll
    for (int r = 0; r < TR; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) o[r][c] = zero;
#pragma unroll 8
    for (int k = 0; k < C2; ++k) {
      const float4 w01 = *reinterpret_cast<const float4*>(&W[k][4 * cg]);
      const float4 w23 = *reinterpret_cast<const float4*>(&W[k][4 * cg + 2]);
      const float2 wv[4] = {make_float2(w01.x, w01.y), make_float2(w01.z, w01.w), make_float2(w23.x, w23.y),
                            make_float2(w23.z, w23.w)};
#pragma unroll
      for (int r = 0; r < TR; ++r) {
        const float2 x = buf[ch & 1][slot + SLOTS * r][k];
#pragma unroll
        for (int c = 0; c < 4; ++c) o[r][c] = f_fma(x, wv[c], o[r][c]);
      }
    }
#pragma unroll
    for (int r = 0; r < TR; ++r) {
      const int row = r0 + slot + SLOTS * r;
      if (row < rows) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int gc = cols[4 * cg + c];
          if (gc >= 0) M[(size_t)row + (size_t)gc * rows] = o[r][c];
        }
      }
    }
    if (ch + 1 < nch && !at_v) stash((ch + 1) & 1);
    __syncthreads();
    if (at_v) {
      // A_I, A_J are final: the next round may read them. V_I, V_J: wait
      // until every earlier round has finished with them.
      if (tid == 0) {
        __threadfence();
        st_release_gpu(rel->aver + I, rel->step + 1);
        st_release_gpu(rel->aver + J, rel->step + 1);
        need = wait_at_least(rel->vver + I, rel->step, rel->err) && wait_at_least(rel->vver + J, rel->step, rel->err)
                   ? 2
                   : 3;
      }
      __syncthreads();
      if (need == 3) return;  // a wait ran out: the launch is abandoned
      fetch(Vm, Nw, 0);
      stash((ch + 1) & 1);
      __syncthreads();
    }
  }
  if (tid == 0) {
    mt.rotated = 1;
    if (flops)
      atomicAdd(flops, 4ull * nv * (nv + 1) * (unsigned long long)Mw + 60ull * C2 * (unsigned long long)nrot +
                           8ull * nv * C2 * (unsigned long long)(Mw + Nw));
  }
}

// One launch per round-robin round: blockIdx.y = task, blockIdx.x = pair.
template <int BW, bool FUSED>
__global__ void __launch_bounds__(256, 3)
    k_jacobi_pair_f32(const GateTask* tasks, TaskMeta* meta, int round, unsigned long long* flops) {
  extern __shared__ __align__(16) unsigned char jsm_raw[];
  pair_f32<BW, FUSED>(tasks, meta, blockIdx.y, round, blockIdx.x, flops, jsm_raw, true);
}

// ---- Scheduled sweeps: every fp32 sweep of every task in one launch
//
// The work items (sweep s, round r, task t, pair p) are numbered sweep-major,
// then by round, task and pair. A CTA takes the next number from a counter
// (the number after that already while it runs the current item), waits until
// the item's inputs are final, runs the pair (steps 1-4) and reports it.
//
// An item depends on the two items of the previous round of its own task that
// last wrote its blocks I and J, and, in the first round of a sweep, on the
// decision taken at the end of the task's previous sweep. The dependency on A
// and on V is tracked apart (per-block round counters of each, qver): a pair
// releases A_I, A_J as soon as it has rotated them, so the next round's Gram
// can start while it rotates V_I, V_J, which it does once the previous round
// has finished with them.
//
// The numbering is a topological order of these dependencies, and a CTA
// takes numbers only while it runs and runs its items in the order taken. So
// the unfinished item with the smallest number always has its inputs final
// and every wait ends. Each wait is bounded all the same (kSchedWaitNs by
// %globaltimer): one that runs out sets the error word and every CTA of the
// launch returns.
//
// Per task, q_done counts the finished pairs of all its sweeps. The CTA that
// finishes the last pair of a sweep takes the end-of-sweep decision (the task
// stops when no pair rotated, or at the sweep limit) and then publishes it in
// q_sweep: the next sweep's number, or kSweepStopped, which ends the wait of
// any later item of the task (such items are skipped). Tasks that do not
// sweep at all start at kSweepStopped.
//
// Each task runs the pairs, rounds and sweeps of the per-round launches on the
// same data, so the results are the same bit for bit; only the order in which
// independent pairs run differs. What this removes is the launch per round and
// the partly filled last wave of every round (a saturated round of 32 tasks is
// 512 CTAs against 456 resident); and a task's next round no longer waits for
// the slowest pair of every other task's round.
struct F32Sched {
  unsigned long long head;  // next work item
  int n_active;             // tasks still sweeping
  int pad;
};
static_assert(sizeof(F32Sched) <= 16, "fits the handle's counter words 4..7");

// One CTA per task: resets its counters and counts it if it sweeps (the
// launcher zeroes the F32Sched words first).
template <int BW>
__global__ void k_f32_sched_setup(const GateTask* tasks, TaskMeta* meta, F32Sched* q) {
  TaskMeta& mt = meta[blockIdx.x];
  const int nb = (mt.Nw + BW - 1) / BW, nbe = nb + (nb & 1);
  int* ver = tasks[blockIdx.x].qver;  // [0, nbe): rounds done on A; [nbe, 2 nbe): on V
  for (int b = threadIdx.x; b < 2 * nbe; b += blockDim.x) ver[b] = 0;
  if (threadIdx.x == 0) {
    mt.q_done = 0;
    if (mt.active && mt.Nw < 1) {  // no pair: one empty sweep, as the per-round launches
      mt.sweeps += 1;
      mt.sweeps_total += 1;
      mt.active = 0;
      mt.rotated = 0;
      mt.maxoff = 0u;
    }
    mt.q_sweep = mt.active ? 0 : kSweepStopped;
    if (mt.active) atomicAdd(&q->n_active, 1);
  }
}

// NTHR threads per CTA: 256 (three CTAs per SM) or 384 (two per SM: the same
// warps per SM in fewer pairs at a time; measured slower at Nw = 512 and a
// little faster at Nw = 256, so the tuner chooses).
template <int BW, int NTHR>
__global__ void __launch_bounds__(NTHR, NTHR == 256 ? 3 : 2)
    k_jacobi_f32_sched(const GateTask* tasks, TaskMeta* meta, int ntask, int r_ub, int p_ub, int max_sweeps,
                       unsigned long long total, F32Sched* q, int* err, unsigned long long* flops) {
  using Smem = JacobiSmem<BW, NTHR / 4>;
  extern __shared__ __align__(16) unsigned char jsm_raw[];
  __shared__ int item[4];  // task (-1: nothing left), round, pair, sweep
  {
    Smem& S = *reinterpret_cast<Smem*>(jsm_raw);
    constexpr int C2 = 2 * BW, NP = BW;
    for (int e = threadIdx.x; e < (C2 - 1) * NP; e += blockDim.x) {
      int p, qq;
      rr_pair_f(C2, e / NP, e % NP, p, qq);
      S.prs[e / NP][e % NP][0] = (unsigned char)p;
      S.prs[e / NP][e % NP][1] = (unsigned char)qq;
    }
  }
  constexpr unsigned long long kNone = ~0ull;
  unsigned long long w_next = kNone;  // thread 0: the next item's number, taken ahead
  for (;;) {
    if (threadIdx.x == 0) {
      int t = -1, r = 0, p = 0, s = 0;
      for (;;) {
        t = -1;
        if (*(volatile int*)&q->n_active == 0 || *(volatile int*)err) break;
        const unsigned long long w = w_next != kNone ? w_next : atomicAdd(&q->head, 1ull);
        w_next = kNone;
        if (w >= total) break;
        unsigned long long x = w;
        p = (int)(x % (unsigned)p_ub);
        x /= (unsigned)p_ub;
        const int tt = (int)(x % (unsigned)ntask);
        x /= (unsigned)ntask;
        r = (int)(x % (unsigned)r_ub);
        s = (int)(x / (unsigned)r_ub);
        TaskMeta& mt = meta[tt];
        const int nb = (mt.Nw + BW - 1) / BW, nbe = nb + (nb & 1);
        const int nr = nbe - 1, np = nbe / 2;
        if (r >= nr || p >= np) continue;  // the task has fewer blocks
        if (!wait_at_least(&mt.q_sweep, s, err)) break;
        if (!*(volatile int*)&mt.active) continue;  // stopped at the end of an earlier sweep
        if (r > 0) {  // the round before wrote blocks I and J
          int I, J;
          rr_pair_f(nbe, r, p, I, J);
          const int* ver = tasks[tt].qver;
          if (!wait_at_least(ver + I, s * nr + r, err) || !wait_at_least(ver + J, s * nr + r, err)) break;
        }
        t = tt;
        break;
      }
      item[0] = t;
      item[1] = r;
      item[2] = p;
      item[3] = s;
      // take the next number now: the counter's latency hides behind this
      // item, and the next item's inputs get this item's duration to become
      // final. Items are still run in the order taken, so the argument above
      // holds: a CTA that holds an unfinished item is running an earlier one
      // or waiting on inputs of smaller number.
      if (t >= 0) w_next = atomicAdd(&q->head, 1ull);
    }
    __syncthreads();
    const int t = item[0], r = item[1], p = item[2], s = item[3];
    if (t < 0) return;
    int step = 0, nbe_t = 0;
    {
      const TaskMeta& mt = meta[t];
      const int nb = (mt.Nw + BW - 1) / BW;
      nbe_t = nb + (nb & 1);
      step = s * (nbe_t - 1) + r;
    }
    const PairRelease rel = {tasks[t].qver, tasks[t].qver + nbe_t, step, err};
    pair_f32<BW, true, NTHR>(tasks, meta, t, r, p, flops, jsm_raw, false, &rel);
    __syncthreads();
    if (threadIdx.x == 0) {
      TaskMeta& mt = meta[t];
      const int nr = nbe_t - 1, per_sweep = nr * (nbe_t / 2);
      int I, J;
      rr_pair_f(nbe_t, r, p, I, J);
      const int need = reinterpret_cast<const Smem*>(jsm_raw)->need;
      __threadfence();
      if (need == 0) {  // no rotation: A is released here (a rotating pair released it after rotating A)
        st_release_gpu(rel.aver + I, step + 1);
        st_release_gpu(rel.aver + J, step + 1);
      }
      // V: one more round done on blocks I and J. Counted, not stored: a pair
      // of the next round that does not rotate may count before this one has.
      atomicAdd(rel.vver + I, 1);
      atomicAdd(rel.vver + J, 1);
      if (add_acq_rel_gpu(&mt.q_done, 1) + 1 == (s + 1) * per_sweep) {
        // end of the task's sweep s (the end-of-sweep rule without a failure at the limit)
        mt.sweeps += 1;
        mt.sweeps_total += 1;
        mt.maxoff = 0u;
        const bool stop = !mt.rotated || mt.sweeps >= max_sweeps;
        if (stop) mt.active = 0;
        mt.rotated = 0;
        __threadfence();
        st_release_gpu(&mt.q_sweep, stop ? kSweepStopped : s + 1);
        if (stop) atomicSub(&q->n_active, 1);
      }
    }
  }
}

template <int BW, bool FUSED>
static void launch_pair_f32(const GateTask* t, TaskMeta* m, int ntask, int round, int pairs_ub,
                            unsigned long long* flops, cudaStream_t st) {
  constexpr int bytes = (int)sizeof(JacobiSmem<BW>);
  k_jacobi_pair_f32<BW, FUSED><<<dim3(pairs_ub, ntask), 256, bytes, st>>>(t, m, round, flops);
}

// resident CTAs of the scheduled kernel: [block width 8, 16][256, 384 threads]
static int g_sched_ctas[2][2] = {{0, 0}, {0, 0}};

template <int BW, int NTHR>
static void sched_prepare(int sms) {
  constexpr int bytes = (int)sizeof(JacobiSmem<BW, NTHR / 4>);
  cudaFuncSetAttribute(k_jacobi_f32_sched<BW, NTHR>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_jacobi_f32_sched<BW, NTHR>, NTHR, bytes);
  g_sched_ctas[BW == 8 ? 0 : 1][NTHR == 256 ? 0 : 1] = std::max(1, per) * std::max(1, sms);
}

void jacobi_f32_prepare() {
  static bool done = false;
  if (done) return;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  sched_prepare<8, 256>(sms);
  sched_prepare<16, 256>(sms);
  sched_prepare<8, 384>(sms);
  sched_prepare<16, 384>(sms);
  cudaFuncSetAttribute(k_jacobi_pair_f32<8, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sizeof(JacobiSmem<8>));
  cudaFuncSetAttribute(k_jacobi_pair_f32<16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sizeof(JacobiSmem<16>));
  cudaFuncSetAttribute(k_jacobi_pair_f32<16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sizeof(JacobiSmem<16>));
  done = true;
}

void launch_jacobi_round_f32(const GateTask* t, TaskMeta* m, int ntask, int round, int pairs_ub, int bw, int fused,
                             unsigned long long* flops, cudaStream_t st) {
  jacobi_f32_prepare();
  if (bw == 8)
    launch_pair_f32<8, true>(t, m, ntask, round, pairs_ub, flops, st);
  else if (fused)
    launch_pair_f32<16, true>(t, m, ntask, round, pairs_ub, flops, st);
  else
    launch_pair_f32<16, false>(t, m, ntask, round, pairs_ub, flops, st);
}

// All fp32 sweeps of every task in one scheduled launch (fused rotation),
// after a set-up of the counters (one CTA per task). sched points to four ints of device
// memory (8-byte aligned) the launch may overwrite; err is the handle's error
// word. Returns the number of launches (0 or 2), or -1 when the launch failed.
int launch_jacobi_f32_sched(const GateTask* t, TaskMeta* m, int ntask, int nw_ub, int bw, int nthr, int max_sweeps,
                            void* sched, int* err, unsigned long long* flops, cudaStream_t st) {
  jacobi_f32_prepare();
  if (ntask < 1 || nw_ub < 1 || max_sweeps < 1) return 0;
  const int nb = (nw_ub + bw - 1) / bw, nbe = nb + (nb & 1);
  const int r_ub = nbe - 1, p_ub = nbe / 2;
  const unsigned long long total = (unsigned long long)max_sweeps * r_ub * (unsigned long long)ntask * p_ub;
  F32Sched* q = static_cast<F32Sched*>(sched);
  if (cudaMemsetAsync(q, 0, sizeof(F32Sched), st) != cudaSuccess) return -1;
  if (bw == 8)
    k_f32_sched_setup<8><<<ntask, 128, 0, st>>>(t, m, q);
  else
    k_f32_sched_setup<16><<<ntask, 128, 0, st>>>(t, m, q);
  const bool wide = nthr == 384;
  const unsigned long long cap = (unsigned long long)g_sched_ctas[bw == 8 ? 0 : 1][wide ? 1 : 0];
  // a cooperative launch (every CTA resident at once); the pull order above
  // needs only that a CTA holding an item runs, which any launch gives
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)std::min(total, cap));
  cfg.blockDim = dim3(wide ? 384 : 256);
  cfg.dynamicSmemBytes = bw == 8 ? (wide ? sizeof(JacobiSmem<8, 96>) : sizeof(JacobiSmem<8>))
                                 : (wide ? sizeof(JacobiSmem<16, 96>) : sizeof(JacobiSmem<16>));
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e;
  if (bw == 8)
    e = wide ? cudaLaunchKernelEx(&cfg, k_jacobi_f32_sched<8, 384>, t, m, ntask, r_ub, p_ub, max_sweeps, total, q, err,
                                  flops)
             : cudaLaunchKernelEx(&cfg, k_jacobi_f32_sched<8, 256>, t, m, ntask, r_ub, p_ub, max_sweeps, total, q, err,
                                  flops);
  else
    e = wide ? cudaLaunchKernelEx(&cfg, k_jacobi_f32_sched<16, 384>, t, m, ntask, r_ub, p_ub, max_sweeps, total, q,
                                  err, flops)
             : cudaLaunchKernelEx(&cfg, k_jacobi_f32_sched<16, 256>, t, m, ntask, r_ub, p_ub, max_sweeps, total, q,
                                  err, flops);
  return e == cudaSuccess ? 2 : -1;
}

}  // namespace mpsgb

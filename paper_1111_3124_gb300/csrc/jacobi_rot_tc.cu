// Tensor-core block rotation of the fp32 preconditioning sweep: for every
// block pair (I, J) of a round, [A_I A_J] <- [A_I A_J] W and
// [V_I V_J] <- [V_I V_J] W, with W (2b x 2b, b = 16) the product of the pair's
// inner Jacobi rotations written by k_jacobi_pair_f32. One CTA per 128 rows
// of A32, or of V32, for one pair.
//
// The product runs on the tcgen05 tensor cores as exact integer arithmetic
// (the Ozaki scheme, as in ozaki_tc.cu, at fp32 width):
//   * complex to real: row m of X = [Re x_m0 .. Re x_m31, Im x_m0 .. Im x_m31]
//     (K = 64), column n of W_r = [Re w_:n; -Im w_:n] for n < 32 and
//     [Im w_:n; Re w_:n] for n >= 32, so (X W_r)[m][n] is Re / Im of (x W)[m][n mod 32];
//   * every column k of X gets a power-of-two scale 2^{e_k} from its largest
//     entry in the tile (one per complex column), folded exactly into row k
//     of W_r; every column n of the scaled W_r gets one from its own largest
//     entry; each entry is rounded to 24 bits relative to its scale (to
//     nearest even) and cut into three signed 8-bit digits, exact in bf16.
//     Column scales keep what one-sided Jacobi needs: every column of the
//     rotated A (Sigma-graded, like U Sigma) to fp32 accuracy relative to its
//     own norm (a row scale would round the small columns away);
//   * the nine digit products (p, q) are tcgen05.mma.kind::f16 chains
//     (M = 128, N = 64, K = 16) summed over K = 64 into fp32 TMEM: each product
//     is below 2^16 and each diagonal p + q holds at most three of them, so
//     every sum stays below 2^24 and is exact; the diagonals alternate between
//     two TMEM accumulators that eight warps drain into one 64-bit integer per
//     output while the next diagonal is multiplied;
//   * the result 2^{f_n} sum 2^{-8(p+q)} S_{p+q} is rounded to fp32 once.
// The only roundings are the operands' to 24 bits and the final one, both to
// nearest: the product is as accurate as an fp32 dot product and carries no
// one-sided error that would make the accumulated rotations drift from
// unitary.
#include <cuda_bf16.h>

#include "engine.cuh"
#include "kernels.cuh"
#include "tc_ptx.cuh"

namespace mpsgb {

namespace {

constexpr int kRtRows = 128;                  // rows per CTA (the MMA's M)
constexpr int kRtThreads = 288;               // warps 0-7 split and drain, warp 8 issues the MMAs
constexpr int kRtC2 = 32;                     // columns of a block pair (b = 16)
constexpr int kRtTileA = kRtRows * 64 * 2;    // one digit slice of X: 128 x 64 bf16
constexpr int kRtTileB = 64 * 64 * 2;         // one digit slice of W_r: 64 x 64 bf16
constexpr int kRtSmem = 1024 /*alignment*/ + 3 * kRtTileA + 3 * kRtTileB + 4096 /*small arrays, barriers*/;
constexpr int kRtTmemCols = 128;              // two 64-column fp32 accumulators

// Byte offset of element (row, k) in a K-major tile of 64 bf16 per row with
// the 128-byte swizzle: the 16-byte chunk index is XORed with row mod 8.
__device__ __forceinline__ uint32_t sw128(int row, int k) {
  const uint32_t byte = (uint32_t)k * 2u;
  return (uint32_t)(row >> 3) * 1024u + (uint32_t)(row & 7) * 128u + ((((byte >> 4) ^ (uint32_t)(row & 7)) & 7u) << 4) +
         (byte & 15u);
}

// The 24-bit magnitude of x relative to the biased exponent emax of its row's
// (or column's) largest entry, rounded to nearest even: X = |x| 2^{24 - e} with
// e = emax - 126, so that the largest entry maps to its own significand.
__device__ __forceinline__ int mag24(float x, int emax) {
  const unsigned b = __float_as_uint(x);
  const int E = (int)((b >> 23) & 0xFF);
  if (E == 0) return 0;  // zero (subnormals count as zero)
  const int m = (int)((b & 0x7FFFFF) | 0x800000);
  const int sh = emax - E;  // >= 0
  if (sh == 0) return m;
  if (sh > 24) return 0;
  // round half to even (rounding ties up would bias every product upward)
  const int q = m >> sh, rem = m & ((1 << sh) - 1), half = 1 << (sh - 1);
  return q + ((rem > half || (rem == half && (q & 1))) ? 1 : 0);
}

// Three signed 8-bit digits of x (sign of x on every digit), as bf16 pairs
// (lo = this element, hi = the next one) are written by the caller.
__device__ __forceinline__ void digits3(float x, int emax, int* d) {
  const int X = mag24(x, emax);
  const int s = __float_as_uint(x) >> 31 ? -1 : 1;
  d[0] = s * (X >> 16);
  d[1] = s * ((X >> 8) & 255);
  d[2] = s * (X & 255);
}

__device__ __forceinline__ uint32_t pack_bf16(int lo, int hi) {
  const __nv_bfloat16 a = __float2bfloat16_rn((float)lo), b = __float2bfloat16_rn((float)hi);
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

__device__ __forceinline__ int biased_exp(float x) { return (int)((__float_as_uint(x) >> 23) & 0xFF); }

__device__ __forceinline__ void rr_pair_r(int n, int r, int p, int& I, int& J) {
  if (p == 0) {
    I = n - 1;
    J = r;
  } else {
    I = (r + p) % (n - 1);
    J = (r - p + n - 1) % (n - 1);
  }
}

}  // namespace

__global__ void __launch_bounds__(kRtThreads, 2)
    k_rot_tc(const GateTask* tasks, const TaskMeta* meta, int round, int mt_ub, int* err) {
  constexpr int BW = kRtC2 / 2;
  const TaskMeta& mt = meta[blockIdx.y];
  if (!mt.active) return;
  const GateTask& tk = tasks[blockIdx.y];
  const int Mw = mt.Mw, Nw = mt.Nw;
  const int nb = (Nw + BW - 1) / BW;
  const int nbe = nb + (nb & 1);
  const int pair = blockIdx.x / mt_ub, tile = blockIdx.x % mt_ub;
  if (round >= nbe - 1 || pair >= nbe / 2) return;
  // tiles of A's rows, then tiles of V's rows: a column scale is shared by a
  // tile's rows, and the columns of A (Sigma-graded) and of V (unit) must not
  // share one
  const int tA = (Mw + kRtRows - 1) / kRtRows;
  const bool isA = tile < tA;
  const int row0 = (isA ? tile : tile - tA) * kRtRows;
  const int rows = isA ? Mw : Nw;
  if (row0 >= rows) return;
  if (!tk.Wneed[pair]) return;  // every pair of the block pair already orthogonal: W = I
  int I, J;
  rr_pair_r(nbe, round, pair, I, J);

  extern __shared__ unsigned char rt_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)rt_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = base;                   // 3 slices of X
  unsigned char* sB = base + 3 * kRtTileA;    // 3 slices of W_r
  unsigned char* small = sB + 3 * kRtTileB;
  unsigned int* xmax = reinterpret_cast<unsigned int*>(small);         // [32] bit patterns of X's column maxima
  int* ex = reinterpret_cast<int*>(small + 1024);                      // [32] their biased exponents
  unsigned int* colmax = reinterpret_cast<unsigned int*>(small + 1536);  // [8][32] partial maxima of W~
  int* ecol = reinterpret_cast<int*>(small + 2560);                    // [32] biased exponents of W~'s columns
  int* cols = reinterpret_cast<int*>(small + 2688);                    // [32]
  uint64_t* bars = reinterpret_cast<uint64_t*>(small + 2816);          // accf[2], acce[2]
  uint64_t* accf = bars;
  uint64_t* acce = bars + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(small + 2880);
  float2* stage = reinterpret_cast<float2*>(base);                     // [128][33] after the products

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid < kRtC2) {
    const int blk = tid < BW ? I : J;
    const int j = blk * BW + (tid % BW);
    cols[tid] = (blk < nb && j < Nw) ? j : -1;
  }
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&accf[i], 1);
      mbar_init(&acce[i], 8);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 8) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kRtTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // ---- X: 128 rows of [A32; V32] at the pair's columns, column maxima
  if (tid < kRtC2) xmax[tid] = 0u;
  __syncthreads();
  float2 x[16];
  const int r = tid % kRtRows, hh = (tid / kRtRows) & 1;  // row of the tile; columns [16 hh, 16 hh + 16)
  const int lrow = row0 + r;
  const bool vrow = lrow < rows;
  float2* const Mrow = isA ? tk.A32 : tk.V32;
  const int ld = rows;
  if (tid < 256) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int gc = cols[16 * hh + j];
      x[j] = (vrow && gc >= 0) ? Mrow[(size_t)lrow + (size_t)gc * ld] : make_float2(0.f, 0.f);
      float mx = fmaxf(fabsf(x[j].x), fabsf(x[j].y));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0) atomicMax(&xmax[16 * hh + j], __float_as_uint(mx));
    }
  }
  __syncthreads();
  if (tid < kRtC2) ex[tid] = biased_exp(__uint_as_float(xmax[tid]));
  __syncthreads();
  // ---- W~ = diag(2^{e_k}) W, its column scales and digit slices of W~_r
  const float2* Wg = tk.Wp + (size_t)pair * kRtC2 * kRtC2;  // W[k][c], row-major
  if (tid < 256) {
    const int c = tid % 32, kq = tid / 32;
    float mx = 0.f;
#pragma unroll
    for (int k = 4 * kq; k < 4 * kq + 4; ++k) {
      const float2 w = Wg[k * kRtC2 + c];
      const float sk = ex[k] ? ldexpf(1.f, ex[k] - 126) : 0.f;
      mx = fmaxf(mx, sk * fmaxf(fabsf(w.x), fabsf(w.y)));
    }
    colmax[kq * 32 + c] = __float_as_uint(mx);
  }
  __syncthreads();
  if (tid < 32) {
    unsigned int m = 0u;
    for (int kq = 0; kq < 8; ++kq) m = max(m, colmax[kq * 32 + tid]);
    ecol[tid] = biased_exp(__uint_as_float(m));
  }
  __syncthreads();
  if (tid < 256) {
    const int n = tid % 64, kb = tid / 64;  // column n of W~_r, rows k in [16 kb, 16 kb + 16)
    const int c = n % 32, E = ecol[c];
#pragma unroll
    for (int k = 16 * kb; k < 16 * kb + 16; k += 2) {
      float v[2];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int kk = k + t, kc = kk % 32;
        const float2 w = Wg[kc * kRtC2 + c];
        const float sk = ex[kc] ? ldexpf(1.f, ex[kc] - 126) : 0.f;
        v[t] = sk * (n < 32 ? (kk < 32 ? w.x : -w.y) : (kk < 32 ? w.y : w.x));
      }
      int d0[3], d1[3];
      digits3(v[0], E, d0);
      digits3(v[1], E, d1);
#pragma unroll
      for (int p = 0; p < 3; ++p)
        *reinterpret_cast<uint32_t*>(sB + p * kRtTileB + sw128(n, k)) = pack_bf16(d0[p], d1[p]);
    }
    // ---- X~ = X diag(2^{-e_k}): digit slices
#pragma unroll
    for (int j = 0; j < 16; j += 2) {
      const int c = 16 * hh + j;
      int a0[3], a1[3], b0[3], b1[3];
      digits3(x[j].x, ex[c], a0);
      digits3(x[j + 1].x, ex[c + 1], a1);
      digits3(x[j].y, ex[c], b0);
      digits3(x[j + 1].y, ex[c + 1], b1);
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        *reinterpret_cast<uint32_t*>(sA + p * kRtTileA + sw128(r, c)) = pack_bf16(a0[p], a1[p]);
        *reinterpret_cast<uint32_t*>(sA + p * kRtTileA + sw128(r, 32 + c)) = pack_bf16(b0[p], b1[p]);
      }
    }
  }
  // the tensor cores read the slices through the async proxy
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  long long tot[32];
  bool ok = true;
  if (warp == 8) {
    if (lane == 0) {  // ------------------------------------------- MMA issuer
      const uint32_t idesc = idesc_bf16_f32(kRtRows, 64);
      for (int D = 0; D < 5 && ok; ++D) {  // diagonal p + q = D + 2 (digits 1-based)
        const int acc = D & 1, use = D >> 1;
        if (use > 0 && !mbar_wait(&acce[acc], (uint32_t)((use - 1) & 1), err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t dcol = tmem + (uint32_t)(acc * 64);
        bool first = true;
        for (int p = 0; p < 3; ++p) {
          const int q = D - p;
          if (q < 0 || q > 2) continue;
          const uint64_t da = smem_desc_sw128(sA + p * kRtTileA);
          const uint64_t db = smem_desc_sw128(sB + q * kRtTileB);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            mma_bf16(dcol, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc, first ? 0u : 1u);
            first = false;
          }
        }
        mma_commit(&accf[acc]);
      }
    }
  } else {  // ------------------------------------------------------- drain
    const int quarter = warp & 3, half = warp >> 2;
#pragma unroll
    for (int j = 0; j < 32; ++j) tot[j] = 0;
    for (int D = 0; D < 5; ++D) {
      const int acc = D & 1, use = D >> 1;
      if (!mbar_wait(&accf[acc], (uint32_t)(use & 1), err)) {
        ok = false;
        break;
      }
      tc_fence_after();
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(acc * 64 + 32 * half), v);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[acc]);
      const int sh = 8 * (4 - D);
#pragma unroll
      for (int j = 0; j < 32; ++j) tot[j] += (long long)f2i_exact(v[j]) * (1LL << sh);
    }
    if (ok) {
      // all products are complete (the last diagonal's commit): the slices'
      // shared memory now stages the result
      const int m = 32 * quarter + lane;
      float* st = reinterpret_cast<float*>(stage + (size_t)m * 33);
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int Ec = ecol[j];
        float val = 0.f;
        if (Ec != 0 && tot[j] != 0) val = ldexpf(__ll2float_rn(tot[j]), (Ec - 126) - 48);
        st[2 * j + half] = val;
      }
    }
  }
  __syncthreads();
  if (ok) {
    for (int e = tid; e < kRtRows * kRtC2; e += kRtThreads) {
      const int rr = e % kRtRows, c = e / kRtRows;
      const int g = row0 + rr, gc = cols[c];
      if (g < rows && gc >= 0) Mrow[(size_t)g + (size_t)gc * ld] = stage[(size_t)rr * 33 + c];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 8) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kRtTmemCols));
  }
}

void rot_tc_prepare() {
  static bool done = false;
  if (done) return;
  cudaFuncSetAttribute(k_rot_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kRtSmem);
  done = true;
}

void launch_rot_tc(const GateTask* t, const TaskMeta* m, int ntask, int round, int pairs_ub, int mw_ub, int nw_ub,
                   int* err, cudaStream_t st) {
  rot_tc_prepare();
  const int mt_ub = (mw_ub + kRtRows - 1) / kRtRows + (nw_ub + kRtRows - 1) / kRtRows;
  k_rot_tc<<<dim3(pairs_ub * mt_ub, ntask), kRtThreads, kRtSmem, st>>>(t, m, round, mt_ub, err);
}

}  // namespace mpsgb

// Split-precision complex GEMM on the 5th-generation tensor cores (sm_103a):
// binary64-accurate C = A B from bf16 slice products accumulated in fp32
// (the Ozaki scheme: Ozaki, Ogita, Oishi, Rump, Numer. Algorithms 59, 2012;
// tensor-core form after Mukunoki et al., ISC 2020).
//
// Splitting. Each complex row r of A gets a power-of-two scale 2^{e_r} with
// max_k |Re A_rk|, |Im A_rk| < 2^{e_r}; each entry is cut (truncated toward
// zero) into s signed 7-bit digits, x = 2^{e_r} sum_{p=1..s} d_p 2^{-7p},
// |d_p| <= 127, with integer arithmetic on the binary64 bit pattern. The same
// for the columns of B (scales 2^{f_n}). A digit is exact in bf16.
// Complex to real: row 2r of A^ is [Re A_r, -Im A_r], row 2r+1 is
// [Im A_r, Re A_r]; row n of B^ (K-major) is [Re B_:n, Im B_:n]. Then
// (A^ B^T)[2r][n] = Re C_rn and [2r+1][n] = Im C_rn.
// Products. Every slice pair (p, q) with p + q <= s + 1 is one tcgen05.mma
// chain over K into its own fp32 TMEM accumulator. Each product of digits is
// below 2^14 and 2K <= 1024 terms keep every partial sum below 2^24, so the
// fp32 accumulation is exact; a longer K runs as 512-wide chunks whose
// binary64 results the epilogue accumulates. The epilogue folds the pair results into two
// 64-bit integers per output (diagonals p+q <= 5 and > 5, shifted), and
// converts them to binary64 once, with the scales 2^{e_r + f_n}.
// Pipeline. One CTA per 128 x 64 output tile of A^ B^T: warp 0 issues TMA
// loads (SWIZZLE_128B, 4 stages), warp 1 issues the MMAs (M = 128, K = 16
// per instruction, N = 64 per slice pair of a pass: up to four pairs in one
// instruction of N = 256) alternating between two TMEM accumulator sets,
// warps 2..9 drain a set while the next pass is being multiplied. Every
// wait is bounded (%globaltimer); a timeout sets an error flag and the CTA
// returns after releasing its TMEM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <cstring>

#include "engine.cuh"
#include "kernels.cuh"
#include "ozaki.cuh"
#include "tc_ptx.cuh"

namespace mpsgb {

// --------------------------------------------------------------- splitting ---

__device__ __forceinline__ double2 oz_elem(const OzView& v, int r, int k) {
  const long long ro = v.rb ? (long long)(r / v.rb) * v.s_rb + (long long)(r % v.rb) * v.s_r : (long long)r * v.s_r;
  const long long ko = v.kb ? (long long)(k / v.kb) * v.s_kb + (long long)(k % v.kb) * v.s_k : (long long)k * v.s_k;
  double2 x = v.p[ro + ko];
  double sc = 1.0;
  if (v.rscale) sc *= v.rscale[v.rb ? r % v.rb : r];
  if (v.kscale) sc *= v.kscale[v.kb ? k % v.kb : k];
  x.x *= sc;
  x.y *= v.conj ? -sc : sc;
  return x;
}

// Exponent e with |x| < 2^e for every x whose magnitude is at most mx (e = 0 for mx = 0).
__device__ __forceinline__ int oz_exponent(double mx) {
  if (!(mx > 0.0)) return 0;
  const long long b = __double_as_longlong(mx);
  const int E = (int)((b >> 52) & 0x7FF);
  if (E == 0) return -1022;  // subnormal maximum: scale as the smallest normal
  return E - 1022;           // mx < 2^{E-1023+1}
}

// Digits of x relative to 2^e: x ~ 2^e sum_{p=1..s} d_p 2^{-7p} (truncation toward zero).
__device__ __forceinline__ void oz_digits(double x, int e, int s, int* d) {
  const long long b = __double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  long long X = 0;
  if (E != 0) {
    const long long m = (b & 0x000FFFFFFFFFFFFFLL) | 0x0010000000000000LL;
    const int sh = E - 1019 - e;  // X = |x| 2^{56-e} = m 2^{E-1075+56-e}
    if (sh >= 0) X = m << sh;     // sh <= 3 because |x| < 2^e
    else if (sh > -64) X = m >> (-sh);
  }
  const bool neg = b < 0;
#pragma unroll
  for (int p = 1; p <= 8; ++p) {
    int v = (int)((X >> (56 - 7 * p)) & 127);
    d[p - 1] = p <= s ? (neg ? -v : v) : 0;
  }
}

// One warp per complex row of the view: scale, digits, K-padding zeros.
// Writes rows 2r and 2r+1 of every slice of A^ ([slice][Mp][Kp] bf16).
// mode 0: A operand (row 2r = [Re, -Im], 2r+1 = [Im, Re]);
// mode 1: B operand (row r = [Re, Im]).
__global__ void __launch_bounds__(256) k_oz_split(const OzJob* jobs, int which, __nv_bfloat16* out, int* expo,
                                                  int Mp, int Kp, int s, int k0, int kchunk, int kcap) {
  const OzJob& jb = jobs[blockIdx.y];
  const OzView& v = which == 0 ? jb.a : jb.b;
  const int R = which == 0 ? jb.M : jb.N;
  const int K = max(0, min(jb.K - k0, kchunk));  // this chunk of the inner dimension
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x >> 5) + warp;
  const int rows_out = which == 0 ? 2 : 1;
  const int rows_cap = which == 0 ? Mp / 2 : Mp;
  if (r >= rows_cap) return;
  const size_t slice_stride = (size_t)Mp * Kp;
  __nv_bfloat16* base = out + (size_t)blockIdx.y * s * slice_stride;
  const int kpad = (2 * K + 63) & ~63;
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f);
  if (r >= R) {  // rows beyond R only feed outputs that are never written
    if (lane == 0) expo[(size_t)blockIdx.y * rows_cap + r] = 0;
    return;
  }
  // the row is read once, into this warp's part of shared memory (loads
  // unrolled so that several are in flight), then cut into digits from there
  extern __shared__ double2 oz_rows[];
  double2* row = oz_rows + (size_t)warp * kcap;  // K <= kcap
  double mx = 0.0;
#pragma unroll 4
  for (int k = lane; k < K; k += 32) {
    const double2 x = oz_elem(v, r, k0 + k);
    row[k] = x;
    mx = fmax(mx, fmax(fabs(x.x), fabs(x.y)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __syncwarp();
  const int e = oz_exponent(mx);
  if (lane == 0) expo[(size_t)blockIdx.y * rows_cap + r] = e;
  if ((K & 1) == 0) {
    // two consecutive k per lane: every slice row gets 4-byte bf16-pair stores
    // (both halves start at even offsets because K is even)
    for (int k = 2 * lane; k < K; k += 64) {
      const double2 x0 = row[k], x1 = row[k + 1];
      int r0[8], i0[8], r1[8], i1[8];
      oz_digits(x0.x, e, s, r0);
      oz_digits(x0.y, e, s, i0);
      oz_digits(x1.x, e, s, r1);
      oz_digits(x1.y, e, s, i1);
#pragma unroll
      for (int p = 0; p < 8; ++p) {  // unrolled: the digit arrays stay in registers
        if (p >= s) break;
        __nv_bfloat162* sl = reinterpret_cast<__nv_bfloat162*>(base + p * slice_stride);
        const __nv_bfloat162 re = __floats2bfloat162_rn((float)r0[p], (float)r1[p]);
        const __nv_bfloat162 im = __floats2bfloat162_rn((float)i0[p], (float)i1[p]);
        if (which == 0) {
          const __nv_bfloat162 nim = __floats2bfloat162_rn((float)(-i0[p]), (float)(-i1[p]));
          sl[((size_t)(2 * r) * Kp + k) / 2] = re;
          sl[((size_t)(2 * r) * Kp + K + k) / 2] = nim;
          sl[((size_t)(2 * r + 1) * Kp + k) / 2] = im;
          sl[((size_t)(2 * r + 1) * Kp + K + k) / 2] = re;
        } else {
          sl[((size_t)r * Kp + k) / 2] = re;
          sl[((size_t)r * Kp + K + k) / 2] = im;
        }
      }
    }
  } else {
    for (int k = lane; k < K; k += 32) {
      const double2 x = row[k];
      int dre[8], dim[8];
      oz_digits(x.x, e, s, dre);
      oz_digits(x.y, e, s, dim);
#pragma unroll
      for (int p = 0; p < 8; ++p) {
        if (p >= s) break;
        __nv_bfloat16* sl = base + p * slice_stride;
        if (which == 0) {
          sl[(size_t)(2 * r) * Kp + k] = __float2bfloat16_rn((float)dre[p]);
          sl[(size_t)(2 * r) * Kp + K + k] = __float2bfloat16_rn((float)(-dim[p]));
          sl[(size_t)(2 * r + 1) * Kp + k] = __float2bfloat16_rn((float)dim[p]);
          sl[(size_t)(2 * r + 1) * Kp + K + k] = __float2bfloat16_rn((float)dre[p]);
        } else {
          sl[(size_t)r * Kp + k] = __float2bfloat16_rn((float)dre[p]);
          sl[(size_t)r * Kp + K + k] = __float2bfloat16_rn((float)dim[p]);
        }
      }
    }
  }
  for (int c = 2 * K + lane; c < kpad; c += 32)
    for (int p = 0; p < s; ++p)
      for (int ro = 0; ro < rows_out; ++ro) base[p * slice_stride + (size_t)(rows_out * r + ro) * Kp + c] = zero;
}

// ------------------------------------------------------------------- GEMM ---

constexpr int kOzM = 128, kOzN = 64, kOzK = 64, kOzStages = 4;
constexpr int kOzQ = 4;  // B slices that share one A-slice tile in a pass
constexpr int kOzABytes = kOzM * kOzK * 2, kOzBBytes = kOzN * kOzK * 2;
constexpr int kOzStageBytes = kOzABytes + kOzQ * kOzBBytes;  // 48 KB
constexpr int kOzThreads = 320;  // 10 warps
constexpr int kOzSmem = kOzStages * kOzStageBytes + 1024 /*align*/ + 256 /*barriers*/;
constexpr int kOzTmemCols = 512;  // two sets of kOzQ 64-column fp32 accumulators

// The slice pairs (p, q), p + q < s, are taken in passes: pass (p, q0) runs
// the pairs (p, q0 .. q0 + nq - 1), nq <= kOzQ, so that each k-tile of A's
// slice p is loaded once for nq products (every pair in its own
// accumulator, which keeps each fp32 sum exact). The passes alternate
// between two accumulator sets, so that the epilogue drains one pass while
// the tensor cores run the next.
__device__ __forceinline__ bool oz_next_pass(int s, int& p, int& q0, int& nq) {
  q0 += kOzQ;
  if (q0 >= s - p) {
    ++p;
    q0 = 0;
  }
  if (p >= s) return false;
  nq = min(kOzQ, s - p - q0);
  return true;
}

__global__ void __launch_bounds__(kOzThreads, 1)
    k_oz_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const OzJob* jobs,
              const int* ea, const int* fb, int MpA, int NpB, int s, int* err, int k0, int kchunk) {
  extern __shared__ __align__(1024) unsigned char oz_smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)oz_smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + kOzStages * kOzStageBytes);
  uint64_t* full = bars;                 // [stages]
  uint64_t* empty = bars + kOzStages;    // [stages]
  uint64_t* accf = bars + 2 * kOzStages; // [2]
  uint64_t* acce = accf + 2;             // [2]
  uint32_t* tmem_slot = (uint32_t*)(acce + 2);

  const OzJob& jb = jobs[blockIdx.z];
  const int m0 = blockIdx.y * kOzM;  // rows of A^ (2 per complex row)
  const int n0 = blockIdx.x * kOzN;
  const int Kc = min(jb.K - k0, kchunk);  // this chunk of the inner dimension
  if (m0 >= 2 * jb.M || n0 >= jb.N || Kc <= 0) return;  // uniform across the CTA
  // Hermitian product: the 64 x 64 complex tiles below the diagonal are
  // written by their mirror tiles (128 rows of A^ are 64 complex rows)
  if (jb.herm && blockIdx.y > blockIdx.x) return;
  const bool mirror = jb.herm && blockIdx.y < blockIdx.x;
  const int KT = (2 * Kc + kOzK - 1) / kOzK;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kOzStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&accf[i], 1);
      mbar_init(&acce[i], 8);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kOzTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {  // ---------------------------------------------- TMA producer
      int it = 0;
      int p = 0, q0 = -kOzQ, nq = 0;
      while (oz_next_pass(s, p, q0, nq))
        for (int kt = 0; kt < KT; ++kt, ++it) {
          const int st = it % kOzStages;
          const uint32_t ph = (uint32_t)(it / kOzStages) & 1u;
          if (!mbar_wait(&empty[st], ph ^ 1u, err)) goto producer_done;
          unsigned char* sa = smem + st * kOzStageBytes;
          mbar_expect_tx(&full[st], kOzABytes + nq * kOzBBytes);
          tma_load_4d(sa, &tmA, &full[st], kt * kOzK, m0, p, blockIdx.z);
          for (int qi = 0; qi < nq; ++qi)
            tma_load_4d(sa + kOzABytes + qi * kOzBBytes, &tmB, &full[st], kt * kOzK, n0, q0 + qi, blockIdx.z);
        }
    producer_done:;
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ---------------------------------------------- MMA issuer
      int it = 0, pi = 0;
      int p = 0, q0 = -kOzQ, nq = 0;
      while (oz_next_pass(s, p, q0, nq)) {
        const int acc = pi & 1;
        const uint32_t use = (uint32_t)(pi >> 1);
        if (!mbar_wait(&acce[acc], (use & 1u) ^ 1u, err)) goto mma_done;
        tc_fence_after();
        const uint32_t dset = tmem + (uint32_t)(acc * kOzQ * kOzN);
        // the pass's nq B tiles lie back to back in the stage (64 rows of
        // 128 bytes each, 8-row groups 1024 bytes apart), which is one
        // K-major operand of nq * 64 rows: a single MMA of N = nq * 64 writes
        // every pair's product into its own 64 accumulator columns
        const uint32_t idesc = idesc_bf16_f32(kOzM, nq * kOzN);
        for (int kt = 0; kt < KT; ++kt, ++it) {
          const int st = it % kOzStages;
          const uint32_t ph = (uint32_t)(it / kOzStages) & 1u;
          if (!mbar_wait(&full[st], ph, err)) goto mma_done;
          tc_fence_after();
          unsigned char* sa = smem + st * kOzStageBytes;
          const uint64_t da = smem_desc_sw128(sa);
          const uint64_t db = smem_desc_sw128(sa + kOzABytes);
#pragma unroll
          for (int kk = 0; kk < kOzK / 16; ++kk)
            mma_bf16(dset, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc, (kt | kk) != 0);
          mma_commit(&empty[st]);
        }
        mma_commit(&accf[acc]);
        ++pi;
      }
    mma_done:;
    }
  } else {  // ----------------------------------------------------------- epilogue
    const int quarter = warp & 3;
    const int chalf = (warp - 2) >> 2;  // 0 or 1: columns [32 chalf, 32 chalf + 32)
    const int dh = s < 5 ? s + 1 : 5;   // diagonals d = p+q (1-based) <= dh go to the high word
    long long hi[32], lo[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      hi[j] = 0;
      lo[j] = 0;
    }
    bool ok = true;
    int pi = 0;
    int p = 0, q0 = -kOzQ, nq = 0;
    while (ok && oz_next_pass(s, p, q0, nq)) {
      const int acc = pi & 1;
      const uint32_t use = (uint32_t)(pi >> 1);
      if (!mbar_wait(&accf[acc], use & 1u, err)) {
        ok = false;
        break;
      }
      tc_fence_after();
      for (int qi = 0; qi < nq; ++qi) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * quarter) << 16) +
                      (uint32_t)(acc * kOzQ * kOzN + qi * kOzN + 32 * chalf), v);
        const int d = p + q0 + qi + 2;
        if (d <= dh) {
          const int sh = 7 * (dh - d);
#pragma unroll
          for (int j = 0; j < 32; ++j) hi[j] += (long long)f2i_exact(v[j]) * (1LL << sh);
        } else {
          const int sh = 7 * (s + 1 - d);
#pragma unroll
          for (int j = 0; j < 32; ++j) lo[j] += (long long)f2i_exact(v[j]) * (1LL << sh);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[acc]);
      ++pi;
    }
    if (ok) {
      const int m = m0 + 32 * quarter + lane;  // row of A^
      if (m < 2 * jb.M) {
        const int r = m >> 1, part = m & 1;
        const int er = ea[(size_t)blockIdx.z * (MpA / 2) + r];
        double* C = reinterpret_cast<double*>(jb.C);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int n = n0 + 32 * chalf + j;
          if (n < jb.N) {
            const int e = er + fb[(size_t)blockIdx.z * NpB + n];
            const double val = ldexp((double)hi[j], e - 7 * dh) + ldexp((double)lo[j], e - 7 * (s + 1));
            double* c = &C[2 * ((size_t)r + (size_t)n * jb.ldc) + part];
            *c = k0 > 0 ? *c + jb.alpha * val : jb.alpha * val;  // later K chunks accumulate
            if (mirror) {  // C[n][r] = conj(C[r][n])
              const double mv = part ? -val : val;
              double* cm = &C[2 * ((size_t)n + (size_t)r * jb.ldc) + part];
              *cm = k0 > 0 ? *cm + jb.alpha * mv : jb.alpha * mv;
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kOzTmemCols));
  }
}

// ------------------------------------------------------------ host side ---

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

static int encode_fn() {
  if (g_encode) return 0;
  cudaDriverEntryPointQueryResult q;
  void* fn = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn)
    return -1;
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return 0;
}

// 4-D map over [jobs][slices][rows][Kp] bf16 with a (64 x box_rows) box.
static int make_map(CUtensorMap* map, const __nv_bfloat16* base, int Kp, int rows, int s, int jobs, int box_rows) {
  if (encode_fn()) return -1;
  cuuint64_t dims[4] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)s, (cuuint64_t)jobs};
  cuuint64_t strides[3] = {(cuuint64_t)Kp * 2, (cuuint64_t)Kp * rows * 2, (cuuint64_t)Kp * rows * s * 2};
  cuuint32_t box[4] = {(cuuint32_t)kOzK, (cuuint32_t)box_rows, 1, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16*>(base), dims, strides, box,
                        estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -1;
}

static inline int rup(int a, int b) { return (a + b - 1) / b * b; }

// One-time set-up (the kernel's shared-memory attribute, the tensor-map
// encoder): done before a program records launches into a graph.
int ozaki_prepare() {
  static bool done = false;
  if (done) return 0;
  if (encode_fn()) return -1;
  if (cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, kOzSmem) != cudaSuccess) return -1;
  if (cudaFuncSetAttribute(k_oz_split, cudaFuncAttributeMaxDynamicSharedMemorySize, 8 * 512 * (int)sizeof(double2)) !=
      cudaSuccess)
    return -1;
  done = true;
  return 0;
}

size_t OzBuffers::bytes_needed(int jobs, int M_ub, int N_ub, int K_ub, int s) {
  const size_t Mp = rup(2 * M_ub, kOzM), Np = rup(N_ub, kOzN), Kp = rup(2 * K_ub, kOzK);
  return (size_t)jobs * s * (Mp + Np) * Kp * 2 + (size_t)jobs * (Mp / 2 + Np) * sizeof(int) + 4096;
}

int ozaki_zgemm(const OzJob* d_jobs, int njobs, int M_ub, int N_ub, int K_ub, int s, OzBuffers& buf, int* d_err,
                cudaStream_t st) {
  if (njobs <= 0) return 0;
  if (s < 1 || s > 8 || K_ub < 1) return -1;
  // exact fp32 accumulation needs 2K <= 1024: longer K in chunks of 512,
  // summed in binary64 by the epilogue
  const int kchunk = 512;
  const int Kc_ub = K_ub < kchunk ? K_ub : kchunk;
  const int Mp = rup(2 * M_ub, kOzM), Np = rup(N_ub, kOzN), Kp = rup(2 * Kc_ub, kOzK);
  const size_t need = OzBuffers::bytes_needed(njobs, M_ub, N_ub, Kc_ub, s);
  if (need > buf.bytes) {
    cudaFree(buf.base);
    buf.base = nullptr;
    buf.bytes = 0;
    if (dev_alloc((void**)&buf.base, need) != cudaSuccess) return -2;
    buf.bytes = need;
  }
  unsigned char* p = static_cast<unsigned char*>(buf.base);
  __nv_bfloat16* Ah = reinterpret_cast<__nv_bfloat16*>(p);
  p += (size_t)njobs * s * Mp * Kp * 2;
  __nv_bfloat16* Bh = reinterpret_cast<__nv_bfloat16*>(p);
  p += (size_t)njobs * s * Np * Kp * 2;
  int* ea = reinterpret_cast<int*>(p);
  p += (size_t)njobs * (Mp / 2) * sizeof(int);
  int* fb = reinterpret_cast<int*>(p);
  CUtensorMap mA, mB;
  if (make_map(&mA, Ah, Kp, Mp, s, njobs, kOzM) || make_map(&mB, Bh, Kp, Np, s, njobs, kOzN)) return -3;
  if (ozaki_prepare()) return -4;
  for (int k0 = 0; k0 < K_ub; k0 += kchunk) {
    const size_t rows_smem = (size_t)8 * Kc_ub * sizeof(double2);  // one row of K <= Kc_ub per warp
    k_oz_split<<<dim3((Mp / 2 + 7) / 8, njobs), 256, rows_smem, st>>>(d_jobs, 0, Ah, ea, Mp, Kp, s, k0, kchunk,
                                                                       Kc_ub);
    k_oz_split<<<dim3((Np + 7) / 8, njobs), 256, rows_smem, st>>>(d_jobs, 1, Bh, fb, Np, Kp, s, k0, kchunk, Kc_ub);
    k_oz_gemm<<<dim3(Np / kOzN, Mp / kOzM, njobs), kOzThreads, kOzSmem, st>>>(mA, mB, d_jobs, ea, fb, Mp, Np, s, d_err,
                                                                             k0, kchunk);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -5;
}

}  // namespace mpsgb

// mps_split_zgemm: the split-precision complex GEMM as a C entry point
// (device operands, column-major), the building block of MPS_PREC_SPLIT.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/mps.h"
#include "engine.cuh"
#include "kernels.cuh"
#include "ozaki.cuh"
#include "tc_ptx.cuh"

using namespace mpsgb;

namespace {
std::mutex g_mu;
OzBuffers g_buf;
OzJob* g_job = nullptr;
int* g_err = nullptr;
// Set once a bounded wait ran out: products may have been abandoned in flight,
// so the device state is not trusted and later calls are refused.
bool g_timed_out = false;

int fail_msg(int code, const char* msg) {
  set_error_message(msg);
  return code;
}
}  // namespace

extern "C" int mps_split_zgemm(int M, int N, int K, const double* dA, long long lda, const double* dB, long long ldb,
                               double* dC, long long ldc, int slices, void* stream) {
  if (!dA || !dB || !dC) return fail_msg(MPS_ERR_ARG, "NULL pointer");
  if (M < 1 || N < 1 || K < 1) return fail_msg(MPS_ERR_ARG, "sizes must be >= 1");
  if (slices < 1 || slices > 8) return fail_msg(MPS_ERR_ARG, "slices must be 1..8");
  if (lda < M || ldb < K || ldc < M) return fail_msg(MPS_ERR_ARG, "leading dimension too small");
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_timed_out) return fail_msg(MPS_ERR_TIMEOUT, "an earlier split GEMM timed out; the device state is not trusted");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!g_job) {
    if (dev_alloc((void**)&g_job, sizeof(OzJob)) != cudaSuccess || dev_alloc((void**)&g_err, sizeof(int)) != cudaSuccess)
      return fail_msg(MPS_ERR_NOMEM, "job table");
  }
  OzJob j = {};
  j.a.p = reinterpret_cast<const double2*>(dA);
  j.a.s_r = 1;
  j.a.s_k = lda;
  j.b.p = reinterpret_cast<const double2*>(dB);
  j.b.s_r = ldb;  // view (n, k) = B[k + n ldb]
  j.b.s_k = 1;
  j.M = M;
  j.N = N;
  j.K = K;
  j.C = reinterpret_cast<double2*>(dC);
  j.ldc = ldc;
  j.alpha = 1.0;
  if (cudaMemcpyAsync(g_job, &j, sizeof(j), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(g_err, 0, sizeof(int), st) != cudaSuccess)
    return fail_msg(MPS_ERR_CUDA, "job upload");
  const int rc = ozaki_zgemm(g_job, 1, M, N, K, slices, g_buf, g_err, st);
  if (rc == -2) return fail_msg(MPS_ERR_NOMEM, "slice buffers");
  if (rc) return fail_msg(MPS_ERR_CUDA, "split GEMM launch failed");
  int err = 0;
  if (cudaMemcpyAsync(&err, g_err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail_msg(MPS_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
  if (err) {
    g_timed_out = true;
    return fail_msg(MPS_ERR_TIMEOUT, "split GEMM: a bounded wait ran out; the device state is not trusted");
  }
  return MPS_OK;
}

// ---- test hook: the bounded wait of the tensor-core kernels, made to run out

namespace {

// One warp initialises an mbarrier that expects one arrival and then waits
// for its first phase, which nothing completes: the wait gives up after
// limit_ns, sets *err and the kernel returns. No copy or MMA is in flight,
// so the context stays usable.
__global__ void k_wait_unset_barrier(int* err, unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (threadIdx.x == 0) mbar_wait_for(&bar, 0u, err, limit_ns);
}

}  // namespace

extern "C" int mps_debug_bounded_wait(double limit_ms, void* stream) {
  if (!(limit_ms > 0.0) || limit_ms > 10000.0) return fail_msg(MPS_ERR_ARG, "limit_ms must be in (0, 10000]");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int* d_err = nullptr;
  cudaError_t e = dev_alloc((void**)&d_err, sizeof(int));
  if (e != cudaSuccess) return fail_msg(MPS_ERR_NOMEM, "mps_debug_bounded_wait: flag allocation");
  int h_err = 0;
  e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    k_wait_unset_barrier<<<1, 32, 0, st>>>(d_err, (unsigned long long)(limit_ms * 1e6));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d_err);
  if (e != cudaSuccess) return fail_msg(MPS_ERR_CUDA, cudaGetErrorString(e));
  if (h_err) return fail_msg(MPS_ERR_TIMEOUT, "mps_debug_bounded_wait: the bounded wait ran out (as intended)");
  return MPS_OK;
}

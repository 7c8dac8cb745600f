// mps_gate2_update_noalloc: the two-site gate update on caller-owned device
// tensors, for callers that must not allocate device memory. Some host
// programs reserve the whole device memory budget up front (a caching
// allocator that already holds the GPU's memory, or a fixed-footprint
// service), and others run loops that must not block: cudaMalloc and cudaFree
// can fail there, or stall the whole device while they synchronise. This
// entry point calls neither, nor any allocating library routine: its working
// storage is the file-scope device array below, reserved once per device when
// the library is loaded and held until the process exits.
//
// The update is the same kernel sequence as mps_apply_gate (theta
// contraction, blocked one-sided Jacobi SVD, truncation, rewrite); only the
// scratch comes from the static array instead of the handle's workspace.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/mps.h"
#include "engine.cuh"
#include "kernels.cuh"

using namespace mpsgb;

namespace {

constexpr int kNaCap = 64;  // largest chi_max accepted (theta at most 128 x 128)

// Byte offsets inside the scratch array (each 256-byte aligned).
constexpr size_t kOffA = 0;
constexpr size_t kSzA = sizeof(double2) * 4 * kNaCap * kNaCap;  // working matrix, (2 cap)^2
constexpr size_t kOffV = kOffA + kSzA;
constexpr size_t kSzV = sizeof(double2) * 4 * kNaCap * kNaCap;  // right rotations, (2 cap)^2
constexpr size_t kOffSig = kOffV + kSzV;
constexpr size_t kSzSig = sizeof(double) * 2 * kNaCap;
constexpr size_t kOffPerm = kOffSig + kSzSig;
constexpr size_t kSzPerm = sizeof(int) * 2 * kNaCap;
constexpr size_t kOffU = kOffPerm + kSzPerm;
constexpr size_t kSzU = 256 * ((sizeof(double2) * 16 + 255) / 256);
constexpr size_t kOffTask = kOffU + kSzU;
constexpr size_t kSzTask = 256 * ((sizeof(GateTask) + 255) / 256);
constexpr size_t kOffMeta = kOffTask + kSzTask;
constexpr size_t kSzMeta = 256 * ((sizeof(TaskMeta) + 255) / 256);
constexpr size_t kOffCnt = kOffMeta + kSzMeta;
constexpr size_t kScratchBytes = kOffCnt + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_addr[kMaxDevices] = {nullptr};

int fail_msg(int code, const char* msg) {
  set_error_message(msg);
  return code;
}

// A failed CUDA call: MPS_ERR_CUDA with the step and the runtime's message.
int fail_cuda(const char* step, cudaError_t e = cudaGetLastError()) {
  static thread_local char buf[256];
  snprintf(buf, sizeof(buf), "mps_gate2_update_noalloc: %s: %s", step, cudaGetErrorString(e));
  return fail_msg(MPS_ERR_CUDA, buf);
}

struct Gate4 {
  double2 u[16];
};

// Writes the task table, the gate and zeroed counters into the scratch array.
__global__ void k_noalloc_put(GateTask* dst, GateTask t, double2* du, Gate4 g, int* cnt) {
  if (threadIdx.x == 0) *dst = t;
  if (threadIdx.x < 16) du[threadIdx.x] = g.u[threadIdx.x];
  if (threadIdx.x < 2) cnt[threadIdx.x] = 0;
}

// Device address of this device's scratch array; the first call on a device
// looks it up (cudaGetSymbolAddress with that device current).
cudaError_t scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int mps_gate2_update_noalloc(double* d_gamma_l, double* d_gamma_r, const double* d_lambda_l,
                                        double* d_lambda_m, const double* d_lambda_r, int* d_chi, int chi_max,
                                        double cutoff, const double* U, void* stream) {
  if (!d_gamma_l || !d_gamma_r || !d_lambda_l || !d_lambda_m || !d_lambda_r || !d_chi || !U)
    return fail_msg(MPS_ERR_ARG, "NULL pointer");
  if (chi_max < 1) return fail_msg(MPS_ERR_ARG, "chi_max must be >= 1");
  if (chi_max > kNaCap) return fail_msg(MPS_ERR_TOO_LARGE, "chi_max above the no-allocation limit of 64");
  if (!(cutoff >= 0.0)) return fail_msg(MPS_ERR_ARG, "cutoff must be >= 0");
  unsigned char* base = nullptr;
  const cudaError_t se = scratch_for_current_device(&base);
  if (se != cudaSuccess) return fail_cuda("looking up the scratch array", se);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the bond dimensions live on the device: read the three ints (no allocation)
  int chi_h[3] = {0, 0, 0};
  if (cudaMemcpyAsync(chi_h, d_chi, sizeof(chi_h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail_cuda("reading the bond dimensions");
  for (int i = 0; i < 3; ++i)
    if (chi_h[i] < 1 || chi_h[i] > chi_max) return fail_msg(MPS_ERR_ARG, "bond dimensions outside [1, chi_max]");

  GateTask* d_task = reinterpret_cast<GateTask*>(base + kOffTask);
  TaskMeta* d_meta = reinterpret_cast<TaskMeta*>(base + kOffMeta);
  int* d_cnt = reinterpret_cast<int*>(base + kOffCnt);
  double2* d_u = reinterpret_cast<double2*>(base + kOffU);

  GateTask t = {};
  t.g0 = reinterpret_cast<double2*>(d_gamma_l);
  t.g1 = reinterpret_cast<double2*>(d_gamma_r);
  t.g2 = nullptr;
  t.lamL = const_cast<double*>(d_lambda_l);
  t.lam0 = d_lambda_m;
  t.lam1 = const_cast<double*>(d_lambda_r);
  t.lamR = const_cast<double*>(d_lambda_r);
  t.chi = d_chi;  // [chi_left, chi_mid, chi_right]; chi_mid is rewritten
  t.U = d_u;
  t.site = 0;
  t.k = 2;
  t.cap = chi_max;
  t.cutoff = cutoff;
  t.A = reinterpret_cast<double2*>(base + kOffA);
  t.V = reinterpret_cast<double2*>(base + kOffV);
  t.T = nullptr;
  t.sigma = reinterpret_cast<double*>(base + kOffSig);
  t.perm = reinterpret_cast<int*>(base + kOffPerm);
  Gate4 g;
  for (int e = 0; e < 16; ++e) g.u[e] = make_double2(U[2 * e], U[2 * e + 1]);

  k_noalloc_put<<<1, 32, 0, st>>>(d_task, t, d_u, g, d_cnt);
  launch_setup(d_task, d_meta, 1, 0, st);
  launch_contract2(d_task, d_meta, 1, chi_max, chi_max, st);
  launch_frob(d_task, d_meta, 1, 4LL * chi_max * chi_max, 0, st);
  const int nw_ub = 2 * chi_max;
  launch_init_V(d_task, d_meta, 1, nw_ub, st);
  const int nb = (nw_ub + kBlockW - 1) / kBlockW;
  const int nbe = nb + (nb & 1);
  for (int sw = 0; sw < kMaxSweeps; ++sw) {
    for (int r = 0; r < nbe - 1; ++r) launch_jacobi_round(d_task, d_meta, 1, r, nbe / 2, 0, nullptr, st);
    if (cudaMemsetAsync(d_cnt, 0, sizeof(int), st) != cudaSuccess) return fail_cuda("clearing the sweep counter");
    launch_sweep_end(d_meta, 1, kMaxSweeps, d_cnt, st);
    int active = 0;
    if (cudaMemcpyAsync(&active, d_cnt, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return fail_cuda("reading the sweep counter");
    if (active == 0) break;
  }
  launch_colnorms(d_task, d_meta, 1, nw_ub, 0, st);
  launch_truncate(d_task, d_meta, 1, 0, chi_max, st);
  launch_emit_left(d_task, d_meta, 1, chi_max, chi_max, 0, st);
  launch_emit_right(d_task, d_meta, 1, chi_max, chi_max, 0, st);
  const cudaError_t le = cudaGetLastError();
  if (le != cudaSuccess) return fail_cuda("a kernel launch", le);
  int status = 0;
  if (cudaMemcpyAsync(&status, d_cnt + 1, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail_cuda("reading the status word");
  if (status != 0) return fail_msg(status, "Jacobi SVD did not converge (tensors left unchanged)");
  return MPS_OK;
}

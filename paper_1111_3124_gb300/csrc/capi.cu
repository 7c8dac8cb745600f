// C ABI (include/mps.h) and host orchestration of the gate-update engine.
//
// A handle owns the Vidal-form tensors of one MPS in device memory (layout
// in engine.cuh), a per-gate workspace that grows with the widest layer seen,
// pinned staging buffers for gates and task tables, and a CUDA stream.
// Bond dimensions live on the device; the host keeps upper bounds
// (ub[b+1] >= chi of bond b) to size grids. Within a pass the only
// device-to-host reads are the one-int convergence count after each Jacobi
// sweep and the task metadata after the truncation, which makes the bounds
// of the rewritten bonds exact.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mps.h"
#include "engine.cuh"
#include "kernels.cuh"
#include "mlp.cuh"
#include "ozaki.cuh"
#include "sketch.cuh"

using namespace mpsgb;
typedef std::complex<double> cd;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(e_ == cudaErrorMemoryAllocation ? MPS_ERR_NOMEM : MPS_ERR_CUDA,             \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                        \
  } while (0)

constexpr int kProfKinds = 6;  // see mps_profile in include/mps.h
constexpr int kSplitMaxCap = kMaxCap;  // the split GEMM chunks K beyond 512
constexpr int kF32Sweeps = 30;
constexpr int kGramSteps = 3;  // simultaneous-rotation steps of the split path's Gram polish
// How the fp32 sweeps are launched (mps_set_tuning): one launch per round with
// the rotation in the pair kernel, or on the tensor cores; or every sweep in
// one scheduled launch of 256-thread CTAs (the default), or of 384-thread CTAs.
constexpr int kF32ModePair = 0, kF32ModeTc = 1, kF32ModeSched = 2, kF32ModeSchedWide = 3;

// Memory budget of one batched pass: the tasks of a layer (or of many
// circuits' layers) are processed in chunks whose workspace fits this.
constexpr size_t kArenaBudget = (size_t)48 << 30;
constexpr int kMaxTasksPerPass = 4096;

}  // namespace

void mpsgb::set_error_message(const char* msg) { g_err = msg; }

namespace {
// mps_debug_fail_alloc: allocations that still succeed before one is refused
// (-1: the hook is off).
std::atomic<long long> g_alloc_left{-1};

bool alloc_refused() {
  long long left = g_alloc_left.load();
  while (left >= 0) {
    if (left == 0) return true;
    if (g_alloc_left.compare_exchange_weak(left, left - 1)) return false;
  }
  return false;
}
}  // namespace

cudaError_t mpsgb::dev_alloc(void** p, size_t bytes) {
  if (alloc_refused()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

cudaError_t mpsgb::host_alloc(void** p, size_t bytes) {
  if (alloc_refused()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocHost(p, bytes);
}

struct mps_state {
  int n = 0, cap = 0;
  double cutoff = 0.0;
  int prec = MPS_PREC_FP64, slices = 8, svd_mode = 0;
  int max_sweeps = kMaxSweeps;  // binary64 Jacobi sweep limit (mps_set_limits)
  // per working-matrix width: fp32 block width and launch mode (mps_set_tuning);
  // empty: block width 16, all sweeps in one scheduled launch of 256-thread CTAs
  struct Tune {
    int nw_max, f32_block, mode;  // mode: how the fp32 sweeps are launched (kF32Mode*)
  };
  std::vector<Tune> tune;
  // recording a program (mps_program_create): launches go into a CUDA graph,
  // no host synchronisation, loops become conditional nodes captured on `side`
  int capturing = 0;
  cudaStream_t side = nullptr;
  cudaStream_t own = nullptr, stream = nullptr;
  double2* gamma = nullptr;
  double* lambda = nullptr;
  int* chi = nullptr;
  std::vector<int> ub;                      // n+1 upper bounds of chi
  std::vector<std::array<cd, 4>> pend;      // held-back single-qubit gates
  std::vector<char> has_pend;
  void* arena = nullptr;  // per-task workspace, laid out per pass from the tasks' dimension bounds
  size_t arena_bytes = 0;
  GateTask* d_tasks = nullptr;
  TaskMeta* d_meta = nullptr;
  double2* d_gates = nullptr;
  int task_cap = 0;
  GateTask* h_tasks = nullptr;               // pinned
  double2* h_gates = nullptr;                // pinned
  int* d_counter = nullptr;
  int* h_counter = nullptr;                  // pinned
  SiteTask* d_site = nullptr;
  SiteTask* h_site = nullptr;                // pinned
  double2* d_site_gates = nullptr;
  double2* h_site_gates = nullptr;           // pinned
  int last_ntask = 0;
  int last_k = 0;
  // per-kernel-class profiling (mps_profile)
  int prof = 0;
  std::vector<cudaEvent_t> evs;
  size_t ev_next = 0;
  std::vector<std::array<int, 3>> prof_rec;  // (class, begin event, end event)
  double prof_flops_host[kProfKinds] = {0, 0, 0, 0, 0, 0};
  long long prof_launch[kProfKinds] = {0, 0, 0, 0, 0, 0};
  long long launches_all = 0;
  unsigned long long* d_prof_flops = nullptr;  // device counters, one per class
  // learned rank predictor / sketch SVD
  mps_mlp* predictor = nullptr;
  long long sk_sketched = 0, sk_accepted = 0, sk_routed = 0;
  unsigned long long sk_seed = 0x243F6A8885A308D3ull;
  void* sk_arena = nullptr;  // sketch buffers, laid out per pass
  size_t sk_bytes = 0;
  // split precision
  OzJob* d_oz_jobs = nullptr;
  int oz_cap = 0;
  OzBuffers oz_buf;
  int* d_oz_err = nullptr;
  // A bounded wait of the split GEMM ran out: asynchronous copies or tensor-core
  // products may have been abandoned in flight, so the handle's device state is
  // no longer trusted and every later split-precision product is refused.
  int oz_timed_out = 0;
  // readout workspace (reduced densities, expectations)
  double2* ro_buf = nullptr;
  size_t ro_bytes = 0;
};

// A recorded circuit (mps_program_create): passes of gate updates over one or
// more MPS, replayed as one CUDA graph. The program owns copies of the gates,
// the task tables of every pass, and a workspace (arena, split-GEMM buffers)
// sized for its largest pass.
struct mps_program {
  struct Chunk {
    int k = 0;
    std::vector<int> owner, site;  // the pass's gates: handle index, first site
    GateTask* d_tasks = nullptr;   // k >= 2
    TaskMeta* d_meta = nullptr;
    SiteTask* d_site = nullptr;    // k = 1
  };
  std::vector<mps_state*> hs;
  std::vector<Chunk> chunks;
  std::vector<std::vector<int>> ub_start, ub_end;  // per handle: bond bounds the graph was sized for / leaves
  bool split = false;
  void* mem = nullptr;  // gates and tables
  void* arena = nullptr;
  size_t arena_bytes = 0;
  OzBuffers oz;
  OzJob* d_jobs = nullptr;
  int jobs_cap = 0;
  cudaStream_t side = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long updates = 0;
  long long recorded_launches = 0;  // kernels recorded (a loop body counted once)
};

namespace {

size_t gamma_elems(const mps_state* h) { return (size_t)h->n * 2 * h->cap * h->cap; }
double2* site_ptr(const mps_state* h, int s) { return h->gamma + (size_t)s * 2 * h->cap * h->cap; }
double* bond_ptr(const mps_state* h, int b) { return h->lambda + (size_t)(b + 1) * h->cap; }

// Profiling brackets: pbeg records a start event (profiling on) and returns its
// index; pend records the end event and counts the launches of the class.
int pbeg(mps_state* h) {
  if (!h->prof || h->capturing) return -1;
  if (h->ev_next + 2 > h->evs.size()) {
    for (int i = 0; i < 256; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
      h->evs.push_back(e);
    }
  }
  const int idx = (int)h->ev_next;
  h->ev_next += 2;
  cudaEventRecord(h->evs[idx], h->stream);
  return idx;
}
void pend(mps_state* h, int kind, int idx, int nlaunch, double host_flops = 0.0) {
  h->launches_all += nlaunch;
  if (idx < 0) return;
  cudaEventRecord(h->evs[idx + 1], h->stream);
  h->prof_rec.push_back({kind, idx, idx + 1});
  h->prof_launch[kind] += nlaunch;
  h->prof_flops_host[kind] += host_flops;
}

__global__ void k_reset(double2* gamma, double* lambda, int* chi, int n, int cap) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s <= n; s += gridDim.x * blockDim.x) {
    if (s < n) {
      gamma[(size_t)s * 2 * cap * cap] = make_double2(1.0, 0.0);
      gamma[((size_t)s * 2 + 1) * cap * cap] = make_double2(0.0, 0.0);
    }
    lambda[(size_t)s * cap] = 1.0;
    chi[s] = 1;
  }
}

int reset_state(mps_state* h) {
  k_reset<<<(h->n + 256) / 256, 256, 0, h->stream>>>(h->gamma, h->lambda, h->chi, h->n, h->cap);
  CK(cudaGetLastError());
  h->ub.assign(h->n + 1, 1);
  h->has_pend.assign(h->n, 0);
  return MPS_OK;
}

int ensure_tasks(mps_state* h, int ntask) {
  if (ntask <= h->task_cap) return MPS_OK;
  int cap = std::max(ntask, 2 * h->task_cap);
  cudaFree(h->d_tasks); cudaFree(h->d_meta); cudaFree(h->d_gates);
  cudaFreeHost(h->h_tasks); cudaFreeHost(h->h_gates);
  h->d_tasks = nullptr; h->d_meta = nullptr; h->d_gates = nullptr; h->h_tasks = nullptr; h->h_gates = nullptr;
  h->task_cap = 0;
  CK(dev_alloc((void**)&h->d_tasks, sizeof(GateTask) * cap));
  CK(dev_alloc((void**)&h->d_meta, sizeof(TaskMeta) * cap));
  CK(cudaMemset(h->d_meta, 0, sizeof(TaskMeta) * cap));
  CK(dev_alloc((void**)&h->d_gates, sizeof(double2) * 64 * cap));
  CK(host_alloc((void**)&h->h_tasks, sizeof(GateTask) * cap));
  CK(host_alloc((void**)&h->h_gates, sizeof(double2) * 64 * cap));
  h->task_cap = cap;
  return MPS_OK;
}

// A gate task: one k-site gate of one MPS (several MPS may share a pass).
struct TaskRef {
  mps_state* st;
  int site;
};

// Workspace of one task from its bond-dimension upper bounds (elements):
// A (Mw x Nw), V (Nw x Nw, both splits of a three-site gate), T, sigma/perm,
// and for the split-precision path A32, V32, P, Q, V2.
struct TaskLayout {
  size_t off[13];
  size_t total;
};

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

TaskLayout task_layout(const TaskRef& r, int k, bool split) {
  const mps_state* st = r.st;
  const size_t xl = st->ub[r.site], xr = st->ub[r.site + k], cap = st->cap;
  size_t sz[13] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (k == 3) {
    const size_t m1 = 2 * xl, n1 = 4 * xr;
    const size_t nw1 = std::min(m1, n1), mw1 = std::max(m1, n1);
    const size_t k1 = std::min(cap, nw1);
    const size_t m2 = 2 * k1, n2 = 2 * xr;
    const size_t nw2 = std::min(m2, n2);
    const size_t nw = std::max(nw1, nw2);
    sz[0] = mw1 * nw1 * sizeof(double2);
    sz[1] = nw * nw * sizeof(double2);
    sz[2] = std::max(4 * cap * cap, m2 * n2) * sizeof(double2);  // partial contraction uses capacity strides
    sz[3] = nw * sizeof(double);
    sz[4] = nw * sizeof(int);
    if (split) {
      sz[2] = std::max(sz[2], mw1 * nw1 * sizeof(double2));  // products A V, A W of the first split
      sz[5] = mw1 * nw1 * sizeof(float2);
      sz[6] = nw * nw * sizeof(float2);
      sz[7] = sz[8] = sz[9] = nw * nw * sizeof(double2);
    }
  } else {
    const size_t m = 2 * xl, n = 2 * xr;
    const size_t mw = std::max(m, n), nw = std::min(m, n);
    sz[0] = mw * nw * sizeof(double2);
    sz[1] = nw * nw * sizeof(double2);
    sz[3] = nw * sizeof(double);
    sz[4] = nw * sizeof(int);
    if (split) {
      sz[2] = mw * nw * sizeof(double2);
      sz[5] = mw * nw * sizeof(float2);
      sz[6] = nw * nw * sizeof(float2);
      sz[7] = sz[8] = sz[9] = nw * nw * sizeof(double2);
    }
  }
  if (split) {  // the fp32 sweeps' per-block-pair rotations (b = 16)
    size_t nw = 1;
    if (k == 3) {
      const size_t m1 = 2 * xl, n1 = 4 * xr, k1 = std::min(cap, std::min(m1, n1));
      nw = std::max(std::min(m1, n1), std::min(2 * k1, 2 * xr));
    } else {
      nw = std::min(2 * xl, 2 * xr);
    }
    const size_t pairs = (nw + 31) / 32 + 1;
    sz[10] = pairs * 32 * 32 * sizeof(float2);
    sz[11] = pairs * sizeof(int);
    sz[12] = 2 * ((nw + 7) / 8 + 2) * sizeof(int);  // per-block round counters of A and V (block width 8 or 16)
  }
  TaskLayout L;
  size_t o = 0;
  for (int i = 0; i < 13; ++i) {
    L.off[i] = o;
    o += align256(sz[i]);
  }
  L.total = o;
  return L;
}

int ensure_arena(mps_state* w, size_t bytes) {
  if (bytes <= w->arena_bytes) return MPS_OK;
  CK(cudaStreamSynchronize(w->stream));
  const size_t grow = std::max(bytes, w->arena_bytes + w->arena_bytes / 2);
  cudaFree(w->arena);
  w->arena = nullptr;
  w->arena_bytes = 0;
  if (dev_alloc((void**)&w->arena, grow) != cudaSuccess) {
    cudaGetLastError();
    CK(dev_alloc((void**)&w->arena, bytes));
    w->arena_bytes = bytes;
    return MPS_OK;
  }
  w->arena_bytes = grow;
  return MPS_OK;
}

void free_state(mps_state* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  cudaFree(h->arena);
  cudaFree(h->sk_arena);
  cudaFree(h->ro_buf);
  cudaFree(h->d_oz_jobs); cudaFree(h->d_oz_err); cudaFree(h->oz_buf.base);
  cudaFree(h->gamma); cudaFree(h->lambda); cudaFree(h->chi);
  cudaFree(h->d_tasks); cudaFree(h->d_meta); cudaFree(h->d_gates); cudaFree(h->d_counter);
  cudaFree(h->d_site); cudaFree(h->d_site_gates);
  cudaFreeHost(h->h_tasks); cudaFreeHost(h->h_gates); cudaFreeHost(h->h_counter);
  cudaFreeHost(h->h_site); cudaFreeHost(h->h_site_gates);
  cudaFree(h->d_prof_flops);
  for (cudaEvent_t e : h->evs) cudaEventDestroy(e);
  if (h->own) cudaStreamDestroy(h->own);
  delete h;
}

bool is_unitary(const double* U, int d) {
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      cd acc = 0;
      for (int r = 0; r < d; ++r) acc += std::conj(cd(U[2 * (r * d + i)], U[2 * (r * d + i) + 1])) * cd(U[2 * (r * d + j)], U[2 * (r * d + j) + 1]);
      if (std::abs(acc - cd(i == j ? 1.0 : 0.0)) > 1e-10) return false;
    }
  return true;
}

// U' = U (P_site (x) ... (x) P_{site+k-1}) with the held-back single-qubit gates
// (they stay held back until consume_pending).
void fold_pending(mps_state* h, int site, int k, const double* U, double2* out) {
  const int d = 1 << k;
  std::vector<cd> P((size_t)d * d, cd(0));
  for (int r = 0; r < d; ++r)
    for (int c = 0; c < d; ++c) {
      cd v = 1.0;
      for (int j = 0; j < k; ++j) {
        const int br = (r >> (k - 1 - j)) & 1, bc = (c >> (k - 1 - j)) & 1;
        const int q = site + j;
        if (h->has_pend[q]) v *= h->pend[q][br * 2 + bc];
        else v *= (br == bc) ? 1.0 : 0.0;
      }
      P[(size_t)r * d + c] = v;
    }
  for (int r = 0; r < d; ++r)
    for (int c = 0; c < d; ++c) {
      cd acc = 0;
      for (int m = 0; m < d; ++m) acc += cd(U[2 * (r * d + m)], U[2 * (r * d + m) + 1]) * P[(size_t)m * d + c];
      out[r * d + c] = make_double2(acc.real(), acc.imag());
    }
}

// The held-back single-qubit gates of a gate's qubits are consumed once the
// gate's update has been launched; a call that fails before that keeps them.
void consume_pending(const TaskRef& r, int k) {
  for (int j = 0; j < k; ++j) r.st->has_pend[r.site + j] = 0;
}

// Applies every held-back single-qubit gate (before readouts and exports).
int flush_pending(mps_state* h) {
  int cnt = 0, el_ub = 1;
  for (int s = 0; s < h->n; ++s) cnt += h->has_pend[s];
  if (!cnt) return MPS_OK;
  if (!h->d_site || !h->h_site) {
    CK(dev_alloc((void**)&h->d_site, sizeof(SiteTask) * h->n));
    CK(dev_alloc((void**)&h->d_site_gates, sizeof(double2) * 4 * h->n));
    CK(host_alloc((void**)&h->h_site, sizeof(SiteTask) * h->n));
    CK(host_alloc((void**)&h->h_site_gates, sizeof(double2) * 4 * h->n));
  }
  CK(cudaStreamSynchronize(h->stream));  // pinned staging reuse
  int t = 0;
  for (int s = 0; s < h->n; ++s) {
    if (!h->has_pend[s]) continue;
    for (int e = 0; e < 4; ++e) h->h_site_gates[4 * t + e] = make_double2(h->pend[s][e].real(), h->pend[s][e].imag());
    SiteTask st;
    st.g = site_ptr(h, s);
    st.chi = h->chi;
    st.site = s;
    st.cap = h->cap;
    st.U = h->d_site_gates + 4 * t;
    h->h_site[t] = st;
    el_ub = std::max(el_ub, h->ub[s] * h->ub[s + 1]);
    h->has_pend[s] = 0;
    ++t;
  }
  CK(cudaMemcpyAsync(h->d_site_gates, h->h_site_gates, sizeof(double2) * 4 * t, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->d_site, h->h_site, sizeof(SiteTask) * t, cudaMemcpyHostToDevice, h->stream));
  launch_apply1(h->d_site, t, el_ub, h->stream);
  h->launches_all += 1;
  CK(cudaGetLastError());
  return MPS_OK;
}

// ----------------------------------------------------------- device loops ---

// Sets the condition of a while node from the continuation flag d_counter[0]
// (tasks still active) and an iteration bound: the loop ends when no task is
// active or after max_iter passes, whichever comes first.
__global__ void k_loop_first(cudaGraphConditionalHandle hc, const int* flag, int* iter) {
  *iter = 0;
  cudaGraphSetConditional(hc, *flag > 0 ? 1u : 0u);
}
__global__ void k_loop_next(cudaGraphConditionalHandle hc, const int* flag, int* iter, int max_iter) {
  const int it = ++*iter;
  cudaGraphSetConditional(hc, (*flag > 0 && it < max_iter) ? 1u : 0u);
}

// Runs body() (one pass that leaves the number of still-active tasks in
// d_counter[0]) while that number is non-zero, at most max_iter times.
// first_always: the first pass runs unconditionally; otherwise d_counter[0]
// already holds the count that decides it.
// Eager: the host reads the count back after every pass. While recording a
// program: a conditional while node whose body is one pass, recorded on the
// side stream, with the device setting the node's condition (no host round trip).
template <class F>
int device_loop(mps_state* h, int max_iter, bool first_always, F body) {
  if (!h->capturing) {
    if (!first_always) {
      CK(cudaMemcpyAsync(h->h_counter, h->d_counter, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      if (*h->h_counter == 0) return MPS_OK;
    }
    for (int it = 0; it < max_iter; ++it) {
      const int rc = body();
      if (rc) return rc;
      CK(cudaMemcpyAsync(h->h_counter, h->d_counter, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      if (*h->h_counter == 0) break;
    }
    return MPS_OK;
  }
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  cudaGraphConditionalHandle hc;
  CK(cudaStreamGetCaptureInfo(h->stream, &cs, nullptr, &g, &deps, nullptr, &nd));
  if (cs != cudaStreamCaptureStatusActive) return fail(MPS_ERR_CUDA, "device loop outside an active capture");
  if (first_always) {
    CK(cudaGraphConditionalHandleCreate(&hc, g, 1u, cudaGraphCondAssignDefault));
    CK(cudaMemsetAsync(h->d_counter + 2, 0, sizeof(int), h->stream));
  } else {
    CK(cudaGraphConditionalHandleCreate(&hc, g, 0u, 0));
    k_loop_first<<<1, 1, 0, h->stream>>>(hc, h->d_counter, h->d_counter + 2);
    CK(cudaGetLastError());
  }
  CK(cudaStreamGetCaptureInfo(h->stream, &cs, nullptr, &g, &deps, nullptr, &nd));
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = hc;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, g, deps, nullptr, nd, &np));
  cudaGraph_t body_graph = np.conditional.phGraph_out[0];
  CK(cudaStreamUpdateCaptureDependencies(h->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  CK(cudaStreamBeginCaptureToGraph(h->side, body_graph, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  cudaStream_t main = h->stream;
  h->stream = h->side;
  int rc = body();
  if (!rc) {
    k_loop_next<<<1, 1, 0, h->side>>>(hc, h->d_counter, h->d_counter + 2, max_iter);
    if (cudaGetLastError() != cudaSuccess) rc = fail(MPS_ERR_CUDA, "loop condition launch");
  }
  h->stream = main;
  cudaGraph_t out = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(h->side, &out);
  if (rc) return rc;
  if (ee != cudaSuccess) return fail(MPS_ERR_CUDA, std::string("loop body capture: ") + cudaGetErrorString(ee));
  return MPS_OK;
}

// Blocked one-sided Jacobi on every task's working matrix (A, or T for the
// second split of a three-site update). One launch per round-robin round;
// a sweep ends with a convergence count read back to the host.
int run_svd_on(mps_state* h, const GateTask* dt, TaskMeta* dm, int ntask, int nw_ub, int second, bool init_v,
               bool first_always = true);

int run_svd(mps_state* h, int ntask, int nw_ub, int second, bool init_v = true, bool first_always = true) {
  return run_svd_on(h, h->d_tasks, h->d_meta, ntask, nw_ub, second, init_v, first_always);
}

// Jacobi sweeps on an explicit task/meta array (the layer's tasks, or the
// sketch's small sub-problems).
int run_svd_on(mps_state* h, const GateTask* dt, TaskMeta* dm, int ntask, int nw_ub, int second, bool init_v,
               bool first_always) {
  if (init_v) {
    launch_init_V(dt, dm, ntask, nw_ub, h->stream);
    h->launches_all += 1;
  }
  const int nb = (nw_ub + kBlockW - 1) / kBlockW;
  const int nbe = nb + (nb & 1);
  unsigned long long* fl = h->prof ? h->d_prof_flops : nullptr;
  const int max_sweeps = h->max_sweeps;
  int rc = device_loop(h, max_sweeps, first_always, [&]() -> int {
    for (int r = 0; r < nbe - 1; ++r) {
      const int ev = pbeg(h);
      launch_jacobi_round(dt, dm, ntask, r, nbe / 2, second, fl, h->stream);
      pend(h, 0, ev, 1);
    }
    CK(cudaMemsetAsync(h->d_counter, 0, sizeof(int), h->stream));
    launch_sweep_end(dm, ntask, max_sweeps, h->d_counter, h->stream);
    h->launches_all += 1;
    return MPS_OK;
  });
  if (rc) return rc;
  CK(cudaGetLastError());
  return MPS_OK;
}

int validate_layer(mps_state* h, int k, int ng, const int* sites, const void* Us) {
  if (k < 1 || k > 3) return fail(MPS_ERR_ARG, "k must be 1, 2 or 3");
  if (ng < 0 || (ng > 0 && (!sites || !Us))) return fail(MPS_ERR_ARG, "null sites/gates");
  std::vector<char> used(h->n, 0);
  for (int g = 0; g < ng; ++g) {
    if (sites[g] < 0 || sites[g] + k > h->n) return fail(MPS_ERR_ARG, "gate site out of range");
    for (int j = 0; j < k; ++j) {
      if (used[sites[g] + j]) return fail(MPS_ERR_ARG, "gates of a layer overlap");
      used[sites[g] + j] = 1;
    }
  }
  return MPS_OK;
}

int ensure_oz(mps_state* h, int njobs) {
  if (!h->d_oz_jobs || h->oz_cap < njobs) {
    CK(cudaStreamSynchronize(h->stream));
    cudaFree(h->d_oz_jobs);
    h->d_oz_jobs = nullptr;
    const int cap = std::max(njobs, h->task_cap);
    CK(dev_alloc((void**)&h->d_oz_jobs, sizeof(OzJob) * cap));
    h->oz_cap = cap;
  }
  if (!h->d_oz_err) {
    CK(dev_alloc((void**)&h->d_oz_err, sizeof(int)));
    CK(cudaMemset(h->d_oz_err, 0, sizeof(int)));
  }
  return MPS_OK;
}

// slices > 0 caps the slice count of this product (a product that only needs
// a bounded absolute accuracy); 0 uses the handle's count.
int oz_gemm(mps_state* h, int ng, int kind, int M_ub, int N_ub, int K_ub, int slices = 0) {
  if (h->oz_timed_out) return fail(MPS_ERR_TIMEOUT, "an earlier split GEMM timed out; the handle's device state is not trusted");
  int rc0 = ensure_oz(h, ng);
  if (rc0) return rc0;
  const int sl = slices > 0 ? std::min(slices, h->slices) : h->slices;
  if (h->capturing && OzBuffers::bytes_needed(ng, M_ub, N_ub, std::min(K_ub, 512), sl) > h->oz_buf.bytes)
    return fail(MPS_ERR_CUDA, "recording: the split-GEMM buffers were sized too small");  // never reallocate mid-capture
  launch_oz_jobs(h->d_tasks, h->d_meta, h->d_oz_jobs, ng, kind, sl, h->prof ? h->d_prof_flops + 3 : nullptr,
                 h->stream);
  const int ev = pbeg(h);
  const int rc = ozaki_zgemm(h->d_oz_jobs, ng, M_ub, N_ub, K_ub, sl, h->oz_buf, h->d_oz_err, h->stream);
  pend(h, 3, ev, 3);  // executed flops: counted by k_oz_jobs
  h->launches_all += 1;
  if (rc == -2) return fail(MPS_ERR_NOMEM, "split GEMM buffers");
  if (rc) return fail(MPS_ERR_CUDA, "split GEMM launch failed");
  return MPS_OK;
}

// fp32 preconditioning sweeps on (A32, V32) of every task, then re-arm the
// tasks (the binary64 sweeps reuse the active/sweep counters).
int run_f32_sweeps(mps_state* h, int ng, int mw_ub, int nw_ub) {
  unsigned long long* fl = h->prof ? h->d_prof_flops + 4 : nullptr;
  // the tuned choice for this width (block width; rotation on the tensor
  // cores, or all sweeps in one scheduled launch)
  int bw = kBlockW32;
  int mode = kF32ModeSched;
  for (const mps_state::Tune& t : h->tune) {
    bw = t.f32_block;
    mode = t.mode;
    if (nw_ub <= t.nw_max) break;
  }
  if (mode == kF32ModeSched || mode == kF32ModeSchedWide) {
    const int ev = pbeg(h);
    const int nl = launch_jacobi_f32_sched(h->d_tasks, h->d_meta, ng, nw_ub, bw, mode == kF32ModeSched ? 256 : 384,
                                           kF32Sweeps, h->d_counter + 4,
                                           h->d_oz_err, fl, h->stream);
    if (nl < 0) {
      const cudaError_t e = cudaGetLastError();
      return fail(MPS_ERR_CUDA, std::string("scheduled fp32 sweeps: ") + cudaGetErrorString(e));
    }
    pend(h, 4, ev, nl);
    CK(cudaGetLastError());
    return MPS_OK;
  }
  const bool tc = mode == kF32ModeTc;
  const int nb = (nw_ub + bw - 1) / bw;
  const int nbe = nb + (nb & 1);
  return device_loop(h, kF32Sweeps, true, [&]() -> int {
    for (int r = 0; r < nbe - 1; ++r) {
      const int ev = pbeg(h);
      launch_jacobi_round_f32(h->d_tasks, h->d_meta, ng, r, nbe / 2, bw, tc ? 0 : 1, fl, h->stream);
      if (tc) launch_rot_tc(h->d_tasks, h->d_meta, ng, r, nbe / 2, mw_ub, nw_ub, h->d_oz_err, h->stream);
      pend(h, 4, ev, tc ? 2 : 1);
    }
    CK(cudaMemsetAsync(h->d_counter, 0, sizeof(int), h->stream));
    launch_sweep_end_nofail(h->d_meta, ng, kF32Sweeps, h->d_counter, h->stream);
    h->launches_all += 1;
    return MPS_OK;
  });
}

// Split-precision theta and SVD of a layer of two-site gates (split_path.cu):
// theta by the split GEMM, fp32 preconditioning sweeps, Newton-Schulz
// re-orthonormalisation of V and B = A V by the split GEMM, binary64 sweeps.
// Split-precision SVD of each task's working matrix in A (Mw x Nw, frob2 set):
// fp32 sweeps, V re-orthonormalised, B = A V, Gram polish, and the blocked
// binary64 sweeps for what the polish leaves (split_path.cu).
int run_split_svd(mps_state* h, int ng, int mw_ub, int nw_ub) {
  int ev = pbeg(h);
  launch_to_f32(h->d_tasks, h->d_meta, ng, nw_ub, (long long)mw_ub * nw_ub + (long long)nw_ub * nw_ub, h->stream);
  pend(h, 5, ev, 2);
  int rc = ensure_oz(h, ng);  // its error word also serves the tensor-core rotation
  if (rc) return rc;
  rc = run_f32_sweeps(h, ng, mw_ub, nw_ub);
  if (rc) return rc;
  ev = pbeg(h);
  launch_v_to_f64(h->d_tasks, h->d_meta, ng, (long long)nw_ub * nw_ub, h->stream);
  pend(h, 5, ev, 1);
  for (int it = 0; it < 2; ++it) {  // Newton-Schulz: V <- V (3I - V^H V) / 2
    if ((rc = oz_gemm(h, ng, kOzVhV, nw_ub, nw_ub, nw_ub))) return rc;
    if ((rc = oz_gemm(h, ng, kOzVP, nw_ub, nw_ub, nw_ub))) return rc;
    ev = pbeg(h);
    launch_ns_update(h->d_tasks, h->d_meta, ng, (long long)nw_ub * nw_ub, h->stream);
    pend(h, 5, ev, 1);
  }
  if ((rc = oz_gemm(h, ng, kOzAV, mw_ub, nw_ub, nw_ub))) return rc;
  ev = pbeg(h);
  launch_take_product(h->d_tasks, h->d_meta, ng, (long long)mw_ub * nw_ub, h->stream);
  pend(h, 5, ev, 1);
  // Gram polish: simultaneous first-order rotations from a split-precision
  // Gram, then a last Gram test; what is left goes to the blocked sweeps
  const long long nv = (long long)nw_ub * nw_ub, na = (long long)mw_ub * nw_ub;
  for (int step = 0; step <= kGramSteps; ++step) {
    const bool last = step == kGramSteps;
    rc = oz_gemm(h, ng, kOzAhA, nw_ub, nw_ub, mw_ub);
    if (rc) return rc;
    ev = pbeg(h);
    launch_gram_diag(h->d_tasks, h->d_meta, ng, nw_ub, h->stream);
    launch_gram_x(h->d_tasks, h->d_meta, ng, nv, last ? 0 : 1, h->stream);
    if (last) CK(cudaMemsetAsync(h->d_counter, 0, sizeof(int), h->stream));
    launch_gram_end(h->d_meta, ng, last ? 1 : 0, h->d_counter, h->stream);
    pend(h, 5, ev, 3);
    if (last) break;
    // the powers of X need only an absolute accuracy well below 1e-16: with
    // |x| <= 1e-3 the s-slice error 2^-7s sqrt(Nw) |x|^k stays under 1e-17
    // for s = 6, 4, 3 (k = 2, 3, 4)
    if ((rc = oz_gemm(h, ng, kOzXX, nw_ub, nw_ub, nw_ub, 6))) return rc;  // Q = X^2
    if ((rc = oz_gemm(h, ng, kOzX3, nw_ub, nw_ub, nw_ub, 4))) return rc;  // V2 = X^3
    if ((rc = oz_gemm(h, ng, kOzX4, nw_ub, nw_ub, nw_ub, 3))) return rc;  // T = X^4
    ev = pbeg(h);
    launch_form_w(h->d_tasks, h->d_meta, ng, nv, h->stream);
    launch_gram_scales(h->d_tasks, h->d_meta, ng, nw_ub, h->stream);
    pend(h, 5, ev, 2);
    if ((rc = oz_gemm(h, ng, kOzAW, mw_ub, nw_ub, nw_ub))) return rc;
    if ((rc = oz_gemm(h, ng, kOzVW, nw_ub, nw_ub, nw_ub))) return rc;
    ev = pbeg(h);
    launch_take_t(h->d_tasks, h->d_meta, ng, na + nv, h->stream);
    launch_givens(h->d_tasks, h->d_meta, ng, mw_ub + nw_ub, h->stream);
    pend(h, 5, ev, 2);
  }
  if (h->capturing) {
    // the blocked binary64 sweeps for the tasks the last Gram test left above
    // the tolerance (their count is in d_counter[0]); a bounded wait that ran
    // out is reported by the next synchronising call
    return run_svd(h, ng, nw_ub, 0, false, false);
  }
  int err = 0;
  CK(cudaMemcpyAsync(&err, h->d_oz_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(h->h_counter, h->d_counter, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (err) {
    h->oz_timed_out = 1;  // sticky: see mps_state::oz_timed_out
    return fail(MPS_ERR_TIMEOUT, "split GEMM: a bounded wait ran out; the handle's device state is not trusted");
  }
  if (*h->h_counter == 0) return MPS_OK;
  return run_svd(h, ng, nw_ub, 0, false);
}

// Two-site split-precision update: theta by the split GEMM and the gate mix,
// then the split SVD.
int run_split_theta_svd(mps_state* h, int ng, int xl_ub, int x0_ub, int xr_ub, int nw_ub) {
  const int mw_ub = std::max(2 * xl_ub, 2 * xr_ub);
  int rc = oz_gemm(h, ng, kOzTheta, 2 * xl_ub, 2 * xr_ub, x0_ub);
  if (rc) return rc;
  const int ev = pbeg(h);
  launch_gate_mix2(h->d_tasks, h->d_meta, ng, xl_ub, xr_ub, h->stream);
  launch_frob(h->d_tasks, h->d_meta, ng, (long long)mw_ub * nw_ub, 0, h->stream);
  pend(h, 5, ev, 2);
  return run_split_svd(h, ng, mw_ub, nw_ub);
}

// The update pipeline of one pass of k-site gates (k = 2, 3), possibly from
// several MPS: refs[g] is gate g, its matrix on the device at d_U + g*u_stride.
// `w` owns the workspace, the task tables and the stream.
// Reads the pass's task metadata back (one small copy after the pass's last
// launch) so that the host bounds of the rewritten bonds become the kept
// ranks themselves: the next layer's grids then follow the actual bond
// dimensions instead of the growth bound min(chi_max, 2 chi_l, 2 chi_r).
int read_meta(mps_state* w, int ng, std::vector<TaskMeta>& hm) {
  hm.resize(ng);
  CK(cudaMemcpyAsync(hm.data(), w->d_meta, sizeof(TaskMeta) * ng, cudaMemcpyDeviceToHost, w->stream));
  CK(cudaStreamSynchronize(w->stream));
  return MPS_OK;
}

// Host bounds of the bonds a pass rewrites when the kept ranks are not read
// back: the growth bounds min(chi_max, 2 chi_l, 2 chi_r) (two-site) and
// min(chi_max, 2 chi_l, 4 chi_r), min(chi_max, 2 k1, 2 chi_r) (three-site).
void advance_bounds(const std::vector<TaskRef>& refs, int k) {
  for (const TaskRef& r : refs) {
    mps_state* h = r.st;
    const int s0 = r.site;
    if (k == 2) {
      h->ub[s0 + 1] = std::min(h->cap, std::min(2 * h->ub[s0], 2 * h->ub[s0 + 2]));
    } else if (k == 3) {
      const int k1 = std::min(h->cap, std::min(2 * h->ub[s0], 4 * h->ub[s0 + 3]));
      h->ub[s0 + 1] = k1;
      h->ub[s0 + 2] = std::min(h->cap, std::min(2 * k1, 2 * h->ub[s0 + 3]));
    }
  }
}

// Fills the task table (w->h_tasks) of one pass with workspace carved from
// `arena` by the tasks' layouts (from the current host bounds); returns the
// workspace bytes used.
size_t build_tasks(mps_state* w, int k, const std::vector<TaskRef>& refs, const double2* d_U, int u_stride,
                   bool split, unsigned char* arena, GateTask* out) {
  unsigned char* base = arena;
  for (size_t g = 0; g < refs.size(); ++g) {
    mps_state* h = refs[g].st;
    const int s = refs[g].site;
    const TaskLayout L = task_layout(refs[g], k, split);
    unsigned char* tb = base;
    base += L.total;
    GateTask t;
    std::memset(&t, 0, sizeof(t));
    t.g0 = site_ptr(h, s);
    t.g1 = site_ptr(h, s + 1);
    t.g2 = k == 3 ? site_ptr(h, s + 2) : nullptr;
    t.lamL = bond_ptr(h, s - 1);
    t.lam0 = bond_ptr(h, s);
    t.lam1 = bond_ptr(h, s + 1);
    t.lamR = bond_ptr(h, s + k - 1);
    t.chi = h->chi;
    t.U = d_U + (size_t)u_stride * g;
    t.site = s;
    t.k = k;
    t.cap = h->cap;
    t.cutoff = h->cutoff;
    const size_t* o = L.off;
    t.A = reinterpret_cast<double2*>(tb + o[0]);
    t.V = reinterpret_cast<double2*>(tb + o[1]);
    t.T = reinterpret_cast<double2*>(tb + o[2]);
    t.sigma = reinterpret_cast<double*>(tb + o[3]);
    t.perm = reinterpret_cast<int*>(tb + o[4]);
    t.A32 = reinterpret_cast<float2*>(tb + o[5]);
    t.V32 = reinterpret_cast<float2*>(tb + o[6]);
    t.P = reinterpret_cast<double2*>(tb + o[7]);
    t.Q = reinterpret_cast<double2*>(tb + o[8]);
    t.V2 = reinterpret_cast<double2*>(tb + o[9]);
    t.Wp = reinterpret_cast<float2*>(tb + o[10]);
    t.Wneed = reinterpret_cast<int*>(tb + o[11]);
    t.qver = reinterpret_cast<int*>(tb + o[12]);
    out[g] = t;
  }
  (void)w;
  return (size_t)(base - arena);
}

// The launch sequence of one pass of k-site gate updates (k = 2, 3), possibly
// from several MPS, on tasks already in w->d_tasks: theta, SVD, truncation,
// rewrite. Grids are sized from the host bounds of the tasks' bonds.
// Eager: reads the pass's task metadata back after the truncation (one small
// copy) so that the bounds of the rewritten bonds become the kept ranks
// themselves; the next layer's grids then follow the actual bond dimensions.
// While recording a program: no read-back; the bounds advance by the growth
// rule (advance_bounds).
int emit_pass(mps_state* w, int k, const std::vector<TaskRef>& refs, bool split) {
  const int ng = (int)refs.size();
  int xl_ub = 1, x0_ub = 1, xr_ub = 1, nw_ub = 1, cap_ub = 1;
  double fl_contract = 0.0;
  for (int g = 0; g < ng; ++g) {
    const mps_state* h = refs[g].st;
    const int s = refs[g].site;
    const int xl = h->ub[s], x0 = h->ub[s + 1], xr = h->ub[s + k];
    xl_ub = std::max(xl_ub, xl);
    x0_ub = std::max(x0_ub, x0);
    xr_ub = std::max(xr_ub, xr);
    cap_ub = std::max(cap_ub, h->cap);
    nw_ub = std::max(nw_ub, std::min(2 * xl, (k == 3 ? 4 : 2) * xr));
    if (k == 2) fl_contract += 32.0 * xl * x0 * xr + 128.0 * xl * xr;
    else fl_contract += 32.0 * x0 * h->ub[s + 2] * xr + 64.0 * xl * x0 * xr + 512.0 * xl * xr;
  }
  int rc;
  launch_setup(w->d_tasks, w->d_meta, ng, 0, w->stream);
  w->launches_all += 1;
  if (split && k == 2) {
    rc = run_split_theta_svd(w, ng, xl_ub, x0_ub, xr_ub, nw_ub);
    if (rc) return rc;
  } else {
    int ev = pbeg(w);
    if (k == 2) launch_contract2(w->d_tasks, w->d_meta, ng, xl_ub, xr_ub, w->stream);
    else launch_contract3(w->d_tasks, w->d_meta, ng, x0_ub, xl_ub, xr_ub, w->stream);
    pend(w, 1, ev, k == 2 ? 1 : 2, fl_contract);
    launch_frob(w->d_tasks, w->d_meta, ng, (long long)(2 * xl_ub) * ((k == 3 ? 4 : 2) * xr_ub), 0, w->stream);
    w->launches_all += 1;
    CK(cudaGetLastError());
    // three-site split mode: the binary64 theta (two contraction steps), split SVD
    rc = split ? run_split_svd(w, ng, std::max(2 * xl_ub, 4 * xr_ub), nw_ub) : run_svd(w, ng, nw_ub, 0);
    if (rc) return rc;
  }
  const int k_ub = std::min(cap_ub, nw_ub);
  int ev = pbeg(w);
  launch_colnorms(w->d_tasks, w->d_meta, ng, nw_ub, 0, w->stream);
  launch_truncate(w->d_tasks, w->d_meta, ng, 0, kMaxCap, w->stream);
  if (k == 2) {
    launch_emit_left(w->d_tasks, w->d_meta, ng, xl_ub, k_ub, 0, w->stream);
    launch_emit_right(w->d_tasks, w->d_meta, ng, xr_ub, k_ub, 0, w->stream);
    pend(w, 2, ev, 4);
    if (w->capturing) {
      advance_bounds(refs, 2);
    } else {
      std::vector<TaskMeta> hm;
      if ((rc = read_meta(w, ng, hm))) return rc;
      for (int g = 0; g < ng; ++g) {
        mps_state* h = refs[g].st;
        const int bound = std::min(h->cap, std::min(2 * h->ub[refs[g].site], 2 * h->ub[refs[g].site + 2]));
        h->ub[refs[g].site + 1] = hm[g].status == 0 ? std::max(1, std::min(bound, hm[g].knew)) : bound;
      }
    }
  } else {
    launch_emit_left(w->d_tasks, w->d_meta, ng, xl_ub, k_ub, 0, w->stream);
    launch_form_second(w->d_tasks, w->d_meta, ng, k_ub, xr_ub, w->stream);
    launch_setup(w->d_tasks, w->d_meta, ng, 1, w->stream);
    pend(w, 2, ev, 5);
    std::vector<int> k1s(ng);
    int nw2_ub = 1;
    std::vector<TaskMeta> hm;
    if (!w->capturing && (rc = read_meta(w, ng, hm))) return rc;
    for (int g = 0; g < ng; ++g) {
      const TaskRef& r = refs[g];
      const mps_state* h = r.st;
      const int bound = std::min(h->cap, std::min(2 * h->ub[r.site], 4 * h->ub[r.site + 3]));
      k1s[g] = (!w->capturing && hm[g].status == 0) ? std::max(1, std::min(bound, hm[g].k1)) : bound;
      nw2_ub = std::max(nw2_ub, std::min(2 * k1s[g], 2 * h->ub[r.site + 3]));
    }
    launch_frob(w->d_tasks, w->d_meta, ng, (long long)(2 * k_ub) * (2 * xr_ub), 1, w->stream);
    w->launches_all += 1;
    if (split) {
      // the second working matrix (in T) moves to A for the split SVD and back
      const long long el2 = (long long)(2 * k_ub) * (2 * xr_ub);
      launch_copy_work(w->d_tasks, w->d_meta, ng, el2, 0, w->stream);
      rc = run_split_svd(w, ng, std::max(2 * k_ub, 2 * xr_ub), nw2_ub);
      if (rc) return rc;
      launch_copy_work(w->d_tasks, w->d_meta, ng, el2, 1, w->stream);
      w->launches_all += 2;
    } else {
      rc = run_svd(w, ng, nw2_ub, 1);
      if (rc) return rc;
    }
    const int k2_ub = std::min(cap_ub, nw2_ub);
    ev = pbeg(w);
    launch_colnorms(w->d_tasks, w->d_meta, ng, nw2_ub, 1, w->stream);
    launch_truncate(w->d_tasks, w->d_meta, ng, 1, kMaxCap, w->stream);
    launch_emit_left(w->d_tasks, w->d_meta, ng, k_ub, k2_ub, 1, w->stream);
    launch_emit_right(w->d_tasks, w->d_meta, ng, xr_ub, k2_ub, 1, w->stream);
    pend(w, 2, ev, 4);
    if (w->capturing) {
      advance_bounds(refs, 3);
    } else {
      if ((rc = read_meta(w, ng, hm))) return rc;
      for (int g = 0; g < ng; ++g) {
        mps_state* h = refs[g].st;
        const int s0 = refs[g].site;
        const int bound = std::min(h->cap, std::min(2 * k1s[g], 2 * h->ub[s0 + 3]));
        h->ub[s0 + 1] = k1s[g];
        h->ub[s0 + 2] = hm[g].status == 0 ? std::max(1, std::min(bound, hm[g].knew)) : bound;
      }
    }
  }
  CK(cudaGetLastError());
  w->last_ntask = ng;
  w->last_k = k;
  return MPS_OK;
}

int run_update_refs(mps_state* w, int k, const std::vector<TaskRef>& refs, const double2* d_U, int u_stride,
                    bool split) {
  const int ng = (int)refs.size();
  size_t total = 0;
  for (int g = 0; g < ng; ++g) total += task_layout(refs[g], k, split).total;
  int rc = ensure_arena(w, total);
  if (rc) return rc;
  build_tasks(w, k, refs, d_U, u_stride, split, static_cast<unsigned char*>(w->arena), w->h_tasks);
  CK(cudaMemcpyAsync(w->d_tasks, w->h_tasks, sizeof(GateTask) * ng, cudaMemcpyHostToDevice, w->stream));
  return emit_pass(w, k, refs, split);
}

// ------------------------------------------------------------- sketch path ---

// Split-precision GEMMs whose jobs are built on the host (exact dimensions).
int oz_gemm_host(mps_state* w, const std::vector<OzJob>& jobs, int M_ub, int N_ub, int K_ub) {
  if (jobs.empty()) return MPS_OK;
  if (w->oz_timed_out) return fail(MPS_ERR_TIMEOUT, "an earlier split GEMM timed out; the handle's device state is not trusted");
  const int n = (int)jobs.size();
  int rc0 = ensure_oz(w, n);
  if (rc0) return rc0;
  CK(cudaStreamSynchronize(w->stream));  // the job table is rewritten below
  CK(cudaMemcpy(w->d_oz_jobs, jobs.data(), sizeof(OzJob) * n, cudaMemcpyHostToDevice));
  const int ev = pbeg(w);
  const int rc = ozaki_zgemm(w->d_oz_jobs, n, M_ub, N_ub, K_ub, w->slices, w->oz_buf, w->d_oz_err, w->stream);
  const int npair = w->slices * (w->slices + 1) / 2;
  pend(w, 3, ev, 3, (double)n * npair * 8.0 * M_ub * N_ub * K_ub);
  if (rc == -2) return fail(MPS_ERR_NOMEM, "split GEMM buffers");
  if (rc) return fail(MPS_ERR_CUDA, "split GEMM launch failed");
  return MPS_OK;
}

OzView view(const double2* p, long long s_r, long long s_k, int conj = 0, const double* rscale = nullptr) {
  OzView v = {};
  v.p = p;
  v.s_r = s_r;
  v.s_k = s_k;
  v.conj = conj;
  v.rscale = rscale;
  return v;
}

OzJob job(OzView a, OzView b, int M, int N, int K, double2* C, long long ldc) {
  OzJob j = {};
  j.a = a;
  j.b = b;
  j.M = M;
  j.N = N;
  j.K = K;
  j.C = C;
  j.ldc = ldc;
  j.alpha = 1.0;
  return j;
}

// Predicted sketch rank of each two-site gate (features of the current state,
// the MLP forward kernel on the device).
int predict_ranks(mps_state* w, const std::vector<TaskRef>& refs, const double2* hU, std::vector<double>& rhat) {
  const int n = (int)refs.size();
  std::vector<FeatureTask> ft(n);
  for (int g = 0; g < n; ++g) {
    const TaskRef& r = refs[g];
    double u[32];
    for (int e = 0; e < 16; ++e) {
      u[2 * e] = hU[64 * g + e].x;
      u[2 * e + 1] = hU[64 * g + e].y;
    }
    FeatureTask f;
    f.lamL = bond_ptr(r.st, r.site - 1);
    f.lamR = bond_ptr(r.st, r.site + 1);
    f.chi = r.st->chi;
    f.site = r.site;
    f.k = 2;
    f.ep = (float)entangling_power(u);
    f.cutoff = r.st->cutoff;
    ft[g] = f;
  }
  FeatureTask* d_ft = nullptr;
  float *d_x = nullptr, *d_y = nullptr;
  CK(dev_alloc((void**)&d_ft, sizeof(FeatureTask) * n));
  CK(dev_alloc((void**)&d_x, sizeof(float) * 16 * n));
  CK(dev_alloc((void**)&d_y, sizeof(float) * n));
  std::vector<float> y(n);
  cudaError_t e = cudaMemcpyAsync(d_ft, ft.data(), sizeof(FeatureTask) * n, cudaMemcpyHostToDevice, w->stream);
  if (e == cudaSuccess) {
    launch_features(d_ft, n, d_x, w->stream);
    launch_mlp_fwd(mlp_params(w->predictor), d_x, n, d_y, w->stream);
    w->launches_all += 2;
    e = cudaMemcpyAsync(y.data(), d_y, sizeof(float) * n, cudaMemcpyDeviceToHost, w->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
  cudaFree(d_ft);
  cudaFree(d_x);
  cudaFree(d_y);
  if (e != cudaSuccess) return fail(MPS_ERR_CUDA, "rank prediction");
  rhat.resize(n);
  for (int g = 0; g < n; ++g) rhat[g] = std::exp2(10.0 * std::min(std::max((double)y[g], -1.0), 1.1));
  return MPS_OK;
}

__global__ void k_mark_skip(TaskMeta* meta, const int* idx, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) meta[idx[t]].status = 1;  // left to the full pass: no truncation or rewrite here
}

// One sketch pass over two-site gates S with sketch widths r (host gates hU,
// folded, stride 64). Accepted gates are finished (truncated, rewritten);
// the indices of rejected gates are returned for the full Jacobi pass.
int run_sketch_pass(mps_state* w, const std::vector<TaskRef>& S, const std::vector<int>& rS, const double2* hU,
                    std::vector<int>& rejected) {
  const int ng = (int)S.size();
  const bool split = w->prec == MPS_PREC_SPLIT;
  CK(cudaStreamSynchronize(w->stream));
  int rc = ensure_tasks(w, ng);
  if (rc) return rc;
  std::memcpy(w->h_gates, hU, sizeof(double2) * 64 * ng);
  CK(cudaMemcpyAsync(w->d_gates, w->h_gates, sizeof(double2) * 64 * ng, cudaMemcpyHostToDevice, w->stream));
  // main task layout (A, V, T, sigma, perm) and sketch buffers
  std::vector<TaskLayout> lay(ng);
  size_t total = 0, sk_total = 0;
  int xl_ub = 1, x0_ub = 1, xr_ub = 1, nw_ub = 1, mw_ub = 1, r_ub = 1, cap_ub = 1;
  std::vector<size_t> sk_off(ng);
  for (int g = 0; g < ng; ++g) {
    lay[g] = task_layout(S[g], 2, true);
    total += lay[g].total;
    const mps_state* h = S[g].st;
    const int xl = h->ub[S[g].site], x0 = h->ub[S[g].site + 1], xr = h->ub[S[g].site + 2];
    const size_t mw = std::max(2 * xl, 2 * xr), nw = std::min(2 * xl, 2 * xr), r = rS[g];
    xl_ub = std::max(xl_ub, xl);
    x0_ub = std::max(x0_ub, x0);
    xr_ub = std::max(xr_ub, xr);
    nw_ub = std::max(nw_ub, (int)nw);
    mw_ub = std::max(mw_ub, (int)mw);
    r_ub = std::max(r_ub, rS[g]);
    cap_ub = std::max(cap_ub, h->cap);
    sk_off[g] = sk_total;
    sk_total += align256(sizeof(double2) * (3 * nw * r + mw * r + mw * nw + 2 * r * r));
  }
  rc = ensure_arena(w, total);
  if (rc) return rc;
  const size_t sig_bytes = align256(sizeof(double) * (size_t)r_ub * ng);
  const size_t tab_bytes = align256(sizeof(SketchTask) * ng) + 2 * align256(sizeof(GateTask) * ng) +
                           2 * align256(sizeof(TaskMeta) * ng) + align256(sizeof(double) * ng) +
                           align256(sizeof(int) * ng) * 2;
  if (sk_total + 2 * sig_bytes + tab_bytes > w->sk_bytes) {
    cudaFree(w->sk_arena);
    w->sk_arena = nullptr;
    w->sk_bytes = 0;
    const size_t want = sk_total + 2 * sig_bytes + tab_bytes;
    CK(dev_alloc((void**)&w->sk_arena, want));
    w->sk_bytes = want;
  }
  unsigned char* skb = static_cast<unsigned char*>(w->sk_arena);
  unsigned char* p = skb + sk_total;
  double* d_sigy = reinterpret_cast<double*>(p);
  p += sig_bytes;
  double* d_sigb = reinterpret_cast<double*>(p);
  p += sig_bytes;
  SketchTask* d_sk = reinterpret_cast<SketchTask*>(p);
  p += align256(sizeof(SketchTask) * ng);
  GateTask* d_suby = reinterpret_cast<GateTask*>(p);
  p += align256(sizeof(GateTask) * ng);
  GateTask* d_subb = reinterpret_cast<GateTask*>(p);
  p += align256(sizeof(GateTask) * ng);
  TaskMeta* d_mety = reinterpret_cast<TaskMeta*>(p);
  p += align256(sizeof(TaskMeta) * ng);
  TaskMeta* d_metb = reinterpret_cast<TaskMeta*>(p);
  p += align256(sizeof(TaskMeta) * ng);
  double* d_res = reinterpret_cast<double*>(p);
  p += align256(sizeof(double) * ng);
  int* d_acc = reinterpret_cast<int*>(p);
  p += align256(sizeof(int) * ng);
  int* d_idx = reinterpret_cast<int*>(p);

  // gate tasks, setup, theta, ||A||_F
  unsigned char* base = static_cast<unsigned char*>(w->arena);
  for (int g = 0; g < ng; ++g) {
    mps_state* h = S[g].st;
    const int s0 = S[g].site;
    unsigned char* tb = base;
    base += lay[g].total;
    GateTask t;
    std::memset(&t, 0, sizeof(t));
    t.g0 = site_ptr(h, s0);
    t.g1 = site_ptr(h, s0 + 1);
    t.lamL = bond_ptr(h, s0 - 1);
    t.lam0 = bond_ptr(h, s0);
    t.lam1 = bond_ptr(h, s0 + 1);
    t.lamR = bond_ptr(h, s0 + 1);
    t.chi = h->chi;
    t.U = w->d_gates + 64 * g;
    t.site = s0;
    t.k = 2;
    t.cap = h->cap;
    t.cutoff = h->cutoff;
    const size_t* o = lay[g].off;
    t.A = reinterpret_cast<double2*>(tb + o[0]);
    t.V = reinterpret_cast<double2*>(tb + o[1]);
    t.T = reinterpret_cast<double2*>(tb + o[2]);
    t.sigma = reinterpret_cast<double*>(tb + o[3]);
    t.perm = reinterpret_cast<int*>(tb + o[4]);
    w->h_tasks[g] = t;
  }
  CK(cudaMemcpyAsync(w->d_tasks, w->h_tasks, sizeof(GateTask) * ng, cudaMemcpyHostToDevice, w->stream));
  launch_setup(w->d_tasks, w->d_meta, ng, 0, w->stream);
  if (split) {
    rc = oz_gemm(w, ng, kOzTheta, 2 * xl_ub, 2 * xr_ub, x0_ub);
    if (rc) return rc;
    launch_gate_mix2(w->d_tasks, w->d_meta, ng, xl_ub, xr_ub, w->stream);
  } else {
    const int ev = pbeg(w);
    launch_contract2(w->d_tasks, w->d_meta, ng, xl_ub, xr_ub, w->stream);
    pend(w, 1, ev, 1);
  }
  launch_frob(w->d_tasks, w->d_meta, ng, (long long)mw_ub * nw_ub, 0, w->stream);
  w->launches_all += 3;
  std::vector<TaskMeta> hm(ng);
  CK(cudaMemcpyAsync(hm.data(), w->d_meta, sizeof(TaskMeta) * ng, cudaMemcpyDeviceToHost, w->stream));
  CK(cudaStreamSynchronize(w->stream));

  // sketch tasks with exact dimensions
  std::vector<SketchTask> sk(ng);
  for (int g = 0; g < ng; ++g) {
    SketchTask& q = sk[g];
    q.task = g;
    q.id = (int)(w->sk_sketched + g);
    q.Mw = hm[g].Mw;
    q.Nw = hm[g].Nw;
    q.r = std::min(rS[g], q.Nw);
    q.rcap = r_ub;
    q.cutoff = S[g].st->cutoff;
    q.A = w->h_tasks[g].A;
    q.V = w->h_tasks[g].V;
    double2* b = reinterpret_cast<double2*>(skb + sk_off[g]);
    const size_t nw = q.Nw, mw = q.Mw, r = q.r;
    q.Om = b;
    q.Y = q.Om + nw * r;
    q.Z = q.Y + mw * r;
    q.Bh = q.Z + nw * r;
    q.T2 = q.Bh + nw * r;
    q.Wy = q.T2 + mw * nw;
    q.Wb = q.Wy + r * r;
  }
  CK(cudaMemcpyAsync(d_sk, sk.data(), sizeof(SketchTask) * ng, cudaMemcpyHostToDevice, w->stream));
  CK(cudaMemsetAsync(d_res, 0, sizeof(double) * ng, w->stream));
  launch_omega(d_sk, ng, (long long)nw_ub * r_ub, w->sk_seed, w->stream);
  w->launches_all += 1;
  // Y = A Omega. No power iteration: A (A^H A)^q Omega compresses the spectrum
  // to sigma^(2q+1), which pushes directions far above the cutoff below the
  // resolution of Y's orthonormalisation; the residual test guards acceptance.
  std::vector<OzJob> J1;
  for (const SketchTask& q : sk)
    J1.push_back(job(view(q.A, 1, q.Mw), view(q.Om, q.Nw, 1), q.Mw, q.r, q.Nw, q.Y, q.Mw));
  if ((rc = oz_gemm_host(w, J1, mw_ub, r_ub, nw_ub))) return rc;
  // Q = orth(Y): one-sided Jacobi on Y, columns divided by their norms
  auto sub_problem = [&](GateTask* d_sub, TaskMeta* d_met, double* d_sig, bool of_y, const std::vector<int>& which,
                         int rows_ub) -> int {
    const int ns = (int)which.size();
    std::vector<GateTask> st(ns);
    std::vector<TaskMeta> sm(ns);
    for (int i = 0; i < ns; ++i) {
      const SketchTask& q = sk[which[i]];
      GateTask t;
      std::memset(&t, 0, sizeof(t));
      t.A = of_y ? q.Y : q.Bh;
      t.V = of_y ? q.Wy : q.Wb;
      t.sigma = d_sig + (size_t)which[i] * r_ub;
      st[i] = t;
      TaskMeta m;
      std::memset(&m, 0, sizeof(m));
      m.Mw = of_y ? q.Mw : q.Nw;
      m.Nw = q.r;
      m.M = m.Mw;
      m.N = m.Nw;
      m.tall = 1;
      m.active = 1;
      sm[i] = m;
    }
    CK(cudaMemcpyAsync(d_sub, st.data(), sizeof(GateTask) * ns, cudaMemcpyHostToDevice, w->stream));
    CK(cudaMemcpyAsync(d_met, sm.data(), sizeof(TaskMeta) * ns, cudaMemcpyHostToDevice, w->stream));
    launch_frob(d_sub, d_met, ns, (long long)rows_ub * r_ub, 0, w->stream);
    int rc2 = run_svd_on(w, d_sub, d_met, ns, r_ub, 0, true);
    if (rc2) return rc2;
    launch_colnorms(d_sub, d_met, ns, r_ub, 0, w->stream);
    w->launches_all += 2;
    CK(cudaStreamSynchronize(w->stream));  // the host vectors above are released on return
    return MPS_OK;
  };
  std::vector<int> all(ng);
  for (int g = 0; g < ng; ++g) all[g] = g;
  rc = sub_problem(d_suby, d_mety, d_sigy, true, all, mw_ub);
  if (rc) return rc;
  launch_scale_q(d_sk, ng, (long long)mw_ub * r_ub, d_sigy, d_mety, w->stream);
  // B^H = A^H Q; T2 = Q B; residual ||A - T2||_F^2
  std::vector<OzJob> J4, J5;
  for (const SketchTask& q : sk) {
    J4.push_back(job(view(q.A, q.Mw, 1, 1), view(q.Y, q.Mw, 1), q.Nw, q.r, q.Mw, q.Bh, q.Nw));
    J5.push_back(job(view(q.Y, 1, q.Mw), view(q.Bh, 1, q.Nw, 1), q.Mw, q.Nw, q.r, q.T2, q.Mw));
  }
  if ((rc = oz_gemm_host(w, J4, nw_ub, r_ub, mw_ub)) || (rc = oz_gemm_host(w, J5, mw_ub, nw_ub, r_ub))) return rc;
  launch_residual(d_sk, ng, (long long)mw_ub * nw_ub, d_res, w->stream);
  launch_sketch_mark(d_sk, ng, d_res, d_acc, w->d_meta, w->stream);
  w->launches_all += 3;
  std::vector<int> acc(ng);
  CK(cudaMemcpyAsync(acc.data(), d_acc, sizeof(int) * ng, cudaMemcpyDeviceToHost, w->stream));
  CK(cudaStreamSynchronize(w->stream));
  std::vector<int> yes;
  rejected.clear();
  for (int g = 0; g < ng; ++g) (acc[g] ? yes : rejected).push_back(g);
  w->sk_sketched += ng;
  w->sk_accepted += (long long)yes.size();
  if (!yes.empty()) {
    // SVD of B: Jacobi on B^H; A[:, j < r] = Q Wb diag(sigma_b); V = B^H Wb / sigma_b
    rc = sub_problem(d_subb, d_metb, d_sigb, false, yes, nw_ub);
    if (rc) return rc;
    std::vector<OzJob> J6;
    for (int g : yes) {
      const SketchTask& q = sk[g];
      J6.push_back(job(view(q.Y, 1, q.Mw), view(q.Wb, q.r, 1, 0, d_sigb + (size_t)g * r_ub), q.Mw, q.r, q.r, q.A,
                       q.Mw));
    }
    if ((rc = oz_gemm_host(w, J6, mw_ub, r_ub, r_ub))) return rc;
    launch_sketch_finish(d_sk, ng, (long long)nw_ub * nw_ub + (long long)mw_ub * nw_ub, d_sigb, d_acc, w->stream);
    w->launches_all += 1;
  }
  if (!rejected.empty()) {
    CK(cudaMemcpyAsync(d_idx, rejected.data(), sizeof(int) * rejected.size(), cudaMemcpyHostToDevice, w->stream));
    k_mark_skip<<<((int)rejected.size() + 127) / 128, 128, 0, w->stream>>>(w->d_meta, d_idx, (int)rejected.size());
    w->launches_all += 1;
  }
  // truncation and rewrite of the accepted gates
  const int k_ub = std::min(cap_ub, r_ub);
  const int ev = pbeg(w);
  launch_colnorms(w->d_tasks, w->d_meta, ng, nw_ub, 0, w->stream);
  launch_truncate(w->d_tasks, w->d_meta, ng, 0, kMaxCap, w->stream);
  launch_emit_left(w->d_tasks, w->d_meta, ng, xl_ub, k_ub, 0, w->stream);
  launch_emit_right(w->d_tasks, w->d_meta, ng, xr_ub, k_ub, 0, w->stream);
  pend(w, 2, ev, 4);
  std::vector<TaskMeta> hm2;
  if ((rc = read_meta(w, ng, hm2))) return rc;
  for (int g : yes) {
    mps_state* h = S[g].st;
    const int s0 = S[g].site;
    const int bound = std::min(sk[g].r, std::min(h->cap, std::min(2 * h->ub[s0], 2 * h->ub[s0 + 2])));
    h->ub[s0 + 1] = hm2[g].status == 0 ? std::max(1, std::min(bound, hm2[g].knew)) : bound;
  }
  CK(cudaGetLastError());
  return MPS_OK;
}

// Runs a list of gate tasks in passes whose workspace fits the budget. The
// host gates (already folded with held-back single-qubit gates) are in
// h_U (2^k x 2^k complex128 each, stride 64 double2), or, for device gates,
// d_U with stride u_stride.
int run_refs_chunked(mps_state* w, int k, std::vector<TaskRef>& refs, const double2* h_U, const double2* d_U,
                     int u_stride) {
  if (k == 2 && w->svd_mode == MPS_SVD_SKETCH_MLP && w->predictor && h_U && !refs.empty()) {
    // rank prediction; gates predicted near full rank go straight to the full SVD
    std::vector<double> rhat;
      int rc = predict_ranks(w, refs, h_U, rhat);
    if (rc) return rc;
      std::vector<TaskRef> S, F;
    std::vector<int> rS;
    std::vector<double2> hS, hF;
    for (size_t g = 0; g < refs.size(); ++g) {
      const mps_state* h = refs[g].st;
      const int nw = std::min(2 * h->ub[refs[g].site], 2 * h->ub[refs[g].site + 2]);
      // the sketch pays off only well below full rank; a rank at chi_max is a
      // truncation by rank, whose kept values a sketch does not reproduce exactly
      const int r = std::min(nw, (int)std::ceil(1.1 * rhat[g]) + 10);
      const bool sketch = 4 * r < 3 * nw && r < h->cap && h->cap <= kSplitMaxCap;
      (sketch ? S : F).push_back(refs[g]);
      std::vector<double2>& dst = sketch ? hS : hF;
      dst.insert(dst.end(), h_U + 64 * g, h_U + 64 * (g + 1));
      if (sketch) rS.push_back(std::max(r, 1));
    }
    w->sk_routed += (long long)F.size();
    if (!S.empty()) {
      std::vector<int> rej;
      rc = run_sketch_pass(w, S, rS, hS.data(), rej);
      if (rc) return rc;
      std::vector<char> is_rej(S.size(), 0);
      for (int g : rej) is_rej[g] = 1;
      for (size_t g = 0; g < S.size(); ++g)
        if (!is_rej[g]) consume_pending(S[g], 2);
      for (int g : rej) {
        F.push_back(S[g]);
        hF.insert(hF.end(), hS.begin() + 64 * g, hS.begin() + 64 * (g + 1));
      }
    }
    if (F.empty()) return MPS_OK;
    const int saved = w->svd_mode;
    w->svd_mode = MPS_SVD_JACOBI;
    rc = run_refs_chunked(w, k, F, hF.data(), nullptr, 0);
    w->svd_mode = saved;
      return rc;
  }
  bool split = (k == 2 || k == 3) && w->prec == MPS_PREC_SPLIT;
  for (const TaskRef& r : refs) split = split && r.st->cap <= kSplitMaxCap;
  size_t g0 = 0;
  while (g0 < refs.size()) {
    size_t g1 = g0, bytes = 0;
    while (g1 < refs.size() && (int)(g1 - g0) < kMaxTasksPerPass) {
      const size_t b = task_layout(refs[g1], k, split).total;
      if (g1 > g0 && bytes + b > kArenaBudget) break;
      bytes += b;
      ++g1;
    }
    const int ng = (int)(g1 - g0);
    CK(cudaStreamSynchronize(w->stream));  // task tables and pinned staging are reused
    int rc = ensure_tasks(w, ng);
    if (rc) return rc;
    const double2* dU = d_U;
    int stride = u_stride;
    if (h_U) {
      std::memcpy(w->h_gates, h_U + 64 * g0, sizeof(double2) * 64 * ng);
      CK(cudaMemcpyAsync(w->d_gates, w->h_gates, sizeof(double2) * 64 * ng, cudaMemcpyHostToDevice, w->stream));
      dU = w->d_gates;
      stride = 64;
    } else {
      dU = d_U + (size_t)u_stride * g0;
    }
    std::vector<TaskRef> part(refs.begin() + g0, refs.begin() + g1);
    rc = run_update_refs(w, k, part, dU, stride, split);
    if (rc) return rc;
    if (h_U)
      for (const TaskRef& r : part) consume_pending(r, k);
    g0 = g1;
  }
  return MPS_OK;
}

void hold_single(mps_state* h, int s, const double* u) {
  std::array<cd, 4> nu;
  std::array<cd, 4> p = h->has_pend[s] ? h->pend[s] : std::array<cd, 4>{1.0, 0.0, 0.0, 1.0};
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 2; ++c)
      nu[r * 2 + c] = cd(u[2 * (r * 2)], u[2 * (r * 2) + 1]) * p[c] + cd(u[2 * (r * 2 + 1)], u[2 * (r * 2 + 1) + 1]) * p[2 + c];
  h->pend[s] = nu;
  h->has_pend[s] = 1;
}

int apply_layer_impl(mps_state* h, int k, int ng, const int* sites, const double* Us) {
  int rc = validate_layer(h, k, ng, sites, Us);
  if (rc) return rc;
  if (ng == 0) return MPS_OK;
  const int d = 1 << k;
  for (int g = 0; g < ng; ++g)
    if (!is_unitary(Us + (size_t)2 * d * d * g, d)) return fail(MPS_ERR_NOT_UNITARY, "gate is not unitary");
  if (k == 1) {
    for (int g = 0; g < ng; ++g) hold_single(h, sites[g], Us + 8 * g);
    return MPS_OK;
  }
  std::vector<double2> hu((size_t)64 * ng);
  std::vector<TaskRef> refs(ng);
  for (int g = 0; g < ng; ++g) {
    fold_pending(h, sites[g], k, Us + (size_t)2 * d * d * g, hu.data() + 64 * g);
    refs[g] = TaskRef{h, sites[g]};
  }
  return run_refs_chunked(h, k, refs, hu.data(), nullptr, 0);
}

int apply_layer_device_impl(mps_state* h, int k, int ng, const int* sites, const double* d_Us) {
  int rc = validate_layer(h, k, ng, sites, d_Us);
  if (rc) return rc;
  if (ng == 0) return MPS_OK;
  rc = flush_pending(h);
  if (rc) return rc;
  const int d = 1 << k;
  if (k == 1) {
    if (!h->d_site || !h->h_site) {
      CK(dev_alloc((void**)&h->d_site, sizeof(SiteTask) * h->n));
      CK(dev_alloc((void**)&h->d_site_gates, sizeof(double2) * 4 * h->n));
      CK(host_alloc((void**)&h->h_site, sizeof(SiteTask) * h->n));
      CK(host_alloc((void**)&h->h_site_gates, sizeof(double2) * 4 * h->n));
    }
    CK(cudaStreamSynchronize(h->stream));
    int el_ub = 1;
    for (int g = 0; g < ng; ++g) {
      SiteTask st;
      st.g = site_ptr(h, sites[g]);
      st.chi = h->chi;
      st.site = sites[g];
      st.cap = h->cap;
      st.U = (const double2*)d_Us + 4 * g;
      h->h_site[g] = st;
      el_ub = std::max(el_ub, h->ub[sites[g]] * h->ub[sites[g] + 1]);
    }
    CK(cudaMemcpyAsync(h->d_site, h->h_site, sizeof(SiteTask) * ng, cudaMemcpyHostToDevice, h->stream));
    launch_apply1(h->d_site, ng, el_ub, h->stream);
    h->launches_all += 1;
    CK(cudaGetLastError());
    return MPS_OK;
  }
  std::vector<TaskRef> refs(ng);
  for (int g = 0; g < ng; ++g) refs[g] = TaskRef{h, sites[g]};
  return run_refs_chunked(h, k, refs, nullptr, (const double2*)d_Us, d * d);
}

// Gates of several MPS in shared batched passes (workspace and stream of hs[0]).
int apply_layer_multi_impl(int count, const mps_handle* hs, int k, const int* n_gates, const int* sites,
                           const double* Us) {
  if (count < 1 || !hs || !n_gates || !hs[0]) return fail(MPS_ERR_ARG, "bad arguments");
  if (k < 2 || k > 3) return fail(MPS_ERR_ARG, "k must be 2 or 3");
  mps_state* w = hs[0];
  const int d = 1 << k;
  size_t tot = 0;
  for (int i = 0; i < count; ++i) {
    if (!hs[i] || n_gates[i] < 0) return fail(MPS_ERR_ARG, "bad handle or gate count");
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return fail(MPS_ERR_ARG, "a handle appears twice");
    int rc = validate_layer(hs[i], k, n_gates[i], sites + tot, Us + (size_t)2 * d * d * tot);
    if (rc) return rc;
    tot += n_gates[i];
  }
  for (size_t g = 0; g < tot; ++g)
    if (!is_unitary(Us + (size_t)2 * d * d * g, d)) return fail(MPS_ERR_NOT_UNITARY, "gate is not unitary");
  for (int i = 1; i < count; ++i) CK(cudaStreamSynchronize(hs[i]->stream));
  std::vector<TaskRef> refs;
  std::vector<size_t> src;
  refs.reserve(tot);
  size_t g = 0;
  for (int i = 0; i < count; ++i)
    for (int j = 0; j < n_gates[i]; ++j, ++g) {
      refs.push_back(TaskRef{hs[i], sites[g]});
      src.push_back(g);
    }
  // largest problems first: grids of a pass are sized by its largest task
  std::vector<size_t> order(tot);
  for (size_t i = 0; i < tot; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
    return task_layout(refs[a], k, false).total > task_layout(refs[b], k, false).total;
  });
  std::vector<TaskRef> sorted(tot);
  std::vector<double2> hu((size_t)64 * tot);
  for (size_t i = 0; i < tot; ++i) {
    sorted[i] = refs[order[i]];
    fold_pending(sorted[i].st, sorted[i].site, k, Us + (size_t)2 * d * d * src[order[i]], hu.data() + 64 * i);
  }
  int rc = run_refs_chunked(w, k, sorted, hu.data(), nullptr, 0);
  if (rc) return rc;
  // later calls on the other handles' streams wait for this pass
  cudaEvent_t ev;
  CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  cudaEventRecord(ev, w->stream);
  for (int i = 1; i < count; ++i) cudaStreamWaitEvent(hs[i]->stream, ev, 0);
  cudaEventDestroy(ev);
  return MPS_OK;
}

// Deferred device errors: the sticky status word (d_counter[1]) set by kernels.
int collect_status(mps_state* h) {
  CK(cudaStreamSynchronize(h->stream));
  int st = 0;
  CK(cudaMemcpy(&st, h->d_counter + 1, sizeof(int), cudaMemcpyDeviceToHost));
  if (st == 0) return MPS_OK;
  CK(cudaMemset(h->d_counter + 1, 0, sizeof(int)));
  return fail(st, st == MPS_ERR_NOCONVERGE ? "Jacobi SVD did not converge (gate left unapplied)"
                                           : "device error");
}

int read_chi(mps_state* h, std::vector<int>& chi) {
  chi.resize(h->n + 1);
  CK(cudaMemcpyAsync(chi.data(), h->chi, sizeof(int) * (h->n + 1), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return MPS_OK;
}

// Readout workspace of the handle (grown on demand, kept until destroy).
int ensure_readout(mps_state* h, size_t elems) {
  const size_t bytes = elems * sizeof(double2);
  if (bytes <= h->ro_bytes) return MPS_OK;
  CK(cudaStreamSynchronize(h->stream));
  cudaFree(h->ro_buf);
  h->ro_buf = nullptr;
  h->ro_bytes = 0;
  CK(dev_alloc((void**)&h->ro_buf, bytes));
  h->ro_bytes = bytes;
  return MPS_OK;
}

// Largest working set of a reduced-density contraction (complex entries per
// environment buffer) and of its partial products.
constexpr size_t kRdoBudget = (size_t)1 << 27;

// Reduced density operator of `qubits` by transfer-matrix contraction of
// Eq. (1) (the tracing-out of Sec. 3.2). The environment runs from the end of
// the chain nearer to the listed qubits' far side (left to right or right to
// left, whichever holds fewer entries), opening a (ket, bra) index pair at
// every listed qubit: environments are blocks indexed by the open pairs so far.
int rdo_impl(mps_state* h, const int* qubits, int nq, std::vector<cd>& rho) {
  std::vector<int> pos(h->n, -1);
  for (int t = 0; t < nq; ++t) pos[qubits[t]] = t;
  int rc = flush_pending(h);
  if (rc) return rc;
  std::vector<int> chi;
  rc = read_chi(h, chi);
  if (rc) return rc;
  // working sets of both directions: environments (nblk * bond^2), partial
  // products (2 nblk xl xr), the scaled site (2 xl xr)
  auto sizes = [&](bool l2r, size_t& e_max, size_t& t_max, size_t& s_max) {
    e_max = t_max = s_max = 1;
    size_t nblk = 1;
    for (int k = 0; k < h->n; ++k) {
      const int s = l2r ? k : h->n - 1 - k;
      const size_t xl = chi[s], xr = chi[s + 1];
      const size_t in_b = l2r ? xl : xr, out_b = l2r ? xr : xl;
      t_max = std::max(t_max, (pos[s] >= 0 ? 2 : 1) * nblk * xl * xr);
      if (pos[s] >= 0) nblk *= 4;
      e_max = std::max(e_max, std::max(nblk * out_b * out_b, nblk * in_b * in_b));
      s_max = std::max(s_max, 2 * xl * xr);
    }
  };
  size_t e_l, t_l, s_l, e_r, t_r, s_r;
  sizes(true, e_l, t_l, s_l);
  sizes(false, e_r, t_r, s_r);
  const bool l2r = std::max(e_l, t_l) <= std::max(e_r, t_r);
  const size_t e_max = l2r ? e_l : e_r, t_max = l2r ? t_l : t_r, s_max = l2r ? s_l : s_r;
  if (e_max > kRdoBudget || t_max > kRdoBudget)
    return fail(MPS_ERR_TOO_LARGE, "reduced density: the contraction would hold more than 2^27 entries per buffer");
  if ((rc = ensure_readout(h, 2 * e_max + t_max + s_max))) return rc;
  double2* E0 = h->ro_buf;
  double2* E1 = E0 + e_max;
  double2* Tm = E1 + e_max;
  double2* Sc = Tm + t_max;
  const double2 one = make_double2(1.0, 0.0);
  CK(cudaMemcpyAsync(E0, &one, sizeof(double2), cudaMemcpyHostToDevice, h->stream));
  long long nblk = 1;
  std::vector<int> open;  // open sites in traversal order: block digit t (base 4, least significant first)
  for (int k = 0; k < h->n; ++k) {
    const int s = l2r ? k : h->n - 1 - k;
    const int xl = chi[s], xr = chi[s + 1];
    launch_scale_site(site_ptr(h, s), bond_ptr(h, s), xl, xr, h->cap, Sc, h->stream);
    const double2* A[2] = {Sc, Sc + (size_t)xl * xr};  // A_i[a][c] = Gamma_s[i][a][c] Lambda_s[c]
    if (l2r) {
      // E'[c][c'] = sum_{a a'} A_i[a][c] E[a][a'] conj(A_j[a'][c'])
      const long long sE = (long long)xl * xl, sT = (long long)xr * xl, sN = (long long)xr * xr;
      if (pos[s] < 0) {
        for (int i = 0; i < 2; ++i) {
          launch_zgemm(xr, xl, xl, A[i], xr, 0, 1, E0, xl, sE, 0, 0, Tm, xl, sT, 0, nblk, h->stream);
          launch_zgemm(xr, xr, xl, Tm, xl, sT, 0, A[i], xr, 0, 1, 0, E1, xr, sN, i, nblk, h->stream);
        }
      } else {
        for (int i = 0; i < 2; ++i)
          launch_zgemm(xr, xl, xl, A[i], xr, 0, 1, E0, xl, sE, 0, 0, Tm + (size_t)i * nblk * sT, xl, sT, 0, nblk,
                       h->stream);
        for (int i = 0; i < 2; ++i)
          for (int j = 0; j < 2; ++j)
            launch_zgemm(xr, xr, xl, Tm + (size_t)i * nblk * sT, xl, sT, 0, A[j], xr, 0, 1, 0,
                         E1 + (size_t)(i * 2 + j) * nblk * sN, xr, sN, 0, nblk, h->stream);
      }
    } else {
      // F'[a][a'] = sum_{c c'} A_i[a][c] F[c][c'] conj(A_j[a'][c'])
      const long long sF = (long long)xr * xr, sT = (long long)xl * xr, sN = (long long)xl * xl;
      if (pos[s] < 0) {
        for (int i = 0; i < 2; ++i) {
          launch_zgemm(xl, xr, xr, A[i], xr, 0, 0, E0, xr, sF, 0, 0, Tm, xr, sT, 0, nblk, h->stream);
          launch_zgemm(xl, xl, xr, Tm, xr, sT, 0, A[i], xr, 0, 1, 1, E1, xl, sN, i, nblk, h->stream);
        }
      } else {
        for (int i = 0; i < 2; ++i)
          launch_zgemm(xl, xr, xr, A[i], xr, 0, 0, E0, xr, sF, 0, 0, Tm + (size_t)i * nblk * sT, xr, sT, 0, nblk,
                       h->stream);
        for (int i = 0; i < 2; ++i)
          for (int j = 0; j < 2; ++j)
            launch_zgemm(xl, xl, xr, Tm + (size_t)i * nblk * sT, xr, sT, 0, A[j], xr, 0, 1, 1,
                         E1 + (size_t)(i * 2 + j) * nblk * sN, xl, sN, 0, nblk, h->stream);
      }
    }
    if (pos[s] >= 0) {
      nblk *= 4;
      open.push_back(s);
    }
    std::swap(E0, E1);
  }
  std::vector<double2> vals(nblk);
  cudaError_t ce = cudaMemcpyAsync(vals.data(), E0, sizeof(double2) * nblk, cudaMemcpyDeviceToHost, h->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
  if (ce == cudaSuccess) ce = cudaGetLastError();
  if (ce != cudaSuccess) return fail(MPS_ERR_CUDA, std::string("reduced density: ") + cudaGetErrorString(ce));
  const int dim = 1 << nq;
  rho.assign((size_t)dim * dim, cd(0));
  cd tr = 0;
  for (long long blk = 0; blk < nblk; ++blk) {
    int x = 0, y = 0;
    bool diag = true;
    for (int t = 0; t < nq; ++t) {
      const int pr = (int)((blk >> (2 * t)) & 3), i = pr >> 1, j = pr & 1;
      const int sh = nq - 1 - pos[open[t]];
      x |= i << sh;
      y |= j << sh;
      diag = diag && (i == j);
    }
    rho[(size_t)x * dim + y] = cd(vals[blk].x, vals[blk].y);
    if (diag) tr += cd(vals[blk].x, vals[blk].y);
  }
  for (cd& v : rho) v /= tr.real();
  return MPS_OK;
}

// --------------------------------------------------- sampling, Pauli strings ---

constexpr int kSampleChunk = 4096;  // samples per pass of the sequential sampler

// Bit strings by sequential conditional sampling of |<b|psi>|^2 / <psi|psi>:
// right environments R_s of the stored tensors (built once, right to left),
// then per site the weights of b_s = 0, 1 for every sample's chosen prefix
// (row vectors V, GEMM-shaped over the samples), the draw against the
// caller's uniform, and V renormalised.
int sample_impl(mps_state* h, int count, const double* u, unsigned char* bits) {
  int rc = flush_pending(h);
  if (rc) return rc;
  std::vector<int> chi;
  if ((rc = read_chi(h, chi))) return rc;
  const int n = h->n;
  std::vector<size_t> env_off(n + 1);
  size_t env_elems = 0, s_max = 1, t_max = 1;
  int x_max = 1;
  for (int s = 0; s <= n; ++s) {
    env_off[s] = env_elems;
    env_elems += (size_t)chi[s] * chi[s];
  }
  for (int s = 0; s < n; ++s) {
    s_max = std::max(s_max, (size_t)2 * chi[s] * chi[s + 1]);
    t_max = std::max(t_max, (size_t)chi[s] * chi[s + 1]);
    x_max = std::max(x_max, chi[s + 1]);
  }
  const int S = std::min(count, kSampleChunk);
  const size_t per = (size_t)S * x_max;
  const size_t u_elems = ((size_t)S * n * sizeof(double) + sizeof(double2) - 1) / sizeof(double2);
  const size_t b_elems = ((size_t)S * n + sizeof(double2) - 1) / sizeof(double2);
  if ((rc = ensure_readout(h, env_elems + s_max + t_max + 5 * per + u_elems + b_elems))) return rc;
  double2* env = h->ro_buf;
  double2* Sc = env + env_elems;
  double2* Tm = Sc + s_max;
  double2* V = Tm + t_max;
  double2* W[2] = {V + per, V + 2 * per};
  double2* T[2] = {V + 3 * per, V + 4 * per};
  double* d_u = reinterpret_cast<double*>(V + 5 * per);
  unsigned char* d_bits = reinterpret_cast<unsigned char*>(V + 5 * per + u_elems);
  // right environments: R_n = [1]; R_s = sum_i A_i R_{s+1} A_i^H, A_i = Gamma_s[i] Lambda_s
  launch_fill_one(env + env_off[n], 1, h->stream);
  for (int s = n - 1; s >= 0; --s) {
    const int xl = chi[s], xr = chi[s + 1];
    launch_scale_site(site_ptr(h, s), bond_ptr(h, s), xl, xr, h->cap, Sc, h->stream);
    for (int i = 0; i < 2; ++i) {
      const double2* Ai = Sc + (size_t)i * xl * xr;
      launch_zgemm(xl, xr, xr, Ai, xr, 0, 0, env + env_off[s + 1], xr, 0, 0, 0, Tm, xr, 0, 0, 1, h->stream);
      launch_zgemm(xl, xl, xr, Tm, xr, 0, 0, Ai, xr, 0, 1, 1, env + env_off[s], xl, 0, i, 1, h->stream);
    }
  }
  for (int c0 = 0; c0 < count; c0 += S) {
    const int m = std::min(S, count - c0);
    CK(cudaMemcpyAsync(d_u, u + (size_t)c0 * n, sizeof(double) * m * n, cudaMemcpyHostToDevice, h->stream));
    launch_fill_one(V, m, h->stream);  // V = [1] per sample (bond -1 has dimension 1)
    for (int s = 0; s < n; ++s) {
      const int xl = chi[s], xr = chi[s + 1];
      launch_scale_site(site_ptr(h, s), bond_ptr(h, s), xl, xr, h->cap, Sc, h->stream);
      for (int i = 0; i < 2; ++i) {
        launch_zgemm(m, xr, xl, V, xl, 0, 0, Sc + (size_t)i * xl * xr, xr, 0, 0, 0, W[i], xr, 0, 0, 1, h->stream);
        launch_zgemm(m, xr, xr, W[i], xr, 0, 0, env + env_off[s + 1], xr, 0, 0, 0, T[i], xr, 0, 0, 1, h->stream);
      }
      launch_sample_step(m, xr, W[0], W[1], T[0], T[1], d_u + s, n, d_bits + s, V, h->stream);
    }
    CK(cudaMemcpyAsync(bits + (size_t)c0 * n, d_bits, (size_t)m * n, cudaMemcpyDeviceToHost, h->stream));
  }
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaGetLastError());
  return MPS_OK;
}

// <psi|P|psi> / <psi|psi> for Pauli strings P: transfer contractions left to
// right with the Pauli matrix as the physical weight (and once with identities
// for the norm).
int pauli_impl(mps_state* h, int count, const char* ps, double* out) {
  int rc = flush_pending(h);
  if (rc) return rc;
  std::vector<int> chi;
  if ((rc = read_chi(h, chi))) return rc;
  const int n = h->n;
  size_t e_max = 1, s_max = 1;
  for (int s = 0; s < n; ++s) {
    e_max = std::max(e_max, (size_t)std::max(chi[s], chi[s + 1]) * std::max(chi[s], chi[s + 1]));
    s_max = std::max(s_max, (size_t)2 * chi[s] * chi[s + 1]);
  }
  if ((rc = ensure_readout(h, 5 * e_max + s_max))) return rc;
  double2* E0 = h->ro_buf;
  double2* E1 = E0 + e_max;
  double2* Tp[2] = {E1 + e_max, E1 + 2 * e_max};
  double2* Tc = E1 + 3 * e_max;
  double2* Sc = E1 + 4 * e_max;
  const double2 z = make_double2(0.0, 0.0), one = make_double2(1.0, 0.0), mone = make_double2(-1.0, 0.0);
  const double2 pi = make_double2(0.0, 1.0), mi = make_double2(0.0, -1.0);
  auto contract = [&](const char* p, double2* val) -> int {
    launch_fill_one(E0, 1, h->stream);
    for (int s = 0; s < n; ++s) {
      const int xl = chi[s], xr = chi[s + 1];
      launch_scale_site(site_ptr(h, s), bond_ptr(h, s), xl, xr, h->cap, Sc, h->stream);
      const double2* A[2] = {Sc, Sc + (size_t)xl * xr};
      // Tp_i = A_i^T E (xr x xl)
      for (int i = 0; i < 2; ++i) launch_zgemm(xr, xl, xl, A[i], xr, 0, 1, E0, xl, 0, 0, 0, Tp[i], xl, 0, 0, 1, h->stream);
      // E' = sum_j (sum_i P[j][i] Tp_i) conj(A_j): ket index i, bra index j
      const char c = p ? p[s] : 'I';
      double2 P[2][2] = {{one, z}, {z, one}};
      if (c == 'X') { P[0][0] = z; P[0][1] = one; P[1][0] = one; P[1][1] = z; }
      if (c == 'Y') { P[0][0] = z; P[0][1] = mi; P[1][0] = pi; P[1][1] = z; }
      if (c == 'Z') { P[1][1] = mone; }
      for (int j = 0; j < 2; ++j) {
        launch_combine2((long long)xr * xl, P[j][0], Tp[0], P[j][1], Tp[1], Tc, h->stream);
        launch_zgemm(xr, xr, xl, Tc, xl, 0, 0, A[j], xr, 0, 1, 0, E1, xr, 0, j, 1, h->stream);
      }
      std::swap(E0, E1);
    }
    CK(cudaMemcpyAsync(val, E0, sizeof(double2), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return MPS_OK;
  };
  double2 norm;
  if ((rc = contract(nullptr, &norm))) return rc;
  for (int q = 0; q < count; ++q) {
    double2 v;
    if ((rc = contract(ps + (size_t)q * n, &v))) return rc;
    out[2 * q] = v.x / norm.x;
    out[2 * q + 1] = v.y / norm.x;
  }
  CK(cudaGetLastError());
  return MPS_OK;
}

// ---------------------------------------------------------------- programs ---

constexpr int kProgMaxTasks = 512;  // gate tasks per recorded pass (bounds the split-GEMM buffers)

void free_program(mps_program* p) {
  if (!p) return;
  // the handles may already be destroyed (their stream with them): wait for
  // the whole device rather than touch them
  cudaDeviceSynchronize();
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  cudaFree(p->mem);
  cudaFree(p->arena);
  cudaFree(p->oz.base);
  cudaFree(p->d_jobs);
  if (p->side) cudaStreamDestroy(p->side);
  delete p;
}

// Upper bound of the split-GEMM buffers one pass needs (every product of the
// split SVD, and theta for two-site gates, at the pass's bounds).
size_t oz_bytes_for_pass(const std::vector<TaskRef>& refs, int k) {
  int xl_ub = 1, x0_ub = 1, xr_ub = 1, nw_ub = 1, cap_ub = 1;
  for (const TaskRef& r : refs) {
    const mps_state* h = r.st;
    xl_ub = std::max(xl_ub, h->ub[r.site]);
    x0_ub = std::max(x0_ub, h->ub[r.site + 1]);
    xr_ub = std::max(xr_ub, h->ub[r.site + k]);
    cap_ub = std::max(cap_ub, h->cap);
    nw_ub = std::max(nw_ub, std::min(2 * h->ub[r.site], (k == 3 ? 4 : 2) * h->ub[r.site + k]));
  }
  const int mw_ub = k == 3 ? std::max(2 * xl_ub, 4 * xr_ub) : std::max(2 * xl_ub, 2 * xr_ub);
  const int M = std::max(std::max(2 * xl_ub, mw_ub), nw_ub);
  const int N = std::max(2 * xr_ub, nw_ub);
  const int K = std::min(512, std::max(std::max(x0_ub, nw_ub), mw_ub));
  return OzBuffers::bytes_needed((int)refs.size(), M, N, K, 8);
}

int program_create(int count, const mps_handle* hs, int n_passes, const int* k, const int* n_gates, const int* sites,
                   const int* owners, const double* d_Us, mps_program** out) {
  if (!out) return fail(MPS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (count < 1 || !hs || n_passes < 0 || (n_passes > 0 && (!k || !n_gates || !sites || !d_Us)))
    return fail(MPS_ERR_ARG, "bad arguments");
  if (count > 1 && !owners) return fail(MPS_ERR_ARG, "owners is NULL for several handles");
  for (int i = 0; i < count; ++i) {
    if (!hs[i]) return fail(MPS_ERR_ARG, "NULL handle");
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return fail(MPS_ERR_ARG, "a handle appears twice");
  }
  mps_state* w = hs[0];
  // ---- the passes, validated per handle
  size_t tot = 0, gate_doubles = 0;
  std::vector<size_t> gate_off(n_passes);
  for (int p = 0; p < n_passes; ++p) {
    if (k[p] < 1 || k[p] > 3 || n_gates[p] < 0) return fail(MPS_ERR_ARG, "bad pass");
    std::vector<std::vector<char>> used(count);
    for (int i = 0; i < count; ++i) used[i].assign(hs[i]->n, 0);
    for (int g = 0; g < n_gates[p]; ++g) {
      const int o = owners ? owners[tot + g] : 0, s0 = sites[tot + g];
      if (o < 0 || o >= count) return fail(MPS_ERR_ARG, "owner out of range");
      if (s0 < 0 || s0 + k[p] > hs[o]->n) return fail(MPS_ERR_ARG, "gate site out of range");
      for (int j = 0; j < k[p]; ++j) {
        if (used[o][s0 + j]) return fail(MPS_ERR_ARG, "gates of a pass overlap");
        used[o][s0 + j] = 1;
      }
    }
    gate_off[p] = gate_doubles;
    gate_doubles += (size_t)n_gates[p] * 2 * (1 << k[p]) * (1 << k[p]);
    tot += n_gates[p];
  }
  mps_program* P = new mps_program();
  P->hs.assign(hs, hs + count);
  P->split = w->prec == MPS_PREC_SPLIT;
  for (int i = 0; i < count; ++i) P->split = P->split && hs[i]->cap <= kSplitMaxCap;
  for (int i = 0; i < count; ++i) P->ub_start.push_back(hs[i]->ub);
  auto restore_ub = [&]() {
    for (int i = 0; i < count; ++i) hs[i]->ub = P->ub_start[i];
  };
  auto bad = [&](int rc) {
    restore_ub();
    free_program(P);
    return rc;
  };
  // ---- planning: chunks, their bounds, the workspace they need
  size_t g0 = 0, arena_max = 0, oz_max = 0, table_bytes = 0;
  int tasks_max = 1;
  for (int p = 0; p < n_passes; ++p) {
    std::vector<TaskRef> refs;
    std::vector<int> own, st;
    for (int g = 0; g < n_gates[p]; ++g) {
      const int o = owners ? owners[g0 + g] : 0;
      refs.push_back(TaskRef{hs[o], sites[g0 + g]});
      own.push_back(o);
      st.push_back(sites[g0 + g]);
    }
    g0 += n_gates[p];
    for (size_t c0 = 0; c0 < refs.size();) {
      size_t c1 = c0, bytes = 0;
      while (c1 < refs.size() && (int)(c1 - c0) < kProgMaxTasks) {
        const size_t b = k[p] >= 2 ? task_layout(refs[c1], k[p], P->split).total : 0;
        if (c1 > c0 && bytes + b > kArenaBudget) break;
        bytes += b;
        ++c1;
      }
      mps_program::Chunk ch;
      ch.k = k[p];
      ch.owner.assign(own.begin() + c0, own.begin() + c1);
      ch.site.assign(st.begin() + c0, st.begin() + c1);
      std::vector<TaskRef> part(refs.begin() + c0, refs.begin() + c1);
      if (k[p] >= 2) {
        arena_max = std::max(arena_max, bytes);
        if (P->split) oz_max = std::max(oz_max, oz_bytes_for_pass(part, k[p]));
        tasks_max = std::max(tasks_max, (int)part.size());
        table_bytes += align256(sizeof(GateTask) * part.size()) + align256(sizeof(TaskMeta) * part.size());
        advance_bounds(part, k[p]);
        P->updates += (long long)part.size();
      } else {
        table_bytes += align256(sizeof(SiteTask) * part.size());
      }
      P->chunks.push_back(ch);
      c0 = c1;
    }
  }
  for (int i = 0; i < count; ++i) P->ub_end.push_back(hs[i]->ub);
  restore_ub();
  // ---- memory: gates, tables, workspace, split-GEMM buffers
  const size_t gate_bytes = align256(sizeof(double) * std::max<size_t>(gate_doubles, 2));
  cudaError_t e = dev_alloc(&P->mem, gate_bytes + table_bytes + 256);
  if (e == cudaSuccess && arena_max) e = dev_alloc(&P->arena, arena_max);
  if (e == cudaSuccess && oz_max) e = dev_alloc(&P->oz.base, oz_max);
  if (e == cudaSuccess && P->split) e = dev_alloc((void**)&P->d_jobs, sizeof(OzJob) * tasks_max);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->side, cudaStreamNonBlocking);
  if (e != cudaSuccess)
    return bad(fail(e == cudaErrorMemoryAllocation ? MPS_ERR_NOMEM : MPS_ERR_CUDA,
                    std::string("program memory: ") + cudaGetErrorString(e)));
  P->arena_bytes = arena_max;
  P->oz.bytes = oz_max;
  P->jobs_cap = tasks_max;
  if (!w->d_oz_err) {
    if ((e = dev_alloc((void**)&w->d_oz_err, sizeof(int))) != cudaSuccess || (e = cudaMemset(w->d_oz_err, 0, sizeof(int))) != cudaSuccess)
      return bad(fail(MPS_ERR_NOMEM, "split GEMM error word"));
  }
  double2* gates = static_cast<double2*>(P->mem);
  if (gate_doubles &&
      (e = cudaMemcpy(gates, d_Us, sizeof(double) * gate_doubles, cudaMemcpyDeviceToDevice)) != cudaSuccess)
    return bad(fail(MPS_ERR_CUDA, std::string("copying the gates: ") + cudaGetErrorString(e)));
  // ---- task tables (built with the bounds each chunk will see)
  unsigned char* tab = static_cast<unsigned char*>(P->mem) + gate_bytes;
  {
    size_t ci = 0, gsum = 0;
    for (int p = 0; p < n_passes; ++p) {
      const int d = 1 << k[p];
      size_t in_pass = 0;
      while (in_pass < (size_t)n_gates[p]) {
        mps_program::Chunk& ch = P->chunks[ci++];
        const size_t ng = ch.site.size();
        const double2* gU = gates + gate_off[p] / 2 + (size_t)d * d * in_pass;
        std::vector<TaskRef> refs;
        for (size_t g = 0; g < ng; ++g) refs.push_back(TaskRef{hs[ch.owner[g]], ch.site[g]});
        if (ch.k >= 2) {
          std::vector<GateTask> ht(ng);
          build_tasks(w, ch.k, refs, gU, d * d, P->split, static_cast<unsigned char*>(P->arena), ht.data());
          ch.d_tasks = reinterpret_cast<GateTask*>(tab);
          tab += align256(sizeof(GateTask) * ng);
          ch.d_meta = reinterpret_cast<TaskMeta*>(tab);
          tab += align256(sizeof(TaskMeta) * ng);
          if ((e = cudaMemcpy(ch.d_tasks, ht.data(), sizeof(GateTask) * ng, cudaMemcpyHostToDevice)) != cudaSuccess ||
              (e = cudaMemset(ch.d_meta, 0, sizeof(TaskMeta) * ng)) != cudaSuccess)
            return bad(fail(MPS_ERR_CUDA, "task tables"));
          advance_bounds(refs, ch.k);
        } else {
          std::vector<SiteTask> hsite(ng);
          for (size_t g = 0; g < ng; ++g) {
            mps_state* h = refs[g].st;
            hsite[g].g = site_ptr(h, refs[g].site);
            hsite[g].chi = h->chi;
            hsite[g].site = refs[g].site;
            hsite[g].cap = h->cap;
            hsite[g].U = gU + 4 * g;
          }
          ch.d_site = reinterpret_cast<SiteTask*>(tab);
          tab += align256(sizeof(SiteTask) * ng);
          if ((e = cudaMemcpy(ch.d_site, hsite.data(), sizeof(SiteTask) * ng, cudaMemcpyHostToDevice)) != cudaSuccess)
            return bad(fail(MPS_ERR_CUDA, "site tables"));
        }
        in_pass += ng;
        gsum += ng;
      }
    }
    (void)gsum;
  }
  restore_ub();
  // ---- record: every launch of every chunk into one graph on the worker's stream
  jacobi_f32_prepare();
  rot_tc_prepare();
  if (ozaki_prepare()) return bad(fail(MPS_ERR_CUDA, "split GEMM set-up"));
  int rc = flush_pending(w);
  for (int i = 1; i < count && !rc; ++i) rc = flush_pending(hs[i]);
  if (rc) return bad(rc);
  for (int i = 0; i < count; ++i)
    if ((e = cudaStreamSynchronize(hs[i]->stream)) != cudaSuccess) return bad(fail(MPS_ERR_CUDA, "stream sync"));
  GateTask* saved_tasks = w->d_tasks;
  TaskMeta* saved_meta = w->d_meta;
  void* saved_arena = w->arena;
  const size_t saved_arena_bytes = w->arena_bytes;
  OzJob* saved_jobs = w->d_oz_jobs;
  const int saved_oz_cap = w->oz_cap;
  const OzBuffers saved_oz = w->oz_buf;
  const int saved_prof = w->prof;
  const int saved_ntask = w->last_ntask;
  const long long saved_launches = w->launches_all;
  w->arena = P->arena;
  w->arena_bytes = P->arena_bytes;
  w->d_oz_jobs = P->d_jobs;
  w->oz_cap = P->jobs_cap;
  w->oz_buf = P->oz;
  w->prof = 0;
  w->side = P->side;
  w->capturing = 1;
  e = cudaStreamBeginCapture(w->stream, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    for (const mps_program::Chunk& ch : P->chunks) {
      std::vector<TaskRef> refs;
      for (size_t g = 0; g < ch.site.size(); ++g) refs.push_back(TaskRef{hs[ch.owner[g]], ch.site[g]});
      if (ch.k == 1) {
        int el_ub = 1;
        for (const TaskRef& r : refs) el_ub = std::max(el_ub, r.st->ub[r.site] * r.st->ub[r.site + 1]);
        launch_apply1(ch.d_site, (int)refs.size(), el_ub, w->stream);
      } else {
        w->d_tasks = ch.d_tasks;
        w->d_meta = ch.d_meta;
        rc = emit_pass(w, ch.k, refs, P->split);
        if (rc) break;
      }
    }
    const cudaError_t ee = cudaStreamEndCapture(w->stream, &P->graph);
    if (!rc && ee != cudaSuccess) rc = fail(MPS_ERR_CUDA, std::string("recording: ") + cudaGetErrorString(ee));
  } else {
    rc = fail(MPS_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
  }
  w->capturing = 0;
  w->side = nullptr;
  w->d_tasks = saved_tasks;
  w->d_meta = saved_meta;
  w->arena = saved_arena;
  w->arena_bytes = saved_arena_bytes;
  w->d_oz_jobs = saved_jobs;
  w->oz_cap = saved_oz_cap;
  w->oz_buf = saved_oz;
  w->prof = saved_prof;
  w->last_ntask = saved_ntask;
  P->recorded_launches = w->launches_all - saved_launches;
  w->launches_all = saved_launches;
  restore_ub();
  cudaGetLastError();
  if (rc) return bad(rc);
  if ((e = cudaGraphInstantiate(&P->exec, P->graph, 0)) != cudaSuccess)
    return bad(fail(MPS_ERR_CUDA, std::string("graph instantiation: ") + cudaGetErrorString(e)));
  *out = P;
  return MPS_OK;
}

int program_run(mps_program* P) {
  if (!P) return fail(MPS_ERR_ARG, "NULL program");
  const int count = (int)P->hs.size();
  for (int i = 0; i < count; ++i) {
    const mps_state* h = P->hs[i];
    for (int b = 0; b <= h->n; ++b)
      if (h->ub[b] > P->ub_start[i][b])
        return fail(MPS_ERR_ARG, "a bond is above the bound the program was recorded with (reset the state)");
  }
  for (int i = 0; i < count; ++i) {
    const int rc = flush_pending(P->hs[i]);
    if (rc) return rc;
  }
  mps_state* w = P->hs[0];
  cudaEvent_t ev;
  CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  for (int i = 1; i < count; ++i) {
    cudaEventRecord(ev, P->hs[i]->stream);
    cudaStreamWaitEvent(w->stream, ev, 0);
  }
  const cudaError_t e = cudaGraphLaunch(P->exec, w->stream);
  if (e == cudaSuccess) {
    cudaEventRecord(ev, w->stream);
    for (int i = 1; i < count; ++i) cudaStreamWaitEvent(P->hs[i]->stream, ev, 0);
  }
  cudaEventDestroy(ev);
  if (e != cudaSuccess) return fail(MPS_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
  for (int i = 0; i < count; ++i) {
    P->hs[i]->ub = P->ub_end[i];
    P->hs[i]->last_ntask = 0;
  }
  w->launches_all += P->recorded_launches;
  return MPS_OK;
}

}  // namespace

// ================================================================= C ABI ===

extern "C" {

const char* mps_last_error(void) { return g_err.c_str(); }

int mps_create(int n, int chi_max, double cutoff, mps_handle* out) {
  if (!out) return fail(MPS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n < 1 || n > 4096) return fail(MPS_ERR_ARG, "n out of range");
  if (chi_max < 1 || chi_max > kMaxCap) return fail(MPS_ERR_ARG, "chi_max out of range");
  if (!(cutoff >= 0.0) || !std::isfinite(cutoff)) return fail(MPS_ERR_ARG, "cutoff must be finite and >= 0");
  mps_state* h = new mps_state();
  h->n = n;
  h->cap = chi_max;
  h->cutoff = cutoff;
  h->pend.assign(n, std::array<cd, 4>{1.0, 0.0, 0.0, 1.0});
  h->has_pend.assign(n, 0);
  auto bad = [&](cudaError_t e) {
    const int code = e == cudaErrorMemoryAllocation ? MPS_ERR_NOMEM : MPS_ERR_CUDA;
    g_err = std::string("mps_create: ") + cudaGetErrorString(e);
    free_state(h);
    return code;
  };
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking)) != cudaSuccess) return bad(e);
  h->stream = h->own;
  if ((e = dev_alloc((void**)&h->gamma, sizeof(double2) * gamma_elems(h))) != cudaSuccess) return bad(e);
  if ((e = dev_alloc((void**)&h->lambda, sizeof(double) * (size_t)(n + 1) * chi_max)) != cudaSuccess) return bad(e);
  if ((e = dev_alloc((void**)&h->chi, sizeof(int) * (n + 1))) != cudaSuccess) return bad(e);
  // words 0-2: active count, sticky status, loop iteration; 4-7: the scheduled fp32 sweeps' counters
  if ((e = dev_alloc((void**)&h->d_counter, 8 * sizeof(int))) != cudaSuccess) return bad(e);
  if ((e = cudaMemset(h->d_counter, 0, 8 * sizeof(int))) != cudaSuccess) return bad(e);
  if ((e = host_alloc((void**)&h->h_counter, sizeof(int))) != cudaSuccess) return bad(e);
  int rc = reset_state(h);
  if (rc) { free_state(h); return rc; }
  if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return bad(e);
  *out = h;
  return MPS_OK;
}

int mps_destroy(mps_handle h) {
  free_state(h);
  return MPS_OK;
}

int mps_set_stream(mps_handle h, void* s) {
  if (!h) return fail(MPS_ERR_ARG, "NULL handle");
  CK(cudaStreamSynchronize(h->stream));
  h->stream = s ? (cudaStream_t)s : h->own;
  return MPS_OK;
}

int mps_set_mode(mps_handle h, int prec, int slices, int svd_mode) {
  if (!h) return fail(MPS_ERR_ARG, "NULL handle");
  if (prec != MPS_PREC_FP64 && prec != MPS_PREC_SPLIT) return fail(MPS_ERR_ARG, "unknown precision mode");
  if (slices != 0 && (slices < 3 || slices > 8)) return fail(MPS_ERR_ARG, "slices must be 0 or 3..8");
  if (svd_mode != MPS_SVD_JACOBI && svd_mode != MPS_SVD_SKETCH_MLP) return fail(MPS_ERR_ARG, "unknown svd_mode");
  CK(cudaStreamSynchronize(h->stream));
  h->prec = prec;
  h->slices = slices ? slices : 8;
  h->svd_mode = svd_mode;
  return MPS_OK;
}

int mps_set_limits(mps_handle h, int max_sweeps) {
  if (!h) return fail(MPS_ERR_ARG, "NULL handle");
  if (max_sweeps < 1 || max_sweeps > kMaxSweeps) return fail(MPS_ERR_ARG, "max_sweeps must be 1..60");
  CK(cudaStreamSynchronize(h->stream));
  h->max_sweeps = max_sweeps;
  return MPS_OK;
}

int mps_set_tuning(mps_handle h, int n, const int* nw_max, const int* f32_block, const int* f32_mode) {
  if (!h) return fail(MPS_ERR_ARG, "NULL handle");
  if (n < 0 || (n > 0 && (!nw_max || !f32_block || !f32_mode))) return fail(MPS_ERR_ARG, "bad table");
  std::vector<mps_state::Tune> t(n);
  for (int i = 0; i < n; ++i) {
    if (f32_block[i] != 8 && f32_block[i] != 16) return fail(MPS_ERR_ARG, "fp32 block width must be 8 or 16");
    if (f32_mode[i] < kF32ModePair || f32_mode[i] > kF32ModeSchedWide)
      return fail(MPS_ERR_ARG, "fp32 mode must be 0, 1, 2 or 3");
    if (f32_mode[i] == kF32ModeTc && f32_block[i] != 16)
      return fail(MPS_ERR_ARG, "the tensor-core rotation needs block width 16");
    if (i > 0 && nw_max[i] <= nw_max[i - 1]) return fail(MPS_ERR_ARG, "widths must increase");
    t[i] = mps_state::Tune{nw_max[i], f32_block[i], f32_mode[i]};
  }
  CK(cudaStreamSynchronize(h->stream));
  h->tune = t;
  return MPS_OK;
}

int mps_debug_fail_alloc(long long after) {
  g_alloc_left.store(after < 0 ? -1 : after);
  return MPS_OK;
}

int mps_debug_mark_timed_out(mps_handle h) {
  if (!h) return fail(MPS_ERR_ARG, "null handle");
  h->oz_timed_out = 1;  // as a bounded wait of the split GEMM that ran out would
  return MPS_OK;
}

int mps_reset(mps_handle h) {
  if (!h) return fail(MPS_ERR_ARG, "NULL handle");
  return reset_state(h);
}

int mps_apply_gate(mps_handle h, int site, int k, const double* U) {
  if (!h) return fail(MPS_ERR_ARG, "NULL handle");
  return apply_layer_impl(h, k, 1, &site, U);
}

int mps_apply_layer(mps_handle h, int k, int n_gates, const int* sites, const double* Us) {
  if (!h) return fail(MPS_ERR_ARG, "NULL handle");
  return apply_layer_impl(h, k, n_gates, sites, Us);
}

int mps_apply_layer_device(mps_handle h, int k, int n_gates, const int* sites, const double* d_Us) {
  if (!h) return fail(MPS_ERR_ARG, "NULL handle");
  return apply_layer_device_impl(h, k, n_gates, sites, d_Us);
}

int mps_apply_layer_multi(int count, const mps_handle* handles, int k, const int* n_gates, const int* sites,
                          const double* Us) {
  return apply_layer_multi_impl(count, handles, k, n_gates, sites, Us);
}

int mps_layer_features(mps_handle h, int k, int n_gates, const int* sites, const double* Us, float* X) {
  if (!h) return fail(MPS_ERR_ARG, "NULL handle");
  if (k != 2) return fail(MPS_ERR_ARG, "features are defined for two-site gates");
  int rc = validate_layer(h, k, n_gates, sites, Us);
  if (rc) return rc;
  if (n_gates == 0) return MPS_OK;
  if (!X) return fail(MPS_ERR_ARG, "X is NULL");
  std::vector<FeatureTask> ft(n_gates);
  for (int g = 0; g < n_gates; ++g) {
    FeatureTask f;
    f.lamL = bond_ptr(h, sites[g] - 1);
    f.lamR = bond_ptr(h, sites[g] + 1);
    f.chi = h->chi;
    f.site = sites[g];
    f.k = 2;
    f.ep = (float)entangling_power(Us + 32 * g);
    f.cutoff = h->cutoff;
    ft[g] = f;
  }
  FeatureTask* d_ft = nullptr;
  float* d_x = nullptr;
  CK(dev_alloc((void**)&d_ft, sizeof(FeatureTask) * n_gates));
  if (dev_alloc((void**)&d_x, sizeof(float) * 16 * n_gates) != cudaSuccess) {
    cudaFree(d_ft);
    return fail(MPS_ERR_NOMEM, "feature buffer");
  }
  cudaError_t e = cudaMemcpyAsync(d_ft, ft.data(), sizeof(FeatureTask) * n_gates, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) {
    launch_features(d_ft, n_gates, d_x, h->stream);
    e = cudaMemcpyAsync(X, d_x, sizeof(float) * 16 * n_gates, cudaMemcpyDeviceToHost, h->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(d_ft);
  cudaFree(d_x);
  return e == cudaSuccess ? MPS_OK : fail(MPS_ERR_CUDA, "features");
}

int mps_apply_gate_on(mps_handle h, int nq, const int* qubits, const double* U, int route) {
  if (!h || !qubits || !U) return fail(MPS_ERR_ARG, "bad arguments");
  if (nq < 1 || nq > 2) return fail(MPS_ERR_ARG, "nq must be 1 or 2");
  if (route != 0 && route != 1) return fail(MPS_ERR_ARG, "route must be 0 or 1");
  for (int t = 0; t < nq; ++t)
    if (qubits[t] < 0 || qubits[t] >= h->n) return fail(MPS_ERR_ARG, "qubit out of range");
  if (nq == 1) return apply_layer_impl(h, 1, 1, qubits, U);
  const int a = qubits[0], b = qubits[1];
  if (a == b) return fail(MPS_ERR_ARG, "the two qubits must differ");
  if (!is_unitary(U, 4)) return fail(MPS_ERR_NOT_UNITARY, "gate is not unitary");
  // the gate with its index bits in increasing qubit order: V = S U S when
  // the first listed qubit is the higher one (S swaps the two index bits)
  double V[32];
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      const int rr = a < b ? r : ((r & 1) << 1 | r >> 1), cc = a < b ? c : ((c & 1) << 1 | c >> 1);
      V[2 * (r * 4 + c)] = U[2 * (rr * 4 + cc)];
      V[2 * (r * 4 + c) + 1] = U[2 * (rr * 4 + cc) + 1];
    }
  const int lo = std::min(a, b), hi = std::max(a, b), d = hi - lo;
  if (d == 1) return apply_layer_impl(h, 2, 1, &lo, V);
  if (d == 2 && route == 0) {
    // U(8) on (lo, lo+1, lo+2) with the identity on the middle qubit
    double W[128];
    std::memset(W, 0, sizeof(W));
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j)
        for (int k = 0; k < 2; ++k)
          for (int l = 0; l < 2; ++l)
            for (int m = 0; m < 2; ++m) {
              const int r = i * 4 + m * 2 + j, c = k * 4 + m * 2 + l, src = (i * 2 + j) * 4 + (k * 2 + l);
              W[2 * (r * 8 + c)] = V[2 * src];
              W[2 * (r * 8 + c) + 1] = V[2 * src + 1];
            }
    return apply_layer_impl(h, 3, 1, &lo, W);
  }
  // SWAP updates carry qubit hi down to lo+1, the gate acts there, and SWAPs
  // carry it back (each SWAP is a two-site update with its own truncation)
  static const double S[32] = {1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0, 0, 0,
                               0, 0, 1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0};
  int rc;
  for (int t = hi - 1; t > lo; --t)
    if ((rc = apply_layer_impl(h, 2, 1, &t, S))) return rc;
  if ((rc = apply_layer_impl(h, 2, 1, &lo, V))) return rc;
  for (int t = lo + 1; t < hi; ++t)
    if ((rc = apply_layer_impl(h, 2, 1, &t, S))) return rc;
  return MPS_OK;
}

int mps_set_predictor(mps_handle h, mps_mlp_handle m) {
  if (!h) return fail(MPS_ERR_ARG, "NULL handle");
  h->predictor = m;
  return MPS_OK;
}

int mps_sketch_stats(mps_handle h, long long* sketched, long long* accepted, long long* routed_full) {
  if (!h) return fail(MPS_ERR_ARG, "NULL handle");
  if (sketched) *sketched = h->sk_sketched;
  if (accepted) *accepted = h->sk_accepted;
  if (routed_full) *routed_full = h->sk_routed;
  return MPS_OK;
}

int mps_profile(mps_handle h, int enable) {
  if (!h) return fail(MPS_ERR_ARG, "NULL handle");
  CK(cudaStreamSynchronize(h->stream));
  if (!h->d_prof_flops) CK(dev_alloc((void**)&h->d_prof_flops, kProfKinds * sizeof(unsigned long long)));
  CK(cudaMemset(h->d_prof_flops, 0, kProfKinds * sizeof(unsigned long long)));
  h->prof = enable ? 1 : 0;
  h->ev_next = 0;
  h->prof_rec.clear();
  for (int i = 0; i < kProfKinds; ++i) {
    h->prof_flops_host[i] = 0.0;
    h->prof_launch[i] = 0;
  }
  h->launches_all = 0;
  return MPS_OK;
}

int mps_profile_read(mps_handle h, int kernel, double* ms, long long* launches, double* flops,
                     long long* launches_all) {
  if (!h || kernel < 0 || kernel >= kProfKinds) return fail(MPS_ERR_ARG, "bad arguments");
  CK(cudaStreamSynchronize(h->stream));
  double tot = 0.0;
  for (const auto& r : h->prof_rec) {
    if (r[0] != kernel) continue;
    float m = 0.f;
    CK(cudaEventElapsedTime(&m, h->evs[r[1]], h->evs[r[2]]));
    tot += m;
  }
  unsigned long long dev[kProfKinds] = {0, 0, 0, 0, 0, 0};
  if (h->d_prof_flops) CK(cudaMemcpy(dev, h->d_prof_flops, sizeof(dev), cudaMemcpyDeviceToHost));
  if (ms) *ms = tot;
  if (launches) *launches = h->prof_launch[kernel];
  if (flops) *flops = (double)dev[kernel] + h->prof_flops_host[kernel];
  if (launches_all) *launches_all = h->launches_all;
  return MPS_OK;
}

int mps_amplitudes(mps_handle h, int count, const unsigned char* bits, double* out) {
  if (!h || !bits || !out || count < 0) return fail(MPS_ERR_ARG, "bad arguments");
  if (count == 0) return MPS_OK;
  int rc = flush_pending(h);
  if (rc) return rc;
  unsigned char* d_bits = nullptr;
  double2* d_out = nullptr;
  CK(dev_alloc((void**)&d_bits, (size_t)count * h->n));
  if (dev_alloc((void**)&d_out, sizeof(double2) * count) != cudaSuccess) {
    cudaFree(d_bits);
    return fail(MPS_ERR_NOMEM, "amplitude buffers");
  }
  cudaError_t e = cudaMemcpyAsync(d_bits, bits, (size_t)count * h->n, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) {
    launch_amplitudes(h->gamma, h->lambda, h->chi, h->n, h->cap, d_bits, count, d_out, h->stream);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_out, sizeof(double2) * count, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(d_bits);
  cudaFree(d_out);
  if (e != cudaSuccess) return fail(MPS_ERR_CUDA, std::string("amplitudes: ") + cudaGetErrorString(e));
  return collect_status(h);
}

int mps_amplitude(mps_handle h, const unsigned char* bits, double* out) { return mps_amplitudes(h, 1, bits, out); }

int mps_reduced_density(mps_handle h, const int* qubits, int nq, double* rho) {
  if (!h || !qubits || !rho) return fail(MPS_ERR_ARG, "bad arguments");
  if (nq < 1) return fail(MPS_ERR_ARG, "nq must be >= 1");
  if (nq > 12) return fail(MPS_ERR_TOO_LARGE, "nq > 12");
  std::vector<char> seen(h->n, 0);
  for (int t = 0; t < nq; ++t) {
    if (qubits[t] < 0 || qubits[t] >= h->n || seen[qubits[t]]) return fail(MPS_ERR_ARG, "bad qubit list");
    seen[qubits[t]] = 1;
  }
  std::vector<cd> r;
  int rc = rdo_impl(h, qubits, nq, r);
  if (rc) return rc;
  for (size_t e = 0; e < r.size(); ++e) {
    rho[2 * e] = r[e].real();
    rho[2 * e + 1] = r[e].imag();
  }
  return collect_status(h);
}

int mps_expectation(mps_handle h, int site, int k, const double* O, double* out) {
  if (!h || !O || !out) return fail(MPS_ERR_ARG, "bad arguments");
  if (k < 1 || k > 3 || site < 0 || site + k > h->n) return fail(MPS_ERR_ARG, "operator range");
  int q[3];
  for (int j = 0; j < k; ++j) q[j] = site + j;
  std::vector<cd> r;
  int rc = rdo_impl(h, q, k, r);
  if (rc) return rc;
  const int d = 1 << k;
  cd acc = 0;
  for (int x = 0; x < d; ++x)
    for (int y = 0; y < d; ++y) acc += r[(size_t)x * d + y] * cd(O[2 * (y * d + x)], O[2 * (y * d + x) + 1]);
  out[0] = acc.real();
  out[1] = acc.imag();
  return collect_status(h);
}

int mps_sample(mps_handle h, int count, const double* u, unsigned char* bits) {
  if (!h || count < 0 || (count > 0 && (!u || !bits))) return fail(MPS_ERR_ARG, "bad arguments");
  if (count == 0) return MPS_OK;
  for (size_t e = 0; e < (size_t)count * h->n; ++e)
    if (!(u[e] >= 0.0 && u[e] < 1.0)) return fail(MPS_ERR_ARG, "uniforms must lie in [0, 1)");
  int rc = sample_impl(h, count, u, bits);
  if (rc) return rc;
  return collect_status(h);
}

int mps_pauli_expectations(mps_handle h, int count, const char* paulis, double* out) {
  if (!h || count < 0 || (count > 0 && (!paulis || !out))) return fail(MPS_ERR_ARG, "bad arguments");
  for (size_t e = 0; e < (size_t)count * h->n; ++e) {
    const char c = paulis[e];
    if (c != 'I' && c != 'X' && c != 'Y' && c != 'Z') return fail(MPS_ERR_ARG, "Pauli strings use I, X, Y, Z");
  }
  if (count == 0) return MPS_OK;
  int rc = pauli_impl(h, count, paulis, out);
  if (rc) return rc;
  return collect_status(h);
}

int mps_get_schmidt(mps_handle h, int bond, double* lambda, int* len) {
  if (!h || !lambda || !len) return fail(MPS_ERR_ARG, "bad arguments");
  if (bond < 0 || bond > h->n - 2) return fail(MPS_ERR_ARG, "bond out of range");
  int c = 0;
  CK(cudaMemcpyAsync(&c, h->chi + bond + 1, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaMemcpy(lambda, bond_ptr(h, bond), sizeof(double) * c, cudaMemcpyDeviceToHost));
  *len = c;
  return collect_status(h);
}

int mps_bond_dims(mps_handle h, int* chi) {
  if (!h || !chi) return fail(MPS_ERR_ARG, "bad arguments");
  std::vector<int> c;
  int rc = read_chi(h, c);
  if (rc) return rc;
  for (int b = 0; b < h->n - 1; ++b) chi[b] = c[b + 1];
  return collect_status(h);
}

int mps_export(mps_handle h, int* chi, double* gammas, double* lambdas) {
  if (!h || !chi) return fail(MPS_ERR_ARG, "bad arguments");
  int rc = flush_pending(h);
  if (rc) return rc;
  std::vector<int> c;
  rc = read_chi(h, c);
  if (rc) return rc;
  for (int b = 0; b <= h->n; ++b) chi[b] = c[b];
  if (gammas) {
    size_t off = 0;
    for (int s = 0; s < h->n; ++s)
      for (int i = 0; i < 2; ++i) {
        const size_t xl = c[s], xr = c[s + 1];
        CK(cudaMemcpy2DAsync(gammas + 2 * off, xr * sizeof(double2), site_ptr(h, s) + (size_t)i * h->cap * h->cap,
                             h->cap * sizeof(double2), xr * sizeof(double2), xl, cudaMemcpyDeviceToHost, h->stream));
        off += xl * xr;
      }
  }
  if (lambdas) {
    size_t off = 0;
    for (int b = 0; b < h->n - 1; ++b) {
      CK(cudaMemcpyAsync(lambdas + off, bond_ptr(h, b), sizeof(double) * c[b + 1], cudaMemcpyDeviceToHost, h->stream));
      off += c[b + 1];
    }
  }
  CK(cudaStreamSynchronize(h->stream));
  return collect_status(h);
}

int mps_import(mps_handle h, const int* chi, const double* gammas, const double* lambdas) {
  if (!h || !chi || !gammas || (h->n > 1 && !lambdas)) return fail(MPS_ERR_ARG, "bad arguments");
  if (chi[0] != 1 || chi[h->n] != 1) return fail(MPS_ERR_ARG, "boundary bonds must be 1");
  for (int b = 0; b <= h->n; ++b)
    if (chi[b] < 1 || chi[b] > h->cap) return fail(MPS_ERR_ARG, "bond dimension out of [1, chi_max]");
  CK(cudaStreamSynchronize(h->stream));
  int rc = reset_state(h);
  if (rc) return rc;
  size_t off = 0;
  for (int s = 0; s < h->n; ++s)
    for (int i = 0; i < 2; ++i) {
      const size_t xl = chi[s], xr = chi[s + 1];
      CK(cudaMemcpy2DAsync(site_ptr(h, s) + (size_t)i * h->cap * h->cap, h->cap * sizeof(double2), gammas + 2 * off,
                           xr * sizeof(double2), xr * sizeof(double2), xl, cudaMemcpyHostToDevice, h->stream));
      off += xl * xr;
    }
  size_t lo = 0;
  for (int b = 0; b < h->n - 1; ++b) {
    CK(cudaMemcpyAsync(bond_ptr(h, b), lambdas + lo, sizeof(double) * chi[b + 1], cudaMemcpyHostToDevice, h->stream));
    lo += chi[b + 1];
  }
  CK(cudaMemcpyAsync(h->chi, chi, sizeof(int) * (h->n + 1), cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->ub.assign(chi, chi + h->n + 1);
  return MPS_OK;
}

int mps_diag(mps_handle h, int cap, int* count, int* k, double* discarded, int* sweeps, int* k_sketch) {
  if (!h || !count || cap < 0) return fail(MPS_ERR_ARG, "bad arguments");
  CK(cudaStreamSynchronize(h->stream));
  *count = h->last_ntask;
  const int m = std::min(cap, h->last_ntask);
  if (m > 0) {
    std::vector<TaskMeta> t(m);
    CK(cudaMemcpy(t.data(), h->d_meta, sizeof(TaskMeta) * m, cudaMemcpyDeviceToHost));
    for (int i = 0; i < m; ++i) {
      if (k) k[i] = t[i].knew;
      if (discarded) discarded[i] = t[i].disc;
      if (sweeps) sweeps[i] = t[i].sweeps_total;
      if (k_sketch) k_sketch[i] = t[i].ksk;
    }
  }
  return MPS_OK;
}

int mps_program_create(int count, const mps_handle* handles, int n_passes, const int* k, const int* n_gates,
                       const int* sites, const int* owners, const double* d_Us, mps_program_handle* out) {
  return program_create(count, handles, n_passes, k, n_gates, sites, owners, d_Us, out);
}

int mps_program_run(mps_program_handle p) { return program_run(p); }

int mps_program_updates(mps_program_handle p, long long* updates) {
  if (!p || !updates) return fail(MPS_ERR_ARG, "bad arguments");
  *updates = p->updates;
  return MPS_OK;
}

int mps_program_destroy(mps_program_handle p) {
  free_program(p);
  return MPS_OK;
}

int mps_sync(mps_handle h) {
  if (!h) return fail(MPS_ERR_ARG, "NULL handle");
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaGetLastError());
  return collect_status(h);
}

}  // extern "C"

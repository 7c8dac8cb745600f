// Host-side launch wrappers of the engine's kernels (all asynchronous on `st`).
#pragma once
#include "engine.cuh"

namespace mpsgb {

constexpr int kBlockW = 8;     // Jacobi block width b (columns per block), binary64 sweeps
constexpr int kBlockW32 = 16;  // block width of the fp32 preconditioning sweeps
constexpr int kF32InnerSweeps = 1;  // inner Hermitian Jacobi sweeps per block pair in the fp32 sweeps
constexpr float kQuadStop = 1e-8f;  // binary64 sweeps stop after one whose max scaled off-diagonal < this
constexpr int kInnerSweepsFar = 1;  // inner sweeps of a block pair whose off-diagonal is above kQuadStop ...
constexpr int kInnerFarSweeps = 30;  // ... during a task's first sweeps
constexpr int kMaxSweeps = 60;       // binary64 sweep limit of one SVD (MPS_ERR_NOCONVERGE beyond it)

// Sets the message returned by mps_last_error() on the calling thread.
void set_error_message(const char* msg);

// Every device and pinned-host allocation of the library goes through these,
// so that a test can make the n-th one fail (mps_debug_fail_alloc) and check
// the MPS_ERR_NOMEM path without exhausting a shared GPU.
cudaError_t dev_alloc(void** p, size_t bytes);
cudaError_t host_alloc(void** p, size_t bytes);

void launch_setup(const GateTask* t, TaskMeta* m, int ntask, int stage, cudaStream_t st);
void launch_contract2(const GateTask* t, const TaskMeta* m, int ntask, int a_ub, int b_ub, cudaStream_t st);
void launch_contract3(const GateTask* t, const TaskMeta* m, int ntask, int x0_ub, int xl_ub, int xr_ub,
                      cudaStream_t st);
void launch_frob(const GateTask* t, TaskMeta* m, int ntask, long long el_ub, int second, cudaStream_t st);
void launch_init_V(const GateTask* t, const TaskMeta* m, int ntask, int nw_ub, cudaStream_t st);
void launch_jacobi_round(const GateTask* t, TaskMeta* m, int ntask, int round, int pairs_ub, int second,
                         unsigned long long* flops, cudaStream_t st);
void launch_sweep_end(TaskMeta* m, int ntask, int max_sweeps, int* active_count, cudaStream_t st);
void launch_sweep_end_nofail(TaskMeta* m, int ntask, int max_sweeps, int* active_count, cudaStream_t st);
// fp32 preconditioning round (jacobi_f32.cu), block width bw = 8 or 16. With
// fused = 0 (bw = 16 only) the pair kernel writes W and launch_rot_tc
// (jacobi_rot_tc.cu) applies it to the rows of A32 and V32 on the tensor cores.
void launch_jacobi_round_f32(const GateTask* t, TaskMeta* m, int ntask, int round, int pairs_ub, int bw, int fused,
                             unsigned long long* flops, cudaStream_t st);
// Every fp32 preconditioning sweep of every task in one scheduled launch
// (fused rotation, bw = 8 or 16, nthr = 256 or 384 threads per CTA, at most
// max_sweeps sweeps per task): the same
// pairs, rounds and sweeps as launch_jacobi_round_f32 with the end-of-sweep
// rule of launch_sweep_end_nofail, taken per task on the device. sched: four
// ints of device scratch (8-byte aligned); err: the handle's error word (set
// when a bounded dependency wait runs out). Returns the launches made, or -1
// when the (cooperative) launch failed.
int launch_jacobi_f32_sched(const GateTask* t, TaskMeta* m, int ntask, int nw_ub, int bw, int nthr, int max_sweeps,
                            void* sched, int* err, unsigned long long* flops, cudaStream_t st);
// One-time kernel attributes (shared-memory sizes), set before a program
// records launches into a graph; the launchers call them too.
void jacobi_f32_prepare();
void rot_tc_prepare();
void launch_rot_tc(const GateTask* t, const TaskMeta* m, int ntask, int round, int pairs_ub, int mw_ub, int nw_ub,
                   int* err, cudaStream_t st);
void launch_colnorms(const GateTask* t, const TaskMeta* m, int ntask, int nw_ub, int second, cudaStream_t st);
void launch_truncate(const GateTask* t, TaskMeta* m, int ntask, int stage, int chi_cap, cudaStream_t st);
void launch_emit_left(const GateTask* t, const TaskMeta* m, int ntask, int r_ub, int k_ub, int stage,
                      cudaStream_t st);
void launch_emit_right(const GateTask* t, const TaskMeta* m, int ntask, int cn_ub, int k_ub, int stage,
                       cudaStream_t st);
void launch_form_second(const GateTask* t, const TaskMeta* m, int ntask, int k1_ub, int xr_ub, cudaStream_t st);
void launch_apply1(const SiteTask* t, int ntask, int el_ub, cudaStream_t st);

void launch_amplitudes(const double2* gamma, const double* lambda, const int* chi, int n, int cap,
                       const unsigned char* bits, int count, double2* out, cudaStream_t st);
void launch_sample_step(int S, int xr, const double2* W0, const double2* W1, const double2* T0, const double2* T1,
                        const double* u, int ustride, unsigned char* bits, double2* V, cudaStream_t st);
void launch_combine2(long long n, double2 a0, const double2* X0, double2 a1, const double2* X1, double2* out,
                     cudaStream_t st);
void launch_fill_one(double2* v, int count, cudaStream_t st);
void launch_scale_site(const double2* g, const double* lam, int xl, int xr, int cap, double2* out, cudaStream_t st);
void launch_zgemm(int M, int N, int K, const double2* A, int lda, long long sA, int transA, const double2* B,
                  int ldb, long long sB, int conjB, int transB, double2* C, int ldc, long long sC, int accumulate,
                  long long batch, cudaStream_t st);

}  // namespace mpsgb

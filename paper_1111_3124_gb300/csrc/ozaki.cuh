// Split-precision (Ozaki scheme) complex GEMM on tcgen05 tensor cores.
#pragma once
#include <cuda_runtime.h>

namespace mpsgb {

// A complex matrix view X(r, k), r < rows, k < K, element at
//   p[(r / rb) * s_rb + (r % rb) * s_r + (k / kb) * s_kb + (k % kb) * s_k]
// (rb = 0 or kb = 0: no blocking), optionally scaled by rscale[r % rb] and
// kscale[k % kb] and conjugated. For the B operand the view is indexed
// (n, k), i.e. it describes B^T.
struct OzView {
  const double2* p;
  long long s_rb, s_r, s_kb, s_k;
  int rb, kb;
  const double* rscale;
  const double* kscale;
  int conj;
};

// One GEMM C = alpha * A B (A: M x K view a, B: K x N given as the N x K view
// b); C is complex binary64, column-major: C[r + n * ldc].
// herm = 1 declares row r of A to be conj(column r of B) up to one common
// sign (A^H A, V^H V, X X with X skew-Hermitian, Q Q with Q Hermitian; M = N):
// every slice of row r of A is then the conjugate of the same slice of column
// r of B with the same scale, the set of slice pairs is symmetric and every
// sum is an exact integer, so the computed C is exactly Hermitian. Only the
// tiles on and above the diagonal are multiplied; each one above writes its
// conjugate transpose below as well, which is the value that tile would have
// produced, bit for bit.
struct OzJob {
  OzView a, b;
  int M, N, K;
  double2* C;
  long long ldc;
  double alpha;
  int herm;
};

// Device scratch for slices and scales, grown on demand by ozaki_zgemm.
struct OzBuffers {
  void* base = nullptr;
  size_t bytes = 0;
  static size_t bytes_needed(int jobs, int M_ub, int N_ub, int K_ub, int s);
};

// Runs njobs GEMMs (job table on the device; dims on the device, bounded by
// M_ub, N_ub, K_ub) with s slices per operand. Returns 0 or a negative code.
// K above 512 runs in 512-wide chunks accumulated in binary64.
// d_err: device int set to 1 if a bounded wait ran out.
// One-time set-up of the GEMM kernel (0 on success); ozaki_zgemm calls it.
int ozaki_prepare();

int ozaki_zgemm(const OzJob* d_jobs, int njobs, int M_ub, int N_ub, int K_ub, int s, OzBuffers& buf, int* d_err,
                cudaStream_t st);

// Products of the split-precision two-site update (split_path.cu):
// kOzTheta: T = X Y (theta); kOzVhV: P = V^H V; kOzVP: Q = V P; kOzAV: T = A V.
// Gram polish (tasks still active and without an overflow of near-degenerate
// pairs): kOzAhA: P = A^H A; kOzXX: Q = P P; kOzX3: V2 = P Q; kOzX4: T = Q Q;
// kOzAW: T = A P; kOzVW: Q = V P.
enum {
  kOzTheta = 0, kOzVhV = 1, kOzVP = 2, kOzAV = 3,
  kOzAhA = 5, kOzXX = 6, kOzX3 = 7, kOzX4 = 8, kOzAW = 9, kOzVW = 10
};
struct GateTask;
struct TaskMeta;
// Fills the job table of product `kind` (a job whose task is finished, or
// left to the blocked sweeps, is empty); with `flops` non-null, adds the
// tensor-core flops of the jobs that run (s slices) to it.
void launch_oz_jobs(const GateTask* t, const TaskMeta* m, OzJob* jobs, int ntask, int kind, int s,
                    unsigned long long* flops, cudaStream_t st);
void launch_gate_mix2(const GateTask* t, const TaskMeta* m, int ntask, int xl_ub, int xr_ub, cudaStream_t st);
// Ranks the working matrix's columns by norm (k_sort_cols), then A32 = fp32(A P), V32 = P.
void launch_to_f32(const GateTask* t, const TaskMeta* m, int ntask, int nw_ub, long long el_ub, cudaStream_t st);
void launch_v_to_f64(const GateTask* t, const TaskMeta* m, int ntask, long long el_ub, cudaStream_t st);
void launch_ns_update(const GateTask* t, const TaskMeta* m, int ntask, long long el_ub, cudaStream_t st);
void launch_take_product(const GateTask* t, TaskMeta* m, int ntask, long long el_ub, cudaStream_t st);
void launch_gram_diag(const GateTask* t, TaskMeta* m, int ntask, int nw_ub, cudaStream_t st);
void launch_givens(const GateTask* t, const TaskMeta* m, int ntask, int rows_ub, cudaStream_t st);
void launch_copy_work(const GateTask* t, const TaskMeta* m, int ntask, long long el_ub, int to_t, cudaStream_t st);
void launch_gram_x(const GateTask* t, TaskMeta* m, int ntask, long long el_ub, int form_x, cudaStream_t st);
void launch_gram_end(TaskMeta* m, int ntask, int final_step, int* active_count, cudaStream_t st);
void launch_form_w(const GateTask* t, const TaskMeta* m, int ntask, long long el_ub, cudaStream_t st);
void launch_gram_scales(const GateTask* t, const TaskMeta* m, int ntask, int nw_ub, cudaStream_t st);
void launch_take_t(const GateTask* t, const TaskMeta* m, int ntask, long long el_ub, cudaStream_t st);

}  // namespace mpsgb

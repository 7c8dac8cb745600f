// Split-precision form of the two-site update (MPS_PREC_SPLIT).
//
//   1. theta: T = X Y with X[(k,a),c] = Lambda_{s-1}[a] Gamma_s[k,a,c] Lambda_s[c]
//      and Y[c,(l,b)] = Gamma_{s+1}[l,c,b] Lambda_{s+1}[b] by the split-precision
//      GEMM (ozaki_tc.cu); the gate mixes the four (k,l) blocks (k_gate_mix2).
//   2. fp32 blocked one-sided Jacobi on a copy of the working matrix
//      (rotation angles in binary64): an approximate right factor V32.
//   3. V = V32 in binary64, re-orthonormalised by two Newton-Schulz steps
//      V <- V (3 I - V^H V) / 2, products by the split-precision GEMM.
//   4. B = A V (split-precision GEMM).
//   5. A second fp32 pass on B (whose columns are nearly orthogonal, so the
//      small rotation angles keep every column's rounding relative to its own
//      norm, small singular values included), V2 re-orthonormalised,
//      B <- B V2 and V <- V V2 by the split-precision GEMM.
//   6. binary64 Jacobi sweeps on B finish the decomposition (quadratic
//      convergence from an O(1e-6) start), keeping the column norms, the
//      orthogonality test and the rotation angles in binary64.
// Truncation and the Lambda^-1 rewrite are those of the binary64 path.
#include "engine.cuh"
#include "kernels.cuh"
#include "ozaki.cuh"

namespace mpsgb {

// Fills one OzJob per task for the product `kind`.
__global__ void k_oz_jobs(const GateTask* tasks, const TaskMeta* meta, OzJob* jobs, int ntask, int kind) {
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
  double2* Vs = (kind & kOzOnV2) ? tk.V2 : tk.V;
  switch (kind & ~kOzOnV2) {
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
      j.a.p = Vs;
      j.a.s_r = mt.Nw;
      j.a.s_k = 1;
      j.a.conj = 1;
      j.b.p = Vs;
      j.b.s_r = mt.Nw;
      j.b.s_k = 1;
      j.M = j.N = j.K = mt.Nw;
      j.C = tk.P;
      j.ldc = mt.Nw;
      break;
    case kOzVP:  // Q = V P
      j.a.p = Vs;
      j.a.s_r = 1;
      j.a.s_k = mt.Nw;
      j.b.p = tk.P;
      j.b.s_r = mt.Nw;
      j.b.s_k = 1;
      j.M = j.N = j.K = mt.Nw;
      j.C = tk.Q;
      j.ldc = mt.Nw;
      break;
    case kOzVV2:  // Q = V V2
      j.a.p = tk.V;
      j.a.s_r = 1;
      j.a.s_k = mt.Nw;
      j.b.p = tk.V2;
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
      j.b.p = Vs;
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

// A32 = fp32(A), V32 = I
__global__ void k_to_f32(const GateTask* tasks, const TaskMeta* meta) {
  const GateTask& tk = tasks[blockIdx.y];
  const TaskMeta& mt = meta[blockIdx.y];
  if (mt.status) return;
  const size_t na = (size_t)mt.Mw * mt.Nw, nv = (size_t)mt.Nw * mt.Nw;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < na + nv; e += (size_t)gridDim.x * blockDim.x) {
    if (e < na) {
      const double2 v = tk.A[e];
      tk.A32[e] = make_float2((float)v.x, (float)v.y);
    } else {
      const size_t f = e - na;
      tk.V32[f] = make_float2((f % mt.Nw) == (f / mt.Nw) ? 1.f : 0.f, 0.f);
    }
  }
}

// V (or V2) = binary64(V32)
__global__ void k_v_to_f64(const GateTask* tasks, const TaskMeta* meta, int to_v2) {
  const GateTask& tk = tasks[blockIdx.y];
  const TaskMeta& mt = meta[blockIdx.y];
  if (mt.status) return;
  double2* V = to_v2 ? tk.V2 : tk.V;
  const size_t nv = (size_t)mt.Nw * mt.Nw;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nv; e += (size_t)gridDim.x * blockDim.x) {
    const float2 v = tk.V32[e];
    V[e] = make_double2((double)v.x, (double)v.y);
  }
}

// Newton-Schulz step V <- (3 V - V (V^H V)) / 2 = 1.5 V - 0.5 Q (on V or V2)
__global__ void k_ns_update(const GateTask* tasks, const TaskMeta* meta, int on_v2) {
  const GateTask& tk = tasks[blockIdx.y];
  const TaskMeta& mt = meta[blockIdx.y];
  if (mt.status) return;
  double2* V = on_v2 ? tk.V2 : tk.V;
  const size_t nv = (size_t)mt.Nw * mt.Nw;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nv; e += (size_t)gridDim.x * blockDim.x) {
    const double2 v = V[e], q = tk.Q[e];
    V[e] = make_double2(fma(1.5, v.x, -0.5 * q.x), fma(1.5, v.y, -0.5 * q.y));
  }
}

// V = Q (after Q = V V2)
__global__ void k_take_q(const GateTask* tasks, const TaskMeta* meta) {
  const GateTask& tk = tasks[blockIdx.y];
  const TaskMeta& mt = meta[blockIdx.y];
  if (mt.status) return;
  const size_t nv = (size_t)mt.Nw * mt.Nw;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nv; e += (size_t)gridDim.x * blockDim.x)
    tk.V[e] = tk.Q[e];
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
  }
}

static inline int grid_for(long long el) {
  long long b = (el + 255) / 256;
  if (b > 1024) b = 1024;
  if (b < 1) b = 1;
  return (int)b;
}

void launch_oz_jobs(const GateTask* t, const TaskMeta* m, OzJob* jobs, int ntask, int kind, cudaStream_t st) {
  k_oz_jobs<<<(ntask + 127) / 128, 128, 0, st>>>(t, m, jobs, ntask, kind);
}
void launch_gate_mix2(const GateTask* t, const TaskMeta* m, int ntask, int xl_ub, int xr_ub, cudaStream_t st) {
  k_gate_mix2<<<dim3(grid_for((long long)xl_ub * xr_ub), ntask), 256, 0, st>>>(t, m);
}
void launch_to_f32(const GateTask* t, const TaskMeta* m, int ntask, long long el_ub, cudaStream_t st) {
  k_to_f32<<<dim3(grid_for(el_ub), ntask), 256, 0, st>>>(t, m);
}
void launch_v_to_f64(const GateTask* t, const TaskMeta* m, int ntask, long long el_ub, int to_v2, cudaStream_t st) {
  k_v_to_f64<<<dim3(grid_for(el_ub), ntask), 256, 0, st>>>(t, m, to_v2);
}
void launch_ns_update(const GateTask* t, const TaskMeta* m, int ntask, long long el_ub, int on_v2, cudaStream_t st) {
  k_ns_update<<<dim3(grid_for(el_ub), ntask), 256, 0, st>>>(t, m, on_v2);
}
void launch_take_q(const GateTask* t, const TaskMeta* m, int ntask, long long el_ub, cudaStream_t st) {
  k_take_q<<<dim3(grid_for(el_ub), ntask), 256, 0, st>>>(t, m);
}
void launch_take_product(const GateTask* t, TaskMeta* m, int ntask, long long el_ub, cudaStream_t st) {
  k_take_product<<<dim3(grid_for(el_ub), ntask), 256, 0, st>>>(t, m);
}

}  // namespace mpsgb

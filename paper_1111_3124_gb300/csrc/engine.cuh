// Device-side data structures and kernel entry points of the gate-update
// engine. Host orchestration lives in capi.cu; kernels in update_fp64.cu,
// readout.cu and (split precision) ozaki_tc.cu.
//
// Layout in HBM (one MPS of n qubits, capacity cap = chi_max):
//   gamma  : n blocks of [2][cap][cap] complex128 (double2); site s, physical
//            index i, left bond a, right bond c at ((s*2 + i)*cap + a)*cap + c.
//            Only the leading chi_{s-1} x chi_s corner of each [cap][cap]
//            block is meaningful.
//   lambda : (n+1) x cap doubles; Lambda_b (bond b = -1..n-1) at (b+1)*cap.
//            The two boundary entries hold [1].
//   chi    : n+1 ints; chi[b+1] = dimension of bond b (chi[0] = chi[n] = 1).
// Bond dimensions live on the device and are read by every kernel, so a
// launch sequence never needs the host to know the current dimensions; the
// host only tracks upper bounds to size grids.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace mpsgb {

constexpr int kMaxCap = 1024;  // largest chi_max accepted by mps_create
constexpr int kMaxGivens = 16;  // near-degenerate pairs the Gram polish rotates exactly, per task

// One gate update (k = 2 or 3) of one MPS.
struct GateTask {
  double2* g0;          // Gamma_s
  double2* g1;          // Gamma_{s+1}
  double2* g2;          // Gamma_{s+2} (k = 3), else nullptr
  double* lamL;         // Lambda_{s-1}
  double* lam0;         // Lambda_s
  double* lam1;         // Lambda_{s+1}
  double* lamR;         // Lambda_{s+k-1} (outer right bond)
  int* chi;             // chi array of the state
  const double2* U;     // 2^k x 2^k gate, row-major, device
  int site, k, cap;
  double cutoff;
  // workspace (device)
  double2* A;           // working matrix of the SVD, column-major
  double2* V;           // accumulated right rotations
  double2* T;           // [4][cap][cap] scratch (3-site partial contraction / second split)
  double* sigma;        // column norms
  int* perm;            // sorted column order
  // split-precision workspace (MPS_PREC_SPLIT)
  float2* A32;          // fp32 copy of the working matrix (preconditioning sweeps)
  float2* V32;          // fp32 right rotations
  double2* P;           // Nw x Nw scratch: V^H V; the Gram polish's G, X, W
  double2* Q;           // Nw x Nw scratch: V P; X^2; V W
  double2* V2;          // Nw x Nw scratch: X^3, then the column scales of A W
  float2* Wp;           // fp32 sweeps: each block pair's 32 x 32 rotation W (for the tensor-core rotation)
  int* Wneed;           //   and whether that pair rotated in this round
  int* qver;            // scheduled fp32 sweeps: rounds finished on each block of A, then of V (2 (nb + 1) entries)
};

// Per-task state written and read by kernels only.
struct TaskMeta {
  int xl, x0, x1, xr;   // chi_{s-1}, chi_s, chi_{s+1}, chi_{s+k-1}
  int M, N;             // theta is M x N
  int Mw, Nw, tall;     // working matrix: Mw x Nw (tall ? theta : theta^H)
  int active;           // Jacobi still sweeping
  int rotated;          // a rotation happened in the current sweep
  int sweeps;           // sweeps done for the current split
  int sweeps_total;     // both splits (k = 3)
  int status;           // 0 or an mps_status code
  int knew;             // kept rank of the current split
  int k1;               // kept rank of the first split (k = 3)
  int ksk;              // singular values above max(cutoff/100, Mw eps) ||sigma||: the rank a sketch must capture
  int hard;             // Gram polish: left to the blocked binary64 sweeps (too many near-degenerate pairs)
  int nhard;            // Gram polish: near-degenerate pairs found by the last test (rotated exactly, <= kMaxGivens kept)
  int hp[kMaxGivens], hq[kMaxGivens];  //   their columns p < q
  double hc[kMaxGivens];               //   cos t of the exact Jacobi rotation
  double2 hs[kMaxGivens];              //   sin t e^{i phi}
  double disc;          // discarded weight (summed over splits)
  double kept_norm;     // sqrt(sum of kept sigma^2) of the current split
  double frob2;         // ||A||_F^2 of the current working matrix
  unsigned int maxoff;  // float bits: largest |g_pq|/sqrt(g_pp g_qq) seen in this sweep
  int q_done;           // scheduled fp32 sweeps: block pairs finished (all sweeps)
  int q_sweep;          //   sweeps whose end-of-sweep decision is published
};

// Readout / single-site tasks.
struct SiteTask {
  double2* g;           // Gamma_s
  int* chi;
  int site, cap;
  const double2* U;     // 2x2
};

}  // namespace mpsgb

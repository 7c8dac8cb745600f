// Randomized range-finder SVD of a gate update (sketch.cu).
#pragma once
#include <cuda_runtime.h>

#include "engine.cuh"

namespace mpsgb {

struct SketchTask {
  int task;        // index of the gate task in its pass
  int id;          // counter of the random generator
  int Mw, Nw, r;   // working matrix Mw x Nw, sketch width r
  int rcap;        // stride of the per-task sigma arrays
  double cutoff;
  double2* A;      // the task's working matrix (Mw x Nw, column-major)
  double2* V;      // the task's right factor (Nw x Nw)
  double2* Om;     // Nw x r Gaussian test matrix
  double2* Y;      // Mw x r range sample, then Q
  double2* Z;      // Nw x r
  double2* Bh;     // Nw x r: A^H Q, then rotated by the SVD of B
  double2* T2;     // Mw x Nw: Q B
  double2* Wy;     // r x r right rotations of Y's Jacobi
  double2* Wb;     // r x r right rotations of B^H's Jacobi
};

void launch_omega(const SketchTask* st, int n, long long el_ub, unsigned long long seed, cudaStream_t s);
void launch_scale_q(const SketchTask* st, int n, long long el_ub, const double* sig, const TaskMeta* mety,
                    cudaStream_t s);
void launch_residual(const SketchTask* st, int n, long long el_ub, double* res, cudaStream_t s);
void launch_sketch_mark(const SketchTask* st, int n, const double* res, int* accept, TaskMeta* meta, cudaStream_t s);
void launch_sketch_finish(const SketchTask* st, int n, long long el_ub, const double* sigb, const int* accept,
                          cudaStream_t s);

}  // namespace mpsgb

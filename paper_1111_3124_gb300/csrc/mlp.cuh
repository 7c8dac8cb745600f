// Rank-predictor MLP (mlp.cu): sizes, parameter layout, feature tasks.
#pragma once
#include <cuda_runtime.h>

struct mps_mlp;

namespace mpsgb {

constexpr int kMlpIn = 16, kMlpHid = 64;
constexpr int kMlpW1 = 0;
constexpr int kMlpB1 = kMlpW1 + kMlpHid * kMlpIn;
constexpr int kMlpW2 = kMlpB1 + kMlpHid;
constexpr int kMlpB2 = kMlpW2 + kMlpHid;
constexpr int kMlpParams = kMlpB2 + 1;  // 1153

// Inputs of the feature kernel for one gate task.
struct FeatureTask {
  const double* lamL;  // Lambda of the left outer bond
  const double* lamR;  // Lambda of the right outer bond
  const int* chi;      // bond dimensions of the state
  int site, k;
  float ep;            // entangling power of the gate
  double cutoff;
};

void launch_mlp_fwd(const float* P, const float* X, int B, float* Y, cudaStream_t st);
void launch_features(const FeatureTask* ft, int n, float* X, cudaStream_t st);
double entangling_power(const double* U);  // two-qubit gate, complex128 row-major
const float* mlp_params(const mps_mlp* m);

}  // namespace mpsgb

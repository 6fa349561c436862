// Launch parameters of the Dirichlet lift (dirichlet.cu).
#pragma once
#include "common.cuh"

namespace hofem {

constexpr int kLiftLocal = (kMaxN + 1) * (kMaxN + 1);

struct LiftParams {
  const double* vb;           // (nrhs, P_1, .., P_N) full grid, P_i = n_i K_i + 1
  double* f;                  // (nrhs, M_1, .., M_N), M_i = P_i - 2
  int N, nrhs;
  int n[3], P[3], M[3];
  double coef[3];             // 4 h_i^-2
  double alpha;
  double A[3][kLiftLocal];    // local stiffness and mass per axis, (n_i + 1)^2, row-major
  double C[3][kLiftLocal];
};

// f -= (full-space operator, interior rows x boundary columns) vb
cudaError_t launch_lift(const LiftParams& p, cudaStream_t s);

}  // namespace hofem

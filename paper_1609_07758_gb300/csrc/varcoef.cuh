// Launch parameters of the variable-coefficient operator (varcoef.cu).
#pragma once
#include "common.cuh"

namespace hofem {

struct VarcoefParams {
  const double* u;            // (M0, M1)
  double* r;                  // (M0, M1), accumulated with atomics (zero it first)
  const double* aq;           // (K0 (n+1), K1 (n+1)) coefficient at the Gauss points
  const double* B;            // (n+1) x (n+1): B[g][a] = e_a(xi_g)
  const double* D;            //                D[g][a] = e_a'(xi_g)
  const double* w;            // n+1 Gauss weights
  int K0, K1, M0, M1, n;
  double s0, s1;              // 4 h_1^-2, 4 h_2^-2
};

cudaError_t launch_varcoef(const VarcoefParams& p, cudaStream_t s);
// *out += x . y (zero *out first)
cudaError_t launch_dot(const double* x, const double* y, long long count, double* out, cudaStream_t s);

}  // namespace hofem

// Launch parameters of the matrix-free FP64 operator sweep (residual.cu).
#pragma once
#include "common.cuh"

namespace hofem {

struct ApplyParams {
  long long outer, inner, outer_per_rhs;   // same geometry as the transform sweeps
  long long tiles_per_outer, seg_per_line, ntiles;
  int M, n, K, W, E;                       // W lines per CTA, E elements per segment
  const double* P;
  const double* Q;                         // may be null
  double* out1;                            // P x C (may be null)
  double* out2;                            // cA P x A + cCP P x C + cCQ Q x C
  const double* f;                         // if set: out2 = f - out2
  double cA, cCP, cCQ;
  int needPC, needPA;                      // which products of P are used
  const double* Aloc;                      // (n+1)^2, device (FP64 part of the stiffness)
  const float* AlocLo;                     // (n+1)^2 remainder of the double-double stiffness
  const double* Cloc;
  int threads;
  size_t smem_bytes;
};

size_t apply_smem_bytes(int n, int W, int E, bool twoInputs);
cudaError_t apply_set_smem_limits();
cudaError_t launch_apply(const ApplyParams& p, cudaStream_t s);

}  // namespace hofem

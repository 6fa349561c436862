// Launch parameters of the matrix-free FP64 operator sweep (residual.cu).
#pragma once
#include "common.cuh"

namespace hofem {

// Folded element tables, sized for the largest order: even part (n/2 + 1)^2, odd part
// ((n+1)/2)^2, row-major with the order's own row length.
constexpr int kFoldE = (kMaxN / 2 + 1) * (kMaxN / 2 + 1);
constexpr int kFoldO = ((kMaxN + 1) / 2) * ((kMaxN + 1) / 2);

// What one sweep computes (all products along the sweep's axis, Q's coefficient is 1):
//   kApplyFirst: out1 = P x C,  out2 = cA (P x A) + cCP (P x C)
//   kApplyMid:   out1 = P x C,  out2 = cA (P x A) + cCP (P x C) + Q x C
//   kApplyLast:                 out2 = [f -] (cA (P x A) + Q x C)
// With `uniform` set (every axis has the coefficient cA, exact integer stiffness tables):
//   kApplyFirst: out1 = P x C,  out2 = P x A + cCP (P x C)       (cCP = alpha / cA)
//   kApplyMid:   out1 = P x C,  out2 = P x A + Q x C
//   kApplyLast:                 out2 = [f -] cA (P x A + Q x C)
enum ApplyMode { kApplyFirst = 0, kApplyMid = 1, kApplyLast = 2 };

constexpr int kApplyThreads = 256;
constexpr int kApplyLines = 32;            // lines per CTA (W)
constexpr int kApplyMinb3MaxN = 9;         // orders compiled for three CTAs per SM
constexpr size_t kApplySmem3 = 232448 / 3 - 1024;   // shared memory per CTA at three per SM

struct ApplyParams {
  long long outer, inner, outer_per_rhs;   // same geometry as the transform sweeps
  long long tiles_per_outer, seg_per_line, ntiles;
  int M, n, K, W, E;                       // W lines per CTA, E elements per segment
  int mode;                                // ApplyMode
  int uniform;                             // every axis has the same stiffness coefficient:
                                           // out2 unscaled, cA applied by the last sweep
  int out2_f32;                            // kApplyLast: out2 is an FP32 array (the right-hand
                                           // side of an FP32 correction solve)
  // Lines that hold only part of the grid along the sweep's axis (a slab of x_1 rows of a
  // problem split over GPUs).  Input line l holds global dofs q0 .. q0 + in_rows - 1, output
  // lines (out1, out2, f) dofs out0 .. out0 + out_rows - 1; segment 0 starts at element e0.
  // The whole-grid sweep: q0 = out0 = e0 = 0, in_rows = out_rows = M.
  long long blk_q0, blk_in_rows, blk_e0, blk_out0, blk_out_rows;
  const double* P;
  const double* Q;                         // kApplyMid, kApplyLast
  double* out1;                            // kApplyFirst, kApplyMid
  double* out2;
  const double* f;                         // kApplyLast, may be null: out2 = f - (...)
  double cA, cCP;
  size_t smem_bytes;
  // folded local matrices (centro-symmetry R M R = M), as kernel parameters so that the
  // unrolled products read them as constant operands
  double CE[kFoldE], CO[kFoldO];           // mass
  double AE[kFoldE], AO[kFoldO];           // stiffness (scaled integers for n <= 9, else hi)
  float AEl[kFoldE], AOl[kFoldO];          // stiffness lo parts (n > 9)
};

size_t apply_smem_bytes(int n, int E);
cudaError_t apply_set_smem_limits();
cudaError_t launch_apply(const ApplyParams& p, cudaStream_t s);

}  // namespace hofem

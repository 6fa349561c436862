// Launch parameters of the load-vector quadrature pass (load.cu).
#pragma once
#include "common.cuh"

namespace hofem {

constexpr int kLoadTab = (kMaxN + 1) * (kMaxN + 1);

struct LoadParams {
  const double* in;           // (outer, K (n+1), inner): samples at the quadrature points
  double* out;                // (outer, M, inner): load-vector entries along this axis
  long long outer, inner;
  int K, n, M;
  double T[kLoadTab];         // T[a (n+1) + g] = w_g e_a(xi_g), as kernel parameters
};

cudaError_t launch_load(const LoadParams& p, cudaStream_t s);
// y = a y + g (g may be null: y = a y), count doubles
cudaError_t launch_axpby(double* y, double a, const double* g, long long count, cudaStream_t s);
// y += c x
cudaError_t launch_axpy(double* y, double c, const double* x, long long count, cudaStream_t s);
// dst[b][r][c] = src[b][r][c], b < batch, r < rows, c < cols (leading dimensions per side)
cudaError_t launch_copy_block(const double* src, double* dst, long long batch, long long rows, long long cols,
                              long long src_ld, long long dst_ld, long long src_bs, long long dst_bs,
                              cudaStream_t s);

}  // namespace hofem

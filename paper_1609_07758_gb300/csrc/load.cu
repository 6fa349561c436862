// FEM average f^h of the right-hand side (Sect. 2 par. 4), by the (n+1)-point
// Gauss-Legendre rule on every element along every axis (Sect. 2 par. 5).  On an element
// the map x = x_{e} + (xi + 1) h / 2 turns (2/h) int f e_a into sum_g w_g e_a(xi_g) f(x_g),
// so one axis maps K (n+1) samples per line to M = nK - 1 entries:
//   interior a = 1..n-1 of element e:  sum_g T[a][g] q_{e,g}
//   node between elements e and e+1:   sum_g T[n][g] q_{e,g} + sum_g T[0][g] q_{e+1,g}
// (the outer nodes are Dirichlet and dropped).  The tensor product is applied one axis at
// a time; one thread per (line, element) writes that element's n owned entries.
#include <algorithm>

#include "common.cuh"
#include "load.cuh"

namespace hofem {

namespace {

template <int N>
__global__ void __launch_bounds__(256) load_axis_kernel(const __grid_constant__ LoadParams P) {
  constexpr int G = N + 1;
  const long long inner = P.inner, K = P.K, total = P.outer * K * inner;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long c = idx % inner, rest = idx / inner;
    const long long e = rest % K, o = rest / K;
    const double* q = P.in + (o * K * G + e * G) * inner + c;
    double* out = P.out + (o * P.M) * inner + c;
    double v[G];
#pragma unroll
    for (int g = 0; g < G; ++g) v[g] = __ldg(q + (long long)g * inner);
#pragma unroll
    for (int a = 1; a < N; ++a) {
      double s = 0.0;
#pragma unroll
      for (int g = 0; g < G; ++g) s = fma(P.T[a * G + g], v[g], s);
      out[(e * N + a - 1) * inner] = s;
    }
    if (e + 1 < K) {
      double s = 0.0;
#pragma unroll
      for (int g = 0; g < G; ++g) s = fma(P.T[N * G + g], v[g], s);
      const double* qn = q + (long long)G * inner;
#pragma unroll
      for (int g = 0; g < G; ++g) s = fma(P.T[g], __ldg(qn + (long long)g * inner), s);
      out[((e + 1) * N - 1) * inner] = s;
    }
  }
}

template <int N> cudaError_t launch_n(const LoadParams& p, cudaStream_t s) {
  const long long total = p.outer * p.K * p.inner;
  const long long blocks = std::min<long long>((total + 255) / 256, 152LL * 16);
  load_axis_kernel<N><<<(unsigned)std::max<long long>(blocks, 1), 256, 0, s>>>(p);
  return cudaGetLastError();
}

__global__ void axpby_kernel(double* __restrict__ y, double a, const double* __restrict__ g, long long count) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    y[i] = g ? fma(a, y[i], __ldg(g + i)) : a * y[i];
}

__global__ void axpy_kernel(double* __restrict__ y, double c, const double* __restrict__ x, long long count) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    y[i] = fma(c, __ldg(x + i), y[i]);
}

// dst[b][r][c] = src[b][r][c] for a batch of row blocks with their own leading dimensions
__global__ void copy_block_kernel(const double* __restrict__ src, double* __restrict__ dst, long long batch,
                                  long long rows, long long cols, long long src_ld, long long dst_ld,
                                  long long src_bs, long long dst_bs) {
  const long long total = batch * rows * cols;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long c = i % cols, t = i / cols, r = t % rows, b = t / rows;
    dst[b * dst_bs + r * dst_ld + c] = __ldg(src + b * src_bs + r * src_ld + c);
  }
}

}  // namespace

cudaError_t launch_copy_block(const double* src, double* dst, long long batch, long long rows, long long cols,
                              long long src_ld, long long dst_ld, long long src_bs, long long dst_bs,
                              cudaStream_t s) {
  const long long total = batch * rows * cols;
  if (total <= 0) return cudaSuccess;
  const long long blocks = std::min<long long>((total + 255) / 256, 152LL * 16);
  copy_block_kernel<<<(unsigned)blocks, 256, 0, s>>>(src, dst, batch, rows, cols, src_ld, dst_ld, src_bs, dst_bs);
  return cudaGetLastError();
}

cudaError_t launch_axpy(double* y, double c, const double* x, long long count, cudaStream_t s) {
  const long long blocks = std::min<long long>((count + 255) / 256, 152LL * 16);
  axpy_kernel<<<(unsigned)std::max<long long>(blocks, 1), 256, 0, s>>>(y, c, x, count);
  return cudaGetLastError();
}

cudaError_t launch_axpby(double* y, double a, const double* g, long long count, cudaStream_t s) {
  const long long blocks = std::min<long long>((count + 255) / 256, 152LL * 16);
  axpby_kernel<<<(unsigned)std::max<long long>(blocks, 1), 256, 0, s>>>(y, a, g, count);
  return cudaGetLastError();
}

cudaError_t launch_load(const LoadParams& p, cudaStream_t s) {
  switch (p.n) {
#define HOFEM_LD_CASE(NN) \
  case NN: return launch_n<NN>(p, s);
    HOFEM_LD_CASE(1) HOFEM_LD_CASE(2) HOFEM_LD_CASE(3) HOFEM_LD_CASE(4) HOFEM_LD_CASE(5) HOFEM_LD_CASE(6)
    HOFEM_LD_CASE(7) HOFEM_LD_CASE(8) HOFEM_LD_CASE(9) HOFEM_LD_CASE(10) HOFEM_LD_CASE(11) HOFEM_LD_CASE(12)
    HOFEM_LD_CASE(13) HOFEM_LD_CASE(14) HOFEM_LD_CASE(15) HOFEM_LD_CASE(16)
#undef HOFEM_LD_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace hofem

// Matrix-free variable-coefficient operator -div(a grad u) on the 2D tensor-product mesh,
// in the scaling of Eq. bvp glob 2 (the problem the solver preconditions, Sect. 1): on every
// element, with a given at the (n+1) x (n+1) Gauss-Legendre points (Sect. 2 par. 5),
//   R = sum_{g,h} w_g w_h a_gh [4 h_1^-2 (D x B)^T (D x B) + 4 h_2^-2 (B x D)^T (B x D)] U,
// B[g][a] = e_a(xi_g), D[g][a] = e_a'(xi_g), by sum factorisation (8 (n+1)^3 FP64 FMAs per
// element) and scatter-added into the shared dofs.  One thread per element; the tables
// sit in shared memory.  Also the FP64 dot product of the conjugate-gradient loop.
#include <algorithm>

#include "common.cuh"
#include "varcoef.cuh"

namespace hofem {

namespace {

template <int N>
__global__ void __launch_bounds__(128) varcoef_kernel(const VarcoefParams P) {
  constexpr int n = N, G = N + 1;
  __shared__ double sB[G * G], sD[G * G], sW[G];
  for (int i = threadIdx.x; i < G * G; i += blockDim.x) {
    sB[i] = P.B[i];
    sD[i] = P.D[i];
  }
  for (int i = threadIdx.x; i < G; i += blockDim.x) sW[i] = P.w[i];
  __syncthreads();
  const long long el = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (el >= (long long)P.K0 * P.K1) return;
  const int e0 = (int)(el / P.K1), e1 = (int)(el - (long long)e0 * P.K1);
  const long long M0 = P.M0, M1 = P.M1;
  double U[G][G], Tx[G][G], Ty[G][G];
#pragma unroll
  for (int a = 0; a < G; ++a) {
    const long long p0 = (long long)e0 * n + a - 1;
#pragma unroll
    for (int b = 0; b < G; ++b) {
      const long long p1 = (long long)e1 * n + b - 1;
      U[a][b] = (p0 >= 0 && p0 < M0 && p1 >= 0 && p1 < M1) ? __ldg(P.u + p0 * M1 + p1) : 0.0;
    }
  }
  // derivative / value along x_1 at the points g
#pragma unroll
  for (int g = 0; g < G; ++g)
#pragma unroll
    for (int b = 0; b < G; ++b) {
      double tx = 0.0, ty = 0.0;
#pragma unroll
      for (int a = 0; a < G; ++a) {
        tx = fma(sD[g * G + a], U[a][b], tx);
        ty = fma(sB[g * G + a], U[a][b], ty);
      }
      Tx[g][b] = tx;
      Ty[g][b] = ty;
    }
  // fluxes at (g, h): gradients weighted by w_g w_h a_gh and the axis scales (U, no longer
  // needed, holds the x_1 flux; Fy the x_2 flux)
  double Fy[G][G];
  const double* aq = P.aq + ((long long)e0 * G) * ((long long)P.K1 * G) + (long long)e1 * G;
#pragma unroll
  for (int g = 0; g < G; ++g)
#pragma unroll
    for (int h = 0; h < G; ++h) {
      double gx = 0.0, gy = 0.0;
#pragma unroll
      for (int b = 0; b < G; ++b) {
        gx = fma(Tx[g][b], sB[h * G + b], gx);
        gy = fma(Ty[g][b], sD[h * G + b], gy);
      }
      const double wa = sW[g] * sW[h] * __ldg(aq + (long long)g * P.K1 * G + h);
      U[g][h] = P.s0 * wa * gx;
      Fy[g][h] = P.s1 * wa * gy;
    }
  // back along x_2: Tx <- flux_1 B, Ty <- flux_2 D (Tx, Ty are free)
#pragma unroll
  for (int g = 0; g < G; ++g)
#pragma unroll
    for (int b = 0; b < G; ++b) {
      double vx = 0.0, vy = 0.0;
#pragma unroll
      for (int h = 0; h < G; ++h) {
        vx = fma(U[g][h], sB[h * G + b], vx);
        vy = fma(Fy[g][h], sD[h * G + b], vy);
      }
      Tx[g][b] = vx;
      Ty[g][b] = vy;
    }
  // back along x_1 and scatter: R[a][b] = sum_g D[g][a] Tx[g][b] + B[g][a] Ty[g][b]
#pragma unroll
  for (int a = 0; a < G; ++a) {
    const long long p0 = (long long)e0 * n + a - 1;
    if (p0 < 0 || p0 >= M0) continue;
#pragma unroll
    for (int b = 0; b < G; ++b) {
      const long long p1 = (long long)e1 * n + b - 1;
      if (p1 < 0 || p1 >= M1) continue;
      double r = 0.0;
#pragma unroll
      for (int g = 0; g < G; ++g) r = fma(sD[g * G + a], Tx[g][b], fma(sB[g * G + a], Ty[g][b], r));
      atomicAdd(P.r + p0 * M1 + p1, r);
    }
  }
}

__global__ void dot_kernel(const double* __restrict__ x, const double* __restrict__ y, long long count,
                           double* out) {
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    s = fma(__ldg(x + i), __ldg(y + i), s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += part[i];
    atomicAdd(out, t);
  }
}

template <int N> cudaError_t launch_n(const VarcoefParams& p, cudaStream_t s) {
  const long long els = (long long)p.K0 * p.K1;
  varcoef_kernel<N><<<(unsigned)((els + 127) / 128), 128, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_varcoef(const VarcoefParams& p, cudaStream_t s) {
  switch (p.n) {
#define HOFEM_VC_CASE(NN) \
  case NN: return launch_n<NN>(p, s);
    HOFEM_VC_CASE(1) HOFEM_VC_CASE(2) HOFEM_VC_CASE(3) HOFEM_VC_CASE(4) HOFEM_VC_CASE(5) HOFEM_VC_CASE(6)
    HOFEM_VC_CASE(7) HOFEM_VC_CASE(8) HOFEM_VC_CASE(9)
#undef HOFEM_VC_CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_dot(const double* x, const double* y, long long count, double* out, cudaStream_t s) {
  const long long blocks = std::min<long long>((count + 255) / 256, 152LL * 4);
  dot_kernel<<<(unsigned)std::max<long long>(blocks, 1), 256, 0, s>>>(x, y, count, out);
  return cudaGetLastError();
}

}  // namespace hofem

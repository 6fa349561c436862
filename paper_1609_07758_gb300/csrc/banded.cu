// The banded solve of algorithm (b) (Sect. 2 par. 4): after the F_n-transforms along
// x_2..x_N, every mode (one column c of the remaining axes) is a 1D FEM problem along x_1,
//   (4 h^-2 A + sigma C) v = f,   sigma = sum_{i >= 2} 4 h_i^-2 lambda_i + alpha,
// symmetric positive definite with the element-block structure of Eq. eig_glob.  It is
// solved by static condensation: the element matrix E = 4 h^-2 A + sigma C is the same in
// every element, so its interior block E_II is factored once per mode (Cholesky), the
// element interiors are eliminated, and the nodal Schur complement is a constant-
// coefficient tridiagonal system (diagonal S_00 + S_nn, off-diagonal S_0n) solved by the
// Thomas algorithm; back-substitution then recovers the interiors.  All arithmetic is FP64.
//
// Only the nodal system is sequential along a mode.  For n >= 2 the solve runs as three
// kernels: the interiors of every chunk of CH elements of every mode are condensed in
// parallel (one thread per (chunk, mode), which also forms the node right-hand sides inside
// its chunk and leaves the two chunk-boundary contributions in scratch); one thread per mode
// runs the Thomas algorithm on the K - 1 nodes; the interiors are back-substituted in
// parallel again.  Threads of consecutive modes are neighbours, so every access is
// coalesced.  n = 1 (no interiors) keeps the single pass of one thread per mode.
#include <algorithm>
#include <cmath>

#include "banded.cuh"
#include "common.cuh"

namespace hofem {

namespace {

template <int N>
__global__ void __launch_bounds__(128) banded_kernel(const __grid_constant__ BandParams P) {
  constexpr int n = N, NI = N - 1, G = N + 1, NL = NI > 0 ? NI : 1;
  const long long lines = P.outer * P.inner;
  const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= lines) return;
  const long long o = l / P.inner, c = l - o * P.inner;
  const long long st = P.inner;
  double* u = P.u + o * P.M * st + c;            // dof p of this mode at u[p * st]
  double* cs = P.scratch + l;                    // Thomas multiplier of node j at cs[(j - 1) lines]
  const int K = P.K;
  double sigma = P.alpha;
  if (P.lamA) {
    const long long qa = P.lamB ? c / P.MB : c;
    sigma += P.lamA[qa];
    if (P.lamB) sigma += P.lamB[c - qa * P.MB];
  }
  auto E = [&](int a, int b) { return P.sA * P.A[a * G + b] + sigma * P.C[a * G + b]; };
  // Cholesky E_II = L L^T of the interior block (local points 1..n-1)
  double L[NL][NL];
#pragma unroll
  for (int i = 0; i < NI; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      double s = E(i + 1, j + 1);
#pragma unroll
      for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
      L[i][j] = (i == j) ? sqrt(s) : s / L[j][j];
    }
  auto solve_II = [&](double (&x)[NL]) {          // x := E_II^{-1} x
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      double s = x[i];
#pragma unroll
      for (int k = 0; k < i; ++k) s -= L[i][k] * x[k];
      x[i] = s / L[i][i];
    }
#pragma unroll
    for (int i = NI - 1; i >= 0; --i) {
      double s = x[i];
#pragma unroll
      for (int k = i + 1; k < NI; ++k) s -= L[k][i] * x[k];
      x[i] = s / L[i][i];
    }
  };
  // Z = E_II^{-1} E_{I,b} for the element's two nodes b = 0, n; nodal Schur complement
  double z0[NL], zn[NL], e0[NL], en[NL];
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    e0[i] = E(0, i + 1);
    en[i] = E(n, i + 1);
    z0[i] = e0[i];
    zn[i] = en[i];
  }
  solve_II(z0);
  solve_II(zn);
  double S00 = E(0, 0), S0n = E(0, n), Snn = E(n, n);
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    S00 -= e0[i] * z0[i];
    S0n -= e0[i] * zn[i];
    Snn -= en[i] * zn[i];
  }
  const double d = S00 + Snn, e = S0n;
  // forward: eliminate the interiors element by element, Thomas elimination on the nodes
  double yp[NL], cprev = 0.0, gprev = 0.0;
  for (int el = 1; el <= K; ++el) {
    double y[NL];
    const long long pi = (long long)(el - 1) * n;  // dof of local point 1
#pragma unroll
    for (int i = 0; i < NI; ++i) y[i] = u[(pi + i) * st];
    solve_II(y);
#pragma unroll
    for (int i = 0; i < NI; ++i) u[(pi + i) * st] = y[i];
    if (el >= 2) {                                  // node j = el - 1 is complete
      const int j = el - 1;
      const long long pn = (long long)j * n - 1;
      double g = u[pn * st];
#pragma unroll
      for (int i = 0; i < NI; ++i) g -= en[i] * yp[i] + e0[i] * y[i];
      const double den = (j == 1) ? d : d - e * cprev;
      cprev = e / den;
      gprev = (j == 1 ? g : g - e * gprev) / den;
      cs[(long long)(j - 1) * lines] = cprev;
      u[pn * st] = gprev;
    }
#pragma unroll
    for (int i = 0; i < NI; ++i) yp[i] = y[i];
  }
  // backward: nodal values, then the interiors u_I = y - z0 x_left - zn x_right
  double xr = 0.0;                                  // node K (Dirichlet)
  for (int el = K; el >= 1; --el) {
    double xl = 0.0;                                // node el - 1
    if (el - 1 >= 1) {
      const long long pn = (long long)(el - 1) * n - 1;
      xl = u[pn * st] - cs[(long long)(el - 2) * lines] * xr;
      u[pn * st] = xl;
    }
    const long long pi = (long long)(el - 1) * n;
#pragma unroll
    for (int i = 0; i < NI; ++i) u[(pi + i) * st] -= z0[i] * xl + zn[i] * xr;
    xr = xl;
  }
}

constexpr int kChunk = 32;   // elements per condensation thread

// Per-mode factors shared by the three kernels: E = sA A + sigma C, the Cholesky factor of
// E_II with reciprocal diagonal, and the couplings e0 = E_{0,I}, en = E_{n,I}.
template <int N> struct ModeFactors {
  static constexpr int NI = N - 1, G = N + 1, NL = NI > 0 ? NI : 1;
  double L[NL][NL], rd[NL], e0[NL], en[NL];
  double E00, E0n, Enn;
  __device__ __forceinline__ void init(const BandParams& P, long long c) {
    double sigma = P.alpha;
    if (P.lamA) {
      const long long qa = P.lamB ? c / P.MB : c;
      sigma += P.lamA[qa];
      if (P.lamB) sigma += P.lamB[c - qa * P.MB];
    }
    auto E = [&](int a, int b) { return P.sA * P.A[a * G + b] + sigma * P.C[a * G + b]; };
#pragma unroll
    for (int i = 0; i < NI; ++i)
#pragma unroll
      for (int j = 0; j <= i; ++j) {
        double v = E(i + 1, j + 1);
#pragma unroll
        for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
        if (i == j) {
          L[i][i] = sqrt(v);
          rd[i] = 1.0 / L[i][i];
        } else {
          L[i][j] = v * rd[j];
        }
      }
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      e0[i] = E(0, i + 1);
      en[i] = E(N, i + 1);
    }
    E00 = E(0, 0);
    E0n = E(0, N);
    Enn = E(N, N);
  }
  __device__ __forceinline__ void solve(double (&x)[NL]) const {   // x := E_II^{-1} x
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      double v = x[i];
#pragma unroll
      for (int k = 0; k < i; ++k) v -= L[i][k] * x[k];
      x[i] = v * rd[i];
    }
#pragma unroll
    for (int i = NI - 1; i >= 0; --i) {
      double v = x[i];
#pragma unroll
      for (int k = i + 1; k < NI; ++k) v -= L[k][i] * x[k];
      x[i] = v * rd[i];
    }
  }
};

// scratch layout: Thomas multipliers cs[(j - 1) lines + l], then the chunk-boundary node
// contributions left[q lines + l] (c0 of the chunk's first element, for node q CH) and
// right[q lines + l] (cn of its last element, for node min((q + 1) CH, K))
template <int N>
__global__ void __launch_bounds__(128) condense_kernel(const __grid_constant__ BandParams P) {
  constexpr int n = N, NI = N - 1;
  const long long lines = P.outer * P.inner;
  const int K = P.K, nch = (K + kChunk - 1) / kChunk;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= lines * nch) return;
  const int q = (int)(t / lines);
  const long long l = t - (long long)q * lines;
  const long long o = l / P.inner, c = l - o * P.inner, st = P.inner;
  double* u = P.u + o * P.M * st + c;
  ModeFactors<N> F;
  F.init(P, c);
  const int el0 = q * kChunk + 1, el1 = min((q + 1) * kChunk, K);
  double cn_prev = 0.0;
  for (int el = el0; el <= el1; ++el) {
    double y[NI];
    const long long pi = (long long)(el - 1) * n;
#pragma unroll
    for (int i = 0; i < NI; ++i) y[i] = u[(pi + i) * st];
    F.solve(y);
    double c0 = 0.0, cn = 0.0;
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      u[(pi + i) * st] = y[i];
      c0 += F.e0[i] * y[i];
      cn += F.en[i] * y[i];
    }
    if (el > el0) u[(pi - 1) * st] -= cn_prev + c0;   // node el - 1, inside the chunk
    else P.scratch[(long long)(K + q) * lines + l] = c0;
    cn_prev = cn;
  }
  P.scratch[(long long)(K + nch + q) * lines + l] = cn_prev;
}

template <int N>
__global__ void __launch_bounds__(128) nodes_kernel(const __grid_constant__ BandParams P) {
  constexpr int n = N, NI = N - 1, NL = NI > 0 ? NI : 1;
  const long long lines = P.outer * P.inner;
  const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= lines) return;
  const int K = P.K, nch = (K + kChunk - 1) / kChunk;
  const long long o = l / P.inner, c = l - o * P.inner, st = P.inner;
  double* u = P.u + o * P.M * st + c;
  double* cs = P.scratch + l;
  ModeFactors<N> F;
  F.init(P, c);
  double z0[NL], zn[NL];
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    z0[i] = F.e0[i];
    zn[i] = F.en[i];
  }
  F.solve(z0);
  F.solve(zn);
  double S00 = F.E00, S0n = F.E0n, Snn = F.Enn;
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    S00 -= F.e0[i] * z0[i];
    S0n -= F.e0[i] * zn[i];
    Snn -= F.en[i] * zn[i];
  }
  const double d = S00 + Snn, e = S0n;
  double cprev = 0.0, gprev = 0.0;
  for (int j = 1; j <= K - 1; ++j) {
    const long long pn = (long long)j * n - 1;
    double g = u[pn * st];
    if (j % kChunk == 0) {   // chunk boundary: the contributions left in scratch
      const int q = j / kChunk;
      g -= P.scratch[(long long)(K + nch + q - 1) * lines + l] + P.scratch[(long long)(K + q) * lines + l];
    }
    const double den = (j == 1) ? d : d - e * cprev;
    const double r = 1.0 / den;
    cprev = e * r;
    gprev = (j == 1 ? g : g - e * gprev) * r;
    cs[(long long)(j - 1) * lines] = cprev;
    u[pn * st] = gprev;
  }
  double xr = 0.0;
  for (int j = K - 1; j >= 1; --j) {
    const long long pn = (long long)j * n - 1;
    const double x = u[pn * st] - cs[(long long)(j - 1) * lines] * xr;
    u[pn * st] = x;
    xr = x;
  }
}

template <int N>
__global__ void __launch_bounds__(128) backsub_kernel(const __grid_constant__ BandParams P) {
  constexpr int n = N, NI = N - 1, NL = NI > 0 ? NI : 1;
  const long long lines = P.outer * P.inner;
  const int K = P.K, nch = (K + kChunk - 1) / kChunk;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= lines * nch) return;
  const int q = (int)(t / lines);
  const long long l = t - (long long)q * lines;
  const long long o = l / P.inner, c = l - o * P.inner, st = P.inner;
  double* u = P.u + o * P.M * st + c;
  ModeFactors<N> F;
  F.init(P, c);
  double z0[NL], zn[NL];
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    z0[i] = F.e0[i];
    zn[i] = F.en[i];
  }
  F.solve(z0);
  F.solve(zn);
  const int el0 = q * kChunk + 1, el1 = min((q + 1) * kChunk, K);
  for (int el = el0; el <= el1; ++el) {
    const long long pi = (long long)(el - 1) * n;
    const double xl = el - 1 >= 1 ? u[(pi - 1) * st] : 0.0;
    const double xr = el <= K - 1 ? u[(pi + n - 1) * st] : 0.0;
#pragma unroll
    for (int i = 0; i < NI; ++i) u[(pi + i) * st] -= z0[i] * xl + zn[i] * xr;
  }
}

template <int N> cudaError_t launch_n(const BandParams& p, cudaStream_t s) {
  const long long lines = p.outer * p.inner;
  if constexpr (N == 1) {
    banded_kernel<N><<<(unsigned)((lines + 127) / 128), 128, 0, s>>>(p);
  } else {
    const long long par = lines * ((p.K + kChunk - 1) / kChunk);
    condense_kernel<N><<<(unsigned)((par + 127) / 128), 128, 0, s>>>(p);
    nodes_kernel<N><<<(unsigned)((lines + 127) / 128), 128, 0, s>>>(p);
    backsub_kernel<N><<<(unsigned)((par + 127) / 128), 128, 0, s>>>(p);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_banded(const BandParams& p, cudaStream_t s) {
  if (p.outer * p.inner <= 0) return cudaSuccess;
  switch (p.n) {
#define HOFEM_BD_CASE(NN) \
  case NN: return launch_n<NN>(p, s);
    // orders the API accepts for algorithm (b) (n_1 <= 9)
    HOFEM_BD_CASE(1) HOFEM_BD_CASE(2) HOFEM_BD_CASE(3) HOFEM_BD_CASE(4) HOFEM_BD_CASE(5) HOFEM_BD_CASE(6)
    HOFEM_BD_CASE(7) HOFEM_BD_CASE(8) HOFEM_BD_CASE(9)
#undef HOFEM_BD_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace hofem

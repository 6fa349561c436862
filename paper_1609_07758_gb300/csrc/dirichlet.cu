// Inhomogeneous Dirichlet data u = b on the boundary, moved into the right-hand side of
// Eq. bvp glob 2 (the remark that follows it in Sect. 2 par. 4): with the 1D matrices
// extended by the two boundary nodes of every axis (same local A, C), the full operator
//   L^ = sum_i 4 h_i^-2 A^_i (x) prod_{m != i} C^_m + alpha C^_1 (x) .. (x) C^_N
// applied to the boundary values v_B and restricted to the interior rows is subtracted
// from f^h.  A row couples to a boundary column only if it lies in an element touching
// the boundary along some axis; one thread per interior dof returns at once elsewhere,
// and sums over the boundary columns of its element patch otherwise, the 1D entries
// assembled from the local matrices (a node shared by two elements sums both).
#include <algorithm>

#include "common.cuh"
#include "dirichlet.cuh"

namespace hofem {

namespace {

constexpr int kPatch = 2 * kMaxN + 1;   // columns of one axis coupled to a dof

// assembled full 1D entry (row fr, column q; full indices) from the local matrix L
__device__ __forceinline__ double entry1d(const double* L, int n, int fr, int q) {
  double s = 0.0;
  const int j1 = fr / n, j0 = (fr % n == 0) ? j1 - 1 : j1;   // the element(s) holding fr
  for (int j = j0; j <= j1; ++j) {
    if (fr % n != 0 && j != j1) continue;
    const int b = j * n;
    if (q >= b && q <= b + n && fr >= b && fr <= b + n) s += L[(fr - b) * (n + 1) + (q - b)];
  }
  return s;
}

template <int N>
__global__ void __launch_bounds__(128) lift_kernel(const __grid_constant__ LiftParams P) {
  long long per = 1;
  for (int m = 0; m < N; ++m) per *= P.M[m];
  const long long total = per * P.nrhs;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long r = idx / per;
    long long rem = idx - r * per;
    int fr[3], lo[3], hi[3];
    bool touch[3], layer = false;
    for (int m = N - 1; m >= 0; --m) {
      const int p = (int)(rem % P.M[m]);
      rem /= P.M[m];
      const int f = p + 1, n = P.n[m];
      fr[m] = f;
      if (f % n == 0) { lo[m] = f - n; hi[m] = f + n; }
      else { lo[m] = (f / n) * n; hi[m] = lo[m] + n; }
      touch[m] = lo[m] == 0 || hi[m] == P.P[m] - 1;
      layer = layer || touch[m];
    }
    if (!layer) continue;
    double eA[3][kPatch], eC[3][kPatch];
    for (int m = 0; m < N; ++m)
      for (int q = lo[m]; q <= hi[m]; ++q) {
        eA[m][q - lo[m]] = entry1d(P.A[m], P.n[m], fr[m], q);
        eC[m][q - lo[m]] = entry1d(P.C[m], P.n[m], fr[m], q);
      }
    const double* vb = P.vb + r * (long long)P.P[0] * P.P[1] * (N == 3 ? P.P[2] : 1);
    double acc = 0.0;
    for (int q0 = lo[0]; q0 <= hi[0]; ++q0) {
      const bool b0 = q0 == 0 || q0 == P.P[0] - 1;
      if (!b0 && !touch[1] && (N < 3 || !touch[2])) continue;
      const double a0 = eA[0][q0 - lo[0]], c0 = eC[0][q0 - lo[0]];
      for (int q1 = lo[1]; q1 <= hi[1]; ++q1) {
        const bool b1 = b0 || q1 == 0 || q1 == P.P[1] - 1;
        const double a1 = eA[1][q1 - lo[1]], c1 = eC[1][q1 - lo[1]];
        if (N == 2) {
          if (!b1) continue;
          const double w = P.coef[0] * a0 * c1 + P.coef[1] * c0 * a1 + P.alpha * c0 * c1;
          acc = fma(w, __ldg(vb + (long long)q0 * P.P[1] + q1), acc);
        } else {
          if (!b1 && !touch[2]) continue;
          for (int q2 = lo[2]; q2 <= hi[2]; ++q2) {
            if (!(b1 || q2 == 0 || q2 == P.P[2] - 1)) continue;
            const double a2 = eA[2][q2 - lo[2]], c2 = eC[2][q2 - lo[2]];
            const double w = P.coef[0] * a0 * c1 * c2 + P.coef[1] * c0 * a1 * c2 + P.coef[2] * c0 * c1 * a2 +
                             P.alpha * c0 * c1 * c2;
            acc = fma(w, __ldg(vb + ((long long)q0 * P.P[1] + q1) * P.P[2] + q2), acc);
          }
        }
      }
    }
    P.f[idx] -= acc;
  }
}

}  // namespace

cudaError_t launch_lift(const LiftParams& p, cudaStream_t s) {
  long long total = p.nrhs;
  for (int m = 0; m < p.N; ++m) total *= p.M[m];
  const long long blocks = std::max<long long>(1, std::min<long long>((total + 127) / 128, 152LL * 32));
  if (p.N == 2) lift_kernel<2><<<(unsigned)blocks, 128, 0, s>>>(p);
  else lift_kernel<3><<<(unsigned)blocks, 128, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace hofem

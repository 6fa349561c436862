// Matrix-free FP64 operator of Eq. bvp glob 2,
//     A u = sum_i 4 h_i^-2 A_i (x) prod_{m!=i} C_m u + alpha C_1 (x) ... (x) C_N u,
// evaluated as one banded 1D sweep per axis (sum factorisation over the tensor product).
// A sweep along axis a reads up to two arrays P, Q and writes
//     out1 = P x_a C,    out2 = cA (P x_a A) + cCP (P x_a C) + cCQ (Q x_a C)
// (optionally out2 := f - out2).  The 1D products are element by element: element j's
// local vector w (n+1 values, Dirichlet nodes = 0) is multiplied by the local C and by
// the local A; unknown p owned by element j (local points 1..n) collects rows 1..n of
// element j plus, for its node, row 0 of element j+1.
// The stiffness is applied to differences, (A w)_a = sum_b A_ab (w_b - w_0): exactly
// zero on constants whatever the rounding of A, which keeps the smallest eigenvalues of
// the operator (O((k/K)^2) against O(n^2) entries) correct -- rounding the plain form
// would shift them by up to ~1e-9 relative for n = 9, K = 1024.  Rounding A to FP64 still
// perturbs the element energy of smooth (locally linear) functions by ~eps |A| relative,
// a systematic error that iterative refinement converges to (~3e-12 for n = 9, K = 1024).
// So A is carried as a double-double hi + lo: sum_b hi_ab d_b in FP64 plus the tiny
// correction sum_b lo_ab d_b in FP32 (it is ~1e-16 of the main term, so ~7 digits are
// plenty), which leaves only the non-systematic FP64 accumulation rounding.
#include "common.cuh"
#include "residual.cuh"

namespace hofem {

__global__ void __launch_bounds__(512, 1) apply_kernel(const ApplyParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = P.n, K = P.K, M = P.M, W = P.W, E = P.E;
  const int n1 = n + 1;
  const int R = (E + 1) * n + 1;       // tile rows: node j0-1 .. node j0+E
  double* tP = reinterpret_cast<double*>(smem_raw);
  double* tQ = tP + (size_t)R * W;
  double* sA = tQ + (P.Q ? (size_t)R * W : 0);
  double* sC = sA + n1 * n1;
  float* sAlo = reinterpret_cast<float*>(sC + n1 * n1);
  for (int i = threadIdx.x; i < n1 * n1; i += blockDim.x) {
    sA[i] = P.Aloc[i];
    sC[i] = P.Cloc[i];
    sAlo[i] = P.AlocLo[i];
  }
  const bool contiguous = (P.inner == 1);
  const long long b = blockIdx.x;
  const long long seg = b % P.seg_per_line;
  const long long rest = b / P.seg_per_line;
  const long long o = rest / P.tiles_per_outer, tix = rest - o * P.tiles_per_outer;
  const long long l0 = tix * W;
  const long long nl = contiguous ? P.outer_per_rhs : P.inner;
  const int wvalid = (int)min((long long)W, nl - l0);
  const int j0 = (int)(seg * E) + 1;   // first element of the segment (1-based)
  const long long p0 = (long long)(j0 - 1) * n - 1;   // dof of tile row 0
  // tile(r, w): contiguous -> [w][r], strided -> [r][w]
  auto tidx = [&](int r, int w) -> size_t { return contiguous ? (size_t)w * R + r : (size_t)r * W + w; };
  auto gidx = [&](long long p, int w) -> size_t {
    return contiguous ? (size_t)(o * P.outer_per_rhs + l0 + w) * M + p
                      : ((size_t)o * M + p) * P.inner + l0 + w;
  };
  for (int it = threadIdx.x; it < R * W; it += blockDim.x) {
    int r, w;
    if (contiguous) { w = it / R; r = it - w * R; } else { r = it / W; w = it - r * W; }
    const long long p = p0 + r;
    double vp = 0.0, vq = 0.0;
    if (w < wvalid && p >= 0 && p < M) {
      vp = __ldg(P.P + gidx(p, w));
      if (P.Q) vq = __ldg(P.Q + gidx(p, w));
    }
    tP[tidx(r, w)] = vp;
    if (P.Q) tQ[tidx(r, w)] = vq;
  }
  __syncthreads();
  const int items = E * W;
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    int e, w;
    if (contiguous) { w = it / E; e = it - w * E; } else { e = it / W; w = it - e * W; }
    const int j = j0 + e;
    if (j > K || w >= wvalid) continue;
    // differences w_t - w_0 of P for element j and element j+1 (stiffness operand)
    double dj[kMaxN + 1], dj1[kMaxN + 1];
    float fj[kMaxN + 1], fj1[kMaxN + 1];   // the same differences in FP32 for the lo term
    const double wp0 = tP[tidx(e * n, w)], xp0 = tP[tidx((e + 1) * n, w)];
#pragma unroll
    for (int t = 0; t <= kMaxN; ++t)
      if (t <= n) {
        dj[t] = tP[tidx(e * n + t, w)] - wp0;
        dj1[t] = tP[tidx((e + 1) * n + t, w)] - xp0;
        if (P.needPA) {
          fj[t] = (float)dj[t];
          fj1[t] = (float)dj1[t];
        }
      }
    const int last = (j == K) ? n - 1 : n;     // node K is a Dirichlet node
    for (int i = 1; i <= last; ++i) {
      double pc = 0.0, pa = 0.0, qc = 0.0;
      const double* cr = sC + i * n1;
      const double* ar = sA + i * n1;
      if (P.needPC) {
        for (int t = 0; t <= n; ++t) pc = fma(cr[t], tP[tidx(e * n + t, w)], pc);
      }
      if (P.needPA) {
        const float* alr = sAlo + i * n1;
        float lo = 0.f;
#pragma unroll
        for (int t = 1; t <= kMaxN; ++t)
          if (t <= n) {
            pa = fma(ar[t], dj[t], pa);
            lo = fmaf(alr[t], fj[t], lo);
          }
        pa += (double)lo;
      }
      if (P.Q) {
        for (int t = 0; t <= n; ++t) qc = fma(cr[t], tQ[tidx(e * n + t, w)], qc);
      }
      if (i == n) {                              // node j: add row 0 of element j+1
        if (P.needPC) {
          for (int t = 0; t <= n; ++t) pc = fma(sC[t], tP[tidx((e + 1) * n + t, w)], pc);
        }
        if (P.needPA) {
          float lo = 0.f;
#pragma unroll
          for (int t = 1; t <= kMaxN; ++t)
            if (t <= n) {
              pa = fma(sA[t], dj1[t], pa);
              lo = fmaf(sAlo[t], fj1[t], lo);
            }
          pa += (double)lo;
        }
        if (P.Q) {
          for (int t = 0; t <= n; ++t) qc = fma(sC[t], tQ[tidx((e + 1) * n + t, w)], qc);
        }
      }
      const long long p = (long long)(j - 1) * n + i - 1;
      const size_t g = gidx(p, w);
      if (P.out1) P.out1[g] = pc;
      double v = P.cA * pa + P.cCP * pc + P.cCQ * qc;
      if (P.f) v = __ldg(P.f + g) - v;
      P.out2[g] = v;
    }
  }
}

size_t apply_smem_bytes(int n, int W, int E, bool twoInputs) {
  const int R = (E + 1) * n + 1;
  return ((size_t)R * W * (twoInputs ? 2 : 1) + 3 * (size_t)(n + 1) * (n + 1)) * sizeof(double);
}

cudaError_t apply_set_smem_limits() {
  return cudaFuncSetAttribute(apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
}

cudaError_t launch_apply(const ApplyParams& p, cudaStream_t s) {
  apply_kernel<<<(unsigned)p.ntiles, p.threads, p.smem_bytes, s>>>(p);
  return cudaGetLastError();
}

}  // namespace hofem

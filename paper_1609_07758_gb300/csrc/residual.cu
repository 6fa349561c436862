// Matrix-free FP64 operator of Eq. bvp glob 2,
//     A u = sum_i 4 h_i^-2 A_i (x) prod_{m!=i} C_m u + alpha C_1 (x) ... (x) C_N u,
// evaluated as one banded 1D sweep per axis (sum factorisation over the tensor product);
// the three sweep kinds are listed with ApplyMode in residual.cuh.  The 1D products are
// element by element: element j's local vector w (n+1 values, Dirichlet nodes = 0) is
// multiplied by the local C and by the local A; unknown p owned by element j (local
// points 1..n) collects rows 1..n of element j plus, for its node, row 0 of element j+1.
//
// The stiffness is applied to differences, (A w)_a = sum_b A_ab (w_b - w_0): exactly
// zero on constants whatever the rounding, which keeps the smallest eigenvalues of the
// operator (O((k/K)^2) against O(n^2) entries) correct.  The table itself must not be
// rounded either: a rounded A perturbs the element energy of smooth (locally linear)
// functions by ~eps |A| relative, a systematic error that iterative refinement converges
// to (~3e-12 for n = 9, K = 1024).  For n <= 9 the table is D A with D the common
// denominator of A's entries -- integers below 2^52, exact in FP64 -- and 1/D is folded
// into the sweep's scalar coefficient, which only rescales the whole term by 1 + O(eps).
// For larger n, A is a double-double hi + lo: sum_b hi_ab d_b in FP64 plus the tiny
// correction sum_b lo_ab d_b in FP32 (~1e-16 of the main term, so ~7 digits suffice).
//
// Folding: with w_e[t] = w_t + w_{n-t}, w_o[t] = w_t - w_{n-t} (t < h = (n+1)/2) and the
// middle value for even n, rows r and n-r of M w are E_r + O_r and E_r - O_r, which
// halves the products.  The odd part of the differences is w_o itself.
//
// Uniform scale (US): when every axis has the same stiffness coefficient c (same h_i and
// exact integer tables of the same order), the operator is c (sum_i A_i x prod C_m) +
// alpha prod C_m, and the sweeps carry the sums unscaled: the first sweep writes P x A
// (+ alpha / c P x C), a middle one P x A + Q x C, and the last one accumulates P x A and
// Q x C in one register per row and writes f - c v (or c v).  That removes one FP64
// multiply per output row of the first sweep and one combining operation per row of the
// later ones.
#include "common.cuh"
#include "convert.cuh"
#include "residual.cuh"

namespace hofem {

namespace {

constexpr int kLd = kApplyLines + 1;   // tile row stride in doubles (odd: no bank conflicts)

// All rows of one element (HALO: only its row 0) for line w; `base` is the tile row of
// the element's left node, `s` its slot index.  The products run column by column
// (outer-product order), so only the row accumulators and one folded pair are live.
// Interior rows are written back into the tiles in place (tP <- P x C, tQ <- out2),
// which only this element reads; rows 0 and n go to the slot arrays for the node sums.
template <int N, int MODE, bool HALO, bool US>
__device__ __forceinline__ void element_rows(const ApplyParams& P, double* tP, double* tQ, int base, int w,
                                             double* sV0, double* sP0, double* sVn, double* sPn, int s) {
  constexpr int n = N, h = (N + 1) / 2, hr = N / 2 + 1;
  constexpr bool has_mid = (N % 2) == 0;
  constexpr bool LO = N > kExactStiffnessMaxN;
  constexpr bool PC = MODE != kApplyLast;    // P x C is wanted
  constexpr bool QC = MODE != kApplyFirst;   // Q x C is wanted
  constexpr bool QS = QC && !US;             // Q x C in accumulators of its own
  static_assert(!(US && LO), "uniform-scale sweeps use exact integer stiffness tables");
  constexpr int rE = HALO ? 1 : hr, rO = HALO ? 1 : h;   // rows computed
  double cE[hr], cO[h], aE[hr], aO[h], qE[hr], qO[h];
  float lE[hr], lO[h];
  const double* cp = tP + (size_t)base * kLd + w;
  const double* cq = tQ + (size_t)base * kLd + w;
  const double w0 = cp[0];
  // column t: folded values pe, po (P), de (differences; their odd part is po), qe, qo (Q)
  auto column = [&](int t, bool middle, double pe, double po, double de, double qe, double qo) {
#pragma unroll
    for (int r = 0; r < rE; ++r) {
      const double ce = P.CE[r * hr + t], ae = P.AE[r * hr + t];
      if (t == 0) {
        if (PC) cE[r] = ce * pe;
        aE[r] = ae * de;
        if (LO) lE[r] = P.AEl[r * hr + t] * (float)de;
        if (QS) qE[r] = ce * qe;
      } else {
        if (PC) cE[r] = fma(ce, pe, cE[r]);
        aE[r] = fma(ae, de, aE[r]);
        if (LO) lE[r] = fmaf(P.AEl[r * hr + t], (float)de, lE[r]);
        if (QS) qE[r] = fma(ce, qe, qE[r]);
      }
      if (US && QC) aE[r] = fma(ce, qe, aE[r]);
    }
    if (middle) return;
#pragma unroll
    for (int r = 0; r < rO; ++r) {
      const double co = P.CO[r * h + t], ao = P.AO[r * h + t];
      if (t == 0) {
        if (PC) cO[r] = co * po;
        aO[r] = ao * po;
        if (LO) lO[r] = P.AOl[r * h + t] * (float)po;
        if (QS) qO[r] = co * qo;
      } else {
        if (PC) cO[r] = fma(co, po, cO[r]);
        aO[r] = fma(ao, po, aO[r]);
        if (LO) lO[r] = fmaf(P.AOl[r * h + t], (float)po, lO[r]);
        if (QS) qO[r] = fma(co, qo, qO[r]);
      }
      if (US && QC) aO[r] = fma(co, qo, aO[r]);
    }
  };
#pragma unroll
  for (int t = 0; t < h; ++t) {
    const double a = cp[t * kLd], c = cp[(n - t) * kLd];
    double qa = 0.0, qc = 0.0;
    if (QC) {
      qa = cq[t * kLd];
      qc = cq[(n - t) * kLd];
    }
    // t = 0: a is w0 itself, so the difference c - w0 is exactly -(a - c), the odd part
    column(t, false, a + c, a - c, t == 0 ? -(a - c) : (a - w0) + (c - w0), qa + qc, qa - qc);
  }
  if (has_mid) {
    const double a = cp[(n / 2) * kLd];
    column(hr - 1, true, a, 0.0, a - w0, QC ? cq[(n / 2) * kLd] : 0.0, 0.0);
  }
  const double cA = P.cA, cCP = P.cCP;
  const bool alpha = PC && cCP != 0.0;
  auto put = [&](int i, double pc, double v) {
    if (i == 0) {
      sV0[s] = v;
      if (PC) sP0[s] = pc;
    } else if (i == n) {
      sVn[s] = v;
      if (PC) sPn[s] = pc;
    } else {
      tQ[(size_t)(base + i) * kLd + w] = v;
      if (PC) tP[(size_t)(base + i) * kLd + w] = pc;
    }
  };
#pragma unroll
  for (int r = 0; r < rE; ++r) {
    double ae = aE[r], ao = r < h ? aO[r] : 0.0;
    if (LO) {
      ae += (double)lE[r];
      if (r < h) ao += (double)lO[r];
    }
    const double ce = PC ? cE[r] : 0.0, co = PC && r < h ? cO[r] : 0.0;
    // even and odd parts of out2 (unscaled sums under a uniform scale)
    double se, so;
    if (US) {
      se = ae;
      so = r < h ? ao : 0.0;
    } else {
      se = QC ? fma(cA, ae, qE[r]) : cA * ae;
      so = r < h ? (QC ? fma(cA, ao, qO[r]) : cA * ao) : 0.0;
    }
    if (alpha) {
      se = fma(cCP, ce, se);
      if (r < h) so = fma(cCP, co, so);
    }
    if (r < h) {
      put(r, ce + co, se + so);
      if (!HALO) put(n - r, ce - co, se - so);
    } else {
      put(r, ce, se);                    // middle row of an even order
    }
  }
}

// One CTA: W lines x E consecutive elements.  The tile holds dofs of tile rows 0..R-1 =
// left node of the segment .. right node of the halo element j0+E (row 0 of which closes
// the segment's last node).  Loads and stores are coalesced along whichever of line or
// dof index is contiguous in memory.
// Orders up to kApplyMinb3MaxN are compiled for three CTAs per SM (at most 85 registers a
// thread, E chosen so that the tile fits a third of shared memory): the FP64 pipe then has
// 24 warps to draw from while some CTAs load or store (measured 7.6% faster than two CTAs
// at n = 9, K = 1024).
template <int N, int MODE, bool US>
__global__ void __launch_bounds__(kApplyThreads, N <= kApplyMinb3MaxN ? 3 : N <= 10 ? 2 : 1) apply_kernel(const __grid_constant__ ApplyParams P) {
  constexpr int n = N, W = kApplyLines;
  constexpr bool PC = MODE != kApplyLast, QC = MODE != kApplyFirst;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int M = P.M, E = P.E;
  const int R = (E + 1) * n + 1;
  double* tP = reinterpret_cast<double*>(smem_raw);
  double* tQ = tP + (size_t)R * kLd;
  double* sV0 = tQ + (size_t)R * kLd;   // [E+1][W]
  double* sP0 = sV0 + (size_t)(E + 1) * W;
  double* sVn = sP0 + (size_t)(E + 1) * W;   // [E][W]
  double* sPn = sVn + (size_t)E * W;
  const bool contiguous = (P.inner == 1);
  const long long b = blockIdx.x;
  const long long seg = b % P.seg_per_line;
  const long long rest = b / P.seg_per_line;
  const long long o = rest / P.tiles_per_outer, tix = rest - o * P.tiles_per_outer;
  const long long l0 = tix * W;
  const long long nl = contiguous ? P.outer_per_rhs : P.inner;
  const int wvalid = (int)min((long long)W, nl - l0);
  const long long p0 = (P.blk_e0 + seg * E) * n - 1;   // global dof of tile row 0
  // element offsets of dof p in the input and the output lines
  const long long Li = P.blk_in_rows, Lo = P.blk_out_rows;
  auto gin = [&](long long p, int w) -> size_t {
    const long long i = p - P.blk_q0;
    return contiguous ? (size_t)(o * P.outer_per_rhs + l0 + w) * Li + i : ((size_t)o * Li + i) * P.inner + l0 + w;
  };
  auto gidx = [&](long long p, int w) -> size_t {
    const long long i = p - P.blk_out0;
    return contiguous ? (size_t)(o * P.outer_per_rhs + l0 + w) * Lo + i : ((size_t)o * Lo + i) * P.inner + l0 + w;
  };
  for (int it = threadIdx.x; it < R * W; it += blockDim.x) {
    int r, w;
    if (contiguous) {
      w = it / R;
      r = it - w * R;
    } else {
      r = it / W;
      w = it - r * W;
    }
    const long long p = p0 + r;
    double vp = 0.0, vq = 0.0;
    if (w < wvalid && p >= 0 && p < M && p >= P.blk_q0 && p < P.blk_q0 + Li) {
      const size_t g = gin(p, w);
      vp = __ldg(P.P + g);
      if (QC) vq = __ldg(P.Q + g);
    }
    tP[(size_t)r * kLd + w] = vp;
    if (QC) tQ[(size_t)r * kLd + w] = vq;
  }
  __syncthreads();
  for (int it = threadIdx.x; it < E * W; it += blockDim.x) {
    const int e = it / W, w = it - e * W;
    element_rows<N, MODE, false, US>(P, tP, tQ, e * n, w, sV0, sP0, sVn, sPn, it);
  }
  for (int w = threadIdx.x; w < W; w += blockDim.x)
    element_rows<N, MODE, true, US>(P, tP, tQ, E * n, w, sV0, sP0, sVn, sPn, E * W + w);
  __syncthreads();
  // node rows (e+1) n: row n of element e + row 0 of element e+1
  for (int it = threadIdx.x; it < E * W; it += blockDim.x) {
    const int e = it / W, w = it - e * W;
    const size_t row = (size_t)(e + 1) * n * kLd + w;
    tQ[row] = sVn[it] + sV0[it + W];
    if (PC) tP[row] = sPn[it] + sP0[it + W];
  }
  __syncthreads();
  // tile rows 1 .. E n are this segment's dofs; f of a group of U entries is read before
  // any of them is stored (clamped valid addresses, masked), so those loads overlap
  const int Rs = E * n, total = Rs * W;
  constexpr int U = 4;
  const bool use_f = MODE == kApplyLast && P.f != nullptr;
  for (int it0 = threadIdx.x; it0 < total; it0 += U * blockDim.x) {
    int rr[U], ww[U];
    bool ok[U];
    size_t gg[U];
    double fv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int it = it0 + u * blockDim.x;
      int r, w;
      if (contiguous) {
        w = it / Rs;
        r = it - w * Rs + 1;
      } else {
        r = it / W + 1;
        w = it - (r - 1) * W;
      }
      const long long p = p0 + r;
      ok[u] = it < total && w < wvalid && p < M && p >= P.blk_out0 && p < P.blk_out0 + Lo;
      rr[u] = r;
      ww[u] = w;
      gg[u] = ok[u] ? gidx(p, w) : 0;
      fv[u] = use_f ? __ldg(P.f + gg[u]) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!ok[u]) continue;
      double v = tQ[(size_t)rr[u] * kLd + ww[u]];
      if (MODE == kApplyLast) {
        if (US) v = use_f ? fma(-P.cA, v, fv[u]) : P.cA * v;
        else if (use_f) v = fv[u] - v;
      }
      if (MODE == kApplyLast && P.out2_f32) reinterpret_cast<float*>(P.out2)[gg[u]] = f64_to_f32_bits(v);
      else P.out2[gg[u]] = v;
      if (PC) P.out1[gg[u]] = tP[(size_t)rr[u] * kLd + ww[u]];
    }
  }
}

}  // namespace

size_t apply_smem_bytes(int n, int E) {
  const size_t R = (size_t)(E + 1) * n + 1;
  return (2 * R * kLd + 2 * (size_t)(E + 1) * kApplyLines + 2 * (size_t)E * kApplyLines) * sizeof(double);
}

template <int N, bool US> static cudaError_t set_limit_us() {
  cudaError_t e = cudaFuncSetAttribute(apply_kernel<N, kApplyFirst, US>, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(apply_kernel<N, kApplyMid, US>, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(apply_kernel<N, kApplyLast, US>, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
  return e;
}

template <int N> static cudaError_t set_limit() {
  cudaError_t e = set_limit_us<N, false>();
  if constexpr (N <= kExactStiffnessMaxN)
    if (e == cudaSuccess) e = set_limit_us<N, true>();
  return e;
}

cudaError_t apply_set_smem_limits() {
  cudaError_t e = cudaSuccess;
#define HOFEM_AP_LIMIT(NN) if (e == cudaSuccess) e = set_limit<NN>();
  HOFEM_AP_LIMIT(1) HOFEM_AP_LIMIT(2) HOFEM_AP_LIMIT(3) HOFEM_AP_LIMIT(4) HOFEM_AP_LIMIT(5) HOFEM_AP_LIMIT(6)
  HOFEM_AP_LIMIT(7) HOFEM_AP_LIMIT(8) HOFEM_AP_LIMIT(9) HOFEM_AP_LIMIT(10) HOFEM_AP_LIMIT(11) HOFEM_AP_LIMIT(12)
  HOFEM_AP_LIMIT(13) HOFEM_AP_LIMIT(14) HOFEM_AP_LIMIT(15) HOFEM_AP_LIMIT(16)
#undef HOFEM_AP_LIMIT
  return e;
}

template <int N, bool US> static void launch_us(const ApplyParams& p, cudaStream_t s) {
  const dim3 grid((unsigned)p.ntiles), block(kApplyThreads);
  switch (p.mode) {
    case kApplyFirst: apply_kernel<N, kApplyFirst, US><<<grid, block, p.smem_bytes, s>>>(p); break;
    case kApplyMid: apply_kernel<N, kApplyMid, US><<<grid, block, p.smem_bytes, s>>>(p); break;
    default: apply_kernel<N, kApplyLast, US><<<grid, block, p.smem_bytes, s>>>(p); break;
  }
}

template <int N> static void launch_n(const ApplyParams& p, cudaStream_t s) {
  if constexpr (N <= kExactStiffnessMaxN) {
    if (p.uniform) {
      launch_us<N, true>(p, s);
      return;
    }
  }
  launch_us<N, false>(p, s);
}

cudaError_t launch_apply(const ApplyParams& p, cudaStream_t s) {
  if (p.mode < kApplyFirst || p.mode > kApplyLast) return cudaErrorInvalidValue;
  if (p.uniform && p.n > kExactStiffnessMaxN) return cudaErrorInvalidValue;
  switch (p.n) {
#define HOFEM_AP_CASE(NN) \
  case NN: launch_n<NN>(p, s); break;
    HOFEM_AP_CASE(1) HOFEM_AP_CASE(2) HOFEM_AP_CASE(3) HOFEM_AP_CASE(4) HOFEM_AP_CASE(5) HOFEM_AP_CASE(6)
    HOFEM_AP_CASE(7) HOFEM_AP_CASE(8) HOFEM_AP_CASE(9) HOFEM_AP_CASE(10) HOFEM_AP_CASE(11) HOFEM_AP_CASE(12)
    HOFEM_AP_CASE(13) HOFEM_AP_CASE(14) HOFEM_AP_CASE(15) HOFEM_AP_CASE(16)
#undef HOFEM_AP_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace hofem

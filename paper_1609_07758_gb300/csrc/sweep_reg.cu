// Register-resident axis sweep (FP32) for element orders and power-of-two K fixed at
// compile time: the direct (Theorem 2 part 2) and inverse (Theorem 2 part 1) F_n-transforms
// of W lines of one axis, optionally fused with the eigenvalue-sum division of algorithm (a)
// (Eq. decomp v 2).  Same line layout, spectral layout and tables as sweep_kernel.
//
// DST-I of a job (two real sequences a, b of length K-1 as x_j = a_j + i b_j, x_0 = 0):
// with X = DFT_K(x) and Z = DFT_K(x_j e^{-i pi j / K}) (the even and odd bins of the
// 2K-point DFT of x zero-padded),
//   2 DST(a)_k = -Im D,  2 DST(b)_k = Re D,   D = X_m - X_{K-m}       (k = 2m)
//                                             D = Z_m - Z_{K-1-m}     (k = 2m + 1).
// Each K-point DFT (K = 32 L) runs on a group of L lanes with 32 complex values per lane in
// registers: lane r holds x_{r + L n2} (n2 < 32); a 32-point DFT over n2 with compile-time
// twiddles, the inter-stage twiddle w_K^{r k2} (w_2K^{r (2 k2 + 1)} for Z), a transpose
// within the group through shared memory, and 32 / L L-point DFTs leave X_{k2 + 32 k1}
// (k2 = r + L t) in register t L + k1.  The partner X_{K-m} of every output sits in lane
// L - r (Z_{K-1-m} in lane L - 1 - r) of the same group at a register fixed at compile
// time, so the DST outputs come out of one shuffle per value.
//
// The pre-combine of the direct transform and the post-combine of the inverse one are
// gathers from the tile (in the DST loads and in the store), so every job works on its
// own slots and no phase needs an in-place update.  Each warp holds one job (K = 1024) or
// 32 / L jobs at a time, transposing through its own area of shared memory; a CTA runs its
// jobs in rounds of one per lane group.
#include <cstdint>
#include <cstdlib>

#include "sweep.cuh"

#ifndef HOFEM_REG_PART
#define HOFEM_REG_PART -1
#endif
#ifndef HOFEM_REG_MIX
#define HOFEM_REG_MIX 0
#endif
#pragma nv_diag_suppress 177   // each part compiles one kernel and uses only some helpers

namespace hofem {
namespace {
// Compile-time shape of one instantiation.
template <int N_, int LOGK_, int W_, int NW_> struct RegCfg {
  static constexpr int N = N_, LOGK = LOGK_, W = W_, NW = NW_;
  static constexpr int K = 1 << LOGK, L = K / 32, T = 32 / L, G = 32 / L;
  static constexpr int M = N * K - 1;
  static constexpr int PAIRS = (N - 1) / 2;
  static constexpr int NJOBS = W * PAIRS + ((N % 2 == 0) ? W : (W + 1) / 2);
  static constexpr int NT = 32 * NW;
  // line stride in the tile: >= M and = 32 / W (mod 32) for W | 32, so that the strided
  // loads (W consecutive lines per row) write distinct banks
  static constexpr int MSR = (W >= 1 && W <= 32 && (32 % W) == 0) ? (32 / W) % 32 : 1;
  static constexpr int MS = M + ((MSR - M % 32) % 32 + 32) % 32;
  static constexpr int WIN = 32 * 33 * 2;          // floats of one warp's transpose area
  static constexpr int TF = (W * MS + 3) & ~3;
  static constexpr int SCR = NW * WIN;
  static constexpr int ROUNDS = (NJOBS + NW * G - 1) / (NW * G);   // job rounds per CTA
  static constexpr int SAVE = ((W * (N > 1 ? N - 1 : 1)) + 3) & ~3;
  static constexpr int LR = (W + 3) & ~3;
  static constexpr size_t SMEM = (size_t)(TF + SCR + SAVE + LR) * 4 + (size_t)NW * 8;
  static_assert(LOGK >= 6 && LOGK <= 10, "K = 64 .. 1024");
  // per-frequency mixing form (HOFEM_REG_MIX): 0 one thread per frequency over all lines,
  // 1 one thread per (frequency, group of up to 4 lines), 2 tensor cores (3xTF32
  // m16n8k8) where n = 8 and the lines come in groups of 16, else form 1
  static constexpr int MIX = HOFEM_REG_MIX == 2 ? ((N == 8 && W % 16 == 0) ? 2 : 1) : HOFEM_REG_MIX;
};

}  // namespace

#if HOFEM_REG_PART != 100
namespace {

// cos(2 pi k / 64), k = 0..16
__host__ __device__ constexpr double cos64_q(int k) {
  switch (k) {
    case 0: return 1.0;
    case 1: return 0.99518472667219688624;
    case 2: return 0.98078528040323044913;
    case 3: return 0.95694033573220886494;
    case 4: return 0.92387953251128675613;
    case 5: return 0.88192126434835502971;
    case 6: return 0.83146961230254523708;
    case 7: return 0.77301045336273696081;
    case 8: return 0.70710678118654752440;
    case 9: return 0.63439328416364549822;
    case 10: return 0.55557023301960222474;
    case 11: return 0.47139673682599764856;
    case 12: return 0.38268343236508977173;
    case 13: return 0.29028467725446236764;
    case 14: return 0.19509032201612826785;
    case 15: return 0.09801714032956060199;
    default: return 0.0;
  }
}

__host__ __device__ constexpr double cos64(int k) {
  k &= 63;
  return k <= 16 ? cos64_q(k) : k <= 32 ? -cos64_q(32 - k) : k <= 48 ? -cos64_q(k - 32) : cos64_q(64 - k);
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// b exp(-2 pi i e / 64) for an exponent known at compile time
__device__ __forceinline__ float2 rot64(float2 b, int e) {
  e &= 63;
  if (e == 0) return b;
  if (e == 16) return make_float2(b.y, -b.x);
  if (e == 32) return make_float2(-b.x, -b.y);
  if (e == 48) return make_float2(-b.y, b.x);
  const float c = (float)cos64(e), s = (float)cos64(e - 16);
  return make_float2(fmaf(b.x, c, b.y * s), fmaf(b.y, c, -b.x * s));
}

// 4-byte asynchronous global -> shared copy; src_bytes = 0 writes a zero (nothing is read)
__device__ __forceinline__ void cp_async4(float* dst, const float* src, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}


// In-register forward DFT of R = 1..32 points (a power of two), natural order in and out:
// split radix (decimation in time), X_k = E_k + w^k O1_k + w^3k O3_k from the R/2-point DFT
// of the even inputs and the R/4-point DFTs of inputs 4m + 1 and 4m + 3, with compile-time
// twiddles (26 general twiddle products at R = 32 against 34 for radix 2).
template <int R> __device__ __forceinline__ void dft(float2 (&v)[R]) {
  if constexpr (R == 2) {
    const float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  } else if constexpr (R >= 4) {
    constexpr int H = R / 2, Q = R / 4;
    float2 e[H], o1[Q], o3[Q];
#pragma unroll
    for (int m = 0; m < H; ++m) e[m] = v[2 * m];
#pragma unroll
    for (int m = 0; m < Q; ++m) {
      o1[m] = v[4 * m + 1];
      o3[m] = v[4 * m + 3];
    }
    dft<H>(e);
    dft<Q>(o1);
    dft<Q>(o3);
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      const float2 z1 = rot64(o1[k], k * (64 / R)), z3 = rot64(o3[k], 3 * k * (64 / R));
      const float2 s = cadd(z1, z3), d = csub(z1, z3);
      v[k] = cadd(e[k], s);
      v[k + H] = csub(e[k], s);
      v[k + Q] = make_float2(e[k + Q].x + d.y, e[k + Q].y - d.x);       // E - i d
      v[k + 3 * Q] = make_float2(e[k + Q].x - d.y, e[k + Q].y + d.x);   // E + i d
    }
  }
}

struct RJob {
  int wa, ca, wb, cb;   // component c of line w; c = 0: nodes; cb < 0: absent
};

template <class C> __device__ __forceinline__ RJob rjob(int jx) {
  if (jx < C::W * C::PAIRS) {
    const int gp = jx / C::W + 1, w = jx % C::W;
    return RJob{w, gp, w, C::N - gp};
  }
  const int r2 = jx - C::W * C::PAIRS;
  if (C::N % 2 == 0) return RJob{r2, 0, r2, C::N / 2};
  return RJob{2 * r2, 0, 2 * r2 + 1 < C::W ? 2 * r2 + 1 : 0, 2 * r2 + 1 < C::W ? 0 : -1};
}

template <class C> __device__ __forceinline__ int slotc(int c) { return c == 0 ? C::N - 1 : c - 1; }

// twt: the pass's inter-stage twiddles, twt[k2 L + r] = w_K^{r k2} (X) or w_2K^{r (2 k2 + 1)}
// (Z), a K-entry table in global memory (L1-resident) laid out so that the lanes of a group
// read consecutive entries.
template <class C, bool Z>
__device__ __forceinline__ void group_fft(float2 (&v)[32], float2* win, int lane, int g, int r,
                                          const float2* twt) {
  constexpr int L = C::L;
  dft<32>(v);
  if (r != 0) {
#pragma unroll
    for (int k2 = Z ? 0 : 1; k2 < 32; ++k2) v[k2] = cmul(v[k2], __ldg(twt + k2 * L + r));
  }
  __syncwarp();
#pragma unroll
  for (int k2 = 0; k2 < 32; ++k2) win[k2 * 33 + lane] = v[k2];
  __syncwarp();
#pragma unroll
  for (int t = 0; t < C::T; ++t) {
    float2 u[L];
    const int row = (r + L * t) * 33 + g * L;
#pragma unroll
    for (int n1 = 0; n1 < L; ++n1) u[n1] = win[row + n1];
    dft<L>(u);
#pragma unroll
    for (int k1 = 0; k1 < L; ++k1) v[t * L + k1] = u[k1];
  }
}

__device__ __forceinline__ float2 shfl2(float2 a, int src) {
  return make_float2(__shfl_sync(0xffffffffu, a.x, src), __shfl_sync(0xffffffffu, a.y, src));
}

// D_m = X_m - X_{K-m} for m = r + L t + 32 k1, k1 < L / 2 (d index t (L/2) + k1)
template <class C> __device__ __forceinline__ void extract_x(const float2 (&v)[32], float2 (&d)[16], int g, int r) {
  constexpr int L = C::L, T = C::T;
  const int src = g * L + ((L - r) & (L - 1));
#pragma unroll
  for (int t = 0; t < T; ++t) {
#pragma unroll
    for (int k1 = 0; k1 < L / 2; ++k1) {
      const float2 pv = shfl2(v[(T - 1 - t) * L + (L - 1 - k1)], src);
      const float2 own = t >= 1 ? v[(T - t) * L + (L - 1 - k1)] : (k1 >= 1 ? v[L - k1] : v[0]);
      d[t * (L / 2) + k1] = csub(v[t * L + k1], r == 0 ? own : pv);
    }
  }
}

// D_m = Z_m - Z_{K-1-m}
template <class C> __device__ __forceinline__ void extract_z(const float2 (&v)[32], float2 (&d)[16], int lane) {
  constexpr int L = C::L, T = C::T;
  const int src = lane ^ (L - 1);
#pragma unroll
  for (int t = 0; t < T; ++t) {
#pragma unroll
    for (int k1 = 0; k1 < L / 2; ++k1) {
      const float2 pv = shfl2(v[(T - 1 - t) * L + (L - 1 - k1)], src);
      d[t * (L / 2) + k1] = csub(v[t * L + k1], pv);
    }
  }
}

// Where job jb reads its inputs: x_j = t[o1 + j N] + wt t[o2 + j N] for each of its two
// sequences (j = 1..K-1).  Forward: the pre-combined physical sequence of component c,
// t[j N + c - 1] + t[j N - c - 1] (the nodes, c = 0: t[j N - 1], weight 0); inverse: the
// spectral slot (weight 0).  Both reads are unconditional, so that the unrolled loads of
// a job issue back to back, and the weight is uniform per job (no select per value).
struct JobIn {
  int a1, a2, b1, b2;
  float wa, wb;
};
template <class C> __device__ __forceinline__ JobIn job_in(const RJob& jb, bool fwd) {
  constexpr int N = C::N, MS = C::MS;
  const int cb = jb.cb >= 0 ? jb.cb : jb.ca;
  auto o1 = [&](int c) { return c == 0 ? -1 : (fwd ? c - 1 : c - 1 - N); };
  auto o2 = [&](int c) { return fwd ? -c - 1 : o1(c); };
  JobIn ji;
  ji.a1 = jb.wa * MS + o1(jb.ca);
  ji.a2 = jb.wa * MS + o2(jb.ca);
  ji.b1 = jb.wb * MS + o1(cb);
  ji.b2 = jb.wb * MS + o2(cb);
  ji.wa = fwd && jb.ca != 0 ? 1.f : 0.f;
  ji.wb = fwd && cb != 0 ? 1.f : 0.f;
  return ji;
}

// Input x_j (j = r + L n2) of a job; zero at j = 0 and for groups without a job.  Reads
// are made at clamped, valid indices and masked afterwards (no branch around a load).
// FWDM: 0 inverse, 1 forward (known at compile time), 2 either (both reads made).
template <class C, int FWDM>
__device__ __forceinline__ float2 job_input(const float* tile, const RJob& jb, const JobIn& ji, bool active, int j) {
  // masks only where the shape needs them (known at compile time): idle lane groups in the
  // last job round, node jobs without a second line; x_0 = 0 is set by the caller
  constexpr bool MASK_ACTIVE = (C::NJOBS % (C::NW * C::G)) != 0;
  constexpr bool MASK_B = (C::N % 2 == 1) && (C::W % 2 == 1);
  const int o = (j > 0 ? j : 1) * C::N;
  float a = tile[ji.a1 + o], b = tile[ji.b1 + o];
  if (FWDM != 0) {
    a = fmaf(ji.wa, tile[ji.a2 + o], a);
    b = fmaf(ji.wb, tile[ji.b2 + o], b);
  }
  if (MASK_ACTIVE) {
    a = active ? a : 0.f;
    b = active ? b : 0.f;
  }
  if (MASK_B) b = jb.cb >= 0 ? b : 0.f;
  return make_float2(a, b);
}

// All DST jobs of the tile.  Forward (FWDM = 1, or 2 with fwd set): pre-combined physical
// sequences -> 2 x DST in the spectral slots.  Inverse (FWDM = 0, or 2 with fwd clear):
// spectral sequences -> 2 x DST (D_j) in the same slots.
// Per job: X from the loaded inputs, its outputs held in registers; the inputs loaded
// again, times w_64^{n2}, for Z; a barrier (every job's reads of the tile are done); the
// X outputs stored; Z, whose outputs are stored as they are extracted.  The transposes
// use the warp's own area of `scr`.
template <class C, int FWDM>
__device__ __forceinline__ void dst_jobs(float* tile, float* scr, const float2* __restrict__ twx,
                                         const float2* __restrict__ twz, bool fwd = FWDM == 1) {
  constexpr int L = C::L, N = C::N;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int g = lane / L, r = lane % L;
  float2* win = reinterpret_cast<float2*>(scr) + wid * (C::WIN / 2);
#pragma unroll 1
  for (int round = 0; round < C::ROUNDS; ++round) {
    // jobs touch disjoint slots of the tile, so a later round's inputs are intact
    const int jx = (round * C::NW + wid) * C::G + g;
    const bool active = jx < C::NJOBS;
    const RJob jb = rjob<C>(active ? jx : 0);
    const JobIn ji = job_in<C>(jb, FWDM == 2 ? fwd : FWDM == 1);
    float2 v[32], d[16];
#pragma unroll
    for (int n2 = 0; n2 < 32; ++n2) v[n2] = job_input<C, FWDM>(tile, jb, ji, active, r + L * n2);
    if (r == 0) v[0] = make_float2(0.f, 0.f);   // x_0 = 0 (j = r + L n2 is 0 only here)
    __syncwarp();    // the previous round's reads of the transpose area are done
    group_fft<C, false>(v, win, lane, g, r, twx);
    extract_x<C>(v, d, g, r);
#pragma unroll
    for (int n2 = 0; n2 < 32; ++n2) v[n2] = rot64(job_input<C, FWDM>(tile, jb, ji, active, r + L * n2), n2);
    if (r == 0) v[0] = make_float2(0.f, 0.f);
    __syncthreads();   // every job of this round has read its inputs
    float* ta = tile + jb.wa * C::MS + slotc<C>(jb.ca);
    float* tb = jb.cb >= 0 ? tile + jb.wb * C::MS + slotc<C>(jb.cb) : nullptr;
    if (active) {
#pragma unroll
      for (int t = 0; t < C::T; ++t) {
#pragma unroll
        for (int k1 = 0; k1 < L / 2; ++k1) {
          const int m = r + L * t + 32 * k1;
          const float2 a = d[t * (L / 2) + k1];
          if (m >= 1) {                               // k = 2m at block k - 1
            ta[(2 * m - 1) * N] = -a.y;
            if (tb) tb[(2 * m - 1) * N] = a.x;
          }
        }
      }
    }
    __syncwarp();    // the first transpose's reads are done before the area is rewritten
    group_fft<C, true>(v, win, lane, g, r, twz);
    extract_z<C>(v, d, lane);
    if (active) {
#pragma unroll
      for (int t = 0; t < C::T; ++t) {
#pragma unroll
        for (int k1 = 0; k1 < L / 2; ++k1) {
          const int m = r + L * t + 32 * k1;
          const float2 b = d[t * (L / 2) + k1];
          ta[(2 * m) * N] = -b.y;                     // k = 2m + 1
          if (tb) tb[(2 * m) * N] = b.x;
        }
      }
    }
  }
  __syncthreads();
}

// Per-frequency mixing, one thread per frequency k and every line of the tile; the k = 0
// block by one thread per line.  MODE: kFwd (w = G x / 2K), kInv (x = G^T w / 2) or
// kFwdScaleInv (both, with the division by lam + rest between them).  G_k is read from the
// frequency-fastest copy of the table (consecutive threads, consecutive addresses) into
// registers and applied to the lines one by one.
// FP32 value as a TF32 operand (round to nearest, ties away) and the TF32 remainder
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(x));
  const float r = x - __uint_as_float(hi);
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lo) : "f"(r));
}

// d += a b for one m16n8k8 TF32 tile (FP32 accumulate)
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// d = a b with a, b split into TF32 hi + lo: hi hi + hi lo + lo hi (the lo lo term and
// the remainders are ~2^-22 relative), small terms first
__device__ __forceinline__ void mma_3xtf32(float (&d)[4], const float (&a)[4], const float (&b)[2]) {
  uint32_t ah[4], al[4], bh[2], bl[2];
#pragma unroll
  for (int i = 0; i < 4; ++i) split_tf32(a[i], ah[i], al[i]);
#pragma unroll
  for (int i = 0; i < 2; ++i) split_tf32(b[i], bh[i], bl[i]);
#pragma unroll
  for (int i = 0; i < 4; ++i) d[i] = 0.f;
  mma_tf32(d, al, bh);
  mma_tf32(d, ah, bl);
  mma_tf32(d, ah, bh);
}

// Per-frequency mixing of n = 8 on the tensor cores: for frequency k and 16 lines, the
// forward Y = X G_k^T / 2K (X: lines x components, A operand from the tile; B[s][l] =
// G_k[l][s]) and the inverse Y = X G_k / 2 (B[l][s] = G_k[l][s]), one warp per
// (frequency, 16 lines).  Fragment layouts of m16n8k8: lane = 4 g + t holds A rows g,
// g + 8 and columns t, t + 4; B row (k) t, t + 4 and column g; C rows g, g + 8 and columns
// 2t, 2t + 1.  The fused sweep divides the C fragment and passes it to the inverse
// product through the warp's own tile slots.
template <class C, int MODE>
__device__ __forceinline__ void mixing_tc(float* tile, const float* lrest, const SweepParams& P) {
  constexpr int N = C::N, K = C::K, KM = C::K - 1;
  static_assert(N == 8 && C::W % 16 == 0, "tensor-core mixing: n = 8, 16 lines per group");
  const float* __restrict__ mt = P.mixT;
  const float* __restrict__ lt = P.lamT;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  for (int item = wid; item < KM * (C::W / 16); item += C::NW) {
    const int kk = item % KM, wb = (item / KM) * 16;
    float* r0 = tile + (wb + g) * C::MS + kk * N;
    float* r1 = r0 + 8 * C::MS;
    float a[4] = {r0[t], r1[t], r0[t + 4], r1[t + 4]};
    float d[4];
    if (MODE & kFwd) {
      const float b[2] = {__ldg(mt + (g * N + t) * KM + kk), __ldg(mt + (g * N + t + 4) * KM + kk)};
      mma_3xtf32(d, a, b);
#pragma unroll
      for (int i = 0; i < 4; ++i) d[i] *= 0.5f / K;
      if (MODE == kFwdScaleInv) {
        const float l0 = __ldg(lt + (2 * t) * KM + kk), l1 = __ldg(lt + (2 * t + 1) * KM + kk);
        const float w0 = lrest[wb + g], w1 = lrest[wb + g + 8];
        d[0] = __fdividef(d[0], l0 + w0);   // ~2 ulp, refined
        d[1] = __fdividef(d[1], l1 + w0);
        d[2] = __fdividef(d[2], l0 + w1);
        d[3] = __fdividef(d[3], l1 + w1);
        __syncwarp();
        r0[2 * t] = d[0];
        r0[2 * t + 1] = d[1];
        r1[2 * t] = d[2];
        r1[2 * t + 1] = d[3];
        __syncwarp();
        a[0] = r0[t];
        a[1] = r1[t];
        a[2] = r0[t + 4];
        a[3] = r1[t + 4];
      }
    }
    if (MODE & kInv) {
      const float b[2] = {__ldg(mt + (t * N + g) * KM + kk), __ldg(mt + ((t + 4) * N + g) * KM + kk)};
      mma_3xtf32(d, a, b);
#pragma unroll
      for (int i = 0; i < 4; ++i) d[i] *= 0.5f;
    }
    __syncwarp();
    r0[2 * t] = d[0];
    r0[2 * t + 1] = d[1];
    r1[2 * t] = d[2];
    r1[2 * t + 1] = d[3];
  }
}

template <class C, int MODE>
__device__ __forceinline__ void mixing(float* tile, float* save, const float* lrest, const SweepParams& P) {
  constexpr int N = C::N, K = C::K, W = C::W, KM = C::K - 1;
  const float* __restrict__ mt = P.mixT;
  const float* __restrict__ lt = P.lamT;
  const float* __restrict__ lam = (const float*)P.lam;
  // lines per work item of the scalar forms
  constexpr int LG = C::MIX == 0 ? W : (W < 4 ? W : 4);
  constexpr int NIT = C::MIX == 2 ? 0 : KM * (W / LG);
  if constexpr (C::MIX == 2) mixing_tc<C, MODE>(tile, lrest, P);
  for (int item = (int)threadIdx.x; item < NIT; item += C::NT) {
    const int kk = item % KM, wl = (item / KM) * LG, base = kk * N;
    float G[N][N], lq[N];
#pragma unroll
    for (int l = 0; l < N; ++l)
#pragma unroll
      for (int s = 0; s < N; ++s) G[l][s] = __ldg(mt + (l * N + s) * KM + kk);
    if (MODE == kFwdScaleInv) {
#pragma unroll
      for (int l = 0; l < N; ++l) lq[l] = __ldg(lt + l * KM + kk);
    }
#pragma unroll(LG <= 4 ? LG : 1)
    for (int w = wl; w < wl + LG; ++w) {
      float x[N], y[N];
#pragma unroll
      for (int s = 0; s < N; ++s) x[s] = tile[w * C::MS + base + s];
      if (MODE & kFwd) {
#pragma unroll
        for (int l = 0; l < N; ++l) {
          float acc = 0.f;
#pragma unroll
          for (int s = 0; s < N; ++s) acc = fmaf(G[l][s], x[s], acc);
          y[l] = acc * (0.5f / K);
        }
        if (MODE == kFwdScaleInv) {
          const float rw = lrest[w];
#pragma unroll
          for (int l = 0; l < N; ++l) x[l] = __fdividef(y[l], lq[l] + rw);   // ~2 ulp, refined
        }
      }
      if (MODE & kInv) {
#pragma unroll
        for (int s = 0; s < N; ++s) y[s] = 0.f;
#pragma unroll
        for (int l = 0; l < N; ++l)
#pragma unroll
          for (int s = 0; s < N; ++s) y[s] = fmaf(G[l][s], x[l], y[s]);
#pragma unroll
        for (int s = 0; s < N; ++s) y[s] *= 0.5f;
      }
#pragma unroll
      for (int s = 0; s < N; ++s) tile[w * C::MS + base + s] = y[s];
    }
  }
  if constexpr (N > 1) {
    constexpr int Mm = N - 1;
    const float* __restrict__ E = (const float*)P.evec;
    for (int w = threadIdx.x; w < W; w += C::NT) {
      const int base = (K - 1) * N;
      float x[Mm], y[Mm];
#pragma unroll
      for (int s = 0; s < Mm; ++s) {
        x[s] = (MODE & kFwd) ? save[w * Mm + s] : tile[w * C::MS + base + s];
        y[s] = 0.f;
      }
      if (MODE & kFwd) {
#pragma unroll
        for (int l = 0; l < Mm; ++l) {
          float acc = 0.f;
#pragma unroll
          for (int s = 0; s < Mm; ++s) acc = fmaf(__ldg(E + l * Mm + s), x[s], acc);
          y[l] = acc * (1.0f / K);
        }
        if (MODE == kFwd) {
#pragma unroll
          for (int l = 0; l < Mm; ++l) tile[w * C::MS + base + l] = y[l];
        } else {
#pragma unroll
          for (int l = 0; l < Mm; ++l) {
            x[l] = y[l] / (__ldg(lam + base + l) + lrest[w]);
            y[l] = 0.f;
          }
        }
      }
      if (MODE & kInv) {
#pragma unroll
        for (int l = 0; l < Mm; ++l)
#pragma unroll
          for (int s = 0; s < Mm; ++s) y[s] = fmaf(__ldg(E + l * Mm + s), x[l], y[s]);
#pragma unroll
        for (int s = 0; s < Mm; ++s) save[w * Mm + s] = y[s];
      }
    }
  }
  __syncthreads();
}

// Where tile b of a sweep lies: outer index o, first line l0, lines present, right-hand
// side and the global offset of its first element.
struct TileGeo {
  long long o, l0, rhs, gbase;
  int wvalid;
};

template <int W, int M, bool CONTIG>
__device__ __forceinline__ TileGeo tile_geo(const SweepParams& P, const long long b) {
  TileGeo g;
  g.o = b / P.tiles_per_outer;
  const long long tix = b - g.o * P.tiles_per_outer;
  g.l0 = tix * W;
  const long long nl = CONTIG ? P.outer_per_rhs : P.inner;
  g.wvalid = (int)(nl - g.l0 < W ? nl - g.l0 : W);
  g.rhs = CONTIG ? g.o : g.o / P.outer_per_rhs;
  g.gbase = CONTIG ? (g.o * P.outer_per_rhs + g.l0) * (long long)M : g.o * (long long)M * P.inner + g.l0;
  return g;
}

// Load W FP64 lines into the FP32 tile (missing lines read as zeros).  Contiguous lines go
// line by line (position p = p0 + u NT, no index division); strided tiles as elements
// e = p W + w.  The loads of an unrolled group are unconditional at clamped valid
// addresses, so that they are all in flight at once.
template <class C, bool CONTIG>
__device__ __forceinline__ void load_f64(const SweepParams& P, const TileGeo& g, float* tile) {
  constexpr int M = C::M, MS = C::MS, NT = C::NT, W = C::W, TOT = W * M, UL = 32;
  constexpr int LW = W == 1 ? 0 : W == 2 ? 1 : W == 4 ? 2 : W == 8 ? 3 : W == 16 ? 4 : 5;
  const int tid = threadIdx.x;
  const double* __restrict__ in = (const double*)P.in;
  if constexpr (CONTIG) {
    for (int w = 0; w < W; ++w) {
      const bool lv = w < g.wvalid;
      const double* src = in + g.gbase + (long long)(lv ? w : 0) * M;
      for (int p0 = tid; p0 < M; p0 += UL * NT) {
        double v[UL];
#pragma unroll
        for (int u = 0; u < UL; ++u) v[u] = __ldg(src + (p0 + u * NT < M ? p0 + u * NT : 0));
#pragma unroll
        for (int u = 0; u < UL; ++u)
          if (p0 + u * NT < M) tile[w * MS + p0 + u * NT] = lv ? (float)v[u] : 0.f;
      }
    }
  } else {
    for (int e0 = tid; e0 < TOT; e0 += UL * NT) {
      double v[UL];
#pragma unroll
      for (int u = 0; u < UL; ++u) {
        const int e = e0 + u * NT, w = e & (W - 1), p = e >> LW;
        v[u] = __ldg(in + ((e < TOT && w < g.wvalid) ? g.gbase + p * P.inner + w : g.gbase));
      }
#pragma unroll
      for (int u = 0; u < UL; ++u) {
        const int e = e0 + u * NT, w = e & (W - 1), p = e >> LW;
        if (e < TOT) tile[w * MS + p] = w < g.wvalid ? (float)v[u] : 0.f;
      }
    }
  }
}

// Issue asynchronous 4-byte copies of W FP32 lines straight into the tile (zero-filled for
// the missing lines), the whole tile in flight at once; the caller commits and waits.
template <class C, bool CONTIG>
__device__ __forceinline__ void load_f32_async(const SweepParams& P, const TileGeo& g, float* tile) {
  constexpr int M = C::M, MS = C::MS, NT = C::NT, W = C::W, TOT = W * M;
  constexpr int LW = W == 1 ? 0 : W == 2 ? 1 : W == 4 ? 2 : W == 8 ? 3 : W == 16 ? 4 : 5;
  const int tid = threadIdx.x;
  const float* __restrict__ in = (const float*)P.in;
  if constexpr (CONTIG) {
    for (int w = 0; w < W; ++w) {
      const bool lv = w < g.wvalid;
      const float* src = in + g.gbase + (long long)(lv ? w : 0) * M;
      for (int p = tid; p < M; p += NT) cp_async4(tile + w * MS + p, src + p, lv ? 4 : 0);
    }
  } else {
    for (int e = tid; e < TOT; e += NT) {
      const int w = e & (W - 1), p = e >> LW;
      const bool ok = w < g.wvalid;
      cp_async4(tile + w * MS + p, in + (ok ? g.gbase + p * P.inner + w : g.gbase), ok ? 4 : 0);
    }
  }
}

// Shared-memory areas of a CTA besides its tile(s).
struct RegAreas {
  float* scr;
  float* save;
  float* lrest;
  double* red;
};

// Everything of tile g after its load has been issued and completed by this thread: the
// per-line eigenvalue rest of the fused sweep, a barrier (the tile and rests visible to all),
// the transforms and mixing, the store (and the norm of the stored update).
template <class C, int MODE, bool CONTIG>
__device__ __forceinline__ void work_tile(const SweepParams& P, const TileGeo& g, float* tile, const RegAreas& a) {
  constexpr int N = C::N, W = C::W, NW = C::NW;
  constexpr int M = C::M, MS = C::MS, NT = C::NT, K = C::K;
  static_assert((W & (W - 1)) == 0, "W is a power of two");
  constexpr int LW = W == 1 ? 0 : W == 2 ? 1 : W == 4 ? 2 : W == 8 ? 3 : W == 16 ? 4 : 5;
  constexpr int TOT = W * M, U = 16;
  float* scr = a.scr;
  float* save = a.save;
  float* lrest = a.lrest;
  double* red = a.red;
  const float2* twx = (const float2*)P.twr;
  const float2* twz = twx + K;
  const int tid = threadIdx.x;
  const long long l0 = g.l0, rhs = g.rhs, gbase = g.gbase, inner = P.inner;
  const int wvalid = g.wvalid;
  if constexpr (MODE == kFwdScaleInv) {
    for (int w = tid; w < W; w += NT) {
      const long long c = P.line_offset + l0 + w;
      float rest = 0.f;
      if (w < wvalid) {
        const long long qa = P.lamB ? c / P.MB : c;
        rest += ((const float*)P.lamA)[qa];
        if (P.lamB) rest += ((const float*)P.lamB)[c - qa * P.MB];
      }
      lrest[w] = (float)P.alpha + rest;
    }
  }
  __syncthreads();

  if constexpr ((MODE & kFwd) != 0) {
    // k = 0 sums t_i = sum_j (-P)^{j-1} y_{j-1/2}, component i, one warp per (line, i)
    if constexpr (N > 1) {
      const int lane = tid & 31, wid = tid >> 5;
      for (int item = wid; item < W * (N - 1); item += NW) {
        const int w = item % W, i = item / W + 1;
        float acc = 0.f;
        for (int j = 1 + lane; j <= K; j += 32) {
          const float v = tile[w * MS + (j - 1) * N + ((j & 1) ? i : N - i) - 1];
          acc += (j & 1) ? v : -v;
        }
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
        if (lane == 0) save[w * (N - 1) + i - 1] = acc;
      }
    }
  }
  if constexpr (MODE == kFwdScaleInv && C::LOGK >= 10) {
    // one copy of the DST code for both transforms: at K = 1024 two copies of the fused
    // sweep's code stall its warps on instruction fetch (measured 1.24 -> 1.15 ms at n = 9,
    // against the inverse's extra read per input); at smaller K the copies are shorter and
    // the extra reads cost more than they save (n = 4, K = 128: 1.14 -> 1.24 ms)
#pragma unroll 1
    for (int ph = 0; ph < 2; ++ph) {
      if (ph == 1) mixing<C, MODE>(tile, save, lrest, P);
      dst_jobs<C, 2>(tile, scr, twx, twz, ph == 0);
    }
  } else {
    if constexpr ((MODE & kFwd) != 0) dst_jobs<C, 1>(tile, scr, twx, twz);
    mixing<C, MODE>(tile, save, lrest, P);
    if constexpr ((MODE & kInv) != 0) dst_jobs<C, 0>(tile, scr, twx, twz);
  }

  // ---- store: spectral tile (direct sweep) or the post-combine of the inverse transform,
  //   v_j = D_j (nodes),  v_{j-1/2,c} = D_{j-1,c} + D_{j,N-c} + (-1)^{j-1} g_{c or N-c}
  constexpr bool inv = (MODE & kInv) != 0;
  const bool want_norm = P.norms != nullptr;
  float s_d = 0.f;
  auto value = [&](int w, int p) -> float {
    const float* t = tile + w * MS;
    if (!inv || N == 1) return t[p];
    const int j = p / N + 1, c = p - (j - 1) * N + 1;
    // clamped reads, masked: D_{j-1, c} (j >= 2), D_{j, N-c} (j <= K-1), g (c < N)
    const int cc = c < N ? c : 1;
    const float d0 = t[j >= 2 ? p - N : p], d1 = t[j <= K - 1 ? p + N - 2 * cc : p];
    const float* gs = save + w * (N > 1 ? N - 1 : 1);
    const float ga = gs[cc - 1], gb = gs[N - cc - 1];
    const float v = (j >= 2 ? d0 : 0.f) + (j <= K - 1 ? d1 : 0.f) + ((j & 1) ? ga : -gb);
    return c == N ? t[p] : v;
  };
  if (P.out_fmt == kFmtF64) {
    double* out = (double*)P.out;
    if constexpr (CONTIG) {
      for (int w = 0; w < wvalid; ++w) {
        double* dst = out + gbase + (long long)w * M;
        for (int p0 = tid; p0 < M; p0 += U * NT) {
          double prev[U];
          if (P.accumulate) {
#pragma unroll
            for (int u = 0; u < U; ++u) prev[u] = dst[p0 + u * NT < M ? p0 + u * NT : 0];
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int p = p0 + u * NT;
            if (p < M) {
              const float tv = value(w, p);
              dst[p] = P.accumulate ? prev[u] + (double)tv : (double)tv;
              if (want_norm) s_d = fmaf(tv, tv, s_d);
            }
          }
        }
      }
    } else {
      for (int e0 = tid; e0 < TOT; e0 += U * NT) {
        double prev[U];
        if (P.accumulate) {
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int e = e0 + u * NT, w = e & (W - 1), p = e >> LW;
            prev[u] = out[(e < TOT && w < wvalid) ? gbase + p * inner + w : gbase];
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int e = e0 + u * NT, w = e & (W - 1), p = e >> LW;
          if (e < TOT && w < wvalid) {
            const float tv = value(w, p);
            out[gbase + p * inner + w] = P.accumulate ? prev[u] + (double)tv : (double)tv;
            if (want_norm) s_d = fmaf(tv, tv, s_d);
          }
        }
      }
    }
  } else {
    float* out = (float*)P.out;
    if constexpr (CONTIG) {
      for (int w = 0; w < wvalid; ++w) {
        float* dst = out + gbase + (long long)w * M;
        for (int p0 = tid; p0 < M; p0 += U * NT) {
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (p0 + u * NT < M) dst[p0 + u * NT] = value(w, p0 + u * NT);
        }
      }
    } else {
      for (int e0 = tid; e0 < TOT; e0 += U * NT) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int e = e0 + u * NT, w = e & (W - 1), p = e >> LW;
          if (e < TOT && w < wvalid) out[gbase + p * inner + w] = value(w, p);
        }
      }
    }
  }
  if (want_norm) {
    const int lane = tid & 31, wid = tid >> 5;
    double sd = (double)s_d;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) sd += __shfl_xor_sync(0xffffffffu, sd, s);
    if (lane == 0) red[wid] = sd;
    __syncthreads();
    if (tid == 0) {
      double a = 0.0;
      for (int i = 0; i < NW; ++i) a += red[i];
      atomicAdd(&P.norms[2 * rhs + P.norm_slot], a);
    }
  }
}

// One sweep of MODE over contiguous (CONTIG) or strided lines: one CTA per tile of W lines.
template <int N, int LOGK, int W, int NW, int MINB, int MODE, bool CONTIG>
__global__ void __launch_bounds__(32 * NW, MINB) sweep_reg_kernel(const SweepParams P) {
  using C = RegCfg<N, LOGK, W, NW>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* tile = reinterpret_cast<float*>(smem_raw);
  float* scr = tile + C::TF;
  float* save = scr + C::SCR;
  float* lrest = save + C::SAVE;
  const RegAreas a{scr, save, lrest, reinterpret_cast<double*>(lrest + C::LR)};
  const TileGeo g = tile_geo<W, C::M, CONTIG>(P, blockIdx.x);
  if (P.in_fmt == kFmtF64) {
    load_f64<C, CONTIG>(P, g, tile);
  } else {
    load_f32_async<C, CONTIG>(P, g, tile);
    cp_async_wait_all();
  }
  work_tile<C, MODE, CONTIG>(P, g, tile, a);
}

}  // namespace
#endif

// ---- instantiations: (id, order, log2 K, lines per CTA, warps per CTA, CTAs per SM), each
// with five kernels: forward on contiguous / strided lines, the fused sweep (always on the
// strided axis 0), inverse on contiguous / strided lines.  The build compiles this file once
// per kernel (HOFEM_REG_PART = 5 id + kernel) and once for the dispatch table
// (HOFEM_REG_PART = 100), so the kernels compile in parallel; without the macro one object
// holds everything.
// (order, log2 K, lines per CTA, warps per CTA, CTAs per SM) of each id.  A build may
// time another launch shape of the n = 9, K = 1024 kernels with -DHOFEM_REG0_W=...,
// -DHOFEM_REG0_NW=..., -DHOFEM_REG0_MB=...
#ifndef HOFEM_REG0_W
#define HOFEM_REG0_W 4
#endif
#ifndef HOFEM_REG0_NW
#define HOFEM_REG0_NW 9
#endif
#ifndef HOFEM_REG0_MB
#define HOFEM_REG0_MB 1
#endif
#define HOFEM_REG_SHAPE0 9, 10, HOFEM_REG0_W, HOFEM_REG0_NW, HOFEM_REG0_MB   /* 2D n = 9, K = 1024 (9215^2 unknowns) */
#define HOFEM_REG_SHAPE1 4, 7, 16, 4, 3                                      /* 3D n = 4, K = 128 */
#define HOFEM_REG_SHAPE2 8, 6, 16, 4, 3                                      /* 3D n = 8, K = 64 */
#define HOFEM_REG_CALL(X, ...) X(__VA_ARGS__)
#define HOFEM_REG_LIST(X) \
  HOFEM_REG_CALL(X, 0, HOFEM_REG_SHAPE0) \
  HOFEM_REG_CALL(X, 1, HOFEM_REG_SHAPE1) \
  HOFEM_REG_CALL(X, 2, HOFEM_REG_SHAPE2)


#define HOFEM_REG_DECL(ID, NN, LK, WW, NWW, MB)                                                \
  cudaError_t reg_attr_##ID##_0(); cudaError_t reg_attr_##ID##_1(); cudaError_t reg_attr_##ID##_2(); \
  cudaError_t reg_attr_##ID##_3(); cudaError_t reg_attr_##ID##_4();                            \
  cudaError_t reg_launch_##ID##_0(const SweepParams& p, cudaStream_t s);                       \
  cudaError_t reg_launch_##ID##_1(const SweepParams& p, cudaStream_t s);                       \
  cudaError_t reg_launch_##ID##_2(const SweepParams& p, cudaStream_t s);                       \
  cudaError_t reg_launch_##ID##_3(const SweepParams& p, cudaStream_t s);                       \
  cudaError_t reg_launch_##ID##_4(const SweepParams& p, cudaStream_t s);
HOFEM_REG_LIST(HOFEM_REG_DECL)
#undef HOFEM_REG_DECL

#define HOFEM_REG_DEF(ID, KI, NN, LK, WW, NWW, MB, MODE, CONTIG)                                          \
  cudaError_t reg_launch_##ID##_##KI(const SweepParams& p, cudaStream_t s) {                           \
    sweep_reg_kernel<NN, LK, WW, NWW, MB, MODE, CONTIG>                                                \
        <<<(unsigned)p.ntiles, 32 * NWW, RegCfg<NN, LK, WW, NWW>::SMEM, s>>>(p);                       \
    return cudaGetLastError();                                                                          \
  }                                                                                                     \
  cudaError_t reg_attr_##ID##_##KI() {                                                                  \
    return cudaFuncSetAttribute(sweep_reg_kernel<NN, LK, WW, NWW, MB, MODE, CONTIG>,                   \
                                cudaFuncAttributeMaxDynamicSharedMemorySize,                            \
                                (int)RegCfg<NN, LK, WW, NWW>::SMEM);                                    \
  }

// the id, kernel index, mode and layout first, so that the shape macro can close the list
#define HOFEM_REG_DEF_S(ID, KI, MODE, CONTIG, NN, LK, WW, NWW, MB) \
  HOFEM_REG_DEF(ID, KI, NN, LK, WW, NWW, MB, MODE, CONTIG)

#if HOFEM_REG_PART < 0 || HOFEM_REG_PART == 0
HOFEM_REG_CALL(HOFEM_REG_DEF_S, 0, 0, kFwd, true, HOFEM_REG_SHAPE0)
#endif
#if HOFEM_REG_PART < 0 || HOFEM_REG_PART == 1
HOFEM_REG_CALL(HOFEM_REG_DEF_S, 0, 1, kFwd, false, HOFEM_REG_SHAPE0)
#endif
#if HOFEM_REG_PART < 0 || HOFEM_REG_PART == 2
HOFEM_REG_CALL(HOFEM_REG_DEF_S, 0, 2, kFwdScaleInv, false, HOFEM_REG_SHAPE0)
#endif
#if HOFEM_REG_PART < 0 || HOFEM_REG_PART == 3
HOFEM_REG_CALL(HOFEM_REG_DEF_S, 0, 3, kInv, true, HOFEM_REG_SHAPE0)
#endif
#if HOFEM_REG_PART < 0 || HOFEM_REG_PART == 4
HOFEM_REG_CALL(HOFEM_REG_DEF_S, 0, 4, kInv, false, HOFEM_REG_SHAPE0)
#endif
#if HOFEM_REG_PART < 0 || HOFEM_REG_PART == 5
HOFEM_REG_CALL(HOFEM_REG_DEF_S, 1, 0, kFwd, true, HOFEM_REG_SHAPE1)
#endif
#if HOFEM_REG_PART < 0 || HOFEM_REG_PART == 6
HOFEM_REG_CALL(HOFEM_REG_DEF_S, 1, 1, kFwd, false, HOFEM_REG_SHAPE1)
#endif
#if HOFEM_REG_PART < 0 || HOFEM_REG_PART == 7
HOFEM_REG_CALL(HOFEM_REG_DEF_S, 1, 2, kFwdScaleInv, false, HOFEM_REG_SHAPE1)
#endif
#if HOFEM_REG_PART < 0 || HOFEM_REG_PART == 8
HOFEM_REG_CALL(HOFEM_REG_DEF_S, 1, 3, kInv, true, HOFEM_REG_SHAPE1)
#endif
#if HOFEM_REG_PART < 0 || HOFEM_REG_PART == 9
HOFEM_REG_CALL(HOFEM_REG_DEF_S, 1, 4, kInv, false, HOFEM_REG_SHAPE1)
#endif
#if HOFEM_REG_PART < 0 || HOFEM_REG_PART == 10
HOFEM_REG_CALL(HOFEM_REG_DEF_S, 2, 0, kFwd, true, HOFEM_REG_SHAPE2)
#endif
#if HOFEM_REG_PART < 0 || HOFEM_REG_PART == 11
HOFEM_REG_CALL(HOFEM_REG_DEF_S, 2, 1, kFwd, false, HOFEM_REG_SHAPE2)
#endif
#if HOFEM_REG_PART < 0 || HOFEM_REG_PART == 12
HOFEM_REG_CALL(HOFEM_REG_DEF_S, 2, 2, kFwdScaleInv, false, HOFEM_REG_SHAPE2)
#endif
#if HOFEM_REG_PART < 0 || HOFEM_REG_PART == 13
HOFEM_REG_CALL(HOFEM_REG_DEF_S, 2, 3, kInv, true, HOFEM_REG_SHAPE2)
#endif
#if HOFEM_REG_PART < 0 || HOFEM_REG_PART == 14
HOFEM_REG_CALL(HOFEM_REG_DEF_S, 2, 4, kInv, false, HOFEM_REG_SHAPE2)
#endif

#if HOFEM_REG_PART < 0 || HOFEM_REG_PART == 100
namespace {

struct RegEntry {
  int n, logK, W, nw;
  size_t smem;
  cudaError_t (*launch[5])(const SweepParams&, cudaStream_t);
  cudaError_t (*attr[5])();
};

#define HOFEM_REG_ENTRY(ID, NN, LK, WW, NWW, MB)                                                  \
  RegEntry{NN, LK, WW, NWW, RegCfg<NN, LK, WW, NWW>::SMEM,                                      \
           {reg_launch_##ID##_0, reg_launch_##ID##_1, reg_launch_##ID##_2, reg_launch_##ID##_3, \
            reg_launch_##ID##_4},                                                               \
           {reg_attr_##ID##_0, reg_attr_##ID##_1, reg_attr_##ID##_2, reg_attr_##ID##_3, reg_attr_##ID##_4}},
const RegEntry kRegTable[] = {HOFEM_REG_LIST(HOFEM_REG_ENTRY)};
#undef HOFEM_REG_ENTRY

const RegEntry* reg_entry(int n, int K) {
  for (const RegEntry& e : kRegTable)
    if (e.n == n && (1 << e.logK) == K) return &e;
  return nullptr;
}

// kernel index of a sweep: forward contiguous / strided, fused (strided), inverse
// contiguous / strided; -1: no kernel (a fused sweep on contiguous lines)
int reg_kernel_index(int mode, bool contiguous) {
  if (mode == kFwd) return contiguous ? 0 : 1;
  if (mode == kFwdScaleInv) return contiguous ? -1 : 2;
  return contiguous ? 3 : 4;
}

}  // namespace

bool sweep_reg_shape(int n, int K, int* W, int* threads, size_t* smem) {
  const RegEntry* e = reg_entry(n, K);
  if (!e) return false;
  *W = e->W;
  *threads = 32 * e->nw;
  *smem = e->smem;
  return true;
}

cudaError_t sweep_reg_set_smem_limits() {
  for (const RegEntry& e : kRegTable)
    for (int k = 0; k < 5; ++k) {
      cudaError_t r = e.attr[k]();
      if (r != cudaSuccess) return r;
    }
  return cudaSuccess;
}

cudaError_t launch_sweep_reg(const SweepParams& p, cudaStream_t s) {
  const RegEntry* e = reg_entry(p.n, p.K);
  const int k = reg_kernel_index(p.mode, p.inner == 1);
  if (!e || e->W != p.W || k < 0) return cudaErrorInvalidValue;
  return e->launch[k](p, s);
}
#endif

}  // namespace hofem

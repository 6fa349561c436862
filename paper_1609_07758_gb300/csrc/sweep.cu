// Axis sweep kernel: direct (Theorem 2 part 2) and inverse (Theorem 2 part 1) F_n-
// transforms of W lines of one axis held in shared memory, optionally fused with the
// eigenvalue-sum scaling of algorithm (a) (Eq. decomp v 2).
//
// Line layout: unknown p = (j-1) n + (i-1) is element j's local point i (i = n: node j).
// Spectral layout after a direct transform: q = (k-1) n + (l-1) for k = 1..K-1 (the n
// modes of frequency k), then q = n (K-1) + (l-1) for the k = 0 modes (Theorem 1 part 2).
//
// Direct transform of y (Theorem 2 part 2, with the eigenvectors of Theorem 1 part 3
// normalised by u^T C_k u = 1, so that ||s||_C^2 = K):
//   nodes      Y_j = y_j,                                j = 1..K-1
//   interiors  z_{j,i} = y_{j+1/2,i} + y_{j-1/2,n-i},    j = 1..K-1  (the even/odd
//              combination of the theorem written without splitting into parts)
//   n DST-I    Yhat_k = sum_j Y_j sin(pi k j / K),  Zhat_{k,i} likewise
//   mixing     w_{k,l} = (c_l Yhat_k + q_l . Zhat_k) / K
//   k = 0      w_{0,l} = e^(l) . sum_j (-P)^{j-1} y_{j-1/2} / K
// Inverse transform (Theorem 2 part 1): a_k = sum_l c_l w_{k,l}, d_k = sum_l q_l w_{k,l},
// g = sum_l w_{0,l} e^(l); A_j, D_j = DST-I of a, d; v_j = A_j and
// v_{j-1/2} = D_{j-1} + P D_j + (-P)^{j-1} g with D_0 = D_K = 0.  The paper's
// [n/2] DST-III + [(n-1)/2] DCT-III of the element-centre values are replaced here by
// n DST-I of the node-aligned sequences, which is the same linear map.
//
// DST-I on the GPU: two real sequences a, b form x = a + i b; the 2K-point DFT of the
// odd extension of x is -2i (DST(a) + i DST(b)).  One radix-2 decimation-in-frequency
// step splits it into two K-point complex FFTs of u_j = x_j - x_{K-j} (even outputs)
// and v_j = (x_j + x_{K-j}) exp(-i pi j / K) (odd outputs), done in shared memory by
// Stockham autosort passes of radix 2..16 with register butterflies.
#include <cstdint>
#include <algorithm>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "sweep.cuh"

// The build compiles this file three times (HOFEM_SWEEP_PART = 0: host helpers and absmax;
// 1: the FP32 kernel instantiations and their launcher; 2: the FP64 ones) so that the
// instantiations compile in parallel; without the macro one object holds everything.
#ifndef HOFEM_SWEEP_PART
#define HOFEM_SWEEP_PART -1
#endif
#define HOFEM_SWEEP_HAS(k) (HOFEM_SWEEP_PART < 0 || HOFEM_SWEEP_PART == (k))

namespace hofem {

template <typename T> struct Cx;
template <> struct Cx<float> { using type = float2; };
template <> struct Cx<double> { using type = double2; };

template <typename C> __device__ __forceinline__ C c_add(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C c_sub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C c_mul(C a, C b) {
  return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

// cos(2 pi k / 32), k = 0..8 (the rest by symmetry)
__host__ __device__ constexpr double cos32_base(int k) {
  switch (k) {
    case 0: return 1.0;
    case 1: return 0.98078528040323043058;
    case 2: return 0.92387953251128673848;
    case 3: return 0.83146961230254523567;
    case 4: return 0.70710678118654757274;
    case 5: return 0.55557023301960228867;
    case 6: return 0.38268343236508983729;
    case 7: return 0.19509032201612833135;
    default: return 0.0;
  }
}

__host__ __device__ constexpr double cos32(int k) {
  k &= 31;
  return k <= 8 ? cos32_base(k) : k <= 16 ? -cos32_base(16 - k) : k <= 24 ? -cos32_base(k - 16) : cos32_base(32 - k);
}

// b * exp(-2 pi i e / 32) for a compile-time-resolvable e
template <typename T, typename C> __device__ __forceinline__ C tw32(C b, int e) {
  e &= 31;
  if (e == 0) return b;
  if (e == 8) return C{b.y, -b.x};
  if (e == 16) return C{-b.x, -b.y};
  if (e == 24) return C{-b.y, b.x};
  const T c = (T)cos32(e), s = (T)cos32(e - 8);
  return C{b.x * c + b.y * s, b.y * c - b.x * s};
}

template <int R> __host__ __device__ constexpr int bitrev(int i) {
  int r = 0;
  for (int b = 1; b < R; b <<= 1) {
    r = (r << 1) | (i & 1);
    i >>= 1;
  }
  return r;
}

// In-register forward DFT of R = 1..32 points (iterative radix-2, natural order out).
template <typename T, int R, typename C> __device__ __forceinline__ void dft_reg(C (&v)[R]) {
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int j = bitrev<R>(i);
    if (j > i) {
      C t = v[i];
      v[i] = v[j];
      v[j] = t;
    }
  }
#pragma unroll
  for (int half = 1; half < R; half <<= 1) {
#pragma unroll
    for (int s = 0; s < R; s += 2 * half) {
#pragma unroll
      for (int k = 0; k < half; ++k) {
        C a = v[s + k];
        C b = tw32<T>(v[s + k + half], k * (32 / (2 * half)));
        v[s + k] = c_add(a, b);
        v[s + k + half] = c_sub(a, b);
      }
    }
  }
}

template <int R> struct Log2;
template <> struct Log2<1> { static constexpr int v = 0; };
template <> struct Log2<32> { static constexpr int v = 5; };
template <> struct Log2<2> { static constexpr int v = 1; };
template <> struct Log2<4> { static constexpr int v = 2; };
template <> struct Log2<8> { static constexpr int v = 3; };
template <> struct Log2<16> { static constexpr int v = 4; };

// Complex registers per thread a pass may hold (R x butterflies per thread).
template <typename T> struct CReg;
template <> struct CReg<float> { static constexpr int v = 32; };
template <> struct CReg<double> { static constexpr int v = 16; };

// Bank-conflict-free layouts.  Tile element e is stored at e + (e >> TileSwz<T>): one pad
// word per 32 banks' worth, so the stride-n and stride-nW walks of the pre-combine, the
// post-combine and the mixing hit distinct banks.  FFT buffer entry e of an FFT is stored
// at e + (e >> FftPad<T>) (one pad complex per 128 bytes), which removes the stride-R
// conflicts of the first Stockham pass.
template <typename T> struct TileSwz;
template <> struct TileSwz<float> { static constexpr int v = 5; };
template <> struct TileSwz<double> { static constexpr int v = 4; };
template <typename T> struct FftPad;
template <> struct FftPad<float> { static constexpr int v = 4; };
template <> struct FftPad<double> { static constexpr int v = 3; };

template <typename T> __host__ __device__ __forceinline__ int fft_stride(int N) {
  return N + (N >> FftPad<T>::v);
}
template <typename T> __device__ __forceinline__ int fpad(int e) { return e + (e >> FftPad<T>::v); }

// One in-place decimation-in-frequency pass (Gentleman-Sande) of radix R over nfft FFTs
// of length N = 2^logN stored back to back (padded) in buf.  Blocks have length
// L = 2^logL; butterfly (block, j) combines the R entries j + r L/R of its block,
// y_q = sum_r x_r exp(-2 pi i r q / R), then twiddles y_q by exp(-2 pi i j q / L) and
// stores it back in the slot of x_q.  Every butterfly reads and writes the same R
// slots, so a pass needs one barrier and one butterfly's registers per thread.  After
// all passes the output is in mixed-radix digit-reversed order (see fft_pos).
// tw[t] = exp(-i pi t / N), t < 2N.
template <typename T, int R>
__device__ __noinline__ void fft_pass(typename Cx<T>::type* buf, int logN, int nfft, int logL,
                                      const typename Cx<T>::type* __restrict__ tw) {
  using C = typename Cx<T>::type;
  constexpr int LR = Log2<R>::v;
  const int N = 1 << logN;
  const int logQ = logL - LR;                  // stride L / R
  const int logB = logN - LR;                  // butterflies per FFT
  const int nb = nfft << logB;
  const int FS = fft_stride<T>(N);
  const int tsh = logN - logL + 1;             // exp(-2 pi i j q / L) = tw[(j q) << tsh]
  const int mask2N = 2 * N - 1;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const int f = b >> logB;
    const int rem = b & ((1 << logB) - 1);
    const int blk = rem >> logQ;
    const int j = rem & ((1 << logQ) - 1);
    C* base = buf + (size_t)f * FS;
    const int e0 = (blk << logL) + j;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = base[fpad<T>(e0 + (r << logQ))];
    dft_reg<T, R>(v);
    if (j != 0) {
#pragma unroll
      for (int q = 1; q < R; ++q) v[q] = c_mul(v[q], tw[((j * q) << tsh) & mask2N]);
    }
#pragma unroll
    for (int q = 0; q < R; ++q) base[fpad<T>(e0 + (q << logQ))] = v[q];
  }
  __syncthreads();
}

// The inverse of one fft_pass up to the factor R, on conjugates: with conj(y) in the
// pass's output slots, z_q = w_L^{jq} conj(y)_{j + qL/R} and the forward R-point DFT of z
// give R conj(x_r) in the input slots j + r L/R.  Run over the passes of a DIF network in
// reverse order, this maps conj(Y) in digit-reversed order to N conj(IDFT(Y)) in natural
// order.
template <typename T, int R>
__device__ __noinline__ void fft_pass_inv(typename Cx<T>::type* buf, int logN, int nfft, int logL,
                                          const typename Cx<T>::type* __restrict__ tw) {
  using C = typename Cx<T>::type;
  constexpr int LR = Log2<R>::v;
  const int N = 1 << logN;
  const int logQ = logL - LR;
  const int logB = logN - LR;
  const int nb = nfft << logB;
  const int FS = fft_stride<T>(N);
  const int tsh = logN - logL + 1;
  const int mask2N = 2 * N - 1;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const int f = b >> logB;
    const int rem = b & ((1 << logB) - 1);
    const int blk = rem >> logQ;
    const int j = rem & ((1 << logQ) - 1);
    C* base = buf + (size_t)f * FS;
    const int e0 = (blk << logL) + j;
    C v[R];
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = base[fpad<T>(e0 + (q << logQ))];
    if (j != 0) {
#pragma unroll
      for (int q = 1; q < R; ++q) v[q] = c_mul(v[q], tw[((j * q) << tsh) & mask2N]);
    }
    dft_reg<T, R>(v);
#pragma unroll
    for (int r = 0; r < R; ++r) base[fpad<T>(e0 + (r << logQ))] = v[r];
  }
  __syncthreads();
}

// DIF passes over nfft FFTs of length 2^logN: the K plan (P.radix) or, NBPLAN, the
// Bluestein length's plan (P.nb_radix); INV runs the inverse network (fft_pass_inv, passes
// in reverse order).
template <typename T, bool NBPLAN = false, bool INV = false>
__device__ void fft_all(typename Cx<T>::type* buf, int logN, int nfft, const SweepParams& P,
                        const typename Cx<T>::type* __restrict__ tw) {
  auto lg = [](int R) { return (R == 16) ? 4 : (R == 8) ? 3 : (R == 4) ? 2 : 1; };
  const int np = NBPLAN ? P.nb_npass : P.npass;
  if constexpr (!INV) {
    int logL = logN;
    for (int ps = 0; ps < np; ++ps) {
      const int R = NBPLAN ? P.nb_radix[ps] : P.radix[ps];
      if (R == 16) fft_pass<T, 16>(buf, logN, nfft, logL, tw);
      else if (R == 8) fft_pass<T, 8>(buf, logN, nfft, logL, tw);
      else if (R == 4) fft_pass<T, 4>(buf, logN, nfft, logL, tw);
      else fft_pass<T, 2>(buf, logN, nfft, logL, tw);
      logL -= lg(R);
    }
  } else {
    int logL = logN;                            // block length of the last pass
    for (int ps = 0; ps + 1 < np; ++ps) logL -= lg((NBPLAN ? P.nb_radix[ps] : P.radix[ps]));
    for (int ps = np - 1; ps >= 0; --ps) {
      const int R = (NBPLAN ? P.nb_radix[ps] : P.radix[ps]);
      if (R == 16) fft_pass_inv<T, 16>(buf, logN, nfft, logL, tw);
      else if (R == 8) fft_pass_inv<T, 8>(buf, logN, nfft, logL, tw);
      else if (R == 4) fft_pass_inv<T, 4>(buf, logN, nfft, logL, tw);
      else fft_pass_inv<T, 2>(buf, logN, nfft, logL, tw);
      if (ps > 0) logL += lg((NBPLAN ? P.nb_radix[ps - 1] : P.radix[ps - 1]));
    }
  }
}

// Bluestein convolution of nfft chirped sequences (stored, zero-padded to nb, by
// dst_load_general): forward DIF FFT, product with the filter's transform (already / nb),
// conjugated, then the inverse network; leaves conj((x c) * conj(c)) in natural order.
template <typename T>
__device__ void bluestein_conv(typename Cx<T>::type* buf, int nfft, const SweepParams& P,
                               const typename Cx<T>::type* __restrict__ twB,
                               const typename Cx<T>::type* __restrict__ filt) {
  using C = typename Cx<T>::type;
  fft_all<T, true, false>(buf, P.nb_log, nfft, P, twB);
  const int FS = fft_stride<T>(P.nb), items = nfft << P.nb_log, mask = P.nb - 1;
  for (int i = threadIdx.x; i < items; i += blockDim.x) {
    const int f = i >> P.nb_log, s = i & mask;
    C* e = buf + (size_t)f * FS + fpad<T>(s);
    const C y = c_mul(*e, filt[s]);
    *e = C{y.x, -y.y};
  }
  __syncthreads();
  fft_all<T, true, true>(buf, P.nb_log, nfft, P, twB);
}

// Memory slot of frequency m after the DIF passes: the low digit of m (base R_1) selects
// the slot's top digit, and so on.
__device__ __forceinline__ int fft_pos(int m, int logN, const SweepParams& P) {
  int pos = 0, sh = logN;
  for (int ps = 0; ps < P.npass; ++ps) {
    const int lb = P.radix_log[ps];
    sh -= lb;
    pos |= (m & ((1 << lb) - 1)) << sh;
    m >>= lb;
  }
  return pos;
}

// ---------------------------------------------------------------------------------
// General K (not a power of two): mixed-radix decimation-in-frequency passes, each out of
// place.  A pass of radix R over blocks of length L (stride Q = L / R) writes
//   dst[b L + j + q Q] = w_L^{j q} sum_r src[b L + j + r Q] w_R^{r q},  w_X = exp(-2 pi i / X),
// one thread per output (R terms); the two buffers alternate between passes.  The
// powers of w_R and w_L are entries 2 x (K / R) and 2 x (K / L) of tw (period 2K).
template <typename T>
__device__ void fft_pass_direct(const typename Cx<T>::type* src, typename Cx<T>::type* dst, int K, int nfft, int L,
                                int R, const typename Cx<T>::type* __restrict__ tw) {
  using C = typename Cx<T>::type;
  const int Q = L / R, FS = fft_stride<T>(K), total = nfft * K;
  const int stepR = 2 * (K / R), stepL = 2 * (K / L);
  for (int o = threadIdx.x; o < total; o += blockDim.x) {
    const int f = o / K, s = o - f * K;
    const int blk = s / L, t = s - blk * L;
    const int q = t / Q, j = t - q * Q;
    const C* in = src + (size_t)f * FS;
    const int e0 = blk * L + j;
    C acc = in[fpad<T>(e0)];
    int x = 0;                                   // r q mod R
    for (int r = 1; r < R; ++r) {
      x += q;
      if (x >= R) x -= R;
      acc = c_add(acc, c_mul(in[fpad<T>(e0 + r * Q)], tw[x * stepR]));
    }
    if (j != 0 && q != 0) acc = c_mul(acc, tw[((j * q) % L) * stepL]);
    dst[(size_t)f * FS + fpad<T>(s)] = acc;
  }
  __syncthreads();
}

// All passes; returns the buffer holding the result (a or b).
template <typename T>
__device__ typename Cx<T>::type* fft_all_general(typename Cx<T>::type* a, typename Cx<T>::type* b, int K, int nfft,
                                                 const SweepParams& P, const typename Cx<T>::type* __restrict__ tw) {
  int L = K;
  for (int ps = 0; ps < P.npass; ++ps) {
    const int R = P.radix[ps];
    fft_pass_direct<T>(a, b, K, nfft, L, R, tw);
    typename Cx<T>::type* t = a;
    a = b;
    b = t;
    L /= R;
  }
  return a;
}

__device__ __forceinline__ int fft_pos_general(int m, const SweepParams& P) {
  int pos = 0;
  for (int ps = 0; ps < P.npass; ++ps) {
    const int R = P.radix[ps], d = m % R;
    m /= R;
    pos += d * P.radix_q[ps];
  }
  return pos;
}

// ---------------------------------------------------------------------------------
// Job = one complex DST pair: real part = component ma of line wa, imaginary part =
// component mb of line wb (mb < 0: absent).  Component 0 = nodes, i = 1..n-1 interior.
struct Job {
  int wa, ma, wb, mb;
};

__device__ __forceinline__ Job job_of(int jx, int W, int logW, int n) {
  const int P = (n - 1) >> 1;  // interior pairs (g, n-g), g = 1..P
  if (jx < (P << logW)) {
    const int g = (jx >> logW) + 1, w = jx & (W - 1);
    return Job{w, g, w, n - g};
  }
  const int r = jx - (P << logW);
  if ((n & 1) == 0) return Job{r, 0, r, n / 2};                 // nodes + middle interior
  return Job{2 * r, 0, 2 * r + 1 < W ? 2 * r + 1 : -1, 2 * r + 1 < W ? 0 : -1};  // nodes of 2 lines
}

__host__ __device__ __forceinline__ int num_jobs(int W, int n) {
  const int P = (n - 1) / 2;
  return W * P + (((n & 1) == 0) ? W : (W + 1) / 2);
}

template <typename T> struct Tile {
  T* t;
  int ps, ws;
  __device__ __forceinline__ T& at(int p, int w) const {
    const int e = p * ps + w * ws;
    return t[e + (e >> TileSwz<T>::v)];
  }
};

// spectral / node-aligned slot of component m inside a frequency block
__device__ __forceinline__ int slot_of(int m, int n) { return m == 0 ? n - 1 : m - 1; }

// forward pre-combined sequence value of component m of line w at j (1..K-1)
template <typename T>
__device__ __forceinline__ T fwd_seq(const Tile<T>& tl, int w, int m, int j, int n) {
  if (m == 0) return tl.at(j * n - 1, w);
  return tl.at(j * n + m - 1, w) + tl.at((j - 1) * n + n - m - 1, w);
}

template <typename T>
__device__ __forceinline__ typename Cx<T>::type pair_x(const Tile<T>& tl, const Job& jb, int j, int n, int K,
                                                      bool inverse) {
  using C = typename Cx<T>::type;
  if (j <= 0 || j >= K) return C{(T)0, (T)0};
  T a, b = (T)0;
  if (!inverse) {
    a = fwd_seq(tl, jb.wa, jb.ma, j, n);
    if (jb.mb >= 0) b = fwd_seq(tl, jb.wb, jb.mb, j, n);
  } else {
    a = tl.at((j - 1) * n + slot_of(jb.ma, n), jb.wa);
    if (jb.mb >= 0) b = tl.at((j - 1) * n + slot_of(jb.mb, n), jb.wb);
  }
  return C{a, b};
}

// Fill the FFT buffer for jobs [j0, j0 + nj): u (even outputs) and v (odd outputs).
template <typename T>
__device__ __noinline__ void dst_load(const Tile<T> tl, typename Cx<T>::type* buf, int j0, int nj, int W, int n,
                                      int K, bool inverse, const typename Cx<T>::type* __restrict__ tw) {
  using C = typename Cx<T>::type;
  const int half = K >> 1;
  const int logH = 30 - __clz(K);           // log2(K / 2)
  const int logW = 31 - __clz(W);
  const int items = nj << logH;
  const int FS = fft_stride<T>(K);
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int jb = it >> logH, t = it & (half - 1);
    const Job job = job_of(j0 + jb, W, logW, n);
    C* U = buf + (size_t)(2 * jb) * FS;
    C* V = U + FS;
    if (t == 0) {
      U[0] = C{(T)0, (T)0};
      V[0] = C{(T)0, (T)0};
      const C xh = pair_x(tl, job, half, n, K, inverse);      // t = K/2: u = 0, v = 2 x w^{K/2}
      U[fpad<T>(half)] = C{(T)0, (T)0};
      V[fpad<T>(half)] = c_mul(c_add(xh, xh), tw[half]);
      continue;
    }
    const C x1 = pair_x(tl, job, t, n, K, inverse);
    const C x2 = pair_x(tl, job, K - t, n, K, inverse);
    const C d = c_sub(x1, x2), sm = c_add(x1, x2);
    U[fpad<T>(t)] = d;
    U[fpad<T>(K - t)] = C{-d.x, -d.y};
    V[fpad<T>(t)] = c_mul(sm, tw[t]);
    V[fpad<T>(K - t)] = c_mul(sm, tw[K - t]);
  }
}

// 2 x DST of the real part (first) and imaginary part (second) at index k (1..K-1).
template <typename T>
__device__ __forceinline__ void dst_out(const typename Cx<T>::type* buf, int jb, int K, int logK, int k, T* a,
                                        T* b, const SweepParams& P) {
  const int FS = fft_stride<T>(K);
  const typename Cx<T>::type* U = buf + (size_t)(2 * jb) * FS;
  const int pos = fpad<T>(fft_pos(k >> 1, logK, P));
  const typename Cx<T>::type R = (k & 1) ? U[FS + pos] : U[pos];
  *a = -R.y;
  *b = R.x;
}

// dst_load for any K: t = 0 .. K/2 fills slots t and K - t of u and v.
// With a Bluestein plan (chirp non-null) every entry t is stored times c_t, the FFTs have
// length (and stride) of P.nb, and entries K .. nb-1 are zeroed.
template <typename T>
__device__ __noinline__ void dst_load_general(const Tile<T> tl, typename Cx<T>::type* buf, int j0, int nj, int W,
                                              int n, int K, bool inverse, const typename Cx<T>::type* __restrict__ tw,
                                              const typename Cx<T>::type* __restrict__ chirp, int NB) {
  using C = typename Cx<T>::type;
  const int per = K / 2 + 1;
  const int logW = 31 - __clz(W);
  const int items = nj * per;
  const int FS = fft_stride<T>(chirp ? NB : K);
  auto ch = [&](C v, int t) { return chirp ? c_mul(v, chirp[t]) : v; };
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int jb = it / per, t = it - jb * per;
    const Job job = job_of(j0 + jb, W, logW, n);
    C* U = buf + (size_t)(2 * jb) * FS;
    C* V = U + FS;
    if (t == 0) {
      U[0] = C{(T)0, (T)0};
      V[0] = C{(T)0, (T)0};
      continue;
    }
    const C x1 = pair_x(tl, job, t, n, K, inverse);
    if (2 * t == K) {                           // u = 0, v = 2 x w^{K/2}
      U[fpad<T>(t)] = C{(T)0, (T)0};
      V[fpad<T>(t)] = ch(c_mul(c_add(x1, x1), tw[t]), t);
      continue;
    }
    const C x2 = pair_x(tl, job, K - t, n, K, inverse);
    const C d = c_sub(x1, x2), sm = c_add(x1, x2);
    U[fpad<T>(t)] = ch(d, t);
    U[fpad<T>(K - t)] = ch(C{-d.x, -d.y}, K - t);
    V[fpad<T>(t)] = ch(c_mul(sm, tw[t]), t);
    V[fpad<T>(K - t)] = ch(c_mul(sm, tw[K - t]), K - t);
  }
  if (chirp) {
    const int pad = NB - K, tail = 2 * nj * pad;
    for (int it = threadIdx.x; it < tail; it += blockDim.x) {
      const int f = it / pad, t = K + (it - f * pad);
      buf[(size_t)f * FS + fpad<T>(t)] = C{(T)0, (T)0};
    }
  }
}

// DST output k of job jb from the FFT results (u at even k, v at odd k): after the direct
// passes in their digit order, after a Bluestein convolution at m = k / 2 in natural order
// as X_m = c_m conj(buf[m]).
template <typename T>
__device__ __forceinline__ void dst_out_general(const typename Cx<T>::type* buf, int jb, int K, int k, T* a, T* b,
                                                const SweepParams& P, const typename Cx<T>::type* __restrict__ chirp) {
  using C = typename Cx<T>::type;
  const int m = k >> 1;
  C R;
  if (chirp) {
    const int FS = fft_stride<T>(P.nb);
    const C y = buf[(size_t)(2 * jb + (k & 1)) * FS + fpad<T>(m)];
    R = c_mul(C{y.x, -y.y}, chirp[m]);
  } else {
    const int FS = fft_stride<T>(K);
    const C* U = buf + (size_t)(2 * jb) * FS;
    const int pos = fpad<T>(fft_pos_general(m, P));
    R = (k & 1) ? U[FS + pos] : U[pos];
  }
  *a = -R.y;
  *b = R.x;
}

// ---------------------------------------------------------------------------------
// Per-frequency n x n mixing, one thread per frequency k looping over the tile's lines
// two at a time; row l of G_k = (q_1..q_{n-1}, c) of mode (k, l) is read with 16-byte
// vector loads from a table whose rows are padded to NP (a multiple of 4) entries.
// Generic-address loads: `row` points into shared memory (staged tables) or global memory.
template <typename T, int N>
__device__ __forceinline__ void load_row(const T* row, T (&g)[N]) {
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int s = 0; s < N; s += 4) {
      const float4 v = reinterpret_cast<const float4*>(row)[s / 4];
      g[s] = v.x;
      if (s + 1 < N) g[s + 1] = v.y;
      if (s + 2 < N) g[s + 2] = v.z;
      if (s + 3 < N) g[s + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int s = 0; s < N; s += 2) {
      const double2 v = reinterpret_cast<const double2*>(row)[s / 2];
      g[s] = v.x;
      if (s + 1 < N) g[s + 1] = v.y;
    }
  }
}

// Block stride (elements of T) of one G_k in the shared staging area: N NP rounded so
// that consecutive blocks start an odd number of 16-byte units apart (conflict-free
// 16-byte loads by consecutive threads).
template <typename T, int N> __device__ __forceinline__ int stage_stride(int NP) {
  constexpr int per16 = 16 / (int)sizeof(T);
  const int b = N * NP;
  return ((b / per16) & 1) ? b : b + per16;
}

template <typename T, int N, bool FWD>
__device__ __forceinline__ void mix_one_k(const Tile<T>& tl, int W, int k, const T* Gk, int NP, T scale) {
  constexpr int LC = 2;
  const int base = (k - 1) * N;
  for (int w0 = 0; w0 < W; w0 += LC) {
    T x[LC][N], y[LC][N];
#pragma unroll
    for (int c = 0; c < LC; ++c)
#pragma unroll
      for (int s = 0; s < N; ++s) {
        x[c][s] = (w0 + c < W) ? tl.at(base + s, w0 + c) : (T)0;
        y[c][s] = (T)0;
      }
#pragma unroll
    for (int l = 0; l < N; ++l) {
      T g[N];
      load_row<T, N>(Gk + l * NP, g);
      if (FWD) {
#pragma unroll
        for (int c = 0; c < LC; ++c) {
          T acc = (T)0;
#pragma unroll
          for (int s = 0; s < N; ++s) acc = fma(g[s], x[c][s], acc);
          y[c][l] = acc * scale;
        }
      } else {
#pragma unroll
        for (int c = 0; c < LC; ++c)
#pragma unroll
          for (int s = 0; s < N; ++s) y[c][s] = fma(g[s], x[c][l], y[c][s]);
      }
    }
#pragma unroll
    for (int c = 0; c < LC; ++c)
      if (w0 + c < W)
#pragma unroll
        for (int s = 0; s < N; ++s) tl.at(base + s, w0 + c) = FWD ? y[c][s] : y[c][s] * scale;
  }
}

// The mixing tables are staged through shared memory (the FFT buffers, idle during the
// mixing) in chunks of frequencies with coalesced 16-byte copies, then read from there;
// reading them straight from L2 thread by thread was latency-bound.
template <typename T, int N, bool FWD>
__device__ __noinline__ void mix_impl(const Tile<T> tl, int W, int K, const T* __restrict__ mix, int NP,
                                      const T* __restrict__ evec, T* save, T scale, T scale0, T* stage,
                                      int stage_cap) {
  const int BS = stage_stride<T, N>(NP);
  const int CK = stage_cap / BS;
  if (CK >= 32) {
    constexpr int per16 = 16 / (int)sizeof(T);
    const int vec_per_block = (N * NP) / per16;
    for (int k0 = 1; k0 < K; k0 += CK) {
      const int nk = min(CK, K - k0);
      const int4* src = reinterpret_cast<const int4*>(mix + (size_t)(k0 - 1) * N * NP);
      const int nvec = nk * vec_per_block;
      for (int v = threadIdx.x; v < nvec; v += blockDim.x) {
        const int kb = v / vec_per_block, r = v - kb * vec_per_block;
        reinterpret_cast<int4*>(stage + (size_t)kb * BS)[r] = __ldg(src + v);
      }
      __syncthreads();
      for (int k = k0 + threadIdx.x; k < k0 + nk; k += blockDim.x)
        mix_one_k<T, N, FWD>(tl, W, k, stage + (size_t)(k - k0) * BS, NP, scale);
      __syncthreads();
    }
  } else {
    for (int k = 1 + threadIdx.x; k < K; k += blockDim.x)
      mix_one_k<T, N, FWD>(tl, W, k, mix + (size_t)(k - 1) * N * NP, NP, scale);
  }
  // k = 0 block: w_0 = E t / K (forward, t in the tile) or g = E^T w_0 (inverse, into save)
  if constexpr (N > 1) {
    constexpr int Mm = N - 1;
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
      const int base = (K - 1) * N;
      T x[Mm], y[Mm];
#pragma unroll
      for (int s = 0; s < Mm; ++s) {
        x[s] = tl.at(base + s, w);
        y[s] = (T)0;
      }
#pragma unroll
      for (int l = 0; l < Mm; ++l)
#pragma unroll
        for (int s = 0; s < Mm; ++s) {
          const T e = __ldg(evec + l * Mm + s);
          if (FWD) y[l] = fma(e, x[s], y[l]);
          else y[s] = fma(e, x[l], y[s]);
        }
#pragma unroll
      for (int s = 0; s < Mm; ++s) {
        if (FWD) tl.at(base + s, w) = y[s] * scale0;
        else save[w * Mm + s] = y[s];
      }
    }
  }
}

template <typename T, bool FWD>
__device__ __forceinline__ void mix_dispatch(const Tile<T> tl, int W, int n, int K, const T* __restrict__ mix, int NP,
                             const T* __restrict__ evec, T* save, T scale, T scale0, T* stage, int stage_cap) {
  switch (n) {
#define HOFEM_MIX_CASE(NN) \
  case NN: mix_impl<T, NN, FWD>(tl, W, K, mix, NP, evec, save, scale, scale0, stage, stage_cap); break;
    HOFEM_MIX_CASE(1) HOFEM_MIX_CASE(2) HOFEM_MIX_CASE(3) HOFEM_MIX_CASE(4)
    HOFEM_MIX_CASE(5) HOFEM_MIX_CASE(6) HOFEM_MIX_CASE(7) HOFEM_MIX_CASE(8)
    HOFEM_MIX_CASE(9) HOFEM_MIX_CASE(10) HOFEM_MIX_CASE(11) HOFEM_MIX_CASE(12)
    HOFEM_MIX_CASE(13) HOFEM_MIX_CASE(14) HOFEM_MIX_CASE(15) HOFEM_MIX_CASE(16)
#undef HOFEM_MIX_CASE
    default: break;
  }
}

template <typename T, bool GK>
__device__ void forward_transform(const Tile<T>& tl, typename Cx<T>::type* fbuf, T* tsave, int W, int n,
                                  int K, const SweepParams& P, const T* __restrict__ mix,
                                  const T* __restrict__ evec, const typename Cx<T>::type* __restrict__ tw) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  // k = 0 sums t_i = sum_j (-P)^{j-1} y_{j-1/2}, component i
  const int logW = 31 - __clz(W);
  for (int item = warp; item < W * (n - 1); item += nwarp) {
    const int w = item & (W - 1), i = (item >> logW) + 1;
    T acc = (T)0;
    for (int j = 1 + lane; j <= K; j += 32) {
      const T v = tl.at((j - 1) * n + ((j & 1) ? i : n - i) - 1, w);
      acc += (j & 1) ? v : -v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) tsave[w * (n - 1) + i - 1] = acc;
  }
  __syncthreads();
  // DST jobs, batch by batch
  const int logK = 31 - __clz(K);
  const int nj_tot = num_jobs(W, n), J = P.jobs_per_batch;
  for (int j0 = 0; j0 < nj_tot; j0 += J) {
    const int nj = min(J, nj_tot - j0);
    if constexpr (!GK) {
      dst_load<T>(tl, fbuf, j0, nj, W, n, K, false, tw);
      __syncthreads();
      fft_all<T>(fbuf, logK, 2 * nj, P, tw);
      const int items = nj << logK;
      for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int jb = it >> logK, k = it & (K - 1);
        if (k == 0) continue;
        const Job job = job_of(j0 + jb, W, logW, n);
        T a, b;
        dst_out<T>(fbuf, jb, K, logK, k, &a, &b, P);
        tl.at((k - 1) * n + slot_of(job.ma, n), job.wa) = a;
        if (job.mb >= 0) tl.at((k - 1) * n + slot_of(job.mb, n), job.wb) = b;
      }
    } else {
      const typename Cx<T>::type* chirp = P.nb ? tw + 2 * K + 2 * P.nb : nullptr;
      dst_load_general<T>(tl, fbuf, j0, nj, W, n, K, false, tw, chirp, P.nb);
      __syncthreads();
      const typename Cx<T>::type* res = fbuf;
      if (P.nb) bluestein_conv<T>(fbuf, 2 * nj, P, tw + 2 * K, chirp + K);
      else res = fft_all_general<T>(fbuf, fbuf + (size_t)J * 2 * fft_stride<T>(K), K, 2 * nj, P, tw);
      const int items = nj * K;
      for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int jb = it / K, k = it - jb * K;
        if (k == 0) continue;
        const Job job = job_of(j0 + jb, W, logW, n);
        T a, b;
        dst_out_general<T>(res, jb, K, k, &a, &b, P, chirp);
        tl.at((k - 1) * n + slot_of(job.ma, n), job.wa) = a;
        if (job.mb >= 0) tl.at((k - 1) * n + slot_of(job.mb, n), job.wb) = b;
      }
    }
    __syncthreads();
  }
  // k = 0 block
  for (int it = threadIdx.x; it < W * (n - 1); it += blockDim.x) {
    const int w = it & (W - 1), i = it >> logW;
    tl.at((K - 1) * n + i, w) = tsave[w * (n - 1) + i];
  }
  __syncthreads();
  // mixing: w_k = G_k xhat_k / (2K)  (the DST outputs above are 2 x DST)
  mix_dispatch<T, true>(tl, W, n, K, mix, P.mixNP, evec, tsave, (T)(0.5 / K), (T)(1.0 / K),
                        reinterpret_cast<T*>(fbuf), P.mix_direct ? 0 : 2 * P.fbuf_complex);
  __syncthreads();
}

template <typename T, bool GK>
__device__ void inverse_transform(const Tile<T>& tl, typename Cx<T>::type* fbuf, T* gsave, int W, int n,
                                  int K, const SweepParams& P, const T* __restrict__ mix,
                                  const T* __restrict__ evec, const typename Cx<T>::type* __restrict__ tw) {
  // mixing: xhat_k = G_k^T w_k / 2 (the DST below returns 2 x DST); g = E^T w_0
  mix_dispatch<T, false>(tl, W, n, K, mix, P.mixNP, evec, gsave, (T)0.5, (T)1.0,
                         reinterpret_cast<T*>(fbuf), P.mix_direct ? 0 : 2 * P.fbuf_complex);
  __syncthreads();
  const int logK = 31 - __clz(K);
  const int logW = 31 - __clz(W);
  const int nj_tot = num_jobs(W, n), J = P.jobs_per_batch;
  for (int j0 = 0; j0 < nj_tot; j0 += J) {
    const int nj = min(J, nj_tot - j0);
    const typename Cx<T>::type* res = fbuf;
    const typename Cx<T>::type* chirp = (GK && P.nb) ? tw + 2 * K + 2 * P.nb : nullptr;
    if constexpr (!GK) {
      dst_load<T>(tl, fbuf, j0, nj, W, n, K, true, tw);
      __syncthreads();
      fft_all<T>(fbuf, logK, 2 * nj, P, tw);
    } else {
      dst_load_general<T>(tl, fbuf, j0, nj, W, n, K, true, tw, chirp, P.nb);
      __syncthreads();
      if (P.nb) bluestein_conv<T>(fbuf, 2 * nj, P, tw + 2 * K, chirp + K);
      else res = fft_all_general<T>(fbuf, fbuf + (size_t)J * 2 * fft_stride<T>(K), K, 2 * nj, P, tw);
    }
    // post-combine into physical rows
    const int items = nj * K;
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
      int jb, j;
      if constexpr (!GK) {
        jb = it >> logK;
        j = (it & (K - 1)) + 1;                        // j = 1..K
      } else {
        jb = it / K;
        j = it - jb * K + 1;
      }
      const Job job = job_of(j0 + jb, W, logW, n);
      T a0 = (T)0, b0 = (T)0, a1 = (T)0, b1 = (T)0;   // D at j-1 and at j
      if constexpr (!GK) {
        if (j - 1 >= 1) dst_out<T>(res, jb, K, logK, j - 1, &a0, &b0, P);
        if (j <= K - 1) dst_out<T>(res, jb, K, logK, j, &a1, &b1, P);
      } else {
        if (j - 1 >= 1) dst_out_general<T>(res, jb, K, j - 1, &a0, &b0, P, chirp);
        if (j <= K - 1) dst_out_general<T>(res, jb, K, j, &a1, &b1, P, chirp);
      }
      if (job.ma == 0) {                        // nodes of line wa (and maybe wb)
        if (j <= K - 1) {
          tl.at(j * n - 1, job.wa) = a1;
          if (job.mb == 0) tl.at(j * n - 1, job.wb) = b1;
        }
        if (job.mb > 0) {                        // middle interior component n/2 (n even)
          const int i = job.mb, m = n - 1;
          const T g = gsave[job.wb * m + i - 1];
          tl.at((j - 1) * n + i - 1, job.wb) = b0 + b1 + ((j & 1) ? g : -g);
        }
      } else {                                   // interior pair (i, n-i) of line wa
        const int i = job.ma, ic = job.mb, m = n - 1, w = job.wa;
        const T gi = gsave[w * m + i - 1], gic = gsave[w * m + ic - 1];
        // v_{j-1/2} = D_{j-1} + P D_j + (-P)^{j-1} g
        const T vi = a0 + b1 + ((j & 1) ? gi : -gic);
        const T vic = b0 + a1 + ((j & 1) ? gic : -gi);
        tl.at((j - 1) * n + i - 1, w) = vi;
        tl.at((j - 1) * n + ic - 1, w) = vic;
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------
// Warp-register FFT path (FP32, K = 32 L with L = 1..32 lanes per FFT).
//
// A DST job (pair a + ib) needs the K-point FFTs of u (even outputs) and v (odd
// outputs); each is a "task" run by a group of L lanes with 32 complex values per lane:
// lane r holds x[r + L n2], n2 = 0..31.  With n = r + L n2 and k = k2 + 32 k1,
//   X[k2 + 32 k1] = sum_r w_L^{r k1} [ w_K^{r k2} sum_n2 x[r + L n2] w_32^{n2 k2} ]:
// a 32-point DFT in registers, a twiddle, one transpose through padded shared memory
// within the group, and 32/L L-point DFTs in registers.  The pre-combined sequences of
// every job of the tile are first staged in shared memory (region X); tasks then read
// X and write their outputs straight to the tile, with warp-level synchronisation only.

template <int L> struct WGeom {
  // complex elements of one lane group's transpose area (rows of L + 1, groups offset by
  // an odd multiple of L complex so the groups of a warp use different banks)
  static constexpr int rows = 32 * (L + 1);
  static constexpr int group = ((rows + 31) / 32) * 32 + L;
  static constexpr int warp = L == 1 ? 0 : (32 / L) * group;
};

__host__ __device__ inline int wfft_warp_scratch(int L) {
  switch (L) {
    case 1: return WGeom<1>::warp;
    case 2: return WGeom<2>::warp;
    case 4: return WGeom<4>::warp;
    case 8: return WGeom<8>::warp;
    case 16: return WGeom<16>::warp;
    default: return WGeom<32>::warp;
  }
}

// In place on v: on return v[t L + k1] = X[(r + L t) + 32 k1].
template <int L>
__device__ __forceinline__ void wfft_core(float2 (&v)[32], float2* sg, int r, const float2* __restrict__ tw, int K) {
  dft_reg<float, 32>(v);
  if (L == 1) return;
  if (r != 0) {
    const int m2 = 2 * K - 1;
#pragma unroll
    for (int k2 = 1; k2 < 32; ++k2) v[k2] = c_mul(v[k2], __ldg(tw + ((2 * r * k2) & m2)));
  }
#pragma unroll
  for (int k2 = 0; k2 < 32; ++k2) sg[k2 * (L + 1) + r] = v[k2];
  __syncwarp();
#pragma unroll
  for (int t = 0; t < 32 / L; ++t) {
    const int k2 = r + L * t;
    float2 u[L];
#pragma unroll
    for (int n1 = 0; n1 < L; ++n1) u[n1] = sg[k2 * (L + 1) + n1];
    dft_reg<float, L>(u);
#pragma unroll
    for (int k1 = 0; k1 < L; ++k1) v[t * L + k1] = u[k1];
  }
  __syncwarp();
}

// Stage x_j = (a_j, b_j), j = 0..K-1 (x_0 = 0) of every job into X (row stride XS).
static __device__ void wfft_build_x(const Tile<float> tl, float2* X, int XS, int njobs, int W, int n, int K, bool inverse) {
  const int logK = 31 - __clz(K), logW = 31 - __clz(W);
  const int items = njobs << logK;
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int jb = it >> logK, j = it & (K - 1);
    const Job job = job_of(jb, W, logW, n);
    X[jb * XS + j] = pair_x(tl, job, j, n, K, inverse);
  }
}

// Run every (job, half) task; outputs 2 x DST of a (-Im) and of b (Re) at index k.
template <int L>
__device__ __noinline__ void wfft_tasks(const Tile<float> tl, const float2* X, int XS, float2* scratch, int njobs,
                                        int W, int n, int K, const float2* __restrict__ tw) {
  constexpr int G = 32 / L;                     // tasks per warp at a time
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int grp = lane / L, r = lane - grp * L;
  float2* sg = scratch + (size_t)warp * WGeom<L>::warp + grp * WGeom<L>::group;
  const int ntasks = 2 * njobs, half = K >> 1, logW = 31 - __clz(W);
  for (int base = warp * G; base < ntasks; base += nwarps * G) {
    const int task = base + grp;
    const bool active = task < ntasks;
    const int jb = active ? (task >> 1) : 0, h = task & 1;
    const float2* x = X + jb * XS;
    float2 v[32];
#pragma unroll
    for (int n2 = 0; n2 < 32; ++n2) {
      const int i = r + L * n2;
      float2 val = make_float2(0.f, 0.f);
      if (active && i != 0) {
        const float2 xa = x[i], xb = x[K - i];
        val = h == 0 ? c_sub(xa, xb) : c_mul(c_add(xa, xb), __ldg(tw + i));
      }
      v[n2] = val;
    }
    wfft_core<L>(v, sg, r, tw, K);
    if (!active) continue;
    const Job job = job_of(jb, W, logW, n);
    const int sa = slot_of(job.ma, n), sb = job.mb >= 0 ? slot_of(job.mb, n) : 0;
#pragma unroll
    for (int t = 0; t < G; ++t)
#pragma unroll
      for (int k1 = 0; k1 < L; ++k1) {
        const int m = r + L * t + 32 * k1;
        if (m >= half) continue;
        const int k = 2 * m + h;               // U gives even k, V odd k
        if (k == 0) continue;
        const float2 o = v[t * L + k1];
        tl.at((k - 1) * n + sa, job.wa) = -o.y;
        if (job.mb >= 0) tl.at((k - 1) * n + sb, job.wb) = o.x;
      }
  }
}

// Inverse post-combine of one job (by one warp): D at rows of its components -> physical
// v_{j-1/2} = D_{j-1} + P D_j + (-P)^{j-1} g (nodes are already in place).  Lanes own
// contiguous j ranges and walk them downwards; each first reads the value below its range.
static __device__ void wfft_postcombine(const Tile<float> tl, const float* gsave, int njobs, int W, int n, int K) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int logW = 31 - __clz(W);
  const int per = (K + 31) / 32;                // j values per lane
  for (int jb = warp; jb < njobs; jb += nwarps) {
    const Job job = job_of(jb, W, logW, n);
    if (job.ma == 0 && job.mb <= 0) continue;   // nodes only
    const int m = n - 1;
    int ci, cc, w;                              // components (ci, cc) of line w; cc = ci for the middle one
    if (job.ma == 0) { ci = job.mb; cc = job.mb; w = job.wb; }
    else { ci = job.ma; cc = job.mb; w = job.wa; }
    const float gi = gsave[w * m + ci - 1], gc = gsave[w * m + cc - 1];
    auto Di = [&](int j) -> float { return (j >= 1 && j <= K - 1) ? tl.at((j - 1) * n + ci - 1, w) : 0.f; };
    auto Dc = [&](int j) -> float { return (j >= 1 && j <= K - 1) ? tl.at((j - 1) * n + cc - 1, w) : 0.f; };
    const int jlo = 1 + lane * per, jhi = min(K, jlo + per - 1);
    float below_i = 0.f, below_c = 0.f;
    if (jlo <= K) { below_i = Di(jlo - 1); below_c = Dc(jlo - 1); }
    __syncwarp();
    for (int j = jhi; j >= jlo; --j) {
      const float di_prev = (j == jlo) ? below_i : Di(j - 1);
      const float dc_prev = (j == jlo) ? below_c : Dc(j - 1);
      const float di = Di(j), dc = Dc(j);
      const bool odd = j & 1;
      const float vi = di_prev + dc + (odd ? gi : -gc);
      const float vc = dc_prev + di + (odd ? gc : -gi);
      tl.at((j - 1) * n + ci - 1, w) = vi;
      if (cc != ci) tl.at((j - 1) * n + cc - 1, w) = vc;
    }
    __syncwarp();
  }
}

template <int L>
__device__ void wfft_forward(const Tile<float>& tl, float2* X, int XS, float2* scratch, float* tsave, int W, int n,
                             int K, const SweepParams& P, const float* __restrict__ mix,
                             const float* __restrict__ evec, const float2* __restrict__ tw, int stage_cap) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int logW = 31 - __clz(W);
  for (int item = warp; item < W * (n - 1); item += nwarps) {
    const int w = item & (W - 1), i = (item >> logW) + 1;
    float acc = 0.f;
    for (int j = 1 + lane; j <= K; j += 32) {
      const float v = tl.at((j - 1) * n + ((j & 1) ? i : n - i) - 1, w);
      acc += (j & 1) ? v : -v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) tsave[w * (n - 1) + i - 1] = acc;
  }
  const int njobs = num_jobs(W, n);
  wfft_build_x(tl, X, XS, njobs, W, n, K, false);
  __syncthreads();
  wfft_tasks<L>(tl, X, XS, scratch, njobs, W, n, K, tw);
  __syncthreads();
  for (int it = threadIdx.x; it < W * (n - 1); it += blockDim.x) {
    const int w = it & (W - 1), i = it >> logW;
    tl.at((K - 1) * n + i, w) = tsave[w * (n - 1) + i];
  }
  __syncthreads();
  mix_dispatch<float, true>(tl, W, n, K, mix, P.mixNP, evec, tsave, 0.5f / K, 1.0f / K, reinterpret_cast<float*>(X),
                            stage_cap);
  __syncthreads();
}

template <int L>
__device__ void wfft_inverse(const Tile<float>& tl, float2* X, int XS, float2* scratch, float* gsave, int W, int n,
                             int K, const SweepParams& P, const float* __restrict__ mix,
                             const float* __restrict__ evec, const float2* __restrict__ tw, int stage_cap) {
  mix_dispatch<float, false>(tl, W, n, K, mix, P.mixNP, evec, gsave, 0.5f, 1.0f, reinterpret_cast<float*>(X),
                             stage_cap);
  __syncthreads();
  const int njobs = num_jobs(W, n);
  wfft_build_x(tl, X, XS, njobs, W, n, K, true);
  __syncthreads();
  wfft_tasks<L>(tl, X, XS, scratch, njobs, W, n, K, tw);
  __syncthreads();
  wfft_postcombine(tl, gsave, njobs, W, n, K);
  __syncthreads();
}

template <bool FWD>
__device__ void wfft_dispatch(const Tile<float>& tl, float2* X, int XS, float2* scratch, float* save, int W, int n,
                              int K, const SweepParams& P, const float* mix, const float* evec, const float2* tw,
                              int stage_cap) {
  switch (K >> 5) {
#define HOFEM_WF_CASE(LL)                                                                                   \
  case LL:                                                                                                 \
    if (FWD) wfft_forward<LL>(tl, X, XS, scratch, save, W, n, K, P, mix, evec, tw, stage_cap);            \
    else wfft_inverse<LL>(tl, X, XS, scratch, save, W, n, K, P, mix, evec, tw, stage_cap);                \
    break;
    HOFEM_WF_CASE(1) HOFEM_WF_CASE(2) HOFEM_WF_CASE(4) HOFEM_WF_CASE(8) HOFEM_WF_CASE(16) HOFEM_WF_CASE(32)
#undef HOFEM_WF_CASE
    default: break;
  }
}

// Element i of an array of format FMT (a compile-time constant), times the power of two sc
// when scaled (applied before any narrowing: FP64 inputs far outside FP32's range keep
// their bits).
template <typename T, int FMT> __device__ __forceinline__ T ld_fmt(const void* p, size_t i, bool scaled, double sc) {
  if constexpr (FMT == kFmtF64) {
    const double x = __ldg((const double*)p + i);
    return (T)(scaled ? x * sc : x);
  } else {
    float x;
    if constexpr (FMT == kFmtBF16) x = __bfloat162float(__ldg((const __nv_bfloat16*)p + i));
    else if constexpr (FMT == kFmtF16) x = __half2float(__ldg((const __half*)p + i));
    else x = __ldg((const float*)p + i);
    return scaled ? (T)x * (T)sc : (T)x;
  }
}

// The tile load of a sweep for one input format: the UNR loads of a group are made at
// clamped valid addresses (an element outside the tile reads element g0) and masked
// afterwards, so that no branch separates them and all are in flight at once.
template <typename T, int FMT, typename AddrF, typename ValidF>
__device__ __forceinline__ void load_tile(T* tile, const void* in, int total, AddrF gaddr, ValidF valid, long long g0,
                                          bool scaled, double sc) {
  constexpr int UNR = HOFEM_LOAD_UNROLL;
  for (int e0 = threadIdx.x; e0 < total; e0 += UNR * blockDim.x) {
    T v[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      const int e = e0 + u * blockDim.x;
      const bool ok = e < total && valid(e);
      v[u] = ld_fmt<T, FMT>(in, (size_t)(ok ? gaddr(e) : g0), scaled, sc);
    }
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      const int e = e0 + u * blockDim.x;
      if (e < total) tile[e + (e >> TileSwz<T>::v)] = valid(e) ? v[u] : (T)0;
    }
  }
}

// s with |max| s in [2^(e-1), 2^e), or 1 without a recorded maximum
__device__ __forceinline__ double amax_scale(const unsigned long long* amax, long long rhs, int e) {
  if (!amax) return 1.0;
  const double m = __longlong_as_double((long long)amax[rhs]);
  return m > 0.0 ? ldexp(1.0, e - ilogb(m) - 1) : 1.0;
}

// GK: K is not a power of two (mixed-radix DST passes); a separate instantiation keeps
// the power-of-two kernel free of the general path.
template <typename T, bool WF, bool GK>
__global__ void __launch_bounds__(sizeof(T) == 4 ? HOFEM_F32_THREADS : 512, 1) sweep_kernel(const SweepParams P) {
  using C = typename Cx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int M = P.M, n = P.n, K = P.K, W = P.W;
  // shared-memory carve-up
  T* tile = reinterpret_cast<T*>(smem_raw);
  size_t off = ((size_t)P.tile_elems * sizeof(T) + 15) & ~(size_t)15;
  C* fbuf = reinterpret_cast<C*>(smem_raw + off);
  off += (size_t)P.fbuf_complex * sizeof(C);
  T* save = reinterpret_cast<T*>(smem_raw + off);
  off += ((size_t)W * kMaxN * sizeof(T) + 15) & ~(size_t)15;
  T* lrest = reinterpret_cast<T*>(smem_raw + off);
  off += ((size_t)W * sizeof(T) + 15) & ~(size_t)15;
  T* lfac = reinterpret_cast<T*>(smem_raw + off);   // per-line output factor (lscale)
  off += ((size_t)W * sizeof(T) + 15) & ~(size_t)15;
  double* red = reinterpret_cast<double*>(smem_raw + off);

  const Tile<T> tl{tile, P.ps, P.ws};
  const bool contiguous = (P.inner == 1);
  const long long b = blockIdx.x;
  const long long o = b / P.tiles_per_outer, tix = b - o * P.tiles_per_outer;
  const long long l0 = tix * W;                     // first line (contiguous) or column (strided)
  const long long nl = contiguous ? P.outer_per_rhs : P.inner;
  const int wvalid = (int)min((long long)W, nl - l0);
  const long long rhs = contiguous ? o : o / P.outer_per_rhs;
  const double in_sc = amax_scale(P.in_amax, rhs, P.amax_exp);
  const double out_sc = P.out_amax ? 1.0 / amax_scale(P.out_amax, rhs, P.amax_exp) : 1.0;

  // ---- load: tile element e = (line w, position p) is e = w M + p (contiguous lines) or
  // e = p W + w (strided columns); 8 independent loads per thread are in flight at once.
  const long long gbase = contiguous ? (o * P.outer_per_rhs + l0) * (long long)M : o * (long long)M * P.inner + l0;
  const int total = M * W;
  const int logW = 31 - __clz(W);
  auto gaddr = [&](int e) -> long long {
    if (contiguous) return gbase + e;
    const int p = e >> logW, w = e & (W - 1);
    return gbase + (long long)p * P.inner + w;
  };
  auto valid = [&](int e) -> bool { return contiguous ? (e < wvalid * M) : ((e & (W - 1)) < wvalid); };
  constexpr int UNR = HOFEM_LOAD_UNROLL;
  {
    const bool scaled = P.in_amax != nullptr;
    switch (P.in_fmt) {
      case kFmtF64: load_tile<T, kFmtF64>(tile, P.in, total, gaddr, valid, gbase, scaled, in_sc); break;
      case kFmtBF16: load_tile<T, kFmtBF16>(tile, P.in, total, gaddr, valid, gbase, scaled, in_sc); break;
      case kFmtF16: load_tile<T, kFmtF16>(tile, P.in, total, gaddr, valid, gbase, scaled, in_sc); break;
      default: load_tile<T, kFmtF32>(tile, P.in, total, gaddr, valid, gbase, scaled, in_sc); break;
    }
  }
  if (P.mode == kFwdScaleInv) {
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
      const long long c = P.line_offset + l0 + w;
      double rest = 0.0;
      if (w < wvalid) {
        const long long qa = P.lamB ? c / P.MB : c;
        rest += (double)((const T*)P.lamA)[qa];
        if (P.lamB) rest += (double)((const T*)P.lamB)[c - qa * P.MB];
      }
      lrest[w] = (T)(P.alpha + rest);
      lfac[w] = (T)rest;
    }
  } else if (P.lscale) {
    // inverse sweep of prescaled data: this line's share of the eigenvalue sum
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
      const T r = (P.lamR && w < wvalid) ? ((const T*)P.lamR)[l0 + w] : (T)0;
      lrest[w] = r;
      lfac[w] = r;
    }
  }
  __syncthreads();

  if (P.lscale && P.mode == kInv) {
    // undo the prescale of the previous sweep: value / (lambda_axis(q) + rest of the line)
    const T* lam = (const T*)P.lam;
    for (int it = threadIdx.x; it < M * W; it += blockDim.x) {
      const int w = it & (W - 1), q = it >> logW;
      tl.at(q, w) = tl.at(q, w) / (lam[q] + lrest[w]);
    }
    __syncthreads();
  }
  const T* mix = (const T*)P.mix;
  const T* evec = (const T*)P.evec;
  const C* tw = (const C*)P.tw;
  if constexpr (WF && sizeof(T) == 4) {
    if (P.mode & kFwd)
      wfft_dispatch<true>(tl, fbuf, P.wf_xs, fbuf + (size_t)num_jobs(W, n) * P.wf_xs, save, W, n, K, P, mix, evec,
                          tw, 2 * P.fbuf_complex);
  } else {
    if (P.mode & kFwd) forward_transform<T, GK>(tl, fbuf, save, W, n, K, P, mix, evec, tw);
  }
  if (P.mode == kFwdScaleInv) {
    const T* lam = (const T*)P.lam;
    for (int it = threadIdx.x; it < M * W; it += blockDim.x) {
      const int w = it & (W - 1), q = it >> logW;
      tl.at(q, w) = tl.at(q, w) / (lam[q] + lrest[w]);
    }
    __syncthreads();
  }
  if constexpr (WF && sizeof(T) == 4) {
    if (P.mode & kInv)
      wfft_dispatch<false>(tl, fbuf, P.wf_xs, fbuf + (size_t)num_jobs(W, n) * P.wf_xs, save, W, n, K, P, mix, evec,
                           tw, 2 * P.fbuf_complex);
  } else {
    if (P.mode & kInv) inverse_transform<T, GK>(tl, fbuf, save, W, n, K, P, mix, evec, tw);
  }

  if (P.lscale && P.out_fmt != kFmtF64) {
    // prescale by the eigenvalue sum of the axes still to invert (one factor per line), so
    // that coefficients damped by it stay inside the storage format's exponent range
    for (int it = threadIdx.x; it < M * W; it += blockDim.x) {
      const int w = it & (W - 1), q = it >> logW;
      tl.at(q, w) = tl.at(q, w) * lfac[w];
    }
    __syncthreads();
  }
  // ---- store (same element order as the load); optional sum of squares of the result
  T s_d = (T)0;
  const bool want_norm = P.norms != nullptr, scaled_out = P.out_amax != nullptr;
  for (int e0 = threadIdx.x; e0 < total; e0 += UNR * blockDim.x) {
    if (P.out_fmt == kFmtF64) {
      double* out = (double*)P.out;
      double prev[UNR];
      if (P.accumulate) {
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
          const int e = e0 + u * blockDim.x;
          prev[u] = out[(e < total && valid(e)) ? gaddr(e) : gbase];   // clamped: no branch
        }
      }
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e < total && valid(e)) {
          const T tv = tile[e + (e >> TileSwz<T>::v)];
          double v = (double)tv;
          if (scaled_out) v *= out_sc;
          out[gaddr(e)] = P.accumulate ? prev[u] + v : v;
          if (want_norm) s_d += tv * tv;
        }
      }
    } else {
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e < total && valid(e)) {
          const float v = (float)tile[e + (e >> TileSwz<T>::v)] * (float)out_sc;
          if (P.out_fmt == kFmtBF16) ((__nv_bfloat16*)P.out)[gaddr(e)] = __float2bfloat16_rn(v);
          else if (P.out_fmt == kFmtF16) ((__half*)P.out)[gaddr(e)] = __float2half_rn(v);
          else ((float*)P.out)[gaddr(e)] = v;
        }
      }
    }
  }
  if (want_norm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double sd = (double)s_d * out_sc * out_sc;
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) sd += __shfl_xor_sync(0xffffffffu, sd, o2);
    if (lane == 0) red[warp] = sd;
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0;
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) a += red[i];
      atomicAdd(&P.norms[2 * rhs + P.norm_slot], a);
    }
  }
}

#if HOFEM_SWEEP_HAS(0)
// Per-rhs max |x| (FP64 bit patterns of non-negative values order like the values).
__global__ void absmax_kernel(const double* __restrict__ x, long long per_rhs, unsigned long long* amax) {
  const long long r = blockIdx.y;
  const double* xr = x + r * per_rhs;
  double m = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < per_rhs; i += (long long)gridDim.x * blockDim.x)
    m = fmax(m, fabs(__ldg(xr + i)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(amax + r, (unsigned long long)__double_as_longlong(m));
}

cudaError_t launch_absmax(const double* x, long long per_rhs, int nrhs, unsigned long long* amax, cudaStream_t s) {
  const long long blocks = std::min<long long>((per_rhs + 255) / 256, 4 * 152);
  absmax_kernel<<<dim3((unsigned)std::max<long long>(blocks, 1), (unsigned)nrhs), 256, 0, s>>>(x, per_rhs, amax);
  return cudaGetLastError();
}

int sweep_tile_elems(int M, int W, int tsize) {
  const long long e = (long long)M * W;
  return (int)(e + (e >> (tsize == 4 ? TileSwz<float>::v : TileSwz<double>::v)) + 1);
}

long long sweep_fbuf_complex(int K, int NB, int J, int tsize) {
  if (NB > 0) return (long long)J * 2 * (tsize == 4 ? fft_stride<float>(NB) : fft_stride<double>(NB));
  const int fs = tsize == 4 ? fft_stride<float>(K) : fft_stride<double>(K);
  const bool pow2 = (K & (K - 1)) == 0;
  return (long long)J * 2 * fs * (pow2 ? 1 : 2);
}

int bluestein_pow2(int K) {
  // outputs m = 0 .. H-1 (H = (K - 1) / 2 + 1) are used; the filter needs lags -(K-1) .. H-1
  const int H = (K - 1) / 2 + 1;
  int NB = 1;
  while (NB < K - 1 + H) NB <<= 1;
  return NB;
}

int bluestein_len(int K) {
  if (K < 2 || (K & (K - 1)) == 0) return 0;
  // direct passes: per element R reads and one write per pass (radices as in the plan:
  // 4s, one 2, odd primes)
  double direct = 0.0;
  int r = K;
  while (r % 4 == 0) { direct += 5; r /= 4; }
  if (r % 2 == 0) { direct += 3; r /= 2; }
  for (int p = 3; p <= r; p += 2)
    while (r % p == 0) { direct += p + 1; r /= p; }
  const int NB = bluestein_pow2(K);
  const int lg = 31 - __builtin_clz(NB);
  // Bluestein: two FFTs of (lg + 3) / 4 in-register passes (a read and a write each), the
  // filter product, per entry of NB; the chirp products per entry of K
  const double blue = (double)NB / K * (2.0 * 2.0 * ((lg + 3) / 4) + 2.0) + 2.0;
  return blue < 0.8 * direct ? NB : 0;
}

// Warp-FFT path (FP32, 32 <= K <= 1024): X rows of K + L complex for every job of the
// tile, then one transpose area per warp.
int wfft_row_stride(int K) { return K + (K >> 5); }
long long wfft_fbuf_complex(int W, int n, int K, int nwarps) {
  return (long long)num_jobs(W, n) * wfft_row_stride(K) + (long long)nwarps * wfft_warp_scratch(K >> 5);
}

size_t sweep_smem_bytes_fbuf(int M, int W, long long fbuf_complex, int tsize) {
  size_t off = ((size_t)sweep_tile_elems(M, W, tsize) * tsize + 15) & ~(size_t)15;
  off += (size_t)fbuf_complex * 2 * tsize;
  off += ((size_t)W * kMaxN * tsize + 15) & ~(size_t)15;
  off += 2 * (((size_t)W * tsize + 15) & ~(size_t)15);
  off += 2 * 32 * sizeof(double);
  return off;
}

size_t sweep_smem_bytes(int M, int n, int K, int NB, int W, int J, int tsize, bool strided) {
  (void)n;
  (void)strided;
  size_t off = ((size_t)sweep_tile_elems(M, W, tsize) * tsize + 15) & ~(size_t)15;
  off += (size_t)sweep_fbuf_complex(K, NB, J, tsize) * 2 * tsize;
  off += ((size_t)W * kMaxN * tsize + 15) & ~(size_t)15;
  off += 2 * (((size_t)W * tsize + 15) & ~(size_t)15);
  off += 2 * 32 * sizeof(double);
  return off;
}

// Jobs per batch are limited only by shared memory (each thread loops over butterflies).
int sweep_max_jobs(int K, int tsize, int threads) {
  (void)K;
  (void)tsize;
  (void)threads;
  return 1 << 20;
}

cudaError_t sweep_set_smem_limits_f32();
cudaError_t sweep_set_smem_limits_f64();

cudaError_t sweep_set_smem_limits() {
  cudaError_t e = sweep_set_smem_limits_f32();
  if (e == cudaSuccess) e = sweep_set_smem_limits_f64();
  return e;
}
#endif  // part 0

#if HOFEM_SWEEP_HAS(1)
cudaError_t sweep_set_smem_limits_f32() {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(sweep_kernel<float, false, false>, a, 232448);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(sweep_kernel<float, true, false>, a, 232448);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(sweep_kernel<float, false, true>, a, 232448);
  return e;
}

cudaError_t launch_sweep_f32(const SweepParams& p, cudaStream_t s) {
  if (p.wfft) sweep_kernel<float, true, false><<<(unsigned)p.ntiles, p.threads, p.smem_bytes, s>>>(p);
  else if (p.pow2) sweep_kernel<float, false, false><<<(unsigned)p.ntiles, p.threads, p.smem_bytes, s>>>(p);
  else sweep_kernel<float, false, true><<<(unsigned)p.ntiles, p.threads, p.smem_bytes, s>>>(p);
  return cudaGetLastError();
}
#endif  // part 1

#if HOFEM_SWEEP_HAS(2)
cudaError_t sweep_set_smem_limits_f64() {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(sweep_kernel<double, false, false>, a, 232448);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(sweep_kernel<double, false, true>, a, 232448);
  return e;
}

cudaError_t launch_sweep_f64(const SweepParams& p, cudaStream_t s) {
  if (p.pow2) sweep_kernel<double, false, false><<<(unsigned)p.ntiles, p.threads, p.smem_bytes, s>>>(p);
  else sweep_kernel<double, false, true><<<(unsigned)p.ntiles, p.threads, p.smem_bytes, s>>>(p);
  return cudaGetLastError();
}
#endif  // part 2

}  // namespace hofem

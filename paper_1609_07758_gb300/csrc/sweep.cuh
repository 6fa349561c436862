// Axis sweep: the direct / inverse F_n-transform of Theorem 2 applied to every line of
// one axis of the tensor-product grid, optionally fused with the eigenvalue-sum scaling
// of algorithm (a) (Eq. decomp v 2).  Host-side launch parameters.
#pragma once
#include "common.cuh"

// Threads per CTA of the FP32 sweep (a build-time tuning knob; FP64 sweeps use 512).
#ifndef HOFEM_F32_THREADS
#define HOFEM_F32_THREADS 512
#endif

// Independent global loads in flight per thread in the load/store phases of a sweep
// (bytes in flight per SM bound the achievable HBM bandwidth of these phases).
#ifndef HOFEM_LOAD_UNROLL
#define HOFEM_LOAD_UNROLL 8
#endif

namespace hofem {

enum SweepMode : int { kFwd = 1, kInv = 2, kFwdScaleInv = 3 };
// storage format of a sweep's input or output array
enum StoreFmt : int { kFmtF32 = 0, kFmtF64 = 1, kFmtBF16 = 2, kFmtF16 = 3 };

struct SweepParams {
  // geometry of the sweep: lines along one axis of a C-order array
  long long outer;            // slabs before the axis (rhs x dims before)
  long long inner;            // product of dims after the axis (1 = contiguous lines)
  long long outer_per_rhs;    // slabs per right-hand side
  long long tiles_per_outer;  // ceil(inner / W) (strided) or ceil(outer_per_rhs / W) (contiguous)
  long long ntiles;
  int M, n, K, W;             // line length, order, elements, lines per CTA
  int mode;
  // data
  const void* in;
  int in_fmt;                 // StoreFmt
  void* out;
  int out_fmt;
  int accumulate;             // out (FP64) += result
  // optional per-rhs |max| of the original right-hand side (FP64 bit patterns): the input is
  // multiplied by the power of two s with |max| s in [2^(amax_exp-1), 2^amax_exp) and the
  // output by 1/s, which keeps FP16 intermediates inside their exponent range (exact)
  const unsigned long long* in_amax;
  const unsigned long long* out_amax;
  int amax_exp;
  // FP16 intermediates: the fused sweep stores its lines multiplied by the eigenvalue sum
  // of the other axes; an inverse sweep divides its input by lam(q) + lamR(line) and
  // multiplies its (non-FP64) output by lamR(line), lamR = eigenvalues of the next axis
  // by column (null: 0)
  int lscale;
  const void* lamR;
  double* norms;              // if non-null: norms[2 rhs + norm_slot] += sum result^2 (atomics)
  int norm_slot;
  // axis tables, in the work precision T
  const void* mix;            // (K-1) n NP, rows padded to NP entries
  int mixNP;
  const void* evec;           // (n-1)^2
  const void* tw;             // 2K complex exp(-i pi t / K)
  const void* lam;            // M
  const float* mixT;          // FP32 (K-1) n n, frequency fastest: [(l n + s)(K-1) + k-1]
  const float* lamT;          // FP32 (K-1) n, frequency fastest: [l (K-1) + k-1]
  const float* twr;           // FP32 complex, K = 32 L a power of two >= 64: K entries
                              // w_K^{r k2} at [k2 L + r], then K entries w_2K^{r (2 k2 + 1)}
  // eigenvalue sums of the other axes for the fused sweep (lines are columns c)
  const void* lamA;           // lam_rest(c) = lamA[c / MB] + lamB[c % MB] (lamB may be null)
  const void* lamB;
  long long MB;
  long long line_offset;      // index of the sweep's first line among the columns c (a block
                              // of columns of a problem split over several GPUs; else 0)
  double alpha;
  // FFT plan for length K: radices of the DIF passes (first pass first); pow2 = 1 for
  // K = 2^m (in-place register passes), else out-of-place mixed-radix passes, whose
  // output slot of frequency m = sum_i d_i radix_q[i] (m = d_1 + R_1 d_2 + R_1 R_2 d_3 ..)
  int npass;
  int radix[8];
  int radix_log[8];
  int radix_q[8];
  int pow2;
  // Bluestein (chirp-z) form of a general-K DFT (nb > 0): with c_j = exp(-i pi j^2 / K),
  //   X_m = c_m sum_j (x_j c_j) conj(c_{m-j}),   m < (K - 1) / 2 + 1 (the outputs used),
  // a circular convolution of length nb = 2^nb_log (bluestein_pow2) done by an in-place
  // power-of-two FFT (radices nb_radix), a product with the transformed filter and the
  // inverse network.  Its tables follow the 2K DST twiddles in tw: exp(-i pi t / nb)
  // (2 nb), c_j (K), and the filter's transform / nb in the FFT's output order (nb).
  int nb, nb_log, nb_npass;
  int nb_radix[4];
  int mix_direct;             // 1: mixing rows read from global memory (L2), not staged
  int jobs_per_batch;
  long long fbuf_complex;     // complex elements of the FFT region (batched buffers or X + transposes)
  int wfft;                   // 1: warp-register FFT path (FP32, 32 <= K <= 1024)
  int wf_xs;                  // row stride (complex) of the staged sequences X
  // shared-memory layout (in elements of T)
  int ps, ws;                 // tile(p, w) = tile[p * ps + w * ws]
  int tile_elems;
  int threads;
  size_t smem_bytes;
};

// Register-resident FP32 sweep (sweep_reg.cu) for the element orders and power-of-two K
// it is instantiated for: lines per CTA, threads and dynamic shared memory of (n, K), or
// false when there is no instantiation.  Input FP64 or FP32, output FP32 or FP64 (with
// accumulate and norms); no per-rhs scaling or FP16 prescale.
bool sweep_reg_shape(int n, int K, int* W, int* threads, size_t* smem);
cudaError_t sweep_reg_set_smem_limits();
cudaError_t launch_sweep_reg(const SweepParams& p, cudaStream_t s);

// Launch one sweep; T = float or double work precision.
cudaError_t launch_sweep_f32(const SweepParams& p, cudaStream_t s);
cudaError_t launch_sweep_f64(const SweepParams& p, cudaStream_t s);

// Shared-memory bytes a sweep needs for (M, n, K, W, J) in precision of size tsize; NB is
// the Bluestein length of the sweep's transforms (0: power-of-two or direct passes).
size_t sweep_smem_bytes(int M, int n, int K, int NB, int W, int J, int tsize, bool strided);
int sweep_tile_elems(int M, int W, int tsize);
// complex entries of the FFT region: J jobs x 2 FFTs of K (doubled for the ping-pong of
// the direct passes unless K = 2^m) or of NB (Bluestein, in place)
long long sweep_fbuf_complex(int K, int NB, int J, int tsize);
// Bluestein convolution length for K: the smallest power of two NB >= K - 1 + H, H =
// (K - 1) / 2 + 1, so that the outputs m < H a DST needs are free of circular wrap-around.
int bluestein_pow2(int K);
// Bluestein length chosen for K (0: K is a power of two or its direct mixed-radix passes
// are cheaper): bluestein_pow2(K) when two FFTs of that length cost less than 0.8 x the
// direct passes (counting shared-memory reads and writes per element).
int bluestein_len(int K);
int wfft_row_stride(int K);
long long wfft_fbuf_complex(int W, int n, int K, int nwarps);
size_t sweep_smem_bytes_fbuf(int M, int W, long long fbuf_complex, int tsize);
int sweep_max_jobs(int K, int tsize, int threads);
cudaError_t sweep_set_smem_limits();
// amax[r] = max |x| over right-hand side r (FP64 bit patterns; amax must be zeroed first)
cudaError_t launch_absmax(const double* x, long long per_rhs, int nrhs, unsigned long long* amax, cudaStream_t s);

}  // namespace hofem

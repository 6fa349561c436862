// C ABI of the hofem library: plans, solves, the FP64 operator and test hooks.
// Algorithm (a) of Sect. 2 par. 4: direct F_n-transforms along every axis, division by
// the eigenvalue sums, inverse F_n-transforms; refined dtypes wrap low-precision solves
// in iterative refinement with the FP64 matrix-free residual.
#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "banded.cuh"
#include "dirichlet.cuh"
#include "varcoef.cuh"
#include "load.cuh"
#include "residual.cuh"
#include "sweep.cuh"

using namespace hofem;

namespace {

thread_local std::string g_last_error;

hofem_status fail(hofem_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

hofem_status cuda_fail(cudaError_t e, const char* where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? HOFEM_ERR_OOM : HOFEM_ERR_CUDA;
}

#define HOFEM_CUDA(x, where)                       \
  do {                                             \
    cudaError_t e__ = (x);                         \
    if (e__ != cudaSuccess) return cuda_fail(e__, where); \
  } while (0)

constexpr int kThreads = 512;
constexpr size_t kSmemLimit = 232448;   // 227 KB opt-in per CTA on sm_103
constexpr int kSMs = 152;

struct DevAxis {
  AxisTables h;
  double *lam64 = nullptr, *mix64 = nullptr, *evec64 = nullptr, *tw64 = nullptr;
  float *lam32 = nullptr, *mix32 = nullptr, *evec32 = nullptr, *tw32 = nullptr;
  // frequency-fastest copies for the register sweep: mixT[(l n + s)(K-1) + k-1] = G_k[l][s],
  // lamT[l (K-1) + k-1] = lam[(k-1) n + l] (consecutive threads read consecutive k)
  float *mixT32 = nullptr, *lamT32 = nullptr;
  float* twr32 = nullptr;        // register sweep twiddles (power-of-two K >= 64), see SweepParams::twr
  int npass = 0, radix[8] = {0};
  int nb = 0;                    // Bluestein length of the K-point DFTs (0: direct passes)
  int mixNP = 0;
};

}  // namespace

struct hofem_plan_s {
  int N = 0, n = 0, dtype = 0;
  int K[3] = {0, 0, 0}, M[3] = {0, 0, 0};
  double X[3] = {0, 0, 0};
  double alpha = 0.0;
  long long total = 0;           // unknowns per right-hand side
  DevAxis ax[3];
  // workspace
  int ws_nrhs = 0;
  float* work32 = nullptr;       // low-precision work array of the forward sweeps (FP32)
  void* work16 = nullptr;        // BF16 / FP16 plans: work array after the eigenvalue division
  int wfmt = kFmtF32;            // StoreFmt of the arrays after the division
  bool refined = false;          // *_REFINED dtype
  unsigned long long* amax = nullptr;   // per-rhs max |rhs| (FP16 work arrays only)
  int amax_exp = 10;             // FP16: scaled right-hand sides have |max| in [2^(e-1), 2^e)
  // load-vector quadrature (hofem_load): tables and the two intermediate axis buffers
  std::vector<double> load_T[3], load_xi[3];   // per axis
  double* ld[2] = {nullptr, nullptr};
  size_t ld_count = 0;
  double* heat = nullptr;        // right-hand side of the heat steps (nrhs x unknowns)
  int heat_nrhs = 0;
  // variable-coefficient operator and PCG: device basis tables, r z p q vectors, dot slot
  double *vcB = nullptr, *vcD = nullptr, *vcW = nullptr;
  double* cg[4] = {nullptr, nullptr, nullptr, nullptr};
  double* dot = nullptr;
  double* h_dot = nullptr;
  double* r64 = nullptr;         // residual
  double* tmp64[4] = {nullptr, nullptr, nullptr, nullptr};
  double* norms = nullptr;       // 2 per rhs
  double* h_norms = nullptr;     // pinned mirror
  int refine_iters = 2;          // fixed count (refine_tol = 0) or most corrections
  double refine_tol = 0.0;       // > 0: stop once ||delta|| / ||u|| <= refine_tol
  int capture_iters = 2;         // fixed count of a solve issued into a capturing stream
  hofem_info info{};
  size_t table_bytes = 0;
  // profiling: event pairs recorded around launches, folded into per-kind totals on query
  bool profiling = false;
  struct Pending { int kind; cudaEvent_t a, b; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  double prof_ms[16] = {0};
  int prof_n[16] = {0};
};

namespace {

// kinds 0-5: the general sweep kernel (FP64 / FP32 work), 6: the FP64 operator sweep,
// 7-9: the register-resident FP32 sweep, 10: the banded solves of algorithm (b)
const char* const kKindNames[] = {"sweep_fwd_f64", "sweep_fsi_f64", "sweep_inv_f64", "sweep_fwd_f32",
                                  "sweep_fsi_f32", "sweep_inv_f32", "apply_f64",     "sweep_fwd_reg",
                                  "sweep_fsi_reg", "sweep_inv_reg", "banded_f64"};
constexpr int kNumKinds = 11;

cudaEvent_t pool_event(hofem_plan_s* p) {
  if (!p->pool.empty()) {
    cudaEvent_t e = p->pool.back();
    p->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Launch `fn` on stream s, counting it and bracketing it with events when profiling.
template <typename F>
cudaError_t timed_launch(hofem_plan_s* p, int kind, cudaStream_t s, F fn) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (p->profiling) {
    a = pool_event(p);
    b = pool_event(p);
    cudaEventRecord(a, s);
  }
  cudaError_t e = fn();
  if (p->profiling) {
    cudaEventRecord(b, s);
    p->pending.push_back({kind, a, b});
  }
  if (e == cudaSuccess) ++p->info.kernel_launches;
  return e;
}

void fold_profile(hofem_plan_s* p) {
  for (auto& q : p->pending) {
    float ms = 0.f;
    cudaEventSynchronize(q.b);
    if (cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess) {
      p->prof_ms[q.kind] += ms;
      p->prof_n[q.kind] += 1;
    }
    p->pool.push_back(q.a);
    p->pool.push_back(q.b);
  }
  p->pending.clear();
}

bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

// DIF radices of a length-K FFT, first pass first: 16s (and one smaller power of two) for
// K = 2^m; otherwise the prime factors with pairs of 2s merged to 4s, smallest first.
// Returns false if more than 8 passes would be needed.
bool radix_plan(int K, int* npass, int* radix) {
  int np = 0;
  if (is_pow2(K)) {
    int m = 0;
    while ((1 << m) < K) ++m;
    while (m >= 4) { radix[np++] = 16; m -= 4; }
    if (m > 0) radix[np++] = 1 << m;
    *npass = np;
    return true;
  }
  int r = K;
  while (r % 4 == 0 && np < 8) { radix[np++] = 4; r /= 4; }
  if (r % 2 == 0 && np < 8) { radix[np++] = 2; r /= 2; }
  for (int p = 3; p <= r && np < 8; p += 2)
    while (r % p == 0 && np < 8) { radix[np++] = p; r /= p; }
  *npass = np;
  return r == 1;
}

template <typename T>
hofem_status upload(const std::vector<double>& src, T** dst, size_t* bytes) {
  std::vector<T> tmp(src.size() ? src.size() : 1);
  for (size_t i = 0; i < src.size(); ++i) tmp[i] = (T)src[i];
  HOFEM_CUDA(cudaMalloc(dst, tmp.size() * sizeof(T)), "cudaMalloc(tables)");
  HOFEM_CUDA(cudaMemcpy(*dst, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice), "upload tables");
  *bytes += tmp.size() * sizeof(T);
  return HOFEM_OK;
}

void free_axis(DevAxis& a) {
  cudaFree(a.lam64); cudaFree(a.mix64); cudaFree(a.evec64); cudaFree(a.tw64);
  cudaFree(a.lam32); cudaFree(a.mix32); cudaFree(a.evec32); cudaFree(a.tw32);
  cudaFree(a.mixT32); cudaFree(a.lamT32); cudaFree(a.twr32);
  a = DevAxis{};
}

void free_workspace(hofem_plan_s* p) {
  cudaFree(p->work32); p->work32 = nullptr;
  cudaFree(p->work16); p->work16 = nullptr;
  cudaFree(p->r64); p->r64 = nullptr;
  for (auto& t : p->tmp64) { cudaFree(t); t = nullptr; }
  cudaFree(p->norms); p->norms = nullptr;
  cudaFree(p->amax); p->amax = nullptr;
  if (p->h_norms) cudaFreeHost(p->h_norms);
  p->h_norms = nullptr;
  p->ws_nrhs = 0;
  p->info.workspace_bytes = 0;
}

hofem_status reserve(hofem_plan_s* p, int nrhs) {
  if (nrhs <= p->ws_nrhs) return HOFEM_OK;
  free_workspace(p);
  const size_t cnt = (size_t)nrhs * p->total;
  size_t bytes = 0;
  const bool low = p->dtype != HOFEM_FP64;
  if (low) {
    HOFEM_CUDA(cudaMalloc(&p->work32, cnt * sizeof(float)), "cudaMalloc(work)");
    bytes += cnt * sizeof(float);
  }
  if (p->wfmt != kFmtF32) {
    HOFEM_CUDA(cudaMalloc(&p->work16, cnt * 2), "cudaMalloc(half work)");
    bytes += cnt * 2;
  }
  if (p->wfmt == kFmtF16) {
    HOFEM_CUDA(cudaMalloc(&p->amax, (size_t)nrhs * sizeof(unsigned long long)), "cudaMalloc(amax)");
    bytes += (size_t)nrhs * sizeof(unsigned long long);
  }
  HOFEM_CUDA(cudaMalloc(&p->r64, cnt * sizeof(double)), "cudaMalloc(residual)");
  bytes += cnt * sizeof(double);
  const int ntmp = p->N == 2 ? 2 : 4;
  for (int i = 0; i < ntmp; ++i) {
    HOFEM_CUDA(cudaMalloc(&p->tmp64[i], cnt * sizeof(double)), "cudaMalloc(operator temporaries)");
    bytes += cnt * sizeof(double);
  }
  HOFEM_CUDA(cudaMalloc(&p->norms, 2 * (size_t)nrhs * sizeof(double)), "cudaMalloc(norms)");
  HOFEM_CUDA(cudaMallocHost(&p->h_norms, 2 * (size_t)nrhs * sizeof(double)), "cudaMallocHost(norms)");
  memset(p->h_norms, 0, 2 * (size_t)nrhs * sizeof(double));
  p->ws_nrhs = nrhs;
  p->info.workspace_bytes = bytes;
  return HOFEM_OK;
}

int num_jobs_host(int W, int n) { return W * ((n - 1) / 2) + (((n & 1) == 0) ? W : (W + 1) / 2); }

// Lines per CTA (W, power of two) and DST jobs per batch (J) for one sweep: the fewest
// DST batches (block-wide barrier rounds) per line, then the largest W (more reuse of
// each mixing-table row), keeping >= 2 CTAs per SM when there are enough lines.
bool choose_sweep(int M, int n, int K, int NB, int tsize, long long lines, bool strided, int* W_out, int* J_out) {
  (void)strided;
  // tuning override "W:J" (both must fit; used to explore launch shapes)
  if (const char* env = getenv("HOFEM_SWEEP_CFG")) {
    int W = 0, J = 0;
    if (sscanf(env, "%d:%d", &W, &J) == 2 && W >= 1 && (W & (W - 1)) == 0 && J >= 1 &&
        J <= num_jobs_host(W, n) && sweep_smem_bytes(M, n, K, NB, W, J, tsize, strided) <= kSmemLimit) {
      *W_out = W;
      *J_out = J;
      return true;
    }
  }
  double best = 1e30;
  int bestW = 0, bestJ = 0;
  for (int W = 64; W >= 1; W >>= 1) {
    if (W > 1 && lines / W < 2 * kSMs) continue;
    const int jobs = num_jobs_host(W, n);
    int J = jobs;
    while (J >= 1 && sweep_smem_bytes(M, n, K, NB, W, J, tsize, strided) > kSmemLimit) --J;
    if (J < 1) continue;
    const int batches = (jobs + J - 1) / J;
    const double score = (double)batches / W;
    if (score < best - 1e-12) {
      best = score;
      bestW = W;
      bestJ = J;
    }
  }
  if (bestW == 0) return false;
  *W_out = bestW;
  *J_out = bestJ;
  return true;
}

// Warp-FFT path (FP32, 32 <= K <= 1024): lines per CTA and warps per CTA.  Score = task
// rounds per line (2 tasks per DST job, 32/L tasks per warp at a time), ties to larger W.
bool choose_sweep_wfft(int M, int n, int K, long long lines, int* W_out, int* nw_out) {
  if (const char* env = getenv("HOFEM_SWEEP_WCFG")) {
    int W = 0, nw = 0;
    if (sscanf(env, "%d:%d", &W, &nw) == 2 && W >= 1 && (W & (W - 1)) == 0 && (nw == 4 || nw == 8 || nw == 16) &&
        sweep_smem_bytes_fbuf(M, W, wfft_fbuf_complex(W, n, K, nw), 4) <= kSmemLimit) {
      *W_out = W;
      *nw_out = nw;
      return true;
    }
  }
  const int L = K >> 5;
  double best = 1e30;
  int bW = 0, bN = 0;
  for (int W = 64; W >= 1; W >>= 1) {
    if (W > 1 && lines / W < 2 * kSMs) continue;
    for (int nw : {16, 8}) {
      if (sweep_smem_bytes_fbuf(M, W, wfft_fbuf_complex(W, n, K, nw), 4) > kSmemLimit) continue;
      const int tasks = 2 * num_jobs_host(W, n);
      const int per_round = nw * (32 / L);
      const double score = (double)((tasks + per_round - 1) / per_round) / W;
      if (score < best - 1e-12) {
        best = score;
        bW = W;
        bN = nw;
      }
    }
  }
  if (!bW) return false;
  *W_out = bW;
  *nw_out = bN;
  return true;
}

struct Geo {
  long long outer_per_rhs, inner;
};

Geo geometry(const hofem_plan_s* p, int axis) {
  Geo g{1, 1};
  for (int i = 0; i < axis; ++i) g.outer_per_rhs *= p->M[i];
  for (int i = axis + 1; i < p->N; ++i) g.inner *= p->M[i];
  return g;
}

// ---- measured launch shapes (autotuner): sweep (W, J) and operator E per shape.
// key: kind (0 sweep, 1 operator), M, n, K, element bytes, strided, mode, lines
typedef std::tuple<int, int, int, int, int, int, int, long long> TuneKey;
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, int>> g_tuned;
bool g_tune_loaded = false;
thread_local int g_force_a = 0, g_force_b = 0;   // candidate under measurement (0: none)
// A sweep's launch shape stores the DST batch J plus this flag when the per-frequency
// mixing reads its table rows from global memory (L2) instead of staging the table
// through shared memory in chunks (the better form when a CTA holds few lines).
constexpr int kMixDirectFlag = 1 << 16;

bool tuned_lookup(const TuneKey& k, int* a, int* b) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tuned.find(k);
  if (it == g_tuned.end()) return false;
  *a = it->second.first;
  *b = it->second.second;
  return true;
}

// Bluestein length a sweep of this axis uses at work-precision size tsize: the plan's
// choice when one line and one job of it fit shared memory, else the direct passes.
int sweep_nb(const DevAxis& A, int tsize) {
  if (A.nb > 0 && sweep_smem_bytes(A.h.M, A.h.n, A.h.K, A.nb, 1, 1, tsize, false) <= kSmemLimit) return A.nb;
  return 0;
}

TuneKey sweep_key(const hofem_plan_s* p, int axis, int mode, bool f64, long long nrhs, long long lines_override) {
  const DevAxis& A = p->ax[axis];
  Geo g = geometry(p, axis);
  if (lines_override >= 0) g = Geo{lines_override, 1};
  const int kind = sweep_nb(A, f64 ? 8 : 4) > 0 ? 2 : 0;   // 2: Bluestein sweeps
  return TuneKey{kind, A.h.M, A.h.n, A.h.K, f64 ? 8 : 4, g.inner > 1 ? 1 : 0, mode, nrhs * g.outer_per_rhs * g.inner};
}

TuneKey apply_key(const hofem_plan_s* p, int axis, int mode, long long nrhs) {
  const DevAxis& A = p->ax[axis];
  const Geo g = geometry(p, axis);
  return TuneKey{1, A.h.M, A.h.n, A.h.K, 8, g.inner > 1 ? 1 : 0, mode, nrhs * g.outer_per_rhs * g.inner};
}

// The register-resident FP32 sweep serves this sweep: an instantiation exists for the
// axis' (n, K), the formats are FP32/FP64 without FP16 scaling, and HOFEM_SWEEP_REG is not
// "0" (which forces the general kernel, for comparisons).
bool use_reg_sweep(const DevAxis& A, bool f64, int mode, bool strided, int in_fmt, int out_fmt,
                   const unsigned long long* in_amax, const unsigned long long* out_amax, int* W, int* threads,
                   size_t* smem) {
  if (f64 || in_amax || out_amax || (mode == kFwdScaleInv && !strided)) return false;
  if ((in_fmt != kFmtF64 && in_fmt != kFmtF32) || (out_fmt != kFmtF64 && out_fmt != kFmtF32)) return false;
  const char* env = getenv("HOFEM_SWEEP_REG");
  if (env && env[0] == '0') return false;
  return sweep_reg_shape(A.h.n, A.h.K, W, threads, smem);
}

hofem_status run_sweep(hofem_plan_s* p, int axis, int mode, bool f64, const void* in, int in_fmt, void* out,
                       int out_fmt, bool accumulate, double* norms, long long nrhs, cudaStream_t s,
                       long long lines_override = -1, const unsigned long long* in_amax = nullptr,
                       const unsigned long long* out_amax = nullptr, int norm_slot = 0,
                       const Geo* block = nullptr, long long line_offset = 0) {
  const DevAxis& A = p->ax[axis];
  SweepParams P{};
  Geo g = geometry(p, axis);
  if (lines_override >= 0) g = Geo{lines_override, 1};
  if (block) g = *block;   // a block of lines of its own geometry (nrhs is folded into it)
  P.line_offset = line_offset;
  const int tsize = f64 ? 8 : 4;
  const bool strided = g.inner > 1;
  const long long lines = nrhs * g.outer_per_rhs * g.inner;
  int W = 1, J = 1, nwarps = 0;
  int rthreads = 0;
  size_t rsmem = 0;
  const bool reg = use_reg_sweep(A, f64, mode, strided, in_fmt, out_fmt, in_amax, out_amax, &W, &rthreads, &rsmem);
  // the warp-register FFT path is opt-in (HOFEM_WFFT=1): on GB300 it measured slower than
  // the block-wide DIF path (2.5 vs 2.0 ms per sweep at n = 9, K = 1024)
  const char* wf_env = getenv("HOFEM_WFFT");
  const bool wfft = !reg && !f64 && is_pow2(A.h.K) && A.h.K >= 32 && A.h.K <= 1024 && wf_env && wf_env[0] == '1' &&
                    choose_sweep_wfft(A.h.M, A.h.n, A.h.K, lines, &W, &nwarps);
  const TuneKey key = sweep_key(p, axis, mode, f64, nrhs, lines_override);
  const int NB = sweep_nb(A, tsize);
  if (reg || wfft) {
  } else if (g_force_a > 0) {
    W = g_force_a;
    J = g_force_b;
  } else if (tuned_lookup(key, &W, &J) &&
             sweep_smem_bytes(A.h.M, A.h.n, A.h.K, NB, W, J % kMixDirectFlag, tsize, strided) <= kSmemLimit) {
  } else if (choose_sweep(A.h.M, A.h.n, A.h.K, NB, tsize, lines, strided, &W, &J)) {
    // mixing rows straight from L2 when few lines per CTA would reuse a staged table
    if (W <= 4) J += kMixDirectFlag;
  } else {
    return fail(HOFEM_ERR_UNSUPPORTED, "no launch configuration fits shared memory for this axis");
  }
  // J carries the mixing form: J / kMixDirectFlag = 1 reads the rows from global memory
  int mix_direct = J / kMixDirectFlag;
  J %= kMixDirectFlag;
  if (const char* md = getenv("HOFEM_MIX_DIRECT")) mix_direct = md[0] == '1' ? 1 : 0;
  P.outer = nrhs * g.outer_per_rhs;
  P.inner = g.inner;
  P.outer_per_rhs = g.outer_per_rhs;
  P.tiles_per_outer = strided ? (g.inner + W - 1) / W : (g.outer_per_rhs + W - 1) / W;
  P.ntiles = (strided ? P.outer : nrhs) * P.tiles_per_outer;
  P.M = A.h.M;
  P.n = A.h.n;
  P.K = A.h.K;
  P.W = W;
  P.mode = mode;
  P.in = in;
  P.in_fmt = in_fmt;
  P.out = out;
  P.out_fmt = out_fmt;
  P.in_amax = in_amax;
  P.out_amax = out_amax;
  P.amax_exp = p->amax_exp;
  // FP16 intermediates carry the eigenvalue-sum prescale between the fused and inverse sweeps
  P.lscale = !f64 && ((mode == kFwdScaleInv && out_fmt == kFmtF16) || (mode == kInv && in_fmt == kFmtF16));
  P.lamR = (P.lscale && mode == kInv && axis < p->N - 1) ? (const void*)p->ax[axis + 1].lam32 : nullptr;
  P.accumulate = accumulate;
  P.norms = norms;
  P.norm_slot = norm_slot;
  P.mix = f64 ? (const void*)A.mix64 : (const void*)A.mix32;
  P.mixT = A.mixT32;
  P.lamT = A.lamT32;
  P.twr = A.twr32;
  P.mixNP = A.mixNP;
  P.evec = f64 ? (const void*)A.evec64 : (const void*)A.evec32;
  P.tw = f64 ? (const void*)A.tw64 : (const void*)A.tw32;
  P.lam = f64 ? (const void*)A.lam64 : (const void*)A.lam32;
  P.alpha = p->alpha;
  if (mode == kFwdScaleInv) {
    // the fused axis is axis 0; lines are columns c = (q_1, .., q_{N-1})
    const DevAxis& a1 = p->ax[1];
    P.lamA = f64 ? (const void*)a1.lam64 : (const void*)a1.lam32;
    if (p->N == 3) {
      const DevAxis& a2 = p->ax[2];
      P.lamB = f64 ? (const void*)a2.lam64 : (const void*)a2.lam32;
      P.MB = p->M[2];
    } else {
      P.lamB = nullptr;
      P.MB = 1;
    }
  }
  P.npass = A.npass;
  P.pow2 = is_pow2(A.h.K) ? 1 : 0;
  {
    int q = A.h.K;
    for (int i = 0; i < A.npass; ++i) {
      q /= A.radix[i];
      P.radix_q[i] = q;
    }
  }
  for (int i = 0; i < 8; ++i) {
    P.radix[i] = A.radix[i];
    P.radix_log[i] = A.radix[i] > 0 ? 31 - __builtin_clz(A.radix[i]) : 0;
  }
  P.nb = wfft ? 0 : NB;
  P.nb_log = P.nb_npass = 0;
  for (int i = 0; i < 4; ++i) P.nb_radix[i] = 0;
  if (P.nb > 0) {
    int rb[8] = {0};
    radix_plan(P.nb, &P.nb_npass, rb);
    for (int i = 0; i < P.nb_npass && i < 4; ++i) P.nb_radix[i] = rb[i];
    P.nb_log = 31 - __builtin_clz(P.nb);
  }
  P.jobs_per_batch = J;
  P.mix_direct = mix_direct;
  P.wfft = wfft ? 1 : 0;
  P.wf_xs = wfft ? wfft_row_stride(A.h.K) : 0;
  P.fbuf_complex = wfft ? wfft_fbuf_complex(W, A.h.n, A.h.K, nwarps) : sweep_fbuf_complex(A.h.K, P.nb, J, tsize);
  if (strided) { P.ps = W; P.ws = 1; } else { P.ps = 1; P.ws = A.h.M; }
  P.tile_elems = sweep_tile_elems(A.h.M, W, tsize);
  P.threads = reg ? rthreads : wfft ? 32 * nwarps : (f64 ? 512 : HOFEM_F32_THREADS);
  P.smem_bytes = reg ? rsmem : sweep_smem_bytes_fbuf(A.h.M, W, P.fbuf_complex, tsize);
  p->info.lines_per_cta[axis] = W;
  if (P.ntiles <= 0) return HOFEM_OK;
  const int kind = (reg ? 7 : f64 ? 0 : 3) + (mode == kFwd ? 0 : mode == kFwdScaleInv ? 1 : 2);
  cudaError_t e = timed_launch(p, kind, s, [&]() {
    return reg ? launch_sweep_reg(P, s) : f64 ? launch_sweep_f64(P, s) : launch_sweep_f32(P, s);
  });
  if (e != cudaSuccess) return cuda_fail(e, "sweep launch");
  return HOFEM_OK;
}

// One low- or full-precision solve f -> u (algorithm (a)); accumulate: u += solution.
// Low precision: the forward sweeps keep FP32 intermediates; the fused sweep and the
// inverse sweeps keep the plan's format (FP32, BF16 or FP16).  Rounding an array that is
// still physical along some axis spreads its error over every frequency of that axis,
// where the eigenvalue division amplifies the smooth ones by up to the 1D condition
// number; after the division rounding errors stay relative.  FP16 adds an exact
// power-of-two scale of each right-hand side.
hofem_status solve_once(hofem_plan_s* p, const double* f, double* u, int nrhs, bool f64, bool accumulate,
                        double* norms, int norm_slot, cudaStream_t s, int f_fmt = kFmtF64) {
  hofem_status st;
  void* wa = f64 ? (void*)u : (void*)p->work32;                                   // before the division
  void* wb = f64 ? (void*)u : (p->wfmt == kFmtF32 ? (void*)p->work32 : p->work16);  // after it
  const int fa = f64 ? kFmtF64 : kFmtF32, fb = f64 ? kFmtF64 : p->wfmt;
  if (f64 && accumulate) return fail(HOFEM_ERR_INVALID_ARG, "internal: FP64 solve cannot accumulate");
  const unsigned long long* amax = nullptr;
  if (f_fmt != kFmtF64 && (f64 || p->wfmt == kFmtF16))
    return fail(HOFEM_ERR_INVALID_ARG, "internal: an FP32 right-hand side needs an FP32 or BF16 solve");
  if (!f64 && p->wfmt == kFmtF16) {
    HOFEM_CUDA(cudaMemsetAsync(p->amax, 0, (size_t)nrhs * sizeof(unsigned long long), s), "memset amax");
    HOFEM_CUDA(launch_absmax(f, p->total, nrhs, p->amax, s), "absmax launch");
    amax = p->amax;
  }
  const int N = p->N;
  // forward along the contiguous axis, then the strided ones down to axis 1
  if ((st = run_sweep(p, N - 1, kFwd, f64, f, f_fmt, wa, fa, false, nullptr, nrhs, s, -1, amax)) != HOFEM_OK)
    return st;
  for (int a = N - 2; a >= 1; --a)
    if ((st = run_sweep(p, a, kFwd, f64, wa, fa, wa, fa, false, nullptr, nrhs, s)) != HOFEM_OK) return st;
  if ((st = run_sweep(p, 0, kFwdScaleInv, f64, wa, fa, wb, fb, false, nullptr, nrhs, s)) != HOFEM_OK) return st;
  for (int a = 1; a <= N - 2; ++a)
    if ((st = run_sweep(p, a, kInv, f64, wb, fb, wb, fb, false, nullptr, nrhs, s)) != HOFEM_OK) return st;
  return run_sweep(p, N - 1, kInv, f64, wb, fb, u, kFmtF64, accumulate, norms, nrhs, s, -1, nullptr, amax, norm_slot);
}

// One operator sweep along `axis` (modes in residual.cuh): Q == nullptr is the first
// sweep (out1 required), Q and out1 a middle one, Q without out1 the last one.
// Elements per CTA of an operator sweep without a tuned value: the largest of 16 / 8 / 4
// whose tile lets three CTAs share an SM (orders compiled for it), else 16, halved later to
// fit shared memory (measured best at n = 9, K = 1024: E = 8 at three CTAs per SM).
int apply_default_elems(int n) {
  int E = 16;
  if (n <= kApplyMinb3MaxN)
    while (E > 4 && apply_smem_bytes(n, E) > kApplySmem3) E /= 2;
  return E;
}

// Lines of an operator sweep that are not the plan's grid: the block's geometry (one right-
// hand side's outer lines and inner stride) and, when elems > 0, a stretch of the sweep's
// axis -- input rows from global dof q0 (in_rows of them), output rows from dof out0
// (out_rows), elements e0 .. e0 + elems - 1 (a slab of x_1 rows with its halo rows).
struct ApplyBlock {
  Geo g;
  long long q0 = 0, in_rows = 0, e0 = 0, elems = 0, out0 = 0, out_rows = 0;
};

hofem_status run_apply(hofem_plan_s* p, int axis, const double* P_, const double* Q_, double* out1, double* out2,
                       const double* f, double cA, double cCP, int nrhs, cudaStream_t s, bool uniform = false,
                       bool out_f32 = false, const ApplyBlock* blk = nullptr) {
  const DevAxis& A = p->ax[axis];
  Geo g = blk ? blk->g : geometry(p, axis);
  const bool part = blk && blk->elems > 0;   // a stretch of the axis, not whole lines
  const bool strided = g.inner > 1;
  ApplyParams P{};
  const int W = kApplyLines;
  int E = apply_default_elems(A.h.n);
  {
    int tE = 0, unused = 0;
    const TuneKey key = apply_key(p, axis, Q_ == nullptr ? kApplyFirst : (out1 ? kApplyMid : kApplyLast), nrhs);
    if (g_force_a > 0) E = g_force_a;
    else if (tuned_lookup(key, &tE, &unused)) E = tE;
  }
  if (const char* env = getenv("HOFEM_APPLY_E")) {
    const int e = atoi(env);
    if (e >= 1 && e <= 256) E = e;
  }
  while (apply_smem_bytes(A.h.n, E) > kSmemLimit && E > 1) E /= 2;
  E = std::min<long long>(E, part ? blk->elems : A.h.K);
  P.mode = Q_ == nullptr ? kApplyFirst : (out1 != nullptr ? kApplyMid : kApplyLast);
  if ((P.mode != kApplyLast) != (out1 != nullptr) || (P.mode == kApplyLast && cCP != 0.0) ||
      (P.mode != kApplyLast && f != nullptr))
    return fail(HOFEM_ERR_INVALID_ARG, "operator sweep: inconsistent arguments");
  P.outer = (long long)nrhs * g.outer_per_rhs;
  P.inner = g.inner;
  P.outer_per_rhs = g.outer_per_rhs;
  P.tiles_per_outer = strided ? (g.inner + W - 1) / W : (g.outer_per_rhs + W - 1) / W;
  P.seg_per_line = ((part ? blk->elems : A.h.K) + E - 1) / E;
  P.blk_q0 = part ? blk->q0 : 0;
  P.blk_in_rows = part ? blk->in_rows : A.h.M;
  P.blk_e0 = part ? blk->e0 : 0;
  P.blk_out0 = part ? blk->out0 : 0;
  P.blk_out_rows = part ? blk->out_rows : A.h.M;
  P.ntiles = (strided ? P.outer : nrhs) * P.tiles_per_outer * P.seg_per_line;
  P.M = A.h.M;
  P.n = A.h.n;
  P.K = A.h.K;
  P.W = W;
  P.E = E;
  P.P = P_;
  P.Q = Q_;
  P.out1 = out1;
  P.out2 = out2;
  P.f = f;
  P.cA = cA * A.h.a_scale;
  P.cCP = cCP;
  P.uniform = uniform ? 1 : 0;
  P.out2_f32 = out_f32 && P.mode == kApplyLast ? 1 : 0;
  std::copy(A.h.CfE.begin(), A.h.CfE.end(), P.CE);
  std::copy(A.h.CfO.begin(), A.h.CfO.end(), P.CO);
  std::copy(A.h.AfE.begin(), A.h.AfE.end(), P.AE);
  std::copy(A.h.AfO.begin(), A.h.AfO.end(), P.AO);
  for (size_t i = 0; i < A.h.AfELo.size(); ++i) P.AEl[i] = (float)A.h.AfELo[i];
  for (size_t i = 0; i < A.h.AfOLo.size(); ++i) P.AOl[i] = (float)A.h.AfOLo[i];
  P.smem_bytes = apply_smem_bytes(A.h.n, E);
  if (P.ntiles <= 0) return HOFEM_OK;
  cudaError_t e = timed_launch(p, 6, s, [&]() { return launch_apply(P, s); });
  if (e != cudaSuccess) return cuda_fail(e, "operator launch");
  return HOFEM_OK;
}

// True when every axis has the same stiffness coefficient 4 h_i^-2 / D_i (exact integer
// tables, n_i <= 9): the operator sweeps then carry unscaled sums and the last one scales.
bool uniform_stiffness(const hofem_plan_s* p, const double* sc) {
  const double c0 = sc[0] * p->ax[0].h.a_scale;
  for (int i = 0; i < p->N; ++i) {
    const AxisTables& h = p->ax[i].h;
    if (h.n > kExactStiffnessMaxN || h.a_scale == 1.0 || sc[i] * h.a_scale != c0) return false;
  }
  return c0 != 0.0;
}

// out = A u (f == nullptr) or out = f - A u, Eq. bvp glob 2, by one sweep per axis; with
// out_f32 the result is written as FP32 values into out's memory (a correction's FP32 solve
// rounds it to FP32 on reading anyway).
hofem_status operator_apply(hofem_plan_s* p, const double* u, const double* f, double* out, int nrhs,
                            cudaStream_t s, bool out_f32 = false) {
  hofem_status st = reserve(p, nrhs);
  if (st != HOFEM_OK) return st;
  const int N = p->N;
  double sc[3];
  for (int i = 0; i < N; ++i) sc[i] = 4.0 * (double)p->K[i] * (double)p->K[i] / (p->X[i] * p->X[i]);
  double** t = p->tmp64;
  if (uniform_stiffness(p, sc)) {
    // A u = c (sum_i A_i x prod_{m != i} C_m + alpha / c prod C_m), c applied by the last sweep
    const double c = sc[0] * p->ax[0].h.a_scale, ac = p->alpha / c;
    if (N == 2) {
      if ((st = run_apply(p, 1, u, nullptr, t[0], t[1], nullptr, sc[1], ac, nrhs, s, true)) != HOFEM_OK) return st;
      return run_apply(p, 0, t[0], t[1], nullptr, out, f, sc[0], 0.0, nrhs, s, true, out_f32);
    }
    if ((st = run_apply(p, 2, u, nullptr, t[0], t[1], nullptr, sc[2], ac, nrhs, s, true)) != HOFEM_OK) return st;
    if ((st = run_apply(p, 1, t[0], t[1], t[2], t[3], nullptr, sc[1], 0.0, nrhs, s, true)) != HOFEM_OK) return st;
    return run_apply(p, 0, t[2], t[3], nullptr, out, f, sc[0], 0.0, nrhs, s, true, out_f32);
  }
  if (N == 2) {
    // axis 1: T1 = u xC, T2 = s1 (u xA) + alpha (u xC); axis 0: out = [f -] (s0 T1 xA + T2 xC)
    if ((st = run_apply(p, 1, u, nullptr, t[0], t[1], nullptr, sc[1], p->alpha, nrhs, s)) != HOFEM_OK) return st;
    return run_apply(p, 0, t[0], t[1], nullptr, out, f, sc[0], 0.0, nrhs, s, false, out_f32);
  }
  // N == 3
  if ((st = run_apply(p, 2, u, nullptr, t[0], t[1], nullptr, sc[2], p->alpha, nrhs, s)) != HOFEM_OK) return st;
  if ((st = run_apply(p, 1, t[0], t[1], t[2], t[3], nullptr, sc[1], 0.0, nrhs, s)) != HOFEM_OK) return st;
  return run_apply(p, 0, t[2], t[3], nullptr, out, f, sc[0], 0.0, nrhs, s, false, out_f32);
}


// out = (C_1 x ... x C_N) u: operator sweeps with the stiffness coefficient 0, keeping
// the mass product of each axis (the second output is scratch).
hofem_status mass_apply(hofem_plan_s* p, const double* u, double* out, int nrhs, cudaStream_t s) {
  hofem_status st = reserve(p, nrhs);
  if (st != HOFEM_OK) return st;
  double** t = p->tmp64;
  if (p->N == 2) {
    if ((st = run_apply(p, 1, u, nullptr, t[0], t[1], nullptr, 0.0, 0.0, nrhs, s)) != HOFEM_OK) return st;
    return run_apply(p, 0, t[0], nullptr, out, t[1], nullptr, 0.0, 0.0, nrhs, s);
  }
  if ((st = run_apply(p, 2, u, nullptr, t[0], t[1], nullptr, 0.0, 0.0, nrhs, s)) != HOFEM_OK) return st;
  if ((st = run_apply(p, 1, t[0], nullptr, t[2], t[1], nullptr, 0.0, 0.0, nrhs, s)) != HOFEM_OK) return st;
  return run_apply(p, 0, t[2], nullptr, out, t[1], nullptr, 0.0, 0.0, nrhs, s);
}


// Algorithm (b) once: FP64 transforms along x_2..x_N (f -> u), one banded solve per mode
// along x_1 (scratch: tmp64[0]), inverse transforms.  u must not be tmp64[0].
hofem_status banded_once(hofem_plan_s* p, const double* f, double* u, int nrhs, cudaStream_t s) {
  hofem_status st;
  const int N = p->N;
  // FP64 direct transforms along x_2..x_N (f -> u), in the order of algorithm (a)
  if ((st = run_sweep(p, N - 1, kFwd, true, f, kFmtF64, u, kFmtF64, false, nullptr, nrhs, s)) != HOFEM_OK) return st;
  for (int a = N - 2; a >= 1; --a)
    if ((st = run_sweep(p, a, kFwd, true, u, kFmtF64, u, kFmtF64, false, nullptr, nrhs, s)) != HOFEM_OK) return st;
  // one banded solve per mode along x_1
  const DevAxis& A0 = p->ax[0];
  const Geo g = geometry(p, 0);
  BandParams B{};
  B.u = u;
  B.scratch = p->tmp64[0];
  B.outer = (long long)nrhs * g.outer_per_rhs;
  B.inner = g.inner;
  B.K = A0.h.K;
  B.n = A0.h.n;
  B.M = A0.h.M;
  B.sA = 4.0 * (double)p->K[0] * (double)p->K[0] / (p->X[0] * p->X[0]);
  B.alpha = p->alpha;
  B.lamA = p->ax[1].lam64;
  B.lamB = N == 3 ? p->ax[2].lam64 : nullptr;
  B.MB = N == 3 ? p->M[2] : 1;
  const int G = A0.h.n + 1;
  for (int i = 0; i < G * G; ++i) {
    B.A[i] = A0.h.Aloc[i];
    B.C[i] = A0.h.Cloc[i];
  }
  {
    cudaError_t e = timed_launch(p, 10, s, [&]() { return launch_banded(B, s); });
    if (e != cudaSuccess) return cuda_fail(e, "banded solve launch");
    p->info.kernel_launches += B.n > 1 ? 2 : 0;   // three kernels for n >= 2 (one counted above)
  }
  // FP64 inverse transforms back along x_2..x_N
  for (int a = 1; a <= N - 1; ++a)
    if ((st = run_sweep(p, a, kInv, true, u, kFmtF64, u, kFmtF64, false, nullptr, nrhs, s)) != HOFEM_OK) return st;
  return HOFEM_OK;
}


// Variable-coefficient operator r = A_a u (2D, equal orders): tables uploaded on first use.
hofem_status varcoef_apply(hofem_plan_s* p, const double* aq, const double* u, double* r, cudaStream_t s) {
  if (p->N != 2 || p->ax[0].h.n != p->ax[1].h.n || p->ax[0].h.n > 9)
    return fail(HOFEM_ERR_UNSUPPORTED, "the variable-coefficient operator is 2D with one order n <= 9");
  const int n = p->ax[0].h.n;
  if (!p->vcB) {
    std::vector<double> B, D, w;
    element_basis_tables(n, &B, &D, &w);
    size_t tb = 0;
    hofem_status st;
    if ((st = upload(B, &p->vcB, &tb)) != HOFEM_OK) return st;
    if ((st = upload(D, &p->vcD, &tb)) != HOFEM_OK) return st;
    if ((st = upload(w, &p->vcW, &tb)) != HOFEM_OK) return st;
  }
  VarcoefParams V{};
  V.u = u;
  V.r = r;
  V.aq = aq;
  V.B = p->vcB;
  V.D = p->vcD;
  V.w = p->vcW;
  V.K0 = p->K[0];
  V.K1 = p->K[1];
  V.M0 = p->M[0];
  V.M1 = p->M[1];
  V.n = n;
  V.s0 = 4.0 * (double)p->K[0] * (double)p->K[0] / (p->X[0] * p->X[0]);
  V.s1 = 4.0 * (double)p->K[1] * (double)p->K[1] / (p->X[1] * p->X[1]);
  HOFEM_CUDA(cudaMemsetAsync(r, 0, (size_t)p->total * sizeof(double), s), "memset (varcoef)");
  HOFEM_CUDA(launch_varcoef(V, s), "varcoef launch");
  p->info.kernel_launches += 1;
  return HOFEM_OK;
}

// x . y on the device, returned to the host (synchronises s).
hofem_status device_dot(hofem_plan_s* p, const double* x, const double* y, cudaStream_t s, double* out) {
  HOFEM_CUDA(cudaMemsetAsync(p->dot, 0, sizeof(double), s), "memset (dot)");
  HOFEM_CUDA(launch_dot(x, y, p->total, p->dot, s), "dot launch");
  HOFEM_CUDA(cudaMemcpyAsync(p->h_dot, p->dot, sizeof(double), cudaMemcpyDeviceToHost, s), "copy (dot)");
  HOFEM_CUDA(cudaStreamSynchronize(s), "stream sync (dot)");
  p->info.kernel_launches += 1;
  *out = *p->h_dot;
  return HOFEM_OK;
}

}  // namespace

namespace hofem {
void set_last_error(const std::string& msg) { g_last_error = msg; }
size_t static_scratch_doubles();
cudaError_t static_scratch_pointer(cudaStream_t s, double** out);
}  // namespace hofem

namespace {

// r = A u with the intermediates in the library's fixed device array (no allocation).
hofem_status operator_apply_static(hofem_plan_s* p, const double* u, double* out, int nrhs, cudaStream_t s) {
  const int N = p->N;
  const int ntmp = N == 2 ? 2 : 4;
  const size_t cnt = (size_t)nrhs * p->total;
  if (cnt * ntmp > static_scratch_doubles()) {
    char msg[160];
    snprintf(msg, sizeof msg, "hofem_apply_static: nrhs x unknowns = %zu exceeds the static scratch limit of %zu",
             cnt, static_scratch_doubles() / ntmp);
    return fail(HOFEM_ERR_INVALID_ARG, msg);
  }
  double* base = nullptr;
  cudaError_t e = static_scratch_pointer(s, &base);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
  double* t[4] = {base, base + cnt, base + 2 * cnt, base + 3 * cnt};
  double sc[3];
  for (int i = 0; i < N; ++i) sc[i] = 4.0 * (double)p->K[i] * (double)p->K[i] / (p->X[i] * p->X[i]);
  hofem_status st;
  if (N == 2) {
    if ((st = run_apply(p, 1, u, nullptr, t[0], t[1], nullptr, sc[1], p->alpha, nrhs, s)) != HOFEM_OK) return st;
    return run_apply(p, 0, t[0], t[1], nullptr, out, nullptr, sc[0], 0.0, nrhs, s);
  }
  if ((st = run_apply(p, 2, u, nullptr, t[0], t[1], nullptr, sc[2], p->alpha, nrhs, s)) != HOFEM_OK) return st;
  if ((st = run_apply(p, 1, t[0], t[1], t[2], t[3], nullptr, sc[1], 0.0, nrhs, s)) != HOFEM_OK) return st;
  return run_apply(p, 0, t[2], t[3], nullptr, out, nullptr, sc[0], 0.0, nrhs, s);
}


// ---- autotuner: time every candidate launch shape of this plan's sweeps and operator
// sweeps on its own (zeroed) workspace and keep the fastest per shape.
template <typename F> double time_launches(cudaStream_t s, F&& fn, bool* ok) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  *ok = fn() == HOFEM_OK;                       // warm-up
  double best = 1e30;
  for (int rep = 0; rep < 5 && *ok; ++rep) {
    cudaEventRecord(a, s);
    *ok = fn() == HOFEM_OK;
    cudaEventRecord(b, s);
    if (cudaEventSynchronize(b) != cudaSuccess) *ok = false;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    best = std::min(best, (double)ms);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaGetLastError();
  return best;
}

void tune_cache_io(bool save) {
  const char* path = getenv("HOFEM_TUNE_CACHE");
  if (!path || !*path) return;
  if (!save) {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    FILE* fp = fopen(path, "r");
    if (!fp) return;
    int k, M, n, K, ts, st, mo, a, b;
    long long lines;
    while (fscanf(fp, "%d %d %d %d %d %d %d %lld %d %d", &k, &M, &n, &K, &ts, &st, &mo, &lines, &a, &b) == 10)
      g_tuned[TuneKey{k, M, n, K, ts, st, mo, lines}] = {a, b};
    fclose(fp);
    return;
  }
  FILE* fp = fopen(path, "w");
  if (!fp) return;
  for (const auto& e : g_tuned) {
    const TuneKey& t = e.first;
    fprintf(fp, "%d %d %d %d %d %d %d %lld %d %d\n", std::get<0>(t), std::get<1>(t), std::get<2>(t), std::get<3>(t),
            std::get<4>(t), std::get<5>(t), std::get<6>(t), std::get<7>(t), e.second.first, e.second.second);
  }
  fclose(fp);
}

hofem_status tune_plan(hofem_plan_s* p, int nrhs, cudaStream_t s, int* measured) {
  hofem_status st = reserve(p, nrhs);
  if (st != HOFEM_OK) return st;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_cache_io(false);
  }
  const size_t cnt = (size_t)nrhs * p->total;
  HOFEM_CUDA(cudaMemsetAsync(p->r64, 0, cnt * sizeof(double), s), "memset (tune)");
  for (double* t : p->tmp64)
    if (t) HOFEM_CUDA(cudaMemsetAsync(t, 0, cnt * sizeof(double), s), "memset (tune)");
  if (p->work32) HOFEM_CUDA(cudaMemsetAsync(p->work32, 0, cnt * sizeof(float), s), "memset (tune)");
  if (p->work16) HOFEM_CUDA(cudaMemsetAsync(p->work16, 0, cnt * 2, s), "memset (tune)");
  const bool f64 = p->dtype == HOFEM_FP64;
  const int N = p->N;
  void* wa = f64 ? (void*)p->tmp64[0] : (void*)p->work32;
  void* wb = f64 ? (void*)p->tmp64[0] : (p->wfmt == kFmtF32 ? (void*)p->work32 : p->work16);
  const int fa = f64 ? kFmtF64 : kFmtF32, fb = f64 ? kFmtF64 : p->wfmt;
  // the last inverse sweep is timed as the correction solves run it (accumulating, with norms)
  struct Sw { int axis, mode; const void* in; int in_fmt; void* out; int out_fmt; bool acc; };
  std::vector<Sw> seq;
  seq.push_back({N - 1, kFwd, p->r64, kFmtF64, wa, fa, false});
  for (int a = N - 2; a >= 1; --a) seq.push_back({a, kFwd, wa, fa, wa, fa, false});
  seq.push_back({0, kFwdScaleInv, wa, fa, wb, fb, false});
  for (int a = 1; a <= N - 2; ++a) seq.push_back({a, kInv, wb, fb, wb, fb, false});
  seq.push_back({N - 1, kInv, wb, fb, p->tmp64[1], kFmtF64, !f64});
  const int tsize = f64 ? 8 : 4;
  for (const Sw& w : seq) {
    const TuneKey key = sweep_key(p, w.axis, w.mode, f64, nrhs, -1);
    int a0, b0;
    if (tuned_lookup(key, &a0, &b0)) continue;
    const DevAxis& A = p->ax[w.axis];
    {
      int rw = 0, rt = 0;
      size_t rs = 0;
      const unsigned long long* am = (!f64 && p->wfmt == kFmtF16) ? p->amax : nullptr;
      if (use_reg_sweep(A, f64, w.mode, std::get<5>(key) == 1, w.in_fmt, w.out_fmt, am, am, &rw, &rt, &rs))
        continue;   // fixed shape
    }
    const long long lines = std::get<7>(key);
    const bool strided = std::get<5>(key) == 1;
    double best = 1e30;
    int bw = 0, bj = 0;
    for (int W = 64; W >= 1; W >>= 1) {
      if (W > 1 && lines < W) continue;
      int Jmax = num_jobs_host(W, A.h.n);
      while (Jmax >= 1 && sweep_smem_bytes(A.h.M, A.h.n, A.h.K, sweep_nb(A, tsize), W, Jmax, tsize, strided) >
                              kSmemLimit)
        --Jmax;
      if (Jmax < 1) continue;
      // the largest DST batch, and halves of it (less shared memory, more batches)
      for (int J = Jmax; J >= 1 && J * 4 >= Jmax; J = (J == 1 ? 0 : (J + 1) / 2))
      for (int direct = 0; direct <= 1; ++direct) {
        g_force_a = W;
        g_force_b = J + direct * kMixDirectFlag;
        bool ok = false;
        const double ms = time_launches(s, [&]() {
          return run_sweep(p, w.axis, w.mode, f64, w.in, w.in_fmt, w.out, w.out_fmt, w.acc,
                           w.acc ? p->norms : nullptr, nrhs, s);
        }, &ok);
        g_force_a = g_force_b = 0;
        ++*measured;
        if (ok && ms < best) { best = ms; bw = W; bj = J + direct * kMixDirectFlag; }
      }
    }
    if (bw > 0) {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      g_tuned[key] = {bw, bj};
    }
  }
  // operator sweeps of the residual (refined dtypes) and of hofem_apply
  struct Ap { int axis; const double *P, *Q; double *o1, *o2; double cCP; };
  std::vector<Ap> aps;
  double** t = p->tmp64;
  if (N == 2) {
    aps.push_back({1, p->r64, nullptr, t[0], t[1], p->alpha});
    aps.push_back({0, t[0], t[1], nullptr, p->r64, 0.0});
  } else {
    aps.push_back({2, p->r64, nullptr, t[0], t[1], p->alpha});
    aps.push_back({1, t[0], t[1], t[2], t[3], 0.0});
    aps.push_back({0, t[2], t[3], nullptr, p->r64, 0.0});
  }
  // the kernel form the solves run (uniform scale or not)
  double sc[3];
  for (int i = 0; i < N; ++i) sc[i] = 4.0 * (double)p->K[i] * (double)p->K[i] / (p->X[i] * p->X[i]);
  const bool uni = uniform_stiffness(p, sc);
  for (const Ap& ap : aps) {
    const int mode = ap.Q == nullptr ? kApplyFirst : (ap.o1 ? kApplyMid : kApplyLast);
    const TuneKey key = apply_key(p, ap.axis, mode, nrhs);
    int a0, b0;
    if (tuned_lookup(key, &a0, &b0)) continue;
    const int dE = std::min(apply_default_elems(p->ax[ap.axis].h.n), p->ax[ap.axis].h.K);
    double best = 1e30, t_default = 1e30;
    int bE = 0;
    for (int E : {4, 8, 16, 32}) {
      if (E > p->ax[ap.axis].h.K || apply_smem_bytes(p->ax[ap.axis].h.n, E) > kSmemLimit) continue;
      g_force_a = E;
      bool ok = false;
      const double ms = time_launches(s, [&]() {
        return run_apply(p, ap.axis, ap.P, ap.Q, ap.o1, ap.o2, nullptr, 1.0, ap.cCP, nrhs, s, uni);
      }, &ok);
      g_force_a = 0;
      ++*measured;
      if (ok && ms < best) { best = ms; bE = E; }
      if (ok && E == dE) t_default = ms;
    }
    // the built-in shape unless a candidate is clearly faster: near-equal timings of one
    // sweep in isolation do not rank the shapes for a solve whose copies and neighbouring
    // kernels share the GPU (three CTAs per SM hide more of them)
    if (t_default < 1e30 && best > 0.97 * t_default) bE = dE;
    if (bE > 0) {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      g_tuned[key] = {bE, 0};
    }
  }
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_cache_io(true);
  }
  return HOFEM_OK;
}

}  // namespace

extern "C" {

const char* hofem_status_string(int s) {
  switch (s) {
    case HOFEM_OK: return "HOFEM_OK";
    case HOFEM_ERR_INVALID_ARG: return "HOFEM_ERR_INVALID_ARG";
    case HOFEM_ERR_UNSUPPORTED: return "HOFEM_ERR_UNSUPPORTED";
    case HOFEM_ERR_OOM: return "HOFEM_ERR_OOM";
    case HOFEM_ERR_CUDA: return "HOFEM_ERR_CUDA";
    case HOFEM_ERR_NOT_CONVERGED: return "HOFEM_ERR_NOT_CONVERGED";
    case HOFEM_ERR_TIMEOUT: return "HOFEM_ERR_TIMEOUT";
    default: return "HOFEM_ERR_UNKNOWN";
  }
}

const char* hofem_last_error(void) { return g_last_error.c_str(); }

hofem_status hofem_plan(int N, const int* K, int n, const double* X, int dtype, double alpha, hofem_plan_t* out) {
  const int ns[3] = {n, n, n};
  return hofem_plan_orders(N, K, ns, X, dtype, alpha, out);
}

hofem_status hofem_plan_orders(int N, const int* K, const int* ns, const double* X, int dtype, double alpha,
                               hofem_plan_t* out) {
  auto t0 = std::chrono::steady_clock::now();
  if (!out) return fail(HOFEM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (N != 2 && N != 3) return fail(HOFEM_ERR_INVALID_ARG, "N must be 2 or 3");
  if (!K || !X || !ns) return fail(HOFEM_ERR_INVALID_ARG, "K, n or X is NULL");
  int n = 0;                                     // largest order over the axes
  for (int i = 0; i < N; ++i) {
    if (ns[i] < 1 || ns[i] > kMaxN) return fail(HOFEM_ERR_INVALID_ARG, "order n must be in 1..16");
    n = std::max(n, ns[i]);
  }
  if (dtype < HOFEM_FP64 || dtype > HOFEM_FP16_REFINED) return fail(HOFEM_ERR_UNSUPPORTED, "unknown dtype");
  double lam_bound = 0.0;
  for (int i = 0; i < N; ++i) {
    if (K[i] < 2) return fail(HOFEM_ERR_INVALID_ARG, "K must be >= 2");
    if (K[i] > kMaxK) return fail(HOFEM_ERR_UNSUPPORTED, "K must be <= 8192");
    if (!(X[i] > 0.0) || !std::isfinite(X[i])) return fail(HOFEM_ERR_INVALID_ARG, "X must be positive");
    lam_bound += M_PI * M_PI / (X[i] * X[i]);
  }
  if (!(alpha > -lam_bound) || !std::isfinite(alpha))
    return fail(HOFEM_ERR_INVALID_ARG, "alpha must exceed -pi^2 sum X_i^-2");
  {
    // the dynamic shared-memory opt-in is a per-device function attribute
    static std::mutex mu;
    static std::vector<int> done;
    int dev = 0;
    HOFEM_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    std::lock_guard<std::mutex> lock(mu);
    if (std::find(done.begin(), done.end(), dev) == done.end()) {
      HOFEM_CUDA(sweep_set_smem_limits(), "cudaFuncSetAttribute(sweep)");
      HOFEM_CUDA(sweep_reg_set_smem_limits(), "cudaFuncSetAttribute(sweep_reg)");
      HOFEM_CUDA(apply_set_smem_limits(), "cudaFuncSetAttribute(apply)");
      done.push_back(dev);
    }
  }
  hofem_plan_s* p = new hofem_plan_s();
  p->N = N;
  p->n = n;
  p->dtype = dtype;
  p->refined = dtype == HOFEM_FP32_REFINED || dtype == HOFEM_BF16_REFINED || dtype == HOFEM_FP16_REFINED;
  p->wfmt = (dtype == HOFEM_BF16 || dtype == HOFEM_BF16_REFINED)   ? kFmtBF16
            : (dtype == HOFEM_FP16 || dtype == HOFEM_FP16_REFINED) ? kFmtF16
                                                                   : kFmtF32;
  p->alpha = alpha;
  // FP16 target exponent: high enough that the eigenvalue-damped lines stay above FP16's
  // smallest normal, with 2^6 headroom below its largest value for the transforms' gain
  // (measured: 2^12 overflowed at n = 8 in 3D); higher orders keep more headroom
  p->amax_exp = n <= 9 ? 10 : 6;
  if (const char* env = getenv("HOFEM_F16_EXP")) {   // tuning knob
    const int e = atoi(env);
    if (e >= -4 && e <= 14) p->amax_exp = e;
  }
  p->total = 1;
  for (int i = 0; i < N; ++i) {
    p->K[i] = K[i];
    p->X[i] = X[i];
    p->M[i] = ns[i] * K[i] - 1;
    p->total *= p->M[i];
  }
  hofem_status st = HOFEM_OK;
  for (int i = 0; i < N && st == HOFEM_OK; ++i) {
    DevAxis& a = p->ax[i];
    std::string err;
    int same = -1;
    for (int j = 0; j < i; ++j)
      if (K[j] == K[i] && X[j] == X[i] && ns[j] == ns[i]) same = j;
    // Bluestein form of the DFTs for K with large prime factors (HOFEM_FFT=direct or
    // =bluestein overrides the cost model for every non-power-of-two K)
    a.nb = bluestein_len(K[i]);
    if (const char* fe = getenv("HOFEM_FFT")) {
      if (!strcmp(fe, "direct")) a.nb = 0;
      if (!strcmp(fe, "bluestein") && !is_pow2(K[i])) a.nb = bluestein_pow2(K[i]);
    }
    if (same >= 0 && p->ax[same].nb == a.nb) {
      a.h = p->ax[same].h;
    } else {
      st = build_axis_tables(ns[i], K[i], X[i], &a.h, &err);
      if (st != HOFEM_OK) { g_last_error = err; break; }
      if (a.nb > 0) {
        int np = 0, rb[8] = {0};
        radix_plan(a.nb, &np, rb);
        bluestein_tables(K[i], a.nb, np, rb, &a.h.tw);
      }
    }
    size_t& tb = p->table_bytes;
    if ((st = upload(a.h.lam, &a.lam64, &tb)) != HOFEM_OK) break;
    {
      // mixing rows padded to a multiple of 4 entries for 16-byte vector loads
      const int na = ns[i], np = (na + 3) & ~3;
      std::vector<double> padded((size_t)(K[i] - 1) * na * np, 0.0);
      for (size_t r = 0; r < (size_t)(K[i] - 1) * na; ++r)
        for (int c = 0; c < na; ++c) padded[r * np + c] = a.h.mix[r * na + c];
      a.mixNP = np;
      if ((st = upload(padded, &a.mix64, &tb)) != HOFEM_OK) break;
      if ((st = upload(padded, &a.mix32, &tb)) != HOFEM_OK) break;
    }
    {
      const int na = ns[i], Km = K[i] - 1;
      std::vector<double> mt((size_t)Km * na * na), lt((size_t)Km * na);
      for (int k = 0; k < Km; ++k)
        for (int l = 0; l < na; ++l) {
          lt[(size_t)l * Km + k] = a.h.lam[(size_t)k * na + l];
          for (int c = 0; c < na; ++c) mt[((size_t)l * na + c) * Km + k] = a.h.mix[((size_t)k * na + l) * na + c];
        }
      if ((st = upload(mt, &a.mixT32, &tb)) != HOFEM_OK) break;
      if ((st = upload(lt, &a.lamT32, &tb)) != HOFEM_OK) break;
      if (is_pow2(K[i]) && K[i] >= 64) {
        // from the DST twiddles exp(-i pi t / K): w_K^{r k2} = tw[2 r k2], w_2K^{r (2k2+1)} = tw[r (2k2+1)]
        const int L = K[i] / 32;
        std::vector<double> tr((size_t)4 * K[i]);
        for (int k2 = 0; k2 < 32; ++k2)
          for (int r = 0; r < L; ++r) {
            const size_t ix = (size_t)k2 * L + r, tx = (size_t)2 * r * k2, tz = (size_t)r * (2 * k2 + 1);
            tr[2 * ix] = a.h.tw[2 * tx];
            tr[2 * ix + 1] = a.h.tw[2 * tx + 1];
            tr[2 * (K[i] + ix)] = a.h.tw[2 * tz];
            tr[2 * (K[i] + ix) + 1] = a.h.tw[2 * tz + 1];
          }
        if ((st = upload(tr, &a.twr32, &tb)) != HOFEM_OK) break;
      }
    }
    if ((st = upload(a.h.evec, &a.evec64, &tb)) != HOFEM_OK) break;
    if ((st = upload(a.h.tw, &a.tw64, &tb)) != HOFEM_OK) break;
    if ((st = upload(a.h.lam, &a.lam32, &tb)) != HOFEM_OK) break;
    if ((st = upload(a.h.evec, &a.evec32, &tb)) != HOFEM_OK) break;
    if ((st = upload(a.h.tw, &a.tw32, &tb)) != HOFEM_OK) break;
    if (!radix_plan(K[i], &a.npass, a.radix)) {
      g_last_error = "K has too many prime factors for the FFT plan (more than 8 passes)";
      st = HOFEM_ERR_UNSUPPORTED;
      break;
    }
    // one line and one DST job must fit the 227 KB of shared memory of a CTA at the
    // precision of this plan's sweeps (FP64 plans: FP64; all others: FP32)
    const int tsize = dtype == HOFEM_FP64 ? 8 : 4;
    if (sweep_smem_bytes(p->M[i], ns[i], K[i], sweep_nb(a, tsize), 1, 1, tsize, false) > kSmemLimit) {
      char msg[200];
      snprintf(msg, sizeof msg,
               "axis %d: a line of %d unknowns and its K = %d transform do not fit shared memory in %s "
               "(smaller K, a power of two, or a lower-precision dtype)",
               i, p->M[i], K[i], tsize == 8 ? "FP64" : "FP32");
      g_last_error = msg;
      st = HOFEM_ERR_UNSUPPORTED;
      break;
    }
  }
  if (st != HOFEM_OK) {
    for (int i = 0; i < N; ++i) free_axis(p->ax[i]);
    delete p;
    return st;
  }
  // Default refinement: corrections until ||delta|| / ||u|| <= 1e-12 (measured: the error
  // after a correction stays below its update norm), at most 10 (FP32) or 16 (BF16,
  // FP16).  The contraction per step depends on the right-hand side: a rough residual is
  // solved accurately in its high modes only, a smooth one throughout, so steps alternate
  // between ~0.1-0.9 and ~1e-5 (2D n = 9, K = 1024, N(0,1) RHS: 2.4e-12 after 2, 6e-15
  // after 4; smooth RHS: 4.9e-13 after 2).  A capturing stream cannot be read by the host,
  // so a captured solve runs a fixed count instead: FP32 2 when every K is a power of two,
  // else 3 (512 problems, n = 2..8, K = 32..512, N(0,1): worst 7.5e-14 after 3), BF16 and
  // FP16 8.
  bool all_pow2 = true;
  for (int i = 0; i < N; ++i) all_pow2 = all_pow2 && is_pow2(K[i]);
  const bool half = dtype == HOFEM_BF16_REFINED || dtype == HOFEM_FP16_REFINED;
  p->capture_iters = dtype == HOFEM_FP32_REFINED ? (all_pow2 ? 2 : 3) : half ? 8 : 0;
  p->refine_iters = dtype == HOFEM_FP32_REFINED ? 10 : half ? 16 : 0;
  p->refine_tol = p->refined ? 1e-12 : 0.0;
  for (int i = 0; i < N; ++i) element_load_table(ns[i], &p->load_T[i], &p->load_xi[i]);
  hofem_info& inf = p->info;
  inf.N = N;
  inf.n = n;
  for (int i = 0; i < N; ++i) inf.orders[i] = ns[i];
  for (int i = 0; i < N; ++i) {
    const int nb = sweep_nb(p->ax[i], dtype == HOFEM_FP64 ? 8 : 4);
    inf.fft_len[i] = nb > 0 ? nb : K[i];
  }
  for (int i = 0; i < N; ++i) {
    inf.K[i] = K[i];
    inf.M[i] = p->M[i];
  }
  inf.dtype = dtype;
  inf.refine_iters = p->refine_iters;
  inf.table_bytes = p->table_bytes;
  inf.threads_per_cta = kThreads;
  inf.plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = p;
  return HOFEM_OK;
}

hofem_status hofem_set_refinement(hofem_plan_t p, int iters, double tol) {
  if (!p) return fail(HOFEM_ERR_INVALID_ARG, "plan is NULL");
  if (!p->refined) return fail(HOFEM_ERR_INVALID_ARG, "plan dtype is not refined");
  if (iters < 0 || iters > 100 || !(tol >= 0.0)) return fail(HOFEM_ERR_INVALID_ARG, "iters in 0..100, tol >= 0");
  p->refine_iters = iters;
  p->refine_tol = tol;
  if (tol == 0.0) p->capture_iters = iters;
  p->info.refine_iters = iters;
  return HOFEM_OK;
}

hofem_status hofem_quadrature_points(hofem_plan_t p, int axis, double* x) {
  if (!p || !x) return fail(HOFEM_ERR_INVALID_ARG, "plan or x is NULL");
  if (axis < 0 || axis >= p->N) return fail(HOFEM_ERR_INVALID_ARG, "axis out of range");
  const int G = p->ax[axis].h.n + 1, K = p->K[axis];
  const double h = p->X[axis] / K;
  for (int e = 0; e < K; ++e)
    for (int g = 0; g < G; ++g) x[(size_t)e * G + g] = e * h + (p->load_xi[axis][g] + 1.0) * h / 2.0;
  return HOFEM_OK;
}

hofem_status hofem_lift_dirichlet(hofem_plan_t p, const double* vb, double* f, int nrhs, void* stream) {
  if (!p) return fail(HOFEM_ERR_INVALID_ARG, "plan is NULL");
  if (!vb || !f || nrhs < 1) return fail(HOFEM_ERR_INVALID_ARG, "bad pointers or nrhs");
  if ((const void*)vb == (const void*)f) return fail(HOFEM_ERR_INVALID_ARG, "vb and f must differ");
  LiftParams L{};
  L.vb = vb;
  L.f = f;
  L.N = p->N;
  L.nrhs = nrhs;
  L.alpha = p->alpha;
  for (int i = 0; i < p->N; ++i) {
    const AxisTables& h = p->ax[i].h;
    L.n[i] = h.n;
    L.M[i] = p->M[i];
    L.P[i] = p->M[i] + 2;
    L.coef[i] = 4.0 * (double)p->K[i] * (double)p->K[i] / (p->X[i] * p->X[i]);
    const int m1 = h.n + 1;
    if ((int)h.Aloc.size() != m1 * m1 || (int)h.Cloc.size() != m1 * m1)
      return fail(HOFEM_ERR_UNSUPPORTED, "plan has no local element matrices");
    for (int k = 0; k < m1 * m1; ++k) {
      L.A[i][k] = h.Aloc[k];
      L.C[i][k] = h.Cloc[k];
    }
  }
  cudaError_t e = launch_lift(L, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "lift launch");
  ++p->info.kernel_launches;
  return HOFEM_OK;
}

hofem_status hofem_load(hofem_plan_t p, const double* fq, double* fh, int nrhs, void* stream) {
  if (!p) return fail(HOFEM_ERR_INVALID_ARG, "plan is NULL");
  if (!fq || !fh || nrhs < 1) return fail(HOFEM_ERR_INVALID_ARG, "bad pointers or nrhs");
  if ((const void*)fq == (const void*)fh) return fail(HOFEM_ERR_INVALID_ARG, "fq and fh must differ");
  cudaStream_t s = (cudaStream_t)stream;
  const int N = p->N;
  long long L[3];                                   // current length of every axis
  for (int i = 0; i < N; ++i) L[i] = (long long)p->K[i] * (p->ax[i].h.n + 1);
  // intermediates after axes N-1 .. 1 (axis 0 writes fh)
  size_t need = 0;
  {
    long long Lt[3] = {L[0], L[1], L[2]};
    for (int a = N - 1; a >= 1; --a) {
      Lt[a] = p->M[a];
      size_t cnt = (size_t)nrhs;
      for (int i = 0; i < N; ++i) cnt *= (size_t)Lt[i];
      need = std::max(need, cnt);
    }
  }
  if (need > p->ld_count) {
    cudaFree(p->ld[0]);
    cudaFree(p->ld[1]);
    p->ld[0] = p->ld[1] = nullptr;
    p->ld_count = 0;
    HOFEM_CUDA(cudaMalloc(&p->ld[0], need * sizeof(double)), "cudaMalloc(load buffer)");
    HOFEM_CUDA(cudaMalloc(&p->ld[1], need * sizeof(double)), "cudaMalloc(load buffer)");
    p->ld_count = need;
  }
  LoadParams P{};
  const double* in = fq;
  int buf = 0;
  for (int a = N - 1; a >= 0; --a) {
    const int na = p->ax[a].h.n, G = na + 1;
    P.n = na;
    for (int i = 0; i < G * G; ++i) P.T[i] = p->load_T[a][i];
    P.in = in;
    P.out = a == 0 ? fh : p->ld[buf];
    P.K = p->K[a];
    P.M = p->M[a];
    P.outer = nrhs;
    for (int i = 0; i < a; ++i) P.outer *= L[i];
    P.inner = 1;
    for (int i = a + 1; i < N; ++i) P.inner *= p->M[i];
    HOFEM_CUDA(launch_load(P, s), "load launch");
    p->info.kernel_launches += 1;
    L[a] = p->M[a];
    in = P.out;
    buf ^= 1;
  }
  return HOFEM_OK;
}

hofem_status hofem_solve_banded(hofem_plan_t p, const double* f, double* u, int nrhs, void* stream) {
  if (!p) return fail(HOFEM_ERR_INVALID_ARG, "plan is NULL");
  if (!f || !u || nrhs < 1) return fail(HOFEM_ERR_INVALID_ARG, "bad pointers or nrhs");
  if ((const void*)f == (const void*)u) return fail(HOFEM_ERR_INVALID_ARG, "f and u must differ");
  if (p->ax[0].h.n > kExactStiffnessMaxN)
    return fail(HOFEM_ERR_UNSUPPORTED, "algorithm (b) supports n_1 <= 9 (higher orders: use hofem_solve)");
  cudaStream_t s = (cudaStream_t)stream;
  hofem_status st = reserve(p, nrhs);
  if (st != HOFEM_OK) return st;
  if ((st = banded_once(p, f, u, nrhs, s)) != HOFEM_OK) return st;
  // one correction with the matrix-free FP64 residual: the interior blocks of high-order
  // equispaced elements are ill-conditioned, so a plain banded solve loses ~cond(E_II) eps
  // (measured 2.7e-12 at n = 9, 6e-10 at n = 16); the correction contracts the error by it
  if ((st = operator_apply(p, u, f, p->r64, nrhs, s)) != HOFEM_OK) return st;
  double* delta = p->tmp64[1];
  if ((st = banded_once(p, p->r64, delta, nrhs, s)) != HOFEM_OK) return st;
  HOFEM_CUDA(launch_axpby(u, 1.0, delta, (long long)nrhs * p->total, s), "axpby launch");
  p->info.kernel_launches += 1;
  return HOFEM_OK;
}

hofem_status hofem_apply_varcoef(hofem_plan_t p, const double* aq, const double* u, double* r, void* stream) {
  if (!p) return fail(HOFEM_ERR_INVALID_ARG, "plan is NULL");
  if (!aq || !u || !r || (const void*)u == (const void*)r) return fail(HOFEM_ERR_INVALID_ARG, "bad pointers");
  return varcoef_apply(p, aq, u, r, (cudaStream_t)stream);
}

hofem_status hofem_pcg(hofem_plan_t p, const double* aq, const double* f, double* u, double tol, int maxit,
                       int* iters, double* relres, void* stream) {
  if (!p) return fail(HOFEM_ERR_INVALID_ARG, "plan is NULL");
  if (!aq || !f || !u || (const void*)f == (const void*)u) return fail(HOFEM_ERR_INVALID_ARG, "bad pointers");
  if (!(tol > 0.0) || maxit < 1) return fail(HOFEM_ERR_INVALID_ARG, "tol > 0 and maxit >= 1 required");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t cnt = (size_t)p->total;
  for (double*& v : p->cg)
    if (!v) HOFEM_CUDA(cudaMalloc(&v, cnt * sizeof(double)), "cudaMalloc(pcg vectors)");
  if (!p->dot) HOFEM_CUDA(cudaMalloc(&p->dot, sizeof(double)), "cudaMalloc(dot)");
  if (!p->h_dot) HOFEM_CUDA(cudaMallocHost(&p->h_dot, sizeof(double)), "cudaMallocHost(dot)");
  double *r = p->cg[0], *z = p->cg[1], *d = p->cg[2], *q = p->cg[3];
  hofem_status st;
  // r = f - A_a u; z = P^-1 r (the fast constant-coefficient solve); d = z
  if ((st = varcoef_apply(p, aq, u, r, s)) != HOFEM_OK) return st;
  HOFEM_CUDA(launch_axpby(r, -1.0, f, (long long)cnt, s), "axpby launch");
  double ff, rz, rr;
  if ((st = device_dot(p, f, f, s, &ff)) != HOFEM_OK) return st;
  if ((st = device_dot(p, r, r, s, &rr)) != HOFEM_OK) return st;
  const double fn = std::sqrt(ff) > 0 ? std::sqrt(ff) : 1.0;
  int k = 0;
  double res = std::sqrt(rr) / fn;
  if (res > tol) {
    if ((st = hofem_solve(p, r, z, 1, stream)) != HOFEM_OK) return st;
    HOFEM_CUDA(cudaMemcpyAsync(d, z, cnt * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy (pcg)");
    if ((st = device_dot(p, r, z, s, &rz)) != HOFEM_OK) return st;
    while (k < maxit) {
      ++k;
      if ((st = varcoef_apply(p, aq, d, q, s)) != HOFEM_OK) return st;
      double dq;
      if ((st = device_dot(p, d, q, s, &dq)) != HOFEM_OK) return st;
      const double a = rz / dq;
      HOFEM_CUDA(launch_axpy(u, a, d, (long long)cnt, s), "axpy launch");
      HOFEM_CUDA(launch_axpy(r, -a, q, (long long)cnt, s), "axpy launch");
      if ((st = device_dot(p, r, r, s, &rr)) != HOFEM_OK) return st;
      res = std::sqrt(rr) / fn;
      if (res <= tol) break;
      if ((st = hofem_solve(p, r, z, 1, stream)) != HOFEM_OK) return st;
      double rz_new;
      if ((st = device_dot(p, r, z, s, &rz_new)) != HOFEM_OK) return st;
      HOFEM_CUDA(launch_axpby(d, rz_new / rz, z, (long long)cnt, s), "axpby launch");
      rz = rz_new;
    }
  }
  if (iters) *iters = k;
  if (relres) *relres = res;
  if (res > tol) return fail(HOFEM_ERR_NOT_CONVERGED, "PCG reached maxit before the tolerance");
  return HOFEM_OK;
}

hofem_status hofem_mass(hofem_plan_t p, const double* u, double* out, int nrhs, void* stream) {
  if (!p) return fail(HOFEM_ERR_INVALID_ARG, "plan is NULL");
  if (!u || !out || nrhs < 1) return fail(HOFEM_ERR_INVALID_ARG, "bad pointers or nrhs");
  if ((const void*)u == (const void*)out) return fail(HOFEM_ERR_INVALID_ARG, "u and out must differ");
  return mass_apply(p, u, out, nrhs, (cudaStream_t)stream);
}

hofem_status hofem_heat_steps(hofem_plan_t p, double* u, const double* g, int steps, int nrhs, void* stream) {
  if (!p) return fail(HOFEM_ERR_INVALID_ARG, "plan is NULL");
  if (!u || nrhs < 1 || steps < 0) return fail(HOFEM_ERR_INVALID_ARG, "bad pointers, nrhs or steps");
  if (!(p->alpha > 0.0)) return fail(HOFEM_ERR_INVALID_ARG, "heat steps need a plan with alpha = 1/tau > 0");
  if (g && (const void*)g == (const void*)u) return fail(HOFEM_ERR_INVALID_ARG, "g and u must differ");
  cudaStream_t s = (cudaStream_t)stream;
  hofem_status st = reserve(p, nrhs);
  if (st != HOFEM_OK) return st;
  if (nrhs > p->heat_nrhs) {
    cudaFree(p->heat);
    p->heat = nullptr;
    p->heat_nrhs = 0;
    HOFEM_CUDA(cudaMalloc(&p->heat, (size_t)nrhs * p->total * sizeof(double)), "cudaMalloc(heat rhs)");
    p->heat_nrhs = nrhs;
  }
  const long long cnt = (long long)nrhs * p->total;
  for (int m = 0; m < steps; ++m) {
    if ((st = mass_apply(p, u, p->heat, nrhs, s)) != HOFEM_OK) return st;
    HOFEM_CUDA(launch_axpby(p->heat, p->alpha, g, cnt, s), "axpby launch");
    p->info.kernel_launches += 1;
    if ((st = hofem_solve(p, p->heat, u, nrhs, stream)) != HOFEM_OK) return st;
  }
  return HOFEM_OK;
}

hofem_status hofem_autotune(hofem_plan_t p, int nrhs, void* stream) {
  if (!p) return fail(HOFEM_ERR_INVALID_ARG, "plan is NULL");
  if (nrhs < 1) return fail(HOFEM_ERR_INVALID_ARG, "nrhs must be >= 1");
  cudaStream_t s = (cudaStream_t)stream;
  int measured = 0;
  const hofem_status st = tune_plan(p, nrhs, s, &measured);
  HOFEM_CUDA(cudaStreamSynchronize(s), "stream sync (autotune)");
  p->info.tuned_shapes += measured;
  return st;
}

hofem_status hofem_reserve(hofem_plan_t p, int nrhs) {
  if (!p) return fail(HOFEM_ERR_INVALID_ARG, "plan is NULL");
  if (nrhs < 1) return fail(HOFEM_ERR_INVALID_ARG, "nrhs must be >= 1");
  return reserve(p, nrhs);
}

hofem_status hofem_solve(hofem_plan_t p, const double* f, double* u, int nrhs, void* stream) {
  if (!p) return fail(HOFEM_ERR_INVALID_ARG, "plan is NULL");
  if (!f || !u) return fail(HOFEM_ERR_INVALID_ARG, "f or u is NULL");
  if (nrhs < 1) return fail(HOFEM_ERR_INVALID_ARG, "nrhs must be >= 1");
  cudaStream_t s = (cudaStream_t)stream;
  const bool refined = p->refined;
  if (refined && (const void*)f == (const void*)u)
    return fail(HOFEM_ERR_INVALID_ARG, "f and u must differ for refined solves");
  hofem_status st;
  if (p->dtype == HOFEM_FP64) {
    st = solve_once(p, f, u, nrhs, true, false, nullptr, 0, s);
    p->info.iterations = 0;
    p->info.converged = 1;
    return st;
  }
  if ((st = reserve(p, nrhs)) != HOFEM_OK) return st;
  // the tolerance test reads the norms on the host, which a capturing stream cannot do
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  HOFEM_CUDA(cudaStreamIsCapturing(s, &cap), "cudaStreamIsCapturing");
  const bool adaptive = refined && p->refine_tol > 0.0 && cap == cudaStreamCaptureStatusNone;
  const int iters = !refined ? 0 : (p->refine_tol > 0.0 && !adaptive) ? p->capture_iters : p->refine_iters;
  // norms[2 r + 1] = ||u||^2 of the first solve, norms[2 r] = ||delta||^2 of the last step
  if (iters > 0) HOFEM_CUDA(cudaMemsetAsync(p->norms, 0, 2 * (size_t)nrhs * sizeof(double), s), "memset norms");
  if ((st = solve_once(p, f, u, nrhs, false, false, iters > 0 ? p->norms : nullptr, 1, s)) != HOFEM_OK) return st;
  int done = 0;
  bool converged = false;
  // an FP32 correction solve reads its right-hand side as FP32 values: the residual is
  // written that way (into the residual buffer), which halves its store and the first
  // sweep's load and lets that sweep use the asynchronous FP32 tile path
  const bool r32 = p->wfmt == kFmtF32;
  for (int i = 0; i < iters; ++i) {
    if ((st = operator_apply(p, u, f, p->r64, nrhs, s, r32)) != HOFEM_OK) return st;
    HOFEM_CUDA(cudaMemset2DAsync(p->norms, 2 * sizeof(double), 0, sizeof(double), nrhs, s), "memset norms");
    if ((st = solve_once(p, p->r64, u, nrhs, false, true, p->norms, 0, s, r32 ? kFmtF32 : kFmtF64)) != HOFEM_OK)
      return st;
    ++done;
    if (adaptive) {
      HOFEM_CUDA(cudaMemcpyAsync(p->h_norms, p->norms, 2 * (size_t)nrhs * sizeof(double), cudaMemcpyDeviceToHost, s),
                 "copy norms");
      HOFEM_CUDA(cudaStreamSynchronize(s), "stream sync (refinement tolerance)");
      double worst = 0.0;
      for (int r = 0; r < nrhs; ++r) {
        const double nu = p->h_norms[2 * r + 1];
        worst = std::max(worst, nu > 0 ? std::sqrt(p->h_norms[2 * r] / nu) : 0.0);
      }
      if (worst <= p->refine_tol) { converged = true; break; }
    }
  }
  if (!adaptive) {
    converged = true;   // fixed iteration count
    if (iters > 0)
      HOFEM_CUDA(cudaMemcpyAsync(p->h_norms, p->norms, 2 * (size_t)nrhs * sizeof(double), cudaMemcpyDeviceToHost, s),
                 "copy norms");
  }
  p->info.iterations = done;
  p->info.converged = converged ? 1 : 0;
  if (adaptive && !converged)
    return fail(HOFEM_ERR_NOT_CONVERGED, "refinement did not reach the tolerance");
  return HOFEM_OK;
}

hofem_status hofem_apply(hofem_plan_t p, const double* u, double* r, int nrhs, void* stream) {
  if (!p) return fail(HOFEM_ERR_INVALID_ARG, "plan is NULL");
  if (!u || !r || nrhs < 1) return fail(HOFEM_ERR_INVALID_ARG, "bad pointers or nrhs");
  if ((const void*)u == (const void*)r) return fail(HOFEM_ERR_INVALID_ARG, "u and r must differ");
  return operator_apply(p, u, nullptr, r, nrhs, (cudaStream_t)stream);
}

hofem_status hofem_apply_static(hofem_plan_t p, const double* u, double* r, int nrhs, void* stream) {
  if (!p) return fail(HOFEM_ERR_INVALID_ARG, "plan is NULL");
  if (!u || !r || nrhs < 1) return fail(HOFEM_ERR_INVALID_ARG, "bad pointers or nrhs");
  if ((const void*)u == (const void*)r) return fail(HOFEM_ERR_INVALID_ARG, "u and r must differ");
  return operator_apply_static(p, u, r, nrhs, (cudaStream_t)stream);
}

hofem_status hofem_residual(hofem_plan_t p, const double* f, const double* u, double* r, int nrhs, void* stream) {
  if (!p) return fail(HOFEM_ERR_INVALID_ARG, "plan is NULL");
  if (!f || !u || !r || nrhs < 1) return fail(HOFEM_ERR_INVALID_ARG, "bad pointers or nrhs");
  if ((const void*)u == (const void*)r) return fail(HOFEM_ERR_INVALID_ARG, "u and r must differ");
  return operator_apply(p, u, f, r, nrhs, (cudaStream_t)stream);
}

hofem_status hofem_transform1d(hofem_plan_t p, int axis, int inverse, const double* in, double* out, long lines,
                               void* stream) {
  if (!p) return fail(HOFEM_ERR_INVALID_ARG, "plan is NULL");
  if (axis < 0 || axis >= p->N) return fail(HOFEM_ERR_INVALID_ARG, "axis out of range");
  if (!in || !out || lines < 1) return fail(HOFEM_ERR_INVALID_ARG, "bad pointers or lines");
  const bool f64 = p->dtype == HOFEM_FP64;
  // work in the output buffer: FP64 in place, or via the FP32 path converting on load/store
  return run_sweep(p, axis, inverse ? kInv : kFwd, f64, in, kFmtF64, out, kFmtF64, false, nullptr, 1,
                   (cudaStream_t)stream, lines);
}

hofem_status hofem_sweep(hofem_plan_t p, int axis, int mode, const double* in, double* out, long long outer,
                         long long inner, long long line_offset, void* stream) {
  if (!p) return fail(HOFEM_ERR_INVALID_ARG, "plan is NULL");
  if (axis < 0 || axis >= p->N) return fail(HOFEM_ERR_INVALID_ARG, "axis out of range");
  if (!in || !out || outer < 0 || inner < 1) return fail(HOFEM_ERR_INVALID_ARG, "bad pointers or block sizes");
  if (mode < HOFEM_SWEEP_FORWARD || mode > HOFEM_SWEEP_INVERSE) return fail(HOFEM_ERR_INVALID_ARG, "bad mode");
  long long plane = 1;
  for (int i = 1; i < p->N; ++i) plane *= p->M[i];
  if (mode == HOFEM_SWEEP_FUSED && (axis != 0 || line_offset < 0 || line_offset + inner > plane))
    return fail(HOFEM_ERR_INVALID_ARG, "the fused sweep runs along axis 0 on columns inside the x_2..x_N plane");
  if (outer == 0) return HOFEM_OK;
  const int m = mode == HOFEM_SWEEP_FORWARD ? kFwd : mode == HOFEM_SWEEP_FUSED ? kFwdScaleInv : kInv;
  const Geo block{outer, inner};
  return run_sweep(p, axis, m, p->dtype == HOFEM_FP64, in, kFmtF64, out, kFmtF64, false, nullptr, 1,
                   (cudaStream_t)stream, -1, nullptr, nullptr, 0, &block, mode == HOFEM_SWEEP_FUSED ? line_offset : 0);
}

hofem_status hofem_residual_slab(hofem_plan_t p, int stage, long long e0, long long e1, const double* a,
                                 const double* b, const double* f, double* out0, double* out1, int out_fp32, int nrhs,
                                 void* stream) {
  if (!p) return fail(HOFEM_ERR_INVALID_ARG, "plan is NULL");
  const int N = p->N, n0 = p->ax[0].h.n, K0 = p->K[0];
  const long long M0 = p->M[0];
  if (stage < 0 || stage > 1 || e0 < 0 || e1 <= e0 || e1 > K0 || nrhs < 1 || !a || !out0 ||
      (stage == 0 && !out1) || (stage == 1 && !b))
    return fail(HOFEM_ERR_INVALID_ARG, "bad stage, element range, nrhs or pointers");
  cudaStream_t s = (cudaStream_t)stream;
  hofem_status st = reserve(p, 1);   // scratch of the 3D first pass
  if (st != HOFEM_OK) return st;
  const long long rows = std::min<long long>(e1 * n0, M0) - e0 * n0;
  const long long pre = e0 > 0 ? 1 : 0, post = e1 < K0 ? n0 : 0, ext = pre + rows + post;
  long long plane = 1;
  for (int i = 1; i < N; ++i) plane *= p->M[i];
  double sc[3];
  for (int i = 0; i < N; ++i) sc[i] = 4.0 * (double)p->K[i] * (double)p->K[i] / (p->X[i] * p->X[i]);
  const bool uni = uniform_stiffness(p, sc);
  const double cCP = uni ? p->alpha / (sc[0] * p->ax[0].h.a_scale) : p->alpha;
  if (stage == 0) {
    // the sweeps along x_N .. x_2 of the slab's rows, into the owned rows of the extended arrays
    for (int q = 0; q < nrhs; ++q) {
      const double* uq = a + (size_t)q * rows * plane;
      double* t0 = out0 + ((size_t)q * ext + pre) * plane;
      double* t1 = out1 + ((size_t)q * ext + pre) * plane;
      if (N == 2) {
        ApplyBlock blk;
        blk.g = Geo{rows, 1};
        if ((st = run_apply(p, 1, uq, nullptr, t0, t1, nullptr, sc[1], cCP, 1, s, uni, false, &blk)) != HOFEM_OK)
          return st;
      } else {
        double** t = p->tmp64;
        ApplyBlock b2, b1;
        b2.g = Geo{rows * p->M[1], 1};
        b1.g = Geo{rows, p->M[2]};
        if ((st = run_apply(p, 2, uq, nullptr, t[0], t[1], nullptr, sc[2], cCP, 1, s, uni, false, &b2)) != HOFEM_OK)
          return st;
        if ((st = run_apply(p, 1, t[0], t[1], t0, t1, nullptr, sc[1], 0.0, 1, s, uni, false, &b1)) != HOFEM_OK)
          return st;
      }
    }
    return HOFEM_OK;
  }
  // the sweep along x_1 over the slab's elements, its halo rows read from the extended arrays
  ApplyBlock blk;
  blk.g = Geo{1, plane};
  blk.q0 = e0 * n0 - pre;
  blk.in_rows = ext;
  blk.e0 = e0;
  blk.elems = e1 - e0;
  blk.out0 = e0 * n0;
  blk.out_rows = rows;
  return run_apply(p, 0, a, b, nullptr, out0, f, sc[0], 0.0, nrhs, s, uni, out_fp32 != 0, &blk);
}

hofem_status hofem_axpy(double* y, double c, const double* x, long long count, void* stream) {
  if (count < 0 || (count > 0 && (!y || !x))) return fail(HOFEM_ERR_INVALID_ARG, "bad pointers or count");
  if (count == 0) return HOFEM_OK;
  HOFEM_CUDA(launch_axpy(y, c, x, count, (cudaStream_t)stream), "axpy launch");
  return HOFEM_OK;
}

hofem_status hofem_copy_block(const double* src, double* dst, long long batch, long long rows, long long cols,
                              long long src_ld, long long dst_ld, long long src_bs, long long dst_bs, void* stream) {
  if (batch < 0 || rows < 0 || cols < 0) return fail(HOFEM_ERR_INVALID_ARG, "negative block sizes");
  if (batch * rows * cols == 0) return HOFEM_OK;
  if (!src || !dst || src_ld < cols || dst_ld < cols || (batch > 1 && (src_bs < rows * src_ld || dst_bs < rows * dst_ld)))
    return fail(HOFEM_ERR_INVALID_ARG, "bad pointers or leading dimensions");
  HOFEM_CUDA(launch_copy_block(src, dst, batch, rows, cols, src_ld, dst_ld, src_bs, dst_bs, (cudaStream_t)stream),
             "copy_block launch");
  return HOFEM_OK;
}

hofem_status hofem_get_eigen(hofem_plan_t p, int axis, double* lam, double* mix, double* evec) {
  if (!p) return fail(HOFEM_ERR_INVALID_ARG, "plan is NULL");
  if (axis < 0 || axis >= p->N) return fail(HOFEM_ERR_INVALID_ARG, "axis out of range");
  const AxisTables& h = p->ax[axis].h;
  if (lam) memcpy(lam, h.lam.data(), h.lam.size() * sizeof(double));
  if (mix) memcpy(mix, h.mix.data(), h.mix.size() * sizeof(double));
  if (evec && h.n > 1) memcpy(evec, h.evec.data(), (size_t)(h.n - 1) * (h.n - 1) * sizeof(double));
  return HOFEM_OK;
}

hofem_status hofem_get_info(hofem_plan_t p, hofem_info* out) {
  if (!p || !out) return fail(HOFEM_ERR_INVALID_ARG, "plan or out is NULL");
  hofem_info inf = p->info;
  double worst = 0.0;
  if (p->h_norms)
    for (int r = 0; r < p->ws_nrhs; ++r) {
      const double nu = p->h_norms[2 * r + 1];
      if (nu > 0) worst = std::max(worst, std::sqrt(p->h_norms[2 * r] / nu));
    }
  inf.last_rel_update = worst;
  *out = inf;
  return HOFEM_OK;
}

hofem_status hofem_profile(hofem_plan_t p, int enable) {
  if (!p) return fail(HOFEM_ERR_INVALID_ARG, "plan is NULL");
  fold_profile(p);
  for (int i = 0; i < 16; ++i) {
    p->prof_ms[i] = 0.0;
    p->prof_n[i] = 0;
  }
  p->profiling = enable != 0;
  return HOFEM_OK;
}

hofem_status hofem_get_profile(hofem_plan_t p, hofem_kernel_time* out, int max_entries, int* count) {
  if (!p || !count || (max_entries > 0 && !out)) return fail(HOFEM_ERR_INVALID_ARG, "bad arguments");
  fold_profile(p);
  int c = 0;
  for (int k = 0; k < kNumKinds; ++k) {
    if (p->prof_n[k] == 0) continue;
    if (c < max_entries) {
      memset(out[c].name, 0, sizeof out[c].name);
      strncpy(out[c].name, kKindNames[k], sizeof out[c].name - 1);
      out[c].launches = p->prof_n[k];
      out[c].total_ms = p->prof_ms[k];
    }
    ++c;
  }
  *count = c;
  return HOFEM_OK;
}

void hofem_destroy(hofem_plan_t p) {
  if (!p) return;
  fold_profile(p);
  for (auto e : p->pool) cudaEventDestroy(e);
  p->pool.clear();
  free_workspace(p);
  cudaFree(p->ld[0]);
  cudaFree(p->ld[1]);
  cudaFree(p->heat);
  cudaFree(p->vcB);
  cudaFree(p->vcD);
  cudaFree(p->vcW);
  for (double* v : p->cg) cudaFree(v);
  cudaFree(p->dot);
  if (p->h_dot) cudaFreeHost(p->h_dot);
  for (int i = 0; i < p->N; ++i) free_axis(p->ax[i]);
  delete p;
}

}  // extern "C"

// Batched solves of independent problems (uneven K, n, X, nrhs): one plan per problem,
// all solves captured into one CUDA graph whose branches spread the problems over a pool
// of streams.  Independent problems then run concurrently inside one graph launch, and the
// graph's dependency edges do the phase ordering that a persistent kernel would need a
// device-wide barrier for.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <string>
#include <vector>

#include "common.cuh"
#include "sweep.cuh"

namespace hofem {
void set_last_error(const std::string& msg);
}

struct hofem_batch_s {
  std::vector<hofem_plan_t> plans;
  std::vector<hofem_problem> probs;
  int dtype = 0;
  cudaStream_t capture = nullptr;           // stream the graph is captured on
  std::vector<cudaStream_t> pool;           // branches
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> joins;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<const double*> gf;            // pointers the graph was captured with
  std::vector<double*> gu;
  hofem_batch_info info{};
};

namespace {

constexpr int kMaxBranches = 16;

hofem_status bfail(hofem_status st, const std::string& msg) {
  hofem::set_last_error(msg);
  return st;
}

hofem_status bcuda(cudaError_t e, const char* where) {
  if (e == cudaSuccess) return HOFEM_OK;
  hofem::set_last_error(std::string(where) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? HOFEM_ERR_OOM : HOFEM_ERR_CUDA;
}

void drop_graph(hofem_batch_s* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->gf.clear();
  b->gu.clear();
  b->info.graph_nodes = 0;
}

void free_batch(hofem_batch_s* b) {
  drop_graph(b);
  for (hofem_plan_t p : b->plans) hofem_destroy(p);
  for (cudaStream_t s : b->pool) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->joins) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->capture) cudaStreamDestroy(b->capture);
  delete b;
}

// Capture every problem's solve into b->graph (launched later on any stream).
hofem_status capture(hofem_batch_s* b, const double* const* f, double* const* u) {
  drop_graph(b);
  const int S = (int)b->pool.size();
  hofem_status st = bcuda(cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal), "begin capture");
  if (st != HOFEM_OK) return st;
  st = bcuda(cudaEventRecord(b->fork, b->capture), "record fork");
  for (int j = 0; j < S && st == HOFEM_OK; ++j) st = bcuda(cudaStreamWaitEvent(b->pool[j], b->fork, 0), "fork");
  for (size_t i = 0; i < b->plans.size() && st == HOFEM_OK; ++i) {
    st = hofem_solve(b->plans[i], f[i], u[i], b->probs[i].nrhs, b->pool[i % S]);
    if (st != HOFEM_OK) hofem::set_last_error("problem " + std::to_string(i) + ": " + hofem_last_error());
  }
  for (int j = 0; j < S && st == HOFEM_OK; ++j) {
    st = bcuda(cudaEventRecord(b->joins[j], b->pool[j]), "record join");
    if (st == HOFEM_OK) st = bcuda(cudaStreamWaitEvent(b->capture, b->joins[j], 0), "join");
  }
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->capture, &g);
  if (st == HOFEM_OK) st = bcuda(e, "end capture");
  if (st != HOFEM_OK) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return st;
  }
  b->graph = g;
  st = bcuda(cudaGraphInstantiate(&b->exec, b->graph, 0), "instantiate graph");
  if (st != HOFEM_OK) {
    drop_graph(b);
    return st;
  }
  size_t nodes = 0;
  cudaGraphGetNodes(b->graph, nullptr, &nodes);
  b->info.graph_nodes = (long long)nodes;
  b->info.captures += 1;
  b->gf.assign(f, f + b->plans.size());
  b->gu.assign(u, u + b->plans.size());
  return HOFEM_OK;
}

// Predicted work of one problem, in units of one unknown-RHS through one axis sweep: each
// solve sweeps every axis 2N - 1 times at a cost per value of ~log2 of its FFT length plus
// the order (the per-frequency mixing), and each correction adds the FP64 operator (about
// two folded element products of order n per axis); refined dtypes run the fixed capture
// count of corrections (2 when every K is a power of two, else 3; 8 for BF16 / FP16).
double problem_cost(const hofem_problem& q, int dtype) {
  double unknowns = q.nrhs, per_value = 0.0, residual = 0.0;
  bool pow2 = true;
  for (int i = 0; i < q.N; ++i) {
    const int K = q.K[i], M = q.n * K - 1;
    unknowns *= M;
    pow2 = pow2 && (K & (K - 1)) == 0;
    const int nb = hofem::bluestein_len(K);
    const double L = nb > 0 ? nb : K;
    per_value += std::log2(std::max(L, 2.0)) + q.n;
    residual += 2.0 * q.n;
  }
  const double sweeps = (2.0 * q.N - 1.0) / q.N * per_value;
  int corr = 0;
  if (dtype == HOFEM_FP32_REFINED) corr = pow2 ? 2 : 3;
  if (dtype == HOFEM_BF16_REFINED || dtype == HOFEM_FP16_REFINED) corr = 8;
  return unknowns * ((corr + 1) * sweeps + corr * residual);
}

}  // namespace

extern "C" {

hofem_status hofem_batch_partition(int count, const hofem_problem* probs, int dtype, int parts, int* part_of,
                                   double* cost) {
  if (count < 1 || !probs || !part_of || parts < 1)
    return bfail(HOFEM_ERR_INVALID_ARG, "count, parts must be >= 1 and probs, part_of non-NULL");
  std::vector<double> c(count);
  for (int i = 0; i < count; ++i) {
    if ((probs[i].N != 2 && probs[i].N != 3) || probs[i].nrhs < 1 || probs[i].n < 1)
      return bfail(HOFEM_ERR_INVALID_ARG, "problem " + std::to_string(i) + ": N must be 2 or 3, n and nrhs >= 1");
    for (int a = 0; a < probs[i].N; ++a)
      if (probs[i].K[a] < 2) return bfail(HOFEM_ERR_INVALID_ARG, "problem " + std::to_string(i) + ": K must be >= 2");
    c[i] = problem_cost(probs[i], dtype);
    if (cost) cost[i] = c[i];
  }
  // longest processing time first: problems by decreasing cost (ties by index), each to
  // the part with the least predicted work so far (ties to the lowest part)
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return c[a] > c[b]; });
  std::vector<double> load(parts, 0.0);
  for (int i : order) {
    const int j = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    part_of[i] = j;
    load[j] += c[i];
  }
  return HOFEM_OK;
}

hofem_status hofem_batch_plan(int count, const hofem_problem* probs, int dtype, hofem_batch_t* out) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!out) return bfail(HOFEM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (count < 1 || !probs) return bfail(HOFEM_ERR_INVALID_ARG, "count must be >= 1 and probs non-NULL");
  for (int i = 0; i < count; ++i)
    if ((probs[i].N != 2 && probs[i].N != 3) || probs[i].nrhs < 1)
      return bfail(HOFEM_ERR_INVALID_ARG, "problem " + std::to_string(i) + ": N must be 2 or 3 and nrhs >= 1");
  hofem_batch_s* b = new hofem_batch_s();
  b->dtype = dtype;
  b->probs.assign(probs, probs + count);
  hofem_status st = HOFEM_OK;
  for (int i = 0; i < count && st == HOFEM_OK; ++i) {
    const hofem_problem& q = probs[i];
    hofem_plan_t p = nullptr;
    st = hofem_plan(q.N, q.K, q.n, q.X, dtype, q.alpha, &p);
    if (st == HOFEM_OK) {
      b->plans.push_back(p);
      st = hofem_reserve(p, q.nrhs);
    }
    if (st != HOFEM_OK) hofem::set_last_error("problem " + std::to_string(i) + ": " + hofem_last_error());
  }
  const int S = std::min(count, kMaxBranches);
  if (st == HOFEM_OK) st = bcuda(cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking), "stream");
  if (st == HOFEM_OK) st = bcuda(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "event");
  for (int j = 0; j < S && st == HOFEM_OK; ++j) {
    cudaStream_t s = nullptr;
    cudaEvent_t e = nullptr;
    st = bcuda(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "stream");
    if (st == HOFEM_OK) b->pool.push_back(s);
    if (st == HOFEM_OK) st = bcuda(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
    if (st == HOFEM_OK) b->joins.push_back(e);
  }
  if (st != HOFEM_OK) {
    free_batch(b);
    return st;
  }
  hofem_batch_info& inf = b->info;
  inf.count = count;
  inf.streams = S;
  for (int i = 0; i < count; ++i) {
    hofem_info pi{};
    hofem_get_info(b->plans[i], &pi);
    long long u = probs[i].nrhs;
    for (int a = 0; a < pi.N; ++a) u *= pi.M[a];
    inf.unknowns += u;
    inf.table_bytes += pi.table_bytes;
    inf.workspace_bytes += pi.workspace_bytes;
  }
  inf.plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = b;
  return HOFEM_OK;
}

hofem_status hofem_batch_tune(hofem_batch_t b, void* stream) {
  if (!b) return bfail(HOFEM_ERR_INVALID_ARG, "batch is NULL");
  const auto t0 = std::chrono::steady_clock::now();
  for (size_t i = 0; i < b->plans.size(); ++i) {
    const hofem_status st = hofem_autotune(b->plans[i], b->probs[i].nrhs, stream);
    if (st != HOFEM_OK) return st;
  }
  drop_graph(b);   // the next solve captures the tuned launch shapes
  b->info.tune_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return HOFEM_OK;
}

hofem_status hofem_batch_solve(hofem_batch_t b, const double* const* f, double* const* u, void* stream) {
  if (!b) return bfail(HOFEM_ERR_INVALID_ARG, "batch is NULL");
  if (!f || !u) return bfail(HOFEM_ERR_INVALID_ARG, "f or u is NULL");
  const size_t cnt = b->plans.size();
  for (size_t i = 0; i < cnt; ++i)
    if (!f[i] || !u[i] || (const void*)f[i] == (const void*)u[i])
      return bfail(HOFEM_ERR_INVALID_ARG, "problem " + std::to_string(i) + ": f and u must be distinct and non-NULL");
  const bool same = b->exec && std::equal(f, f + cnt, b->gf.begin()) && std::equal(u, u + cnt, b->gu.begin());
  if (!same) {
    const hofem_status st = capture(b, f, u);
    if (st != HOFEM_OK) return st;
  }
  return bcuda(cudaGraphLaunch(b->exec, (cudaStream_t)stream), "graph launch");
}

hofem_status hofem_batch_get_info(hofem_batch_t b, hofem_batch_info* out) {
  if (!b || !out) return bfail(HOFEM_ERR_INVALID_ARG, "batch or out is NULL");
  *out = b->info;
  return HOFEM_OK;
}

hofem_status hofem_batch_get_plan(hofem_batch_t b, int i, hofem_plan_t* out) {
  if (!b || !out || i < 0 || i >= (int)b->plans.size()) return bfail(HOFEM_ERR_INVALID_ARG, "bad batch, index or out");
  *out = b->plans[i];
  return HOFEM_OK;
}

void hofem_batch_destroy(hofem_batch_t b) {
  if (b) free_batch(b);
}

}  // extern "C"

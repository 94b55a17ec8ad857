// Batched contexts (tc_init_batch / tc_apply_batch): many independent cells
// of uneven box size, k mesh and band count applied by one CUDA-graph launch.
//
// Each cell keeps its own setup and tables.  The workspace (real-space fields,
// per-side fields, scratch) is shared: the batch owns L "lanes" of workspace,
// each as large as the largest cell needs.  Cells are distributed over the
// lanes by estimated cost (longest first, to the least loaded lane); cells of
// one lane run one after the other on that lane's stream, lanes run
// concurrently.  The whole schedule -- occupation uploads and every kernel of
// every cell -- is captured once into a CUDA graph (fork/join over the lane
// streams) and replayed by each tc_apply_batch.  The number of lanes is chosen
// by measurement on the first call: the graph is built for L = 1, 2, 4, 8, 16
// (as memory allows), on a sample of at most 12 cells spread over the cost
// order, and the fastest replay is kept.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "tc_ctx.hpp"

namespace tc {

constexpr int kMaxLanes = 16;
constexpr int kTuneCandidates[] = {1, 2, 4, 8, 16};
constexpr int kNumTune = 5;
constexpr int kTuneCells = 12;   // cells timed per candidate lane count

struct BatchState {
  std::vector<tc_ctx*> cells;
  std::vector<WsLayout> layouts;
  std::vector<double> cost;          // estimated work per cell
  size_t lane_bytes = 0;
  int lanes_max = 1;
  int lanes = 0;                     // chosen lane count (0 until the first tc_apply_batch)
  char* d_ws = nullptr;
  cudaStream_t s0 = nullptr;
  cudaStream_t lane[kMaxLanes] = {};
  cudaEvent_t fork = nullptr, join[kMaxLanes] = {}, t0 = nullptr, t1 = nullptr;
  cudaEvent_t done = nullptr;        // recorded after each replay
  cudaGraphExec_t exec = nullptr;
  std::vector<const void*> key;      // device pointers the graph was captured with
  double tune_ms[kNumTune] = {-1, -1, -1, -1, -1};
};

void destroy_batch(tc_ctx* c) {
  BatchState* B = c->batch;
  if (!B) return;
  if (B->exec) cudaGraphExecDestroy(B->exec);
  for (tc_ctx* cell : B->cells) destroy_context(cell);
  for (int l = 0; l < kMaxLanes; ++l) {
    if (B->lane[l]) cudaStreamDestroy(B->lane[l]);
    if (B->join[l]) cudaEventDestroy(B->join[l]);
  }
  if (B->s0) cudaStreamDestroy(B->s0);
  if (B->fork) cudaEventDestroy(B->fork);
  if (B->t0) cudaEventDestroy(B->t0);
  if (B->t1) cudaEventDestroy(B->t1);
  if (B->done) cudaEventDestroy(B->done);
  if (B->d_ws) cudaFree(B->d_ws);
  delete B;
  c->batch = nullptr;
}

namespace {

// Cell indices in decreasing estimated cost.
std::vector<int> by_cost(const BatchState* B) {
  std::vector<int> order(B->cells.size());
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return B->cost[a] > B->cost[b]; });
  return order;
}

// Captures the cells `order` (decreasing cost) with L lanes into an executable graph.
tc_status capture(tc_ctx* c, int L, const std::vector<int>& order, const double2* const* phi,
                  const double2* const* chi, double2* const* oR, double2* const* oL, cudaGraphExec_t* exec) {
  BatchState* B = c->batch;
  // longest processing time first onto the least loaded lane
  std::vector<std::vector<int>> lanes(L);
  std::vector<double> load(L, 0.0);
  for (int i : order) {
    const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    lanes[l].push_back(i);
    load[l] += B->cost[i];
  }
  cudaError_t e = cudaStreamBeginCapture(B->s0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return fail(c, TC_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  int r = TC_OK;
  e = cudaEventRecord(B->fork, B->s0);
  for (int l = 0; l < L && e == cudaSuccess; ++l) e = cudaStreamWaitEvent(B->lane[l], B->fork, 0);
  for (int l = 0; l < L && e == cudaSuccess && r == TC_OK; ++l) {
    char* base = B->d_ws + (size_t)l * B->lane_bytes;
    for (int i : lanes[l]) {
      tc_ctx* cell = B->cells[i];
      ws_assign(cell, base, B->layouts[i]);
      const size_t nj = (size_t)cell->S.Nk * cell->S.nb;
      e = cudaMemcpyAsync(cell->d_occ, cell->h_occ, nj * sizeof(double), cudaMemcpyHostToDevice, B->lane[l]);
      if (e != cudaSuccess) break;
      r = apply_device(cell, phi[i], chi[i], oR[i], oL[i], B->lane[l]);
      if (r != TC_OK) {
        c->err = "cell " + std::to_string(i) + ": " + cell->err;
        break;
      }
    }
    if (e == cudaSuccess && r == TC_OK) e = cudaEventRecord(B->join[l], B->lane[l]);
    if (e == cudaSuccess && r == TC_OK) e = cudaStreamWaitEvent(B->s0, B->join[l], 0);
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(B->s0, &graph);
  if (e == cudaSuccess) e = e2;
  if (r != TC_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    if (r != TC_OK) return (tc_status)r;
    return fail(c, TC_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  }
  e = cudaGraphInstantiate(exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(c, TC_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  return TC_OK;
}

// Replay time (ms) of exec on s0, after one warm-up replay.
tc_status time_graph(tc_ctx* c, cudaGraphExec_t exec, double* ms) {
  BatchState* B = c->batch;
  cudaError_t e = cudaGraphLaunch(exec, B->s0);
  if (e == cudaSuccess) e = cudaEventRecord(B->t0, B->s0);
  if (e == cudaSuccess) e = cudaGraphLaunch(exec, B->s0);
  if (e == cudaSuccess) e = cudaEventRecord(B->t1, B->s0);
  if (e == cudaSuccess) e = cudaEventSynchronize(B->t1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, B->t0, B->t1);
  if (e != cudaSuccess) return fail(c, TC_ERR_CUDA, std::string("graph timing: ") + cudaGetErrorString(e));
  *ms = t;
  return TC_OK;
}

}  // namespace
}  // namespace tc

using tc::BatchState;

extern "C" {

tc_status tc_init_batch(int ncell, const tc_params* params, tc_ctx** out) {
  if (!params || !out || ncell < 1) return TC_ERR_ARG;
  *out = nullptr;
  for (int i = 1; i < ncell; ++i)
    if (params[i].precision != params[0].precision) {
      tc::set_thread_error("tc_init_batch: every cell must use the same precision");
      return TC_ERR_ARG;
    }
  tc_ctx* c = new (std::nothrow) tc_ctx();
  BatchState* B = new (std::nothrow) BatchState();
  if (!c || !B) {
    delete c;
    delete B;
    return TC_ERR_OOM;
  }
  c->batch = B;
  c->prec = params[0].precision;
  cudaGetDevice(&c->device);
  auto bail = [&](tc_status s, const std::string& msg) {
    tc::set_thread_error("tc_init_batch: " + msg);
    tc::destroy_context(c);
    return s;
  };
  for (int i = 0; i < ncell; ++i) {
    tc_ctx* cell = nullptr;
    std::string err;
    const int r = tc::init_context(&params[i], false, &cell, err);
    if (r != TC_OK) return bail((tc_status)r, "cell " + std::to_string(i) + ": " + err);
    cell->batch_owner = true;
    B->cells.push_back(cell);
    B->layouts.push_back(tc::ws_layout(cell));
    B->lane_bytes = std::max(B->lane_bytes, B->layouts.back().total);
    const tc::Setup& S = cell->S;
    const double pairs = 4.0 * (double)S.Nk * S.nb * (double)S.Nk * S.no;
    B->cost.push_back(pairs * (double)S.N * std::log2((double)S.N));
  }
  size_t free_b = 0, total_b = 0;
  cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
  if (e != cudaSuccess) return bail(TC_ERR_CUDA, cudaGetErrorString(e));
  const size_t budget = free_b / 4;   // at most a quarter of the free memory for the lanes
  B->lanes_max = (int)std::min<size_t>({(size_t)tc::kMaxLanes, (size_t)ncell, std::max<size_t>(1, budget / B->lane_bytes)});
  e = cudaMalloc((void**)&B->d_ws, (size_t)B->lanes_max * B->lane_bytes);
  if (e != cudaSuccess) return bail(e == cudaErrorMemoryAllocation ? TC_ERR_OOM : TC_ERR_CUDA, cudaGetErrorString(e));
  // zeroed once: every later read of the workspace follows a write of the same cell
  e = cudaMemset(B->d_ws, 0, (size_t)B->lanes_max * B->lane_bytes);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B->s0, cudaStreamNonBlocking);
  for (int l = 0; l < B->lanes_max && e == cudaSuccess; ++l) {
    e = cudaStreamCreateWithFlags(&B->lane[l], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->join[l], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreate(&B->t0);
  if (e == cudaSuccess) e = cudaEventCreate(&B->t1);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->done, cudaEventDisableTiming);
  if (e != cudaSuccess) return bail(TC_ERR_CUDA, cudaGetErrorString(e));
  for (int i = 0; i < ncell; ++i) tc::ws_assign(B->cells[i], B->d_ws, B->layouts[i]);
  *out = c;
  return TC_OK;
}

tc_status tc_batch_cell(tc_ctx* c, int i, tc_ctx** cell) {
  if (!c || !c->batch) return TC_ERR_STATE;
  if (!cell || i < 0 || i >= (int)c->batch->cells.size()) return TC_ERR_ARG;
  *cell = c->batch->cells[i];
  return TC_OK;
}

tc_status tc_apply_batch(tc_ctx* c, const void* const* phi_R, const void* const* phi_L, const double* const* occ,
                         void* const* out_R, void* const* out_L, void* stream) {
  if (!c || !c->batch) return TC_ERR_STATE;
  BatchState* B = c->batch;
  if (!phi_R || !phi_L || !occ || !out_R || !out_L) return tc::fail(c, TC_ERR_ARG, "null pointer array");
  if (const int f = tc::injected_fault("launch"))
    return tc::fail(c, (tc_status)f, "injected fault (TC_FAULT): no device work done");
  const int n = (int)B->cells.size();
  std::vector<const void*> key;
  key.reserve(4 * (size_t)n);
  for (int i = 0; i < n; ++i) {
    const void* p[4] = {phi_R[i], phi_L[i], out_R[i], out_L[i]};
    for (const void* q : p) {
      if (!q || !tc::device_ptr(q))
        return tc::fail(c, TC_ERR_ARG, "cell " + std::to_string(i) + ": orbital and output arrays must be device pointers");
      key.push_back(q);
    }
    if (!occ[i]) return tc::fail(c, TC_ERR_ARG, "null occupation array");
    tc_ctx* cell = B->cells[i];
    const size_t nj = (size_t)cell->S.Nk * cell->S.nb;
    for (size_t j = 0; j < nj; ++j)
      if (!(occ[i][j] >= 0.0 && occ[i][j] <= 1.0))
        return tc::fail(c, TC_ERR_ARG, "cell " + std::to_string(i) + ": occupations must lie in [0, 1]");
  }
  auto arr = [&](const void* const* a) { return reinterpret_cast<const double2* const*>(a); };
  auto arr_out = [&](void* const* a) { return reinterpret_cast<double2* const*>(a); };
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the previous replay may still read the pinned occupation buffers: wait for it
  cudaError_t e = cudaEventSynchronize(B->done);
  if (e != cudaSuccess) return tc::fail(c, TC_ERR_CUDA, std::string("tc_apply_batch: ") + cudaGetErrorString(e));
  for (int i = 0; i < n; ++i) {
    tc_ctx* cell = B->cells[i];
    std::memcpy(cell->h_occ, occ[i], (size_t)cell->S.Nk * cell->S.nb * sizeof(double));
  }
  if (!B->exec || key != B->key) {
    if (B->exec) {
      cudaGraphExecDestroy(B->exec);
      B->exec = nullptr;
    }
    const std::vector<int> order = tc::by_cost(B);
    if (B->lanes == 0) {
      // autotune the lane count on this call's inputs, over a sample of at most kTuneCells
      // cells spread evenly over the cost order (the whole batch if it is small)
      std::vector<int> sample;
      if (n <= tc::kTuneCells) {
        sample = order;
      } else {
        for (int i = 0; i < tc::kTuneCells; ++i) sample.push_back(order[(size_t)i * n / tc::kTuneCells]);
      }
      double best = 1e300;
      for (int t = 0; t < tc::kNumTune; ++t) {
        const int L = tc::kTuneCandidates[t];
        if (L > B->lanes_max || L > (int)sample.size()) continue;
        cudaGraphExec_t ex = nullptr;
        tc_status r = tc::capture(c, L, sample, arr(phi_R), arr(phi_L), arr_out(out_R), arr_out(out_L), &ex);
        if (r != TC_OK) return r;
        double ms = 0.0;
        r = tc::time_graph(c, ex, &ms);
        if (r != TC_OK) {
          cudaGraphExecDestroy(ex);
          return r;
        }
        B->tune_ms[t] = ms;
        if (ms < best) {
          best = ms;
          B->lanes = L;
        }
        cudaGraphExecDestroy(ex);
      }
    }
    tc_status r = tc::capture(c, B->lanes, order, arr(phi_R), arr(phi_L), arr_out(out_R), arr_out(out_L), &B->exec);
    if (r != TC_OK) return r;
    B->key = key;
  }
  e = cudaGraphLaunch(B->exec, st);
  if (e == cudaSuccess) e = cudaEventRecord(B->done, st);
  if (e != cudaSuccess) return tc::fail(c, TC_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
  return TC_OK;
}

tc_status tc_batch_info(const tc_ctx* c, int* ncell, int* lanes, int* lanes_max, double* tune_ms) {
  if (!c || !c->batch) return TC_ERR_STATE;
  const BatchState* B = c->batch;
  if (ncell) *ncell = (int)B->cells.size();
  if (lanes) *lanes = B->lanes;
  if (lanes_max) *lanes_max = B->lanes_max;
  if (tune_ms)
    for (int t = 0; t < tc::kNumTune; ++t) tune_ms[t] = B->tune_ms[t];
  return TC_OK;
}

}  // extern "C"

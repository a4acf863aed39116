// Batched randomized QLP: many independent problems of uneven m, n, k in one
// CUDA-graph launch, on one of two engines; and one factorization recorded
// into a graph for replays (rqlp_graph_*, at the end).
//
// Persistent engine (persist.cu): one kernel of one CTA per SM takes
// (problem, stage, tile) work items from an ordered device list; the graph
// holds a zeroing node and that kernel.
//
// Graph engine: rqlp_batched_create() records every problem's whole pipeline
// (the same kernels as rqlp()) into one graph, spread over `branches`
// parallel streams so that independent problems run side by side, and
// instantiates it once; rqlp_batched_launch() replays it with a single
// cudaGraphLaunch.  While recording, launch shapes are lowered so that one
// problem does not claim the whole GPU: the CPQR of B runs as one CTA (its
// exchanges never wait on another CTA), and the split-K targets of the FP64
// and tensor-core products come from the tuning record (picked by the
// autotuner).  Problems of one branch run one after another and share one
// workspace; each problem's status word is copied into a per-problem array.
#include <algorithm>
#include <cstring>
#include <vector>

#include "kernels.cuh"
#include "mixed.cuh"
#include "persist.cuh"

using namespace rqk;

struct rqlp_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int kernels = 0;  // library kernels one replay runs
};

struct rqlp_batch {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int count = 0;
  int branches = 0;
  int kernel_nodes = 0;
  int32_t *d_status = nullptr;
  int engine = RQLP_BATCH_GRAPH;
  PersistLaunch pl = {};
};

namespace {

size_t up256(size_t b) { return (b + 255) / 256 * 256; }

bool valid_problem(const rqlp_problem &p, const rqlp_opts *o) {
  if (!p.A || !p.Omega || !p.Q || !p.L || !p.P) return false;
  if (p.a_dtype != RQLP_F64 && p.a_dtype != RQLP_F32) return false;
  return rqlp_workspace_size(p.m, p.n, p.k, p.p, o) > 0 && p.lda >= p.n && p.ldo >= p.k + p.p;
}

// the engine a batch runs on: RQLP_BATCH_PERSISTENT, RQLP_BATCH_GRAPH, or
// 0 when the requested engine cannot run it
int engine_of(const rqlp_problem *probs, int32_t count, const rqlp_opts *opts,
              const rqlp_batch_tuning *t) {
  const int want = t ? t->engine : RQLP_BATCH_AUTO;
  if (want != RQLP_BATCH_AUTO && want != RQLP_BATCH_GRAPH && want != RQLP_BATCH_PERSISTENT)
    return 0;
  if (want != RQLP_BATCH_GRAPH && persist_ws_bytes(probs, count, opts) > 0)
    return RQLP_BATCH_PERSISTENT;
  return want == RQLP_BATCH_PERSISTENT ? 0 : RQLP_BATCH_GRAPH;
}

int branches_of(const rqlp_batch_tuning *t, int count) {
  int b = (t && t->branches > 0) ? t->branches : 64;
  if (b > count) b = count;
  if (b < 1) b = 1;
  return b;
}

// Persistent engine: plan the work items into the workspace, then capture
// the zeroing and the kernel into a graph of two nodes.
int create_persistent(const rqlp_problem *probs, int32_t count, const rqlp_opts *opts, void *ws,
                      size_t ws_bytes, rqlp_batch_t *out) {
  char *base = reinterpret_cast<char *>(ws);
  int32_t *d_status = reinterpret_cast<int32_t *>(base);
  const size_t head = up256((size_t)count * sizeof(int32_t));
  rqlp_batch *plan = new rqlp_batch;
  plan->count = count;
  plan->branches = 1;
  plan->d_status = d_status;
  plan->engine = RQLP_BATCH_PERSISTENT;
  int rc = persist_setup(probs, count, opts, base + head, ws_bytes - head, d_status, &plan->pl);
  cudaStream_t s0 = nullptr;
  if (rc == RQLP_OK && cudaStreamCreateWithFlags(&s0, cudaStreamNonBlocking) != cudaSuccess)
    rc = RQLP_ERR_CUDA;
  if (rc == RQLP_OK && cudaMemsetAsync(d_status, 0, sizeof(int32_t) * count, s0) != cudaSuccess)
    rc = RQLP_ERR_CUDA;
  if (rc == RQLP_OK && cudaStreamSynchronize(s0) != cudaSuccess) rc = RQLP_ERR_CUDA;
  cudaGraph_t graph = nullptr;
  if (rc == RQLP_OK) {
    if (cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      rc = RQLP_ERR_CUDA;
    } else {
      const int r = persist_enqueue(plan->pl, s0);
      const cudaError_t ec = cudaStreamEndCapture(s0, &graph);
      if (r != RQLP_OK) rc = r;
      else if (ec != cudaSuccess) rc = RQLP_ERR_CUDA;
    }
  }
  if (rc == RQLP_OK && cudaGraphInstantiate(&plan->exec, graph, 0) != cudaSuccess)
    rc = RQLP_ERR_CUDA;
  plan->graph = graph;
  plan->kernel_nodes = 1;
  if (s0) cudaStreamDestroy(s0);
  if (rc != RQLP_OK) {
    rqlp_batched_destroy(plan);
    return rc;
  }
  *out = plan;
  return RQLP_OK;
}

}  // namespace

extern "C" {

size_t rqlp_batched_workspace_size(const rqlp_problem *probs, int32_t count, const rqlp_opts *opts,
                                   const rqlp_batch_tuning *tune) {
  if (!probs || count <= 0 || !opts || opts->block_b != 0) return 0;
  size_t per = 0;
  for (int i = 0; i < count; ++i) {
    if (!valid_problem(probs[i], opts)) return 0;
    per = std::max(per, rqlp_workspace_size(probs[i].m, probs[i].n, probs[i].k, probs[i].p, opts));
  }
  const int eng = engine_of(probs, count, opts, tune);
  if (eng == 0) return 0;
  if (eng == RQLP_BATCH_PERSISTENT)
    return up256((size_t)count * sizeof(int32_t)) + persist_ws_bytes(probs, count, opts) + 256;
  const int b = branches_of(tune, count);
  return up256((size_t)count * sizeof(int32_t)) + (size_t)b * up256(per) + 256;
}

int rqlp_batched_create(const rqlp_problem *probs, int32_t count, const rqlp_opts *opts,
                        const rqlp_batch_tuning *tune, void *ws, size_t ws_bytes,
                        rqlp_batch_t *out) {
  if (!out) return RQLP_ERR_INVALID_ARG;
  *out = nullptr;
  const size_t need = rqlp_batched_workspace_size(probs, count, opts, tune);
  if (need == 0) return RQLP_ERR_INVALID_ARG;
  if (!ws || ws_bytes < need || reinterpret_cast<uintptr_t>(ws) % 256) return RQLP_ERR_WORKSPACE;
  if (engine_of(probs, count, opts, tune) == RQLP_BATCH_PERSISTENT)
    return create_persistent(probs, count, opts, ws, ws_bytes, out);
  size_t per = 0;
  for (int i = 0; i < count; ++i)
    per = std::max(per, rqlp_workspace_size(probs[i].m, probs[i].n, probs[i].k, probs[i].p, opts));
  per = up256(per);
  const int nb = branches_of(tune, count);
  char *base = reinterpret_cast<char *>(ws);
  int32_t *d_status = reinterpret_cast<int32_t *>(base);
  char *wsb = base + up256((size_t)count * sizeof(int32_t));

  rqlp_batch *plan = new rqlp_batch;
  plan->count = count;
  plan->branches = nb;
  plan->d_status = d_status;

  std::vector<cudaStream_t> streams(nb);
  std::vector<cudaEvent_t> joins(nb);
  cudaStream_t s0 = nullptr;
  cudaEvent_t fork = nullptr;
  int rc = RQLP_OK;
  auto cleanup = [&]() {
    for (auto s : streams) if (s) cudaStreamDestroy(s);
    for (auto e : joins) if (e) cudaEventDestroy(e);
    if (fork) cudaEventDestroy(fork);
    if (s0) cudaStreamDestroy(s0);
  };
  for (auto &s : streams) s = nullptr;
  for (auto &e : joins) e = nullptr;
  if (cudaStreamCreateWithFlags(&s0, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess) {
    cleanup();
    delete plan;
    return RQLP_ERR_CUDA;
  }
  for (int b = 0; b < nb; ++b) {
    if (cudaStreamCreateWithFlags(&streams[b], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&joins[b], cudaEventDisableTiming) != cudaSuccess) {
      cleanup();
      delete plan;
      return RQLP_ERR_CUDA;
    }
  }

  // set-up that must not happen inside a capture
  if (chol_init() != cudaSuccess || (opts->prec != RQLP_PREC_FP64 && mixed_init() != RQLP_OK) ||
      ozaki_init() != RQLP_OK) {
    cleanup();
    delete plan;
    return RQLP_ERR_CUDA;
  }
  const Tuning saved = tuning();
  tuning().cpqr_max_ctas = 1;
  tuning().gemm_target_ctas = (tune && tune->gemm_target_ctas > 0) ? tune->gemm_target_ctas
                                                                    : num_sms() / 2;
  tuning().mma_max_splits = (tune && tune->mma_max_splits > 0) ? tune->mma_max_splits : 2;
  // small problems side by side: the FP64 units' kernels share SMs, a digit
  // product's CTAs each hold a whole SM
  tuning().no_digit_products = 1;

  if (cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = RQLP_ERR_CUDA;
  if (rc == RQLP_OK && cudaEventRecord(fork, s0) != cudaSuccess) rc = RQLP_ERR_CUDA;
  for (int b = 0; rc == RQLP_OK && b < nb; ++b)
    if (cudaStreamWaitEvent(streams[b], fork, 0) != cudaSuccess) rc = RQLP_ERR_CUDA;
  // longest-processing-time-first assignment of problems to branches, by an
  // estimate of each problem's work (products with A, then the QR and CPQR
  // terms that run on few SMs)
  std::vector<int> order(count), branch_of(count);
  std::vector<double> cost(count), load(nb, 0.0);
  for (int i = 0; i < count; ++i) {
    const double l = probs[i].k + probs[i].p;
    cost[i] = (2.0 * opts->q + 2.0) * probs[i].m * probs[i].n * l / 64.0 +
              (probs[i].m + probs[i].n) * l * l + 4.0 * probs[i].n * l * l;
    order[i] = i;
  }
  std::sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  for (int i : order) {
    int best = 0;
    for (int b = 1; b < nb; ++b)
      if (load[b] < load[best]) best = b;
    branch_of[i] = best;
    load[best] += cost[i];
  }
  for (int ii = 0; rc == RQLP_OK && ii < count; ++ii) {
    const int i = order[ii];
    const int b = branch_of[i];
    const rqlp_problem &p = probs[i];
    void *wsi = wsb + (size_t)b * per;
    int r = rqlp(p.A, p.a_dtype, p.m, p.n, p.lda, p.k, p.p, p.Omega, p.ldo, opts, p.Q, p.L, p.P,
                 p.Lvalues, p.piv0, p.piv1, wsi, per, reinterpret_cast<rqlp_stream_t>(streams[b]));
    if (r != RQLP_OK) {
      rc = r;
      break;
    }
    // the status word sits at the head of the problem's workspace
    if (cudaMemcpyAsync(d_status + i, wsi, sizeof(int32_t), cudaMemcpyDeviceToDevice,
                        streams[b]) != cudaSuccess)
      rc = RQLP_ERR_CUDA;
  }
  for (int b = 0; b < nb; ++b) {
    cudaEventRecord(joins[b], streams[b]);
    cudaStreamWaitEvent(s0, joins[b], 0);
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(s0, &graph);
  tuning() = saved;
  if (rc == RQLP_OK && ec != cudaSuccess) rc = RQLP_ERR_CUDA;
  if (rc == RQLP_OK && cudaGraphInstantiate(&plan->exec, graph, 0) != cudaSuccess) rc = RQLP_ERR_CUDA;
  if (rc == RQLP_OK) {
    size_t n = 0;
    cudaGraphGetNodes(graph, nullptr, &n);
    std::vector<cudaGraphNode_t> nodes(n);
    cudaGraphGetNodes(graph, nodes.data(), &n);
    int kn = 0;
    for (auto nd : nodes) {
      cudaGraphNodeType t;
      if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kn;
    }
    plan->kernel_nodes = kn;
  }
  plan->graph = graph;
  cleanup();
  if (rc != RQLP_OK) {
    rqlp_batched_destroy(plan);
    return rc;
  }
  *out = plan;
  return RQLP_OK;
}

int rqlp_batched_launch(rqlp_batch_t plan, rqlp_stream_t stream) {
  if (!plan || !plan->exec) return RQLP_ERR_INVALID_ARG;
  return cudaGraphLaunch(plan->exec, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
             ? RQLP_OK
             : RQLP_ERR_CUDA;
}

int rqlp_batched_status(rqlp_batch_t plan, rqlp_stream_t stream, int32_t *statuses) {
  if (!plan) return RQLP_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess)
    return RQLP_ERR_CUDA;
  std::vector<int32_t> h(plan->count);
  if (cudaMemcpy(h.data(), plan->d_status, sizeof(int32_t) * plan->count,
                 cudaMemcpyDeviceToHost) != cudaSuccess)
    return RQLP_ERR_CUDA;
  int worst = RQLP_OK;
  for (int i = 0; i < plan->count; ++i) {
    if (statuses) statuses[i] = h[i];
    if (h[i] < 0 && worst >= 0) worst = h[i];
    else if (h[i] > 0 && worst == RQLP_OK) worst = h[i];
  }
  return worst;
}

int rqlp_batched_kernel_nodes(rqlp_batch_t plan) { return plan ? plan->kernel_nodes : 0; }

int rqlp_batched_engine(rqlp_batch_t plan, int64_t *items) {
  if (!plan) return 0;
  if (items) *items = plan->engine == RQLP_BATCH_PERSISTENT ? plan->pl.items : 0;
  return plan->engine;
}

int rqlp_batched_stage_times(rqlp_batch_t plan, rqlp_stream_t stream, double *busy_us,
                             double *wait_us, int64_t *items) {
  if (!plan || plan->engine != RQLP_BATCH_PERSISTENT) return RQLP_ERR_INVALID_ARG;
  return persist_stats(plan->pl, reinterpret_cast<cudaStream_t>(stream), busy_us, wait_us, items);
}

void rqlp_batched_destroy(rqlp_batch_t plan) {
  if (!plan) return;
  persist_release(&plan->pl);
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  if (plan->graph) cudaGraphDestroy(plan->graph);
  delete plan;
}

// ---- one factorization recorded once, replayed with one launch -------------
// rqlp() enqueues ~110 kernels; a replay of its recording costs one graph
// launch and no host work per kernel.  The recording is made on a private
// stream after one ordinary call on the caller's stream (which checks the
// arguments and does every one-time set-up, none of which may happen inside a
// capture); the private stream's side stream is created before the capture,
// so that the explicit Q0 becomes a branch beside the QR of R0^T.
int rqlp_graph_create(const void *A, int32_t a_dtype, int64_t m, int64_t n, int64_t lda,
                      int32_t k, int32_t p, const double *Omega, int64_t ldo,
                      const rqlp_opts *opts, double *Q, double *L, double *P, double *Lvalues,
                      int32_t *piv0, int32_t *piv1, void *ws, size_t ws_bytes,
                      rqlp_stream_t stream, rqlp_graph_t *out) {
  if (!out) return RQLP_ERR_INVALID_ARG;
  *out = nullptr;
  int rc = rqlp(A, a_dtype, m, n, lda, k, p, Omega, ldo, opts, Q, L, P, Lvalues, piv0, piv1, ws,
                ws_bytes, stream);
  if (rc != RQLP_OK) return rc;
  if (cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess)
    return RQLP_ERR_CUDA;
  cudaStream_t rec = nullptr;
  if (cudaStreamCreateWithFlags(&rec, cudaStreamNonBlocking) != cudaSuccess) return RQLP_ERR_CUDA;
  rqlp_graph *g = new rqlp_graph;
  side_stream_prepare(rec);
  const long long n0 = launch_count();
  if (cudaStreamBeginCapture(rec, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    rc = RQLP_ERR_CUDA;
  } else {
    side_stream_in_capture(true);
    rc = rqlp(A, a_dtype, m, n, lda, k, p, Omega, ldo, opts, Q, L, P, Lvalues, piv0, piv1, ws,
              ws_bytes, reinterpret_cast<rqlp_stream_t>(rec));
    side_stream_in_capture(false);
    const cudaError_t ec = cudaStreamEndCapture(rec, &g->graph);
    if (rc == RQLP_OK && ec != cudaSuccess) rc = RQLP_ERR_CUDA;
  }
  // the launches counted while recording ran nothing; each replay adds them
  g->kernels = (int)(launch_count() - n0);
  count_launch(-g->kernels);
  if (rc == RQLP_OK && cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess) rc = RQLP_ERR_CUDA;
  cudaStreamDestroy(rec);
  if (rc != RQLP_OK) {
    cudaGetLastError();
    rqlp_graph_destroy(g);
    return rc;
  }
  *out = g;
  return RQLP_OK;
}

int rqlp_graph_launch(rqlp_graph_t graph, rqlp_stream_t stream) {
  if (!graph || !graph->exec) return RQLP_ERR_INVALID_ARG;
  if (cudaGraphLaunch(graph->exec, reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess)
    return RQLP_ERR_CUDA;
  count_launch(graph->kernels);
  return RQLP_OK;
}

int rqlp_graph_kernels(rqlp_graph_t graph) { return graph ? graph->kernels : 0; }

void rqlp_graph_destroy(rqlp_graph_t graph) {
  if (!graph) return;
  if (graph->exec) cudaGraphExecDestroy(graph->exec);
  if (graph->graph) cudaGraphDestroy(graph->graph);
  delete graph;
}

}  // extern "C"

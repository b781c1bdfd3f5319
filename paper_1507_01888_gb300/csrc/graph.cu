// graph.cu -- an apply recorded once as a CUDA graph and replayed with one launch.
//
// mra_apply_graph_create runs the apply (plain or batched) once to learn its sizes -- the
// record count P after the screen and the destination count -- and then records the same
// sequence of kernels and library sorts in fixed-size mode on a private stream: no host
// synchronisation, the learned sizes as launch shapes, and device-side checks that the counts a
// replay computes are the recorded ones.  A replay reads the input tree's buffers and writes
// the output tree's buffers at the addresses given at creation; coefficients may change between
// replays, and mra_apply_graph_status reports (and clears) any replay whose sizes differed.
#include <new>

#include "apply_internal.cuh"

namespace mra {
namespace {

struct ApplyGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
  int *d_status = nullptr;
  int64_t *d_in_offsets = nullptr;
  float *d_partial = nullptr;
  FixedSizes fx;
  int64_t n_out = 0;
  long long kernels = 0;
};

void destroy(ApplyGraph *g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->d_status) cudaFree(g->d_status);
  if (g->d_in_offsets) cudaFree(g->d_in_offsets);
  if (g->d_partial) cudaFree(g->d_partial);
  if (g->cap) cudaStreamDestroy(g->cap);
  delete g;
}

}  // namespace
}  // namespace mra

using namespace mra;

extern "C" {

int mra_apply_graph_create(const mra_operator *h, int nfunc, const mra_tree_view *in, const int64_t *in_offsets,
                           const mra_apply_opts *o, mra_tree_view *out, int64_t *out_offsets, void *workspace,
                           size_t workspace_bytes, mra_apply_graph **handle, void *stream) {
  if (!handle) return fail(MRA_ERR_ARG, "mra_apply_graph_create: NULL handle");
  *handle = nullptr;
  if (!h || !in || !o || !out) return fail(MRA_ERR_ARG, "mra_apply_graph_create: NULL argument");
  if (nfunc < 1) return fail(MRA_ERR_ARG, "mra_apply_graph_create: nfunc=%d", nfunc);
  if (in->n == 0) return fail(MRA_ERR_ARG, "mra_apply_graph_create: empty input");
  // the sizing run, through the public entry points (their argument checks included)
  mra_apply_stats st{};
  int rc = nfunc > 1 ? mra_apply_batched(h, nfunc, in, in_offsets, o, out, out_offsets, workspace, workspace_bytes,
                                         &st, stream)
                     : mra_apply(h, in, o, out, workspace, workspace_bytes, &st, stream);
  if (rc != MRA_OK) return rc;
  if (nfunc == 1 && out_offsets) {
    out_offsets[0] = 0;
    out_offsets[1] = out->n;
  }
  ApplyGraph *g = new (std::nothrow) ApplyGraph();
  if (!g) return fail(MRA_ERR_ARG, "mra_apply_graph_create: out of host memory");
  auto bail = [&](int code, const char *what, cudaError_t e) {
    destroy(g);
    return fail(code, "mra_apply_graph_create: %s: %s", what, cudaGetErrorString(e));
  };
  cudaError_t e = cudaMalloc((void **)&g->d_status, sizeof(int));
  if (e != cudaSuccess) return bail(MRA_ERR_CUDA, "status word", e);
  e = cudaMemset(g->d_status, 0, sizeof(int));
  if (e != cudaSuccess) return bail(MRA_ERR_CUDA, "status word", e);
  if (nfunc > 1) {
    e = cudaMalloc((void **)&g->d_in_offsets, (nfunc + 1) * sizeof(int64_t));
    if (e == cudaSuccess)
      e = cudaMemcpy(g->d_in_offsets, in_offsets, (nfunc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bail(MRA_ERR_CUDA, "input offsets", e);
  }
  g->fx.P = st.pairs;
  g->fx.nd = out->n;
  g->fx.status = g->d_status;
  g->fx.d_in_offsets = g->d_in_offsets;
  g->n_out = out->n;
  const Operator *op = reinterpret_cast<const Operator *>(h);
  if (apply_uses_src_path(*op, *o) && st.pairs > 0) {  // the recorded apply's partial sums, owned by the graph
    e = cudaMalloc((void **)&g->d_partial, (size_t)st.pairs * op->k * op->k * op->k * sizeof(float));
    if (e != cudaSuccess) return bail(MRA_ERR_CUDA, "partial-sum buffer", e);
    g->fx.partial = g->d_partial;
  }
  e = cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) return bail(MRA_ERR_CUDA, "capture stream", e);
  const long long k0 = launch_total();
  e = cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return bail(MRA_ERR_CUDA, "begin capture", e);
  mra_tree_view o_view = *out;
  rc = apply_run(*op, *in, *o, o_view, workspace, workspace_bytes, nullptr, g->cap, nfunc,
                 nfunc > 1 ? in_offsets : nullptr, nullptr, &g->fx);
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(g->cap, &graph);
  g->graph = graph;
  if (rc != MRA_OK) {
    destroy(g);
    return rc;
  }
  if (e != cudaSuccess) return bail(MRA_ERR_CUDA, "end capture", e);
  g->kernels = launch_total() - k0;
  e = cudaGraphInstantiate(&g->exec, g->graph, 0);
  if (e != cudaSuccess) return bail(MRA_ERR_CUDA, "instantiate", e);
  *handle = reinterpret_cast<mra_apply_graph *>(g);
  return MRA_OK;
}

int mra_apply_graph_launch(mra_apply_graph *handle, void *stream) {
  ApplyGraph *g = reinterpret_cast<ApplyGraph *>(handle);
  if (!g || !g->exec) return fail(MRA_ERR_ARG, "mra_apply_graph_launch: NULL graph");
  MRA_CUDA_TRY(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
  for (long long i = 0; i < g->kernels; ++i) note_launch();
  return MRA_OK;
}

int mra_apply_graph_status(mra_apply_graph *handle, void *stream) {
  ApplyGraph *g = reinterpret_cast<ApplyGraph *>(handle);
  if (!g) return fail(MRA_ERR_ARG, "mra_apply_graph_status: NULL graph");
  cudaStream_t s = (cudaStream_t)stream;
  int st = 0;
  MRA_CUDA_TRY(cudaMemcpyAsync(&st, g->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  MRA_CUDA_TRY(cudaMemsetAsync(g->d_status, 0, sizeof(int), s));
  MRA_CUDA_TRY(cudaStreamSynchronize(s));
  if (st & 8) return fail(MRA_ERR_TIMEOUT, "mra_apply_graph: a tensor-core completion wait gave up");
  if (st & (1 | 2))
    return fail(MRA_ERR_CAPACITY, "mra_apply_graph: a replay needed other sizes than the recorded ones "
                "(record count %s, destination count %s); create the graph again",
                (st & 1) ? "changed" : "same", (st & 2) ? "changed" : "same");
  if (st & 4) return fail(MRA_ERR_ARG, "mra_apply_graph: an input box lies on a level the operator does not cover");
  if (st) return fail(MRA_ERR_ARG, "mra_apply_graph: inconsistent work list (status %d)", st);
  return MRA_OK;
}

int mra_apply_graph_info(const mra_apply_graph *handle, int64_t *n_out, long long *kernels_per_launch) {
  const ApplyGraph *g = reinterpret_cast<const ApplyGraph *>(handle);
  if (!g) return fail(MRA_ERR_ARG, "mra_apply_graph_info: NULL graph");
  if (n_out) *n_out = g->n_out;
  if (kernels_per_launch) *kernels_per_launch = g->kernels;
  return MRA_OK;
}

int mra_apply_graph_free(mra_apply_graph *handle) {
  destroy(reinterpret_cast<ApplyGraph *>(handle));
  return MRA_OK;
}

}  // extern "C"

// apply_internal.cuh -- declarations shared by the apply translation units.
#pragma once

#include "mra_internal.cuh"

namespace mra {

// Fixed-size mode, used when an apply is recorded into a CUDA graph: no host synchronisation;
// the record count P and destination count nd of an earlier run of the same input are used as
// the sizes, and kernels compare the counts the device computes with them, OR-ing into *status:
// 1 = record count differs, 2 = destination count differs, 4 = a box on a level the operator
// does not cover, 8 = a tensor-core wait gave up, 16 = inconsistent split work list.
struct FixedSizes {
  int64_t P = 0, nd = 0;
  int *status = nullptr;                  // device word
  const int64_t *d_in_offsets = nullptr;  // device copy of the batched input offsets (nfunc + 1)
  float *partial = nullptr;               // the source-stationary kernel's partial sums (P k^3 floats)
};

// The sorted work list handed from the screen/sort stage to an apply kernel.
// Destination d gathers records perm[seg[d]] .. perm[seg[d+1]-1]; record p names
// a source box rec_src[p], a displacement rec_l[p] (three biased bytes) and the
// kept Gaussian terms rec_mask[2p], rec_mask[2p+1] (bit m = term m).
struct ApplyWork {
  int64_t n_dest, P;
  const int64_t *seg;
  const int *perm;
  const int *did;             // 1-based destination index of each dest-sorted record
  const uint64_t *skey;       // dest-sorted destination keys (one per record)
  const int *rec_src;
  const int *rec_l;
  const uint64_t *rec_mask;
  const uint64_t *dest_key;
  const int64_t *rec_cnt;     // records of each source box (source order) and their offsets
  const int64_t *rec_off;
  const int64_t *box_kept;    // kept terms of each source box
  void *split_ws;             // scratch for the tensor-core path's grouping
  size_t split_ws_bytes;
  cudaEvent_t ev0, ev1;       // recorded around the apply kernel when non-null
  cudaEvent_t evk0, evk1;     // around the main kernel alone, where the apply runs more kernels
  const FixedSizes *fx;       // fixed-size (graph) mode when non-null
};

size_t apply_workspace_bytes(const Operator &op, const mra_apply_opts &o, int64_t n_in);
int apply_run(const Operator &op, const mra_tree_view &in, const mra_apply_opts &o,
              mra_tree_view &out, void *ws, size_t ws_bytes, mra_apply_stats *stats,
              cudaStream_t s, int nfunc = 1, const int64_t *in_offsets = nullptr, int64_t *out_offsets = nullptr,
              const FixedSizes *fx = nullptr);
int apply_split_run(const Operator &op, const mra_tree_view &in, const mra_apply_opts &o,
                    mra_tree_view &out, const ApplyWork &wk, mra_apply_stats *stats,
                    cudaStream_t s);
size_t split_workspace_bytes(int64_t P);
// source-stationary tensor-core apply (apply_src.cu): orders and displacement ranges it covers,
// its scratch, and the run (dap: the records' |l|_inf range per absolute level)
bool src_path_supported(int k, int max_rec_disp);
size_t src_workspace_bytes(int64_t n_in);
// *passes (when not null, and not in graph mode): the kernel's passes, each one set of stage-1,
// 2 and 3 MMAs
int apply_src_run(const Operator &op, const mra_tree_view &in, const mra_apply_opts &o, mra_tree_view &out,
                  const ApplyWork &wk, const int *dap, float *partial, cudaStream_t s, int64_t *passes = nullptr);
// whether an apply with these options runs the source-stationary kernel (its partial sums need
// P k^3 floats besides the workspace)
bool apply_uses_src_path(const Operator &op, const mra_apply_opts &o);
// test hook of the failure path (one-shot), and the fixed-size mode's status from a kernel error word
bool take_injected_stall();
void split_fixed_err(const int *err, int *status, cudaStream_t s);
// BF16 pieces of the operator's blocks and of c_m times them (allocated once; rebuild = true
// recomputes them, after the blocks or the coefficients changed)
int split_blocks_build(Operator &op, cudaStream_t s, bool rebuild = false);
int log_terms_run(const Operator &op, const mra_tree_view &in, const mra_apply_opts &o, int64_t max_terms,
                  uint64_t seed, float *features, float *log_norms, int64_t *n_logged, void *ws,
                  size_t ws_bytes, cudaStream_t s);
int norm_run(const mra_tree_view &t, double *per_box, double *total, cudaStream_t s);
int debug_selftest_run(cudaStream_t s);
int compare_run(const mra_tree_view &t, const mra_tree_view &r, mra_compare_result *res,
                cudaStream_t s);

}  // namespace mra

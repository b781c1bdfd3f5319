// apply_split.cu -- split-precision tensor-core apply (tcgen05).  Placeholder
// until the kernel lands: reports the precision as unsupported.
#include "apply_internal.cuh"

namespace mra {

int apply_split_run(const Operator &, const mra_tree_view &, const mra_apply_opts &,
                    mra_tree_view &, const ApplyWork &, mra_apply_stats *, cudaStream_t) {
  return fail(MRA_ERR_UNSUPPORTED, "mra_apply: MRA_PREC_SPLIT_BF16 is not built yet");
}

}  // namespace mra

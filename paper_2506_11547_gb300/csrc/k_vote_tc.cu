// k_vote_tc.cu -- tensor-core (tcgen05) vote.  Not built yet in this revision.
#include "rv_internal.h"

namespace rv {

cudaError_t launch_vote_tc(const VoteItem *, int, const ProbRef *, const LevelRef *, int, int, PairPool, ProbStats *,
                           int, float, int, int *, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace rv

// The vote kernel instantiated at 2 blocks of 256 threads per SM.
#include "trk_vote_kernel.cuh"

namespace trk {
TRK_VOTE_LEVEL_DISPATCH(2)
}  // namespace trk

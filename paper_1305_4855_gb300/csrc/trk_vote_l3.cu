// The vote kernel instantiated at 3 blocks of 256 threads per SM.
#include "trk_vote_kernel.cuh"

namespace trk {
TRK_VOTE_LEVEL_DISPATCH(3)
}  // namespace trk

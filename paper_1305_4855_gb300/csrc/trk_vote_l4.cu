// The vote kernel instantiated at 4 blocks of 256 threads per SM.
#include "trk_vote_kernel.cuh"

namespace trk {
TRK_VOTE_LEVEL_DISPATCH(4)
}  // namespace trk

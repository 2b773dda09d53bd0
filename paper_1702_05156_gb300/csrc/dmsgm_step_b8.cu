// dmsgm_step_b8.cu -- the per-tile frame-step kernel for 8x8 blocks
// (one translation unit per block size, so the builds run in parallel).
#include "dmsgm_step.cuh"

namespace dmsgm {
template cudaError_t launch_step_block<8>(dmsgm_ctx*, const CUtensorMap&, const StreamArgs&,
                                           const Coef&, cudaStream_t, bool);
}  // namespace dmsgm

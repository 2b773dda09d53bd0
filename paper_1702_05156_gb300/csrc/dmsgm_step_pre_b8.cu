// dmsgm_step_pre_b8.cu -- the frame step with fused preprocessing for 8x8
// blocks (its own translation unit, so the builds run in parallel).
#include "dmsgm_step_pre.cuh"

namespace dmsgm {
template cudaError_t launch_step_pre_block<8>(const dmsgm_ctx*, const uint8_t*, const StreamArgs&,
                                               const Coef&, cudaStream_t, bool);
}  // namespace dmsgm

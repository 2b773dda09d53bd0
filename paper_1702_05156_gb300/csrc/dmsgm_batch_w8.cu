// dmsgm_batch_w8.cu -- the batched step's launches for work items of 8
// warps (dmsgm_batch_opts.item_warps = 8), in a translation unit of their own
// so that they compile in parallel with the 4-warp ones.
#include "dmsgm_batch.cuh"

namespace dmsgm {

template <int CAP>
static cudaError_t launch_cap_w8(bool spread, const void* p, int ctas, cudaStream_t s, bool pdl,
                                 int max_block) {
    const BatchParams<CAP>& bp = *static_cast<const BatchParams<CAP>*>(p);
    return spread ? launch_t<CAP, true, 8>(bp, ctas, s, pdl, max_block)
                  : launch_t<CAP, false, 8>(bp, ctas, s, pdl, max_block);
}

cudaError_t batch_launch_w8(int cap, bool spread, const void* p, int ctas, cudaStream_t s,
                            bool pdl, int max_block) {
    switch (cap) {
        case 16: return launch_cap_w8<16>(spread, p, ctas, s, pdl, max_block);
        case 64: return launch_cap_w8<64>(spread, p, ctas, s, pdl, max_block);
        case DMSGM_MAX_BATCH: return launch_cap_w8<DMSGM_MAX_BATCH>(spread, p, ctas, s, pdl, max_block);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace dmsgm

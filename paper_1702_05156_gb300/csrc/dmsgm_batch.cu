// dmsgm_batch.cu -- many streams per launch.
#include "dmsgm_internal.h"

namespace dmsgm {

int launch_batch(int n, const dmsgm_t* hs, const uint8_t* const* frames_dev, const double* Hs,
                 uint32_t* const* masks_dev, cudaStream_t stream) {
    for (int i = 0; i < n; ++i) {
        int rc = dmsgm_process(hs[i], frames_dev[i], Hs + 9 * size_t(i), masks_dev[i], stream);
        if (rc) return rc;
    }
    return DMSGM_OK;
}

}  // namespace dmsgm

// dmsgm_batch.cu -- many streams, one launch per frame step.
//
// Every stream of the batch contributes its frame's 256 x (4 B) tiles (or
// 256 x (8 B) with dmsgm_batch_opts.item_warps = 8) to one (stream, tile) work
// list, grouped by kind (block size, state precision).  The kernels live in
// dmsgm_batch.cuh; the 8-warp launches are instantiated in dmsgm_batch_w8.cu.
// Two kernels run the fused DMSGM step (Sec. 2.2-2.4) over the list:
//  - dmsgm_batch_single_kernel, one work item per CTA (the default: every
//    item gets a CTA at once).  As in the per-frame kernel, the item's
//    pixels, block statistics and back-projections are done before the wait
//    on the previous step; only gathers, update and mask wait for it.
//  - dmsgm_batch_kernel, a persistent grid (when the caller asks for fewer
//    CTAs than items) that walks the list with a static stride and
//    double-buffers its tiles in shared memory.
// A batch of up to 64 streams carries one 2-D tensor map per stream's frame
// in the kernel parameters, so a tile arrives in one TMA copy; a larger
// batch stages a tile by 1-D bulk copies, one per pixel row.  Streams may
// differ in size, block size (4 / 8) and state precision (FP32 / FP16).
//
// The per-stream descriptors travel in the kernel's parameter space, so a
// launch needs no device scratch and no host->device copy, and a stream
// capture bakes each step's descriptors into its graph node.
#include <algorithm>

#include "dmsgm_batch.cuh"

namespace dmsgm {

template <int CAP>
static int run_cap(int n, const dmsgm_t* hs, const uint8_t* const* frames, const double* Hs,
                   uint32_t* const* masks, const dmsgm_batch_opts& o, cudaStream_t s) {
    if (o.reserved != 0) return fail(DMSGM_ERR_INVALID_ARG, "dmsgm_batch_opts.reserved must be 0");
    if (o.item_warps != 0 && o.item_warps != 4 && o.item_warps != 8)
        return fail(DMSGM_ERR_INVALID_ARG, "dmsgm_batch_opts.item_warps must be 0, 4 or 8");
    const int nwb = o.item_warps ? o.item_warps : 4;
    static thread_local BatchParams<CAP> p;   // ~CAP*120 bytes: keep it off the stack
    // the work list holds the streams grouped by kind (block, precision), so
    // that the CTAs resident on an SM mostly run the same code
    int order[DMSGM_MAX_BATCH];
    int m = 0;
    for (int kind = 0; kind < 4; ++kind)
        for (int i = 0; i < n; ++i)
            if (((hs[i]->B == 8 ? 2 : 0) | (hs[i]->prec == DMSGM_STATE_FP16 ? 1 : 0)) == kind)
                order[m++] = i;
    for (int i = 0; i < n; ++i)   // blocks other than 4 and 8 are refused below
        if (hs[i]->B != 4 && hs[i]->B != 8) order[m++] = i;
    int total = 0, max_block = 4;
    bool spread = false;
    for (int q = 0; q < n; ++q) {
        const int i = order[q];
        const dmsgm_ctx* h = hs[i];
        if (h->W > 65535 || h->H > 65535)
            return fail(DMSGM_ERR_INVALID_ARG, "batched streams must be at most 65535 px wide/high");
        if (!((h->B == 4 || h->B == 8) && h->H % h->B == 0))
            return fail(DMSGM_ERR_UNSUPPORTED,
                        "batched streams take blocks 4 and 8 on whole block rows (stream %d)", i);
        if (h->pre_gauss || h->pre_median)
            return fail(DMSGM_ERR_UNSUPPORTED, "batched streams take no preprocessing (stream %d)", i);
        if (h->checked)
            return fail(DMSGM_ERR_UNSUPPORTED, "batched streams take no checked handles (stream %d)", i);
        BatchItem& it = p.item[q];
        max_block = std::max(max_block, h->B);
        if constexpr (CAP <= kMapCap) {
            const int rc = batch_frame_map(const_cast<dmsgm_ctx*>(h), frames[i], nwb * h->B,
                                           &p.map[q]);
            if (rc) return rc;
        }
        it.frame = frames[i];
        it.mask = masks[i];
        it.mem = static_cast<char*>(h->mem);
        int affine = 0;
        if (!make_coef(Hs + 9 * size_t(i), h->B, &it.coef, &affine))
            return fail(DMSGM_ERR_INVALID_ARG, "homography %d is not finite in FP32", i);
        it.affine = uint8_t(affine);
        it.W = uint16_t(h->W);
        it.H = uint16_t(h->H);
        it.B = uint8_t(h->B);
        it.prec = uint8_t(h->prec);
        it.first = h->initialized ? 0 : 1;
        it.parity = uint8_t(h->parity);
        it.theta_s = h->theta_s;
        it.theta_d = h->theta_d;
        it.age_max = uint8_t(h->age_max);
        it.spread = uint8_t(h->mix_spread);
        spread = spread || h->mix_spread;
        it.unused = 0;
        it.tile_begin = total;
        const int th = nwb * h->B;
        total += ((h->W + kTileW - 1) / kTileW) * ((h->H + th - 1) / th);
    }
    p.n = n;
    p.total = total;
    // 0: one work item per CTA (the single-item kernel); otherwise as asked,
    // a persistent grid when fewer than the items (CTAs never wait on one
    // another, so more CTAs than fit at once is fine)
    int ctas = o.ctas > 0 ? o.ctas : total;
    ctas = std::max(1, std::min(ctas, total));
    const bool pdl = o.use_pdl > 0;
    cudaError_t e;
    if (nwb == 8)
        e = batch_launch_w8(CAP, spread, &p, ctas, s, pdl, max_block);
    else
        e = spread ? launch_t<CAP, true, 4>(p, ctas, s, pdl, max_block)
                   : launch_t<CAP, false, 4>(p, ctas, s, pdl, max_block);
    if (e != cudaSuccess)
        return fail(DMSGM_ERR_CUDA, "batch kernel launch failed: %s", cudaGetErrorString(e));
    for (int i = 0; i < n; ++i) advance(hs[i]);
    return DMSGM_OK;
}

int launch_batch(int n, const dmsgm_t* hs, const uint8_t* const* frames_dev, const double* Hs,
                 uint32_t* const* masks_dev, const dmsgm_batch_opts& o, cudaStream_t stream) {
    if (n <= 16) return run_cap<16>(n, hs, frames_dev, Hs, masks_dev, o, stream);
    if (n <= 64) return run_cap<64>(n, hs, frames_dev, Hs, masks_dev, o, stream);
    return run_cap<DMSGM_MAX_BATCH>(n, hs, frames_dev, Hs, masks_dev, o, stream);
}

}  // namespace dmsgm

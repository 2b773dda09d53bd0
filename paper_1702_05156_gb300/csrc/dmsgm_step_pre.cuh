// dmsgm_step_pre.cuh -- the per-tile frame step with the Sec. 2.1
// preprocessing fused in: a CTA stages its tile's source box with the
// filter's halo, blurs and medians it in shared memory (dmsgm_filter.cuh),
// then runs the step of dmsgm_step.cuh on the filtered tile.  The filter
// depends on the frame alone, so it runs before the wait on the previous
// frame's kernel, overlapping its end.  Instantiated for 4x4 blocks with
// 8 warps and 8x8 blocks with 4 warps (32-row tiles both), Gaussian sizes
// up to 7, in dmsgm_step_pre_b<B>.cu.
#pragma once

#include "dmsgm_filter.cuh"
#include "dmsgm_internal.h"

namespace dmsgm {

template <int B, typename T, int NW, int HALF>
__global__ void __launch_bounds__(NW * 32)
    dmsgm_step_pre_kernel(const uint8_t* __restrict__ frame, const StreamArgs a, const Coef k,
                          const FiltArgs f) {
    constexpr int RPT = 1, STRIPS = NW, TILE_H = NW * B, NT = NW * 32;
    static_assert(TILE_H * kTileW <= filt_src_bytes<HALF, TILE_H>(), "tile fits the source box");
    __shared__ __align__(16) uint8_t src[filt_src_bytes<HALF, TILE_H>()];   // then the filtered tile
    __shared__ __align__(16) uint32_t rp[filt_rp_words<TILE_H>()];
    __shared__ Origin orig[2 * STRIPS];
    const int tx0 = blockIdx.x * kTileW;
    const int ty0 = blockIdx.y * TILE_H;
    // The next frame's CTAs may start now: everything before their wait
    // reads only their own frame, and the wait itself still holds until this
    // grid has completed.  Their filtering, the longest part of the kernel,
    // then overlaps this frame's (measured: 1920x1080 at 5.0 us per frame
    // instead of 7.9 with the trigger after the wait).
    pdl_launch_dependents();
    fill_origins<B>(a, k, tx0, ty0, STRIPS, orig);
    filt_stage<HALF, TILE_H, NT>(frame, a.W, a.H, tx0, ty0, src);
    __syncthreads();
    filt_blur<HALF, TILE_H, NT>(f, src, rp);
    __syncthreads();
    uint8_t* tile = src;
    filt_write<TILE_H, NT>(f, rp, tx0, ty0, a.W, a.H, tile, kTileW, TILE_H, kTileW);
    __syncthreads();
    constexpr int BPL = kLaneBlocks<B>;
    const bool xin = tx0 + kLanePx * int(threadIdx.x & 31) < a.W;
    Stats st[RPT][BPL];
    Proj pj[RPT][BPL];
    tile_stats<B, NW, RPT>(a, tile, ty0, xin, st);
    tile_project<B, NW, RPT>(a, k, tx0, ty0, orig, pj);
    pdl_wait();
    float muA[RPT][BPL], thr[RPT][BPL];
    tile_update<B, T, NW, RPT, false, false>(a, tx0, ty0, pj, st, muA, thr);
    tile_mask<B, NW, RPT>(a, tile, tx0, ty0, st, muA, thr);
}

template <int B, typename T, int NW, int HALF>
static cudaError_t launch_step_pre_t(const uint8_t* frame, const StreamArgs& a, const Coef& k,
                                     const FiltArgs& f, cudaStream_t s, bool pdl) {
    constexpr int TILE_H = NW * B;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((a.W + kTileW - 1) / kTileW, (a.H + TILE_H - 1) / TILE_H, 1);
    cfg.blockDim = dim3(NW * 32, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, dmsgm_step_pre_kernel<B, T, NW, HALF>, frame, a, k, f);
}

// 4x4 blocks: 8 warps; 8x8 blocks: 4 warps (both 32-row tiles).
template <int B>
cudaError_t launch_step_pre_block(const dmsgm_ctx* h, const uint8_t* frame, const StreamArgs& a,
                                  const Coef& k, cudaStream_t s, bool pdl) {
    constexpr int NW = 32 / B;
    const bool f16 = h->prec == DMSGM_STATE_FP16;
    const FiltArgs& f = h->filt;
#define DMSGM_PRE(HH)                                                                   \
    case HH:                                                                            \
        return f16 ? launch_step_pre_t<B, __half, NW, HH>(frame, a, k, f, s, pdl)       \
                   : launch_step_pre_t<B, float, NW, HH>(frame, a, k, f, s, pdl);
    switch (h->pre_half) {
        DMSGM_PRE(0) DMSGM_PRE(1) DMSGM_PRE(2) DMSGM_PRE(3)
        default: return cudaErrorInvalidValue;
    }
#undef DMSGM_PRE
}

}  // namespace dmsgm

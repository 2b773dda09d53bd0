// dmsgm_step.cuh -- the per-tile frame-step kernel and its launch, as a
// template over the block size.  Each block size is instantiated in its own
// translation unit (dmsgm_step_b<B>.cu) so that they compile in parallel.
#pragma once

#include <mutex>

#include "dmsgm_internal.h"

namespace dmsgm {

constexpr uint64_t kWaitTimeoutNs = 2000000000ull;   // 2 s: only a broken copy gets here

// 8x8 blocks, one strip row per warp: 32 registers (full occupancy); two
// rows per warp: 64.  4x4 blocks keep the compiler's choice.
// CTAs per SM the kernel is compiled for.  Block 1 (4 warps, one strip row
// each): 6, i.e. at most 80 registers instead of 96; at 3840x2160 that took
// a frame from 113 to 107 us (7 and 8 spill, 131 and 135 us).
template <int B, int NW, int RPT>
constexpr int step_min_blocks() {
    return B == 8 ? (RPT == 1 ? 64 : 32) / NW : (B == 1 && NW == 4 && RPT == 1 ? 6 : 1);
}

template <int B, typename T, int NW, int RPT, bool SPREAD>
__global__ void __launch_bounds__(NW * 32, (step_min_blocks<B, NW, RPT>()))
    dmsgm_step_kernel(const __grid_constant__ CUtensorMap tmap, const StreamArgs a, const Coef k,
                      int* status) {
    constexpr int STRIPS = NW * RPT;          // strip rows per tile
    constexpr int TILE_H = STRIPS * B;
    __shared__ __align__(128) uint8_t tile[TILE_H * kTileW];
    __shared__ __align__(8) uint64_t bar;
    __shared__ Origin orig[2 * STRIPS];
    const int tx0 = blockIdx.x * kTileW;
    const int ty0 = blockIdx.y * TILE_H;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        mbar_arrive_expect_tx(&bar, TILE_H * kTileW);
        tma_load_2d(tile, &tmap, tx0, ty0, &bar);
    }
    fill_origins<B>(a, k, tx0, ty0, STRIPS, orig);
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0, kWaitTimeoutNs);
    if (__syncthreads_or(!ok)) {
        // report, give the copy one more bounded chance to land, and leave
        if (threadIdx.x == 0) atomicOr(status, kStatusWaitTimeout);
        mbar_wait_bounded(&bar, 0, kWaitTimeoutNs);
        return;
    }
    // The pixels, their block statistics and the back-projections do not
    // depend on the previous frame's kernel, so they run before its end;
    // the state does.
    constexpr int BPL = kLaneBlocks<B>;
    const bool xin = tx0 + kLanePx * int(threadIdx.x & 31) < a.W;
    Stats st[RPT][BPL];
    Proj pj[RPT][BPL];
    tile_stats<B, NW, RPT>(a, tile, ty0, xin, st);
    tile_project<B, NW, RPT>(a, k, tx0, ty0, orig, pj);
    pdl_wait();
    // Triggered here, not at entry: an earlier trigger lets the CTAs of
    // several later frames start, and their pixel loads and statistics then
    // compete with this frame's update, the recurrence's critical path.
    pdl_launch_dependents();
    float muA[RPT][BPL], thr[RPT][BPL];
    tile_update<B, T, NW, RPT, false, SPREAD>(a, tx0, ty0, pj, st, muA, thr);
    tile_mask<B, NW, RPT>(a, tile, tx0, ty0, st, muA, thr);
}

// The checked build of the same step (dmsgm_opts.checked): every state load
// and store and every mask byte checks its index; an index out of range is
// skipped and sets kStatusBounds in the status word.  No mixture option.
template <int B, typename T, int NW, int RPT>
__global__ void __launch_bounds__(NW * 32)
    dmsgm_step_checked_kernel(const __grid_constant__ CUtensorMap tmap, const StreamArgs a,
                              const Coef k, int* status) {
    constexpr int STRIPS = NW * RPT;
    constexpr int TILE_H = STRIPS * B;
    __shared__ __align__(128) uint8_t tile[TILE_H * kTileW];
    __shared__ __align__(8) uint64_t bar;
    __shared__ Origin orig[2 * STRIPS];
    const int tx0 = blockIdx.x * kTileW;
    const int ty0 = blockIdx.y * TILE_H;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        mbar_arrive_expect_tx(&bar, TILE_H * kTileW);
        tma_load_2d(tile, &tmap, tx0, ty0, &bar);
    }
    fill_origins<B>(a, k, tx0, ty0, STRIPS, orig);
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0, kWaitTimeoutNs);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) atomicOr(status, kStatusWaitTimeout);
        mbar_wait_bounded(&bar, 0, kWaitTimeoutNs);
        return;
    }
    constexpr int BPL = kLaneBlocks<B>;
    const bool xin = tx0 + kLanePx * int(threadIdx.x & 31) < a.W;
    Stats st[RPT][BPL];
    Proj pj[RPT][BPL];
    tile_stats<B, NW, RPT>(a, tile, ty0, xin, st);
    tile_project<B, NW, RPT>(a, k, tx0, ty0, orig, pj);
    pdl_wait();
    pdl_launch_dependents();
    float muA[RPT][BPL], thr[RPT][BPL];
    const CheckedSrc<T, false> src{global_src<T, false>(a), a.Gx * a.Gy, status, a.Gx};
    auto gather_fn = [&](const Proj& p) { return gather<false>(a, p, src); };
    tile_update_with<B, T, NW, RPT, decltype(gather_fn), true>(a, tx0, ty0, pj, st, muA, thr,
                                                               gather_fn, status);
    tile_mask<B, NW, RPT, true>(a, tile, tx0, ty0, st, muA, thr, status);
}

}  // namespace dmsgm

#include "dmsgm_step_narrow.cuh"

namespace dmsgm {

template <int B, typename T, int NW, int RPT>
static cudaError_t launch_step_t(const CUtensorMap& tmap, const StreamArgs& a, const Coef& k,
                                 int* status, cudaStream_t s, bool pdl, bool checked) {
    // the mixture-variance option and the checked build have their own kernels
    auto kern = checked ? dmsgm_step_checked_kernel<B, T, NW, RPT>
                        : (a.spread ? dmsgm_step_kernel<B, T, NW, RPT, true>
                                    : dmsgm_step_kernel<B, T, NW, RPT, false>);
    constexpr int TILE_H = NW * RPT * B;
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
    return cudaLaunchKernelEx(&cfg, kern, tmap, a, k, status);
}

// How many CTAs of one per-tile kernel shape the GPU holds at once.
template <int B, typename T, int NW, int RPT>
static int step_capacity(int device) {
    static std::mutex mu;
    static int cache[64] = {0};
    std::lock_guard<std::mutex> g(mu);
    if (device < 0 || device >= 64) return 0;
    if (!cache[device]) {
        int per_sm = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dmsgm_step_kernel<B, T, NW, RPT, false>,
                                                          NW * 32, 0) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        cache[device] = per_sm * sms;
    }
    return cache[device];
}

// Strip rows per warp for tile_rows = 8 B: 8 warps x 1 row when the frame's
// CTAs fit the GPU at once; otherwise 4 warps x 2 rows, which holds the
// frame in fewer resident warps (a single wave at 3840 x 2160) instead of
// leaving a partial second wave.
template <int B, typename T>
static int step_rpt_q8(const dmsgm_ctx* h) {
    const int ctas = ((h->W + kTileW - 1) / kTileW) * ((h->H + 8 * B - 1) / (8 * B));
    const int cap = step_capacity<B, T, 8, 1>(h->device);
    return (cap > 0 && ctas > cap) ? 2 : 1;
}

// tile_rows = NW * B * RPT with (NW, RPT) in {(4, 1), (8, 1) or (4, 2), (8, 2)};
// block 4 with 32-row tiles takes the one-block-per-lane kernel
// (dmsgm_step_narrow.cuh) for frames of at most one tile per SM.
template <int B>
cudaError_t launch_step_block(dmsgm_ctx* h, const CUtensorMap& tmap, const StreamArgs& a,
                              const Coef& k, cudaStream_t s, bool pdl) {
    const int q = h->tile_rows / B;   // 4, 8 or 16
    const bool f16 = h->prec == DMSGM_STATE_FP16;
    if constexpr (B == 4) {
        if (q == 8 && !h->checked) {
            if (h->step_narrow == 0) {
                // measured: 320 x 240 2.41 instead of 2.64 us per frame;
                // 1920 x 1080 (272 tiles) 3.60 instead of 3.45 us, so only
                // frames of at most one tile per SM take it
                const int ctas = ((h->W + kTileW - 1) / kTileW) * ((h->H + kNarrowRows - 1) / kNarrowRows);
                int sms = 0;
                if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess)
                    sms = 0;
                const int cap = f16 ? narrow_capacity<__half>(h->device) : narrow_capacity<float>(h->device);
                h->step_narrow = (cap > 0 && ctas <= cap && ctas <= sms) ? 1 : -1;
            }
            if (h->step_narrow > 0)
                return f16 ? launch_narrow_t<__half>(tmap, a, k, h->status_dev, s, pdl)
                           : launch_narrow_t<float>(tmap, a, k, h->status_dev, s, pdl);
        }
    }
    if (q == 8 && h->step_rpt == 0)
        h->step_rpt = f16 ? step_rpt_q8<B, __half>(h) : step_rpt_q8<B, float>(h);
    const int rpt = q == 8 ? h->step_rpt : (q == 16 ? 2 : 1);
    int* st = h->status_dev;
    const bool ck = h->checked != 0;
#define DMSGM_CASE(TT, QQ, NWW, RR) \
    if (q == QQ && rpt == RR) return launch_step_t<B, TT, NWW, RR>(tmap, a, k, st, s, pdl, ck);
    if (!f16) {
        DMSGM_CASE(float, 4, 4, 1) DMSGM_CASE(float, 8, 8, 1) DMSGM_CASE(float, 8, 4, 2)
        DMSGM_CASE(float, 16, 8, 2)
    } else {
        DMSGM_CASE(__half, 4, 4, 1) DMSGM_CASE(__half, 8, 8, 1) DMSGM_CASE(__half, 8, 4, 2)
        DMSGM_CASE(__half, 16, 8, 2)
    }
#undef DMSGM_CASE
    return cudaErrorInvalidValue;
}

}  // namespace dmsgm

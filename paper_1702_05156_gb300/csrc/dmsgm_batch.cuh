// dmsgm_batch.cuh -- the batched step's kernels and launch templates (see
// dmsgm_batch.cu for the work list and the host side).  The launches for
// work items of 4 warps are instantiated in dmsgm_batch.cu, those for 8
// warps in dmsgm_batch_w8.cu, so that the two compile in parallel.
#pragma once

#include <algorithm>

#include "dmsgm_internal.h"

namespace dmsgm {

struct BatchItem {
    const uint8_t* frame;
    uint32_t* mask;
    char* mem;           // the handle's device memory (control block + buffers)
    Coef coef;
    uint16_t W, H;
    uint8_t B, prec, first, parity, affine, age_max, spread, unused;
    float theta_s, theta_d;
    int tile_begin;      // first work-list index of this stream
};
static_assert(sizeof(BatchItem) == 120, "BatchItem layout");

// Batches of up to kMapCap streams also carry one 2-D tensor map per
// stream's frame (box kTileW x the item's rows), so a tile arrives in one TMA copy;
// larger batches stage their tiles by 1-D bulk copies, one per pixel row.
constexpr int kMapCap = 64;

template <int CAP, bool MAPS = (CAP <= kMapCap)>
struct BatchParams {
    int n;
    int total;           // work-list length
    BatchItem item[CAP];
};
template <int CAP>
struct BatchParams<CAP, true> {
    CUtensorMap map[CAP];
    int n;
    int total;
    BatchItem item[CAP];
};
static_assert(sizeof(BatchParams<DMSGM_MAX_BATCH>) <= 32764, "kernel parameter limit");
static_assert(sizeof(BatchParams<kMapCap>) <= 32764, "kernel parameter limit");

// Work items are tiles of kTileW x (NWB * B) pixels, NWB = 4 or 8 warps per
// item (dmsgm_batch_opts.item_warps), one strip row of blocks per warp.  The
// persistent kernel's stage buffers are sized for B = 8.

// Stream whose work items contain t (the last with tile_begin <= t).
template <int CAP>
__device__ __forceinline__ int find_stream(const BatchParams<CAP>& p, int t) {
    int lo = 0, hi = p.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.item[mid].tile_begin <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Tile origin of work item t of stream `si`.
template <int NWB>
__device__ __forceinline__ void item_origin(const BatchItem& it, int t, int& tx0, int& ty0) {
    const int tiles_x = (it.W + kTileW - 1) / kTileW;
    const int lt = t - it.tile_begin;
    tx0 = (lt % tiles_x) * kTileW;
    ty0 = (lt / tiles_x) * (NWB * it.B);
}

// Stage setup (one warp): start the bulk copies of the item's pixel rows and
// compute its affine origins.
template <int CAP, int NWB>
__device__ __forceinline__ void stage_item(const BatchParams<CAP>& p, int t, int* meta,
                                           Origin* orig, uint8_t* tile, uint64_t* bar) {
    const int lane = threadIdx.x & 31;
    const int si = find_stream(p, t);
    const BatchItem& it = p.item[si];
    const int W = it.W, H = it.H, B = it.B;
    int tx0, ty0;
    item_origin<NWB>(it, t, tx0, ty0);
    if constexpr (CAP <= kMapCap) {
        // one 2-D copy of the whole box (rows and columns past the frame
        // arrive as zeros and count as transferred bytes)
        if (lane == 0) {
            meta[0] = si;
            mbar_arrive_expect_tx(bar, kTileW * NWB * B);
            tma_load_2d(tile, &p.map[si], tx0, ty0, bar);
        }
    } else {
        const int rows = min(NWB * B, H - ty0);
        const uint32_t wbytes = static_cast<uint32_t>(min(kTileW, W - tx0));
        if (lane == 0) {
            meta[0] = si;
            mbar_arrive_expect_tx(bar, wbytes * rows);
        }
        __syncwarp();
        for (int r = lane; r < rows; r += 32)
            bulk_load_1d(tile + r * kTileW, it.frame + size_t(ty0 + r) * W + tx0, wbytes, bar);
    }
    if (it.affine && !it.first && lane < 2 * NWB)   // the tile's affine origins
        orig[lane] = affine_origin(it.coef, (tx0 + 128 * (lane & 1)) / B, ty0 / B + (lane >> 1));
}

// The per-frame arguments of a stream, built in registers from the kernel's
// parameters (uniform constant-bank loads).
__device__ __forceinline__ StreamArgs item_args(const BatchItem& it) {
    StreamArgs a;
    const int B = it.B;
    const int s = it.prec == DMSGM_STATE_FP16 ? 2 : 4;
    a.prev = state_buf(it.mem, it.W, it.H, B, s, it.parity);
    a.next = state_buf(it.mem, it.W, it.H, B, s, it.parity ^ 1);
    a.mask = it.mask;
    a.W = it.W;
    a.H = it.H;
    a.Gx = it.W / B;
    a.Gy = grid_rows(it.H, B);
    a.mask_words = (it.W + 31) / 32;
    a.first = it.first;
    a.affine = it.affine;
    a.age_max = it.age_max;
    a.theta_s = it.theta_s;
    a.theta_d = it.theta_d;
    a.spread = it.spread;
    return a;
}

template <int B, typename T, bool SPREAD, int NWB>
__device__ __forceinline__ bool run_item(const BatchItem& it, int t, const Origin* orig,
                                         const uint8_t* tile, uint64_t* bar, uint32_t parity) {
    constexpr int BPL = kLaneBlocks<B>;
    const StreamArgs a = item_args(it);
    int tx0, ty0;
    item_origin<NWB>(it, t, tx0, ty0);
    Proj pj[1][BPL];
    tile_project<B, NWB, 1>(a, it.coef, tx0, ty0, orig, pj);
    const bool ok = mbar_wait_bounded(bar, parity, 2000000000ull);
    if (__syncthreads_or(!ok)) return false;
    const bool xin = tx0 + kLanePx * int(threadIdx.x & 31) < a.W;
    Stats st[1][BPL];
    tile_stats<B, NWB, 1>(a, tile, ty0, xin, st);
    float muA[1][BPL], thr[1][BPL];
    tile_update<B, T, NWB, 1, false, SPREAD>(a, tx0, ty0, pj, st, muA, thr);
    tile_mask<B, NWB, 1>(a, tile, tx0, ty0, st, muA, thr);
    return true;
}

// One work item per CTA: as the per-frame kernel, the item's pixels, block
// statistics and projections run before the previous step's kernel ends;
// only the gathers, update and mask wait for it.
template <int B, typename T, bool SPREAD, int NWB>
__device__ __forceinline__ bool run_single(const BatchItem& it, const StreamArgs& a, int tx0,
                                           int ty0, const Origin* orig, const uint8_t* tile,
                                           uint64_t* bar) {
    constexpr int BPL = kLaneBlocks<B>;
    Proj pj[1][BPL];
    tile_project<B, NWB, 1>(a, it.coef, tx0, ty0, orig, pj);
    const bool ok = mbar_wait_bounded(bar, 0, 2000000000ull);
    if (__syncthreads_or(!ok)) return false;
    const bool xin = tx0 + kLanePx * int(threadIdx.x & 31) < a.W;
    Stats st[1][BPL];
    tile_stats<B, NWB, 1>(a, tile, ty0, xin, st);
    pdl_wait();
    float muA[1][BPL], thr[1][BPL];
    tile_update<B, T, NWB, 1, false, SPREAD>(a, tx0, ty0, pj, st, muA, thr);
    tile_mask<B, NWB, 1>(a, tile, tx0, ty0, st, muA, thr);
    return true;
}

// One work item per CTA, in a kernel of its own: one pixel stage in dynamic
// shared memory sized for the batch's largest block (4 KB when every stream
// has 4x4 blocks, 8 KB with 8x8 ones), and no persistent loop, so more CTAs
// fit an SM.  Compiled for 16 CTAs per SM (32 registers, a small spill):
// measured on 64 mixed streams, 36.0 us per step with two lanes against 38.1
// at 10 CTAs per SM (48 registers) and 36.6 at 12 (40 registers); the warps
// of the other CTAs cover the first warp's per-item setup.  Items of 8 warps
// take 8 CTAs per SM, the same 32 registers.
template <int CAP, bool SPREAD, int NWB>
__global__ void __launch_bounds__(NWB * 32, 64 / NWB)
    dmsgm_batch_single_kernel(const __grid_constant__ BatchParams<CAP> p) {
    extern __shared__ __align__(128) uint8_t stage[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int meta[2];
    __shared__ Origin orig[2 * NWB];
    __shared__ StreamArgs sa;   // the item's arguments, built once per CTA
    __shared__ int sxy[2];      // the item's tile origin
    const int t = blockIdx.x;
    // The next step's CTAs may launch once every CTA of this one has started:
    // a step has far more items than the GPU holds, so they only take the
    // slots that this step's finished CTAs free, and their pixel loads and
    // statistics overlap this step's tail (measured 64 mixed streams: 39.0
    // instead of 40.0 us per step).  The per-frame kernel triggers after its
    // wait instead; there the next frame's CTAs would compete with the frame's
    // own critical path.
    pdl_launch_dependents();
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        stage_item<CAP, NWB>(p, t, meta, orig, stage, &bar);
        if (threadIdx.x == 0) {
            const BatchItem& i0 = p.item[meta[0]];
            sa = item_args(i0);
            item_origin<NWB>(i0, t, sxy[0], sxy[1]);
        }
    }
    __syncthreads();           // the item's stream, arguments and origins are visible
    const BatchItem& it = p.item[meta[0]];
    const StreamArgs a = sa;
    const int tx0 = sxy[0], ty0 = sxy[1];
    const int kind = (it.B == 8 ? 2 : 0) | (it.prec == DMSGM_STATE_FP16 ? 1 : 0);
    bool ok;
    switch (kind) {
        case 0: ok = run_single<4, float, SPREAD, NWB>(it, a, tx0, ty0, orig, stage, &bar); break;
        case 1: ok = run_single<4, __half, SPREAD, NWB>(it, a, tx0, ty0, orig, stage, &bar); break;
        case 2: ok = run_single<8, float, SPREAD, NWB>(it, a, tx0, ty0, orig, stage, &bar); break;
        default: ok = run_single<8, __half, SPREAD, NWB>(it, a, tx0, ty0, orig, stage, &bar); break;
    }
    if (!ok && threadIdx.x == 0) atomicOr(reinterpret_cast<int*>(it.mem), kStatusWaitTimeout);
}

// SPREAD: built to honour the streams' mixture-variance option (each item
// still follows its own flag); without it the option's code is compiled out.
template <int CAP, bool SPREAD, int NWB>
__global__ void __launch_bounds__(NWB * 32, 32 / NWB)
    dmsgm_batch_kernel(const __grid_constant__ BatchParams<CAP> p) {
    __shared__ __align__(128) uint8_t tile[2][NWB * 8 * kTileW];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int meta[2][2];
    __shared__ Origin orig[2][2 * NWB];
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    int t = blockIdx.x;
    // the first tile's pixels do not depend on the previous step
    if (t < p.total && threadIdx.x < 32) stage_item<CAP, NWB>(p, t, meta[0], orig[0], tile[0], &bar[0]);
    pdl_wait();
    pdl_launch_dependents();
    for (int k = 0; t < p.total; t += gridDim.x, ++k) {
        const int st = k & 1;
        __syncthreads();   // stage st staged; stage st^1 free
        const int tn = t + gridDim.x;
        if (tn < p.total && threadIdx.x < 32)
            stage_item<CAP, NWB>(p, tn, meta[st ^ 1], orig[st ^ 1], tile[st ^ 1], &bar[st ^ 1]);
        const int si = meta[st][0];
        const BatchItem& it = p.item[si];
        const uint32_t par = (k >> 1) & 1;
        const int kind = (it.B == 8 ? 2 : 0) | (it.prec == DMSGM_STATE_FP16 ? 1 : 0);
        bool ok;
        switch (kind) {
            case 0: ok = run_item<4, float, SPREAD, NWB>(it, t, orig[st], tile[st], &bar[st], par); break;
            case 1: ok = run_item<4, __half, SPREAD, NWB>(it, t, orig[st], tile[st], &bar[st], par); break;
            case 2: ok = run_item<8, float, SPREAD, NWB>(it, t, orig[st], tile[st], &bar[st], par); break;
            default: ok = run_item<8, __half, SPREAD, NWB>(it, t, orig[st], tile[st], &bar[st], par); break;
        }
        if (!ok) {
            // report on the stream's status word; let in-flight copies land
            if (threadIdx.x == 0) atomicOr(reinterpret_cast<int*>(it.mem), kStatusWaitTimeout);
            if (tn < p.total) mbar_wait_bounded(&bar[st ^ 1], ((k + 1) >> 1) & 1, 2000000000ull);
            return;
        }
    }
}

template <int CAP, bool SPREAD, int NWB>
cudaError_t launch_t(const BatchParams<CAP>& p, int ctas, cudaStream_t s, bool pdl,
                            int max_block) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ctas, 1, 1);
    cfg.blockDim = dim3(NWB * 32, 1, 1);
    cfg.stream = s;
    const bool single = ctas >= p.total;
    if (single) cfg.dynamicSmemBytes = size_t(NWB) * max_block * kTileW;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    if (single) return cudaLaunchKernelEx(&cfg, dmsgm_batch_single_kernel<CAP, SPREAD, NWB>, p);
    return cudaLaunchKernelEx(&cfg, dmsgm_batch_kernel<CAP, SPREAD, NWB>, p);
}



// Launch for work items of 8 warps (dmsgm_batch_w8.cu); p points to a
// BatchParams<cap>, cap 16, 64 or DMSGM_MAX_BATCH.
cudaError_t batch_launch_w8(int cap, bool spread, const void* p, int ctas, cudaStream_t s,
                            bool pdl, int max_block);

}  // namespace dmsgm

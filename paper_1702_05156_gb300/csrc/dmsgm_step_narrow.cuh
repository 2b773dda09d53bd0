// dmsgm_step_narrow.cuh -- the per-tile frame step for 4x4 blocks with ONE
// block per lane, for small frames (at most one 256 x 32 tile per SM).
//
// The default block-4 layout gives a lane two adjacent blocks (8 pixel
// columns, one mask byte per row).  A small frame then fills few warps, and
// the step after the wait on the previous frame (gathers, update, mask) is a
// latency-bound chain per warp.  Here a warp
// covers half a tile row, 32 blocks: warp w takes strip row w / 2, half
// w % 2 (pixel columns [128 h, 128 h + 128) of the tile), lane l the block of
// pixel columns [128 h + 4 l, 128 h + 4 l + 4).  Twice the warps, half the
// work each.  The tile (256 x 32 pixels, one TMA copy), the affine origins
// (one per strip row and half) and every per-block operation are those of
// the default layout, so the results are the same bits.
//
// Mask: a lane tests its 4 pixels of a row at once (the byte interval test)
// and the even lane of each pair writes the byte of both.
#pragma once

#include "dmsgm_internal.h"

namespace dmsgm {

constexpr int kNarrowWarps = 16;                  // 8 strip rows x 2 halves
constexpr int kNarrowRows = kNarrowWarps / 2 * 4;  // tile rows: 32

template <typename T, bool SPREAD>
__global__ void __launch_bounds__(kNarrowWarps * 32)
    dmsgm_step_narrow_kernel(const __grid_constant__ CUtensorMap tmap, const StreamArgs a,
                             const Coef k, int* status) {
    constexpr int B = 4, STRIPS = kNarrowWarps / 2;
    __shared__ __align__(128) uint8_t tile[kNarrowRows * kTileW];
    __shared__ __align__(8) uint64_t bar;
    __shared__ Origin orig[2 * STRIPS];
    const int tx0 = blockIdx.x * kTileW;
    const int ty0 = blockIdx.y * kNarrowRows;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        mbar_arrive_expect_tx(&bar, kNarrowRows * kTileW);
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
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int s = warp >> 1, h = warp & 1;
    const int px = tx0 + 128 * h + 4 * lane;           // first pixel column of the lane
    const int bx = px / B, by = ty0 / B + s;
    const bool in = px < a.W && by < a.Gy;
    const int vr = strip_rows<B>(a, ty0, s);            // rows of the strip inside the frame
    // statistics over the rows inside the frame (a cut bottom block row
    // counts only those), and the back-projection
    uint32_t w[B];
#pragma unroll
    for (int i = 0; i < B; ++i)
        w[i] = *reinterpret_cast<const uint32_t*>(tile + (B * s + i) * kTileW + 128 * h + 4 * lane);
    Stats st;
    {
        uint32_t sm, lo, hi;
        if (vr == B) {
            raw_stats<B>(w, B, sm, lo, hi);
            st = stats_from<B * B>(sm, lo, hi);
        } else {
            raw_stats<B>(w, vr, sm, lo, hi);
            st = stats_from<0>(sm, lo, hi, B * vr);
        }
    }
    const Proj pj = in ? project<B>(a, k, bx, by, (tx0 + 128 * h) / B, orig[(s << 1) | h])
                       : no_proj();
    pdl_wait();
    pdl_launch_dependents();
    // gather, update, store the block's next state
    Comp c = gather<SPREAD>(a, pj, global_src<T, false>(a));
    dual_mode_step<sizeof(T) == 4>(c, st, a);
    if (in) store_block<T>(a, by * a.Gx + bx, c);
    // mask bytes of the strip's rows: lane pairs (2m, 2m + 1) share byte m
    if (by >= a.Gy) return;   // warp-uniform: strip below the frame
    const float thr = a.theta_d * c.A.var;
    const size_t mrow = size_t(a.mask_words) * 4;
    const int mbyte = px >> 3;                          // the pair's mask byte
    const bool writer = (lane & 1) == 0 && mbyte < int(mrow);
    uint8_t* m = reinterpret_cast<uint8_t*>(a.mask) + size_t(ty0 + B * s) * mrow + mbyte;
    const bool flat = !in || block_all_bg(st, c.A.mu, thr);
    if (__all_sync(0xffffffffu, flat)) {
#pragma unroll
        for (int i = 0; i < B; ++i)
            if (i < vr && writer) m[i * mrow] = 0;
        return;
    }
    const Thresh t = bg_interval(c.A.mu, thr);
#pragma unroll
    for (int i = 0; i < B; ++i) {
        if (i >= vr) break;   // warp-uniform
        // bits 0..3: the lane's 4 pixels; zero for lanes past the frame
        const uint32_t nib = flat ? 0u : __umulhi(fg_bits(w[i], t), 0x02040810u);
        const uint32_t hi = __shfl_down_sync(0xffffffffu, nib, 1);
        if (writer) m[i * mrow] = uint8_t(nib | (hi << 4));
    }
}

// How many CTAs of the narrow kernel the GPU holds at once.
template <typename T>
static int narrow_capacity(int device) {
    static std::mutex mu;
    static int cache[64] = {0};
    std::lock_guard<std::mutex> g(mu);
    if (device < 0 || device >= 64) return 0;
    if (!cache[device]) {
        int per_sm = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dmsgm_step_narrow_kernel<T, false>,
                                                          kNarrowWarps * 32, 0) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        cache[device] = per_sm * sms;
    }
    return cache[device];
}

template <typename T>
static cudaError_t launch_narrow_t(const CUtensorMap& tmap, const StreamArgs& a, const Coef& k,
                                   int* status, cudaStream_t s, bool pdl) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((a.W + kTileW - 1) / kTileW, (a.H + kNarrowRows - 1) / kNarrowRows, 1);
    cfg.blockDim = dim3(kNarrowWarps * 32, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    auto kern = a.spread ? dmsgm_step_narrow_kernel<T, true> : dmsgm_step_narrow_kernel<T, false>;
    return cudaLaunchKernelEx(&cfg, kern, tmap, a, k, status);
}

}  // namespace dmsgm

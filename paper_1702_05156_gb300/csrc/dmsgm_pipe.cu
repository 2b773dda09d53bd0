// dmsgm_pipe.cu -- persistent, software-pipelined frame step.
//
// The per-tile kernel (dmsgm_api.cu) runs one CTA per tile, and every CTA
// waits one L2 round trip for its state gathers (Sec. 2.4 compensation)
// before it can update its blocks.  Here a resident CTA runs a strided
// sequence of tiles of the frame in a two-stage pipeline: while it computes
// tile k from shared memory, TMA brings tile k+1's pixels and the box of
// previous-state blocks that tile k+1's back-projected blocks overlap, so the
// gathers read shared memory.
//
// The box comes from the tile's affine origins.  Within a half-warp strip
// the integer part of the block displacement moves by at most one block (the
// host admits the affine form only for |d ex / d bx|, |d ey / d bx| <= 1/31),
// so a strip's blocks read columns [c - 1, c + half + 1] and rows
// [r - 1, r + 2] around its origin block (c, r); the box takes one more block
// of margin on each side and starts at a column that is a multiple of 8 (the
// TMA alignment of the 2-byte age array).  A tile whose box would not fit
// (strong shear) reads global memory, and so does any single block whose
// 2 x 2 group falls outside the box.  Frames in the general projective form
// go to the per-tile kernel.
#include <algorithm>
#include <climits>
#include <mutex>
#include <type_traits>

#include "dmsgm_internal.h"

namespace dmsgm {

constexpr uint64_t kPipeTimeoutNs = 2000000000ull;   // 2 s: only a broken copy gets here

// Tile and state-box geometry (in blocks unless noted).
template <int B, int NW>
struct PipeGeom {
    static constexpr int kTileH = NW * B;              // pixel rows per tile (one strip per warp)
    static constexpr int kHalf = 128 / B;              // blocks per half-warp strip
    static constexpr int kBoxW = B == 4 ? 80 : 48;     // >= 2 * kHalf + 13, a multiple of 8
    static constexpr int kBoxH = NW + 8;               // >= NW + 6
};

template <typename T>
using Pair = typename std::conditional<std::is_same<T, float>::value, float2, __half2>::type;

__device__ __forceinline__ float2 to_f2(float2 v) { return v; }
__device__ __forceinline__ float2 to_f2(__half2 v) { return __half22float2(v); }

// Shared memory of one CTA: two stages of pixels, origins and state box.
// Every array is a multiple of 128 bytes, so each TMA destination stays
// 128-byte aligned.
template <int B, typename T, int NW>
struct PipeSmem {
    using G = PipeGeom<B, NW>;
    uint8_t frame[2][G::kTileH * kTileW];
    Pair<T> mu[2][G::kBoxH * G::kBoxW];
    Pair<T> var[2][G::kBoxH * G::kBoxW];
    uint16_t age[2][G::kBoxH * G::kBoxW];
    Origin orig[2][2 * NW];
    int box[2][3];              // first column, first row, 1 if the box was staged
    uint64_t fbar[2], sbar[2];  // pixels / state box of each stage
};

// The staged box as a gather source.
template <typename T>
struct BoxSrc {
    const Pair<T>* mu;
    const Pair<T>* var;
    const uint16_t* age;
    int pitch;
    int rx0, ry0;
    __device__ __forceinline__ int at(int i, int j) const { return (j - ry0) * pitch + (i - rx0); }
    __device__ __forceinline__ float2 ld_mu(int k) const { return to_f2(mu[k]); }
    __device__ __forceinline__ float2 ld_var(int k) const { return to_f2(var[k]); }
    __device__ __forceinline__ uint32_t ld_ag(int k) const { return age[k]; }
};

template <int B, typename T, int NW>
__global__ void __launch_bounds__(NW * 32, 1)
    dmsgm_pipe_kernel(const __grid_constant__ CUtensorMap fmap,
                      const __grid_constant__ CUtensorMap mumap,
                      const __grid_constant__ CUtensorMap varmap,
                      const __grid_constant__ CUtensorMap agemap, const StreamArgs a,
                      const Coef k, int tiles_x, int n_tiles, int* status) {
    using G = PipeGeom<B, NW>;
    using S = PipeSmem<B, T, NW>;
    constexpr int BPL = kLaneBlocks<B>;
    constexpr uint32_t kFrameBytes = G::kTileH * kTileW;
    constexpr uint32_t kStateBytes = G::kBoxH * G::kBoxW * (2 * sizeof(Pair<T>) + 2);
    extern __shared__ __align__(128) uint8_t dsm[];
    S& sm = *reinterpret_cast<S*>(dsm);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int t0 = blockIdx.x, step = gridDim.x;
    if (t0 >= n_tiles) return;

    auto tile_xy = [&](int tile, int& tx0, int& ty0) {
        tx0 = (tile % tiles_x) * kTileW;
        ty0 = (tile / tiles_x) * G::kTileH;
    };
    // stage s <- pixels (thread 0 starts the copy) and affine origins of `tile`
    auto stage_frame = [&](int s, int tile) {
        int tx0, ty0;
        tile_xy(tile, tx0, ty0);
        if (tid == 0) {
            mbar_arrive_expect_tx(&sm.fbar[s], kFrameBytes);
            tma_load_2d(sm.frame[s], &fmap, tx0, ty0, &sm.fbar[s]);
        }
        fill_origins<B>(a, k, tx0, ty0, NW, sm.orig[s]);
    };
    // warp 0, once stage s's origins are visible: the state box and its copies
    auto stage_state = [&](int s, int tile) {
        int tx0, ty0;
        tile_xy(tile, tx0, ty0);
        bool ok = a.affine && !a.first;   // uniform
        int rx0 = 0, ry0 = 0;
        if (ok) {
            int c = INT_MAX, r = INT_MAX, c2 = INT_MIN, r2 = INT_MIN;
            if (lane < 2 * NW) {
                const Origin o = sm.orig[s][lane];
                c = c2 = (tx0 + 128 * (lane & 1)) / B + o.nx;
                r = r2 = ty0 / B + (lane >> 1) + o.ny;
            }
            const int cmin = __reduce_min_sync(0xffffffffu, c) - 2;
            const int cmax = __reduce_max_sync(0xffffffffu, c2) + G::kHalf + 2;
            const int rmin = __reduce_min_sync(0xffffffffu, r) - 2;
            const int rmax = __reduce_max_sync(0xffffffffu, r2) + 3;
            rx0 = cmin & ~7;   // floor to a multiple of 8
            ry0 = rmin;
            ok = cmax - rx0 < G::kBoxW && rmax - ry0 < G::kBoxH;
        }
        if (lane == 0) {
            sm.box[s][0] = rx0;
            sm.box[s][1] = ry0;
            sm.box[s][2] = ok ? 1 : 0;
            if (ok) {   // out-of-grid parts of the box read as zeros and are never used
                mbar_arrive_expect_tx(&sm.sbar[s], kStateBytes);
                tma_load_2d(sm.mu[s], &mumap, 2 * rx0, ry0, &sm.sbar[s]);
                tma_load_2d(sm.var[s], &varmap, 2 * rx0, ry0, &sm.sbar[s]);
                tma_load_2d(sm.age[s], &agemap, rx0, ry0, &sm.sbar[s]);
            }
        }
    };
    // leave after a timed-out wait: report, and give the copies still in
    // flight one more bounded chance to land
    auto abandon = [&](bool frame_pending, int fs, uint32_t fpar, bool state_pending, int ss,
                       uint32_t spar) {
        if (tid == 0) {
            atomicOr(status, kStatusWaitTimeout);
            if (frame_pending) mbar_wait_bounded(&sm.fbar[fs], fpar, kPipeTimeoutNs);
            if (state_pending) mbar_wait_bounded(&sm.sbar[ss], spar, kPipeTimeoutNs);
        }
    };

    if (tid == 0) {
        mbar_init(&sm.fbar[0], 1);
        mbar_init(&sm.fbar[1], 1);
        mbar_init(&sm.sbar[0], 1);
        mbar_init(&sm.sbar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t ph = 0;   // bit s: next phase of fbar[s]; bit 2 + s: of sbar[s]

    // Prologue: the first tile's pixels, statistics and projections depend on
    // this frame only, so they run before the previous frame's kernel ends.
    stage_frame(0, t0);
    __syncthreads();
    int tx0, ty0;
    tile_xy(t0, tx0, ty0);
    Stats st[1][BPL];
    Proj pj[1][BPL];
    bool ok = mbar_wait_bounded(&sm.fbar[0], ph & 1, kPipeTimeoutNs);
    if (__syncthreads_or(!ok)) {
        abandon(true, 0, ph & 1, false, 0, 0);
        return;
    }
    ph ^= 1;
    tile_stats<B, NW, 1>(a, sm.frame[0], ty0, tx0 + kLanePx * lane < a.W, st);
    tile_project<B, NW, 1>(a, k, tx0, ty0, sm.orig[0], pj);
    pdl_wait();
    pdl_launch_dependents();
    if (warp == 0) stage_state(0, t0);

    for (int it = 0;; ++it) {
        const int s = it & 1;
        const int cur = t0 + it * step, nxt = cur + step;
        const bool more = nxt < n_tiles;
        if (more) stage_frame(s ^ 1, nxt);
        __syncthreads();   // stage s^1's origins and stage s's box are visible
        if (more && warp == 0) stage_state(s ^ 1, nxt);
        tile_xy(cur, tx0, ty0);
        const bool boxed = sm.box[s][2] != 0;
        ok = !boxed || mbar_wait_bounded(&sm.sbar[s], (ph >> (2 + s)) & 1, kPipeTimeoutNs);
        if (__syncthreads_or(!ok)) {
            abandon(more, s ^ 1, (ph >> (s ^ 1)) & 1, more && sm.box[s ^ 1][2], s ^ 1, (ph >> (2 + (s ^ 1))) & 1);
            return;
        }
        if (boxed) ph ^= 4u << s;
        float muA[1][BPL], thr[1][BPL];
        if (boxed) {
            const BoxSrc<T> box{sm.mu[s], sm.var[s], sm.age[s], G::kBoxW, sm.box[s][0], sm.box[s][1]};
            const GlobalSrc<T, false> glob = global_src<T, false>(a);
            tile_update_with<B, T, NW, 1>(a, tx0, ty0, pj, st, muA, thr, [&](const Proj& p) {
                const unsigned li = unsigned(p.i0 - box.rx0), lj = unsigned(p.j0 - box.ry0);
                return (li <= unsigned(G::kBoxW - 2) && lj <= unsigned(G::kBoxH - 2))
                           ? gather<false>(a, p, box)
                           : gather<false>(a, p, glob);
            });
        } else {
            tile_update<B, T, NW, 1, false, false>(a, tx0, ty0, pj, st, muA, thr);
        }
        tile_mask<B, NW, 1>(a, sm.frame[s], tx0, ty0, st, muA, thr);
        if (!more) break;
        // the next tile's statistics and projections; its pixels were copied meanwhile
        ok = mbar_wait_bounded(&sm.fbar[s ^ 1], (ph >> (s ^ 1)) & 1, kPipeTimeoutNs);
        if (__syncthreads_or(!ok)) {   // also: every thread is done with stage s
            abandon(true, s ^ 1, (ph >> (s ^ 1)) & 1, sm.box[s ^ 1][2] != 0, s ^ 1, (ph >> (2 + (s ^ 1))) & 1);
            return;
        }
        ph ^= 1u << (s ^ 1);
        tile_xy(nxt, tx0, ty0);
        tile_stats<B, NW, 1>(a, sm.frame[s ^ 1], ty0, tx0 + kLanePx * lane < a.W, st);
        tile_project<B, NW, 1>(a, k, tx0, ty0, sm.orig[s ^ 1], pj);
    }
}

// ------------------------------------------------------------------ host
// Tensor maps of the previous-state arrays of buffer b: (mu, var) as
// 2 Gx x Gy values of the stored type, age as Gx x Gy uint16.
static bool encode_state_maps(dmsgm_ctx* h, int b, int box_w, int box_h, CUtensorMap out[3]) {
    auto enc = encode_fn();
    if (!enc) return false;
    const bool f16 = h->prec == DMSGM_STATE_FP16;
    const CUtensorMapDataType vt = f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const size_t s = f16 ? 2 : 4;
    const StateBuf& sb = h->buf[b];
    void* ptr[3] = {sb.mu, sb.var, sb.age};
    for (int i = 0; i < 3; ++i) {
        const bool is_age = i == 2;
        cuuint64_t dims[2] = {cuuint64_t(is_age ? h->Gx : 2 * h->Gx), cuuint64_t(h->Gy)};
        cuuint64_t strides[1] = {cuuint64_t(is_age ? 2 * size_t(h->Gx) : 2 * s * h->Gx)};
        cuuint32_t box[2] = {cuuint32_t(is_age ? box_w : 2 * box_w), cuuint32_t(box_h)};
        cuuint32_t estr[2] = {1, 1};
        if (strides[0] % 16 != 0) return false;
        CUresult r = enc(&out[i], is_age ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : vt, 2, ptr[i], dims,
                         strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return false;
    }
    return true;
}

template <int B, typename T, int NW>
static int pipe_capacity(int device) {
    static std::mutex mu;
    static int cache[64] = {0};
    std::lock_guard<std::mutex> g(mu);
    if (device < 0 || device >= 64) return 0;
    if (!cache[device]) {
        const int smem = int(sizeof(PipeSmem<B, T, NW>));
        int per_sm = 0, sms = 0;
        if (cudaFuncSetAttribute(dmsgm_pipe_kernel<B, T, NW>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dmsgm_pipe_kernel<B, T, NW>,
                                                          NW * 32, smem) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        cache[device] = per_sm * sms;
    }
    return cache[device];
}

template <int B, typename T, int NW>
static int launch_pipe_t(dmsgm_ctx* h, const CUtensorMap& fmap, const StreamArgs& a,
                         const Coef& c, cudaStream_t s, bool automatic, bool* launched) {
    using G = PipeGeom<B, NW>;
    if (h->pipe_maps == 0)
        h->pipe_maps = (encode_state_maps(h, 0, G::kBoxW, G::kBoxH, h->smap[0]) &&
                        encode_state_maps(h, 1, G::kBoxW, G::kBoxH, h->smap[1]))
                           ? 1
                           : -1;
    if (h->pipe_maps < 0) return DMSGM_OK;   // not encodable: the caller uses the per-tile kernel
    const int cap = pipe_capacity<B, T, NW>(h->device);
    if (cap <= 0) return DMSGM_OK;
    const int tiles_x = (h->W + kTileW - 1) / kTileW;
    const int n_tiles = tiles_x * ((h->H + G::kTileH - 1) / G::kTileH);
    // automatic: the per-tile kernel, which measures faster on every size so far
    if (automatic) return DMSGM_OK;
    const CUtensorMap* sm = h->smap[h->parity];
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(std::min(n_tiles, cap), 1, 1);
    cfg.blockDim = dim3(NW * 32, 1, 1);
    cfg.dynamicSmemBytes = sizeof(PipeSmem<B, T, NW>);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = h->use_pdl ? 1 : 0;
    cudaError_t e = cudaLaunchKernelEx(&cfg, dmsgm_pipe_kernel<B, T, NW>, fmap, sm[0], sm[1], sm[2],
                                       a, c, tiles_x, n_tiles, h->status_dev);
    if (e != cudaSuccess)
        return fail(DMSGM_ERR_CUDA, "kernel launch failed: %s", cudaGetErrorString(e));
    *launched = true;
    return DMSGM_OK;
}

int launch_pipe(dmsgm_ctx* h, const CUtensorMap& fmap, const StreamArgs& a, const Coef& c,
                cudaStream_t s, bool automatic, bool* launched) {
    *launched = false;
    if (!a.first && !a.affine) return DMSGM_OK;   // general projective form: per-tile kernel
    if (h->H % h->B) return DMSGM_OK;              // a cut bottom block row: per-tile kernel
    if (h->mix_spread) return DMSGM_OK;            // the mixture-variance option: per-tile kernel
    const int q = h->tile_rows / h->B;
    const bool f16 = h->prec == DMSGM_STATE_FP16;
#define DMSGM_PIPE(BB, TT, NWW) return launch_pipe_t<BB, TT, NWW>(h, fmap, a, c, s, automatic, launched);
    if (h->B == 4 && q == 4) { if (f16) DMSGM_PIPE(4, __half, 4) else DMSGM_PIPE(4, float, 4) }
    if (h->B == 4 && q == 8) { if (f16) DMSGM_PIPE(4, __half, 8) else DMSGM_PIPE(4, float, 8) }
    if (h->B == 8 && q == 4) { if (f16) DMSGM_PIPE(8, __half, 4) else DMSGM_PIPE(8, float, 4) }
    if (h->B == 8 && q == 8) { if (f16) DMSGM_PIPE(8, __half, 8) else DMSGM_PIPE(8, float, 8) }
#undef DMSGM_PIPE
    return DMSGM_OK;
}

}  // namespace dmsgm

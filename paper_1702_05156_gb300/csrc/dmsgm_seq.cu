// dmsgm_seq.cu -- T consecutive frames of one stream in one persistent launch.
//
// Frame t+1 of a block needs only the frame-t state of the blocks its
// back-projected square can reach (Sec. 2.4), so a global barrier between
// frames is not needed: each CTA owns one tile for the whole launch and
// starts frame t+1 as soon as the tiles within the dependency radius have
// published frame t.  Per tile and frame the critical path is
//   wait for the neighbours' counters -> gather (L2) -> mix -> update ->
//   store the state -> publish the counter;
// the frame's pixels (3-D TMA, double-buffered: frame t+1 loads while frame
// t runs), the block statistics and the whole mask stage stay off it, so
// they overlap other tiles' critical paths.
//
// All CTAs must be resident at once (they wait on each other): the launch is
// cooperative, sized to the GPU, and every wait is bounded (timeout -> the
// handle's status word, the kernel leaves).  The same ping-pong buffers as
// the single-frame kernel are used: waiting for the neighbours' frame t-1
// also orders this tile's overwrite of the frame t-2 buffer after their
// reads of it.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "dmsgm_internal.h"

namespace dmsgm {

constexpr int kSeqMaxFrames = 256;              // frames per launch (parameter space)
constexpr uint64_t kSeqTimeoutNs = 2000000000ull;

struct SeqParams {
    StateBuf buf[2];        // the handle's two state buffers
    uint32_t* masks;        // mask of frame k at masks + k * frame_words
    int* flags;             // one progress counter per tile (zeroed before the launch)
    int* status;            // the handle's status word
    long long frame_words;  // mask words per frame
    int W, H, Gx, Gy, mask_words;
    int T;                  // frames in this launch
    int p0;                 // buffer holding the state before frame 0
    int first;              // 1: frame 0 has no previous state
    int age_max;
    float theta_s, theta_d;
    int spread;             // mixed variance carries the spread of the mixed means
    int tiles_x, tiles_y;
    int rx, ry;             // dependency radius, in tiles
    uint8_t affine[kSeqMaxFrames];
    Coef coef[kSeqMaxFrames];
};
static_assert(sizeof(SeqParams) + sizeof(CUtensorMap) <= 32764, "kernel parameter limit");

// Bounded wait until counter f reaches `target`.
__device__ __forceinline__ bool wait_counter(const int* f, int target, uint64_t timeout_ns) {
    if (ld_acquire_gpu(f) >= target) return true;
    const uint64_t t0 = global_timer_ns();
    for (uint32_t it = 0;; ++it) {
        __nanosleep(64);
        if (ld_acquire_gpu(f) >= target) return true;
        if ((it & 15u) == 15u && global_timer_ns() - t0 > timeout_ns) return false;
    }
}

template <int B, typename T, int NW, int RPT>
__global__ void __launch_bounds__(NW * 32, (NW == 8 ? 2 : 1))
    dmsgm_seq_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ SeqParams p) {
    constexpr int STRIPS = NW * RPT;
    constexpr int TILE_H = STRIPS * B;
    constexpr int BPL = kLaneBlocks<B>;
    static_assert(TILE_H <= 256, "TMA box rows");
    extern __shared__ __align__(128) uint8_t dyn_smem[];   // two pixel stages
    uint8_t* tile[2] = {dyn_smem, dyn_smem + TILE_H * kTileW};
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ Origin orig[2][2 * STRIPS];

    const int tix = blockIdx.x % p.tiles_x, tiy = blockIdx.x / p.tiles_x;
    const int tx0 = tix * kTileW, ty0 = tiy * TILE_H;
    const bool xin = tx0 + kLanePx * int(threadIdx.x & 31) < p.W;
    constexpr uint32_t kTileBytes = TILE_H * kTileW;

    StreamArgs a;
    a.W = p.W;
    a.H = p.H;
    a.Gx = p.Gx;
    a.Gy = p.Gy;
    a.mask_words = p.mask_words;
    a.age_max = p.age_max;
    a.theta_s = p.theta_s;
    a.theta_d = p.theta_d;
    a.spread = p.spread;

    auto origins = [&](int k, Origin* o) {
        const int t = threadIdx.x;
        if (p.affine[k] && t < 2 * STRIPS)
            o[t] = affine_origin(p.coef[k], (tx0 + 128 * (t & 1)) / B, ty0 / B + (t >> 1));
    };

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        mbar_arrive_expect_tx(&bar[0], kTileBytes);
        tma_load_3d(tile[0], &tmap, tx0, ty0, 0, &bar[0]);
    }
    origins(0, orig[0]);
    __syncthreads();

    // neighbours this tile waits for (excluding itself)
    const int nx = 2 * p.rx + 1, ny = 2 * p.ry + 1;
    const int nn = nx * ny;

    for (int k = 0; k < p.T; ++k) {
        const int st = k & 1;
        if (k + 1 < p.T) {   // next frame's pixels and origins; that stage is free
            if (threadIdx.x == 0) {
                mbar_arrive_expect_tx(&bar[st ^ 1], kTileBytes);
                tma_load_3d(tile[st ^ 1], &tmap, tx0, ty0, k + 1, &bar[st ^ 1]);
            }
            origins(k + 1, orig[st ^ 1]);
        }
        bool ok = mbar_wait_bounded(&bar[st], (k >> 1) & 1, kSeqTimeoutNs);
        a.prev = p.buf[(p.p0 + k) & 1];
        a.next = p.buf[(p.p0 + k + 1) & 1];
        a.first = (k == 0) ? p.first : 0;
        a.affine = p.affine[k];
        a.mask = p.masks + k * p.frame_words;
        // the frame's block statistics and back-projections need no other tile
        Stats sts[RPT][BPL];
        Proj pj[RPT][BPL];
        tile_stats<B, NW, RPT>(a, tile[st], ty0, ok && xin, sts);
        tile_project<B, NW, RPT>(a, p.coef[k], tx0, ty0, orig[st], pj);
        // wait until every neighbour tile has published frame k-1
        if (k > 0) {
            for (int q = threadIdx.x; q < nn; q += NW * 32) {
                const int ntx = tix + q % nx - p.rx, nty = tiy + q / nx - p.ry;
                if (ntx < 0 || ntx >= p.tiles_x || nty < 0 || nty >= p.tiles_y) continue;
                if (ntx == tix && nty == tiy) continue;
                if (!wait_counter(p.flags + nty * p.tiles_x + ntx, k, kSeqTimeoutNs)) ok = false;
            }
        }
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) atomicOr(p.status, kStatusWaitTimeout);
            if (k + 1 < p.T) mbar_wait_bounded(&bar[st ^ 1], ((k + 1) >> 1) & 1, kSeqTimeoutNs);
            return;
        }
        // critical path: gather, mix, update, store the state
        float muA[RPT][BPL], thr[RPT][BPL];
        tile_update<B, T, NW, RPT, true, false>(a, tx0, ty0, pj, sts, muA, thr);
        __syncthreads();
        if (threadIdx.x == 0) {   // publish: this tile's frame-k state is visible
            __threadfence();
            st_release_gpu(p.flags + blockIdx.x, k + 1);
        }
        // off the critical path: the frame's mask bytes
        tile_mask<B, NW, RPT>(a, tile[st], tx0, ty0, sts, muA, thr);
        __syncthreads();   // this stage's pixels and origins are consumed
    }
}

// ------------------------------------------------------------------ host
struct SeqShape {
    int nw, rpt;
};

template <int B, int NW, int RPT>
constexpr size_t seq_smem() { return 2 * size_t(NW * RPT * B) * kTileW; }

// Opt the kernel in to its dynamic shared memory (once per device) and
// return how many of its CTAs the whole GPU holds at once.
template <int B, typename T, int NW, int RPT>
static int seq_capacity(int device) {
    static std::mutex mu;
    static int cache[64] = {0};
    std::lock_guard<std::mutex> g(mu);
    if (device < 0 || device >= 64) return 0;
    if (!cache[device]) {
        constexpr size_t smem = seq_smem<B, NW, RPT>();
        int per_sm = 0, sms = 0;
        if (cudaFuncSetAttribute(dmsgm_seq_kernel<B, T, NW, RPT>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dmsgm_seq_kernel<B, T, NW, RPT>,
                                                          NW * 32, smem) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        cache[device] = per_sm * sms;
    }
    return cache[device];
}

template <int B, typename T, int NW, int RPT>
static cudaError_t launch_seq_t(const CUtensorMap& tm, const SeqParams& p, int ctas,
                                cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ctas, 1, 1);
    cfg.blockDim = dim3(NW * 32, 1, 1);
    cfg.dynamicSmemBytes = seq_smem<B, NW, RPT>();
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, dmsgm_seq_kernel<B, T, NW, RPT>, tm, p);
}

// The shapes the kernel is built for (tile heights 8B .. 256 rows), with
// their capacity (co-resident CTAs).  B = 8 stops at 16 warps x 2 strips.
template <int B, typename T>
static int seq_cap(int nw, int rpt, int dev) {
    if (nw == 8 && rpt == 1) return seq_capacity<B, T, 8, 1>(dev);
    if (nw == 16 && rpt == 1) return seq_capacity<B, T, 16, 1>(dev);
    if (nw == 16 && rpt == 2) return seq_capacity<B, T, 16, 2>(dev);
    if constexpr (B == 4) {
        if (nw == 16 && rpt == 4) return seq_capacity<B, T, 16, 4>(dev);
    }
    return 0;
}

template <int B, typename T>
static cudaError_t seq_launch(int nw, int rpt, const CUtensorMap& tm, const SeqParams& p,
                              int ctas, cudaStream_t s) {
    if (nw == 8 && rpt == 1) return launch_seq_t<B, T, 8, 1>(tm, p, ctas, s);
    if (nw == 16 && rpt == 1) return launch_seq_t<B, T, 16, 1>(tm, p, ctas, s);
    if (nw == 16 && rpt == 2) return launch_seq_t<B, T, 16, 2>(tm, p, ctas, s);
    if constexpr (B == 4) {
        if (nw == 16 && rpt == 4) return launch_seq_t<B, T, 16, 4>(tm, p, ctas, s);
    }
    return cudaErrorInvalidValue;
}

static int capacity(const dmsgm_ctx* h, int nw, int rpt) {
    if (h->B == 4)
        return h->prec == DMSGM_STATE_FP16 ? seq_cap<4, __half>(nw, rpt, h->device)
                                           : seq_cap<4, float>(nw, rpt, h->device);
    return h->prec == DMSGM_STATE_FP16 ? seq_cap<8, __half>(nw, rpt, h->device)
                                       : seq_cap<8, float>(nw, rpt, h->device);
}

// Pick the tile shape: the most tiles that still fit one per SM, else the
// most that fit the GPU at all; {0, 0} if none fits.
static SeqShape pick_shape(const dmsgm_ctx* h, int sms) {
    static const SeqShape shapes[] = {{8, 1}, {16, 1}, {16, 2}, {16, 4}};
    // built for blocks 4 and 8 on whole block rows, without the
    // mixture-variance option or preprocessing (those calls run per frame)
    if (!((h->B == 4 || h->B == 8) && h->H % h->B == 0) || h->mix_spread || h->pre_gauss || h->pre_median || h->checked)
        return SeqShape{0, 0};
    if (h->seq_tile_rows) {   // asked for: use it if the tiles fit the GPU at once
        for (const SeqShape& sh : shapes) {
            if (sh.nw * sh.rpt * h->B != h->seq_tile_rows) continue;
            const int th = h->seq_tile_rows;
            const long tiles = long((h->W + kTileW - 1) / kTileW) * ((h->H + th - 1) / th);
            if (tiles <= capacity(h, sh.nw, sh.rpt)) return sh;
        }
        return SeqShape{0, 0};
    }
    SeqShape best{0, 0};
    long best_tiles = -1;
    bool best_one = false;
    for (const SeqShape& sh : shapes) {
        const int th = sh.nw * sh.rpt * h->B;
        const long tiles = long((h->W + kTileW - 1) / kTileW) * ((h->H + th - 1) / th);
        const int cap = capacity(h, sh.nw, sh.rpt);
        if (tiles > cap) continue;
        const bool one = tiles <= sms;
        if ((one && !best_one) || (one == best_one && tiles > best_tiles)) {
            best = sh;
            best_tiles = tiles;
            best_one = one;
        }
    }
    return best;
}

static int seq_map(dmsgm_ctx* h, const uint8_t* frames, int T, int rows, CUtensorMap* out) {
    auto enc = encode_fn();
    if (!enc) return fail(DMSGM_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    if (h->seqmap.ptr == frames && h->seqmap.frames == T && h->seqmap.rows == rows) {
        *out = h->seqmap.map;
        return DMSGM_OK;
    }
    cuuint64_t dims[3] = {cuuint64_t(h->W), cuuint64_t(h->H), cuuint64_t(T)};
    cuuint64_t strides[2] = {cuuint64_t(h->W), cuuint64_t(h->W) * h->H};
    cuuint32_t box[3] = {cuuint32_t(kTileW), cuuint32_t(rows), 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(out, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<uint8_t*>(frames), dims,
                     strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(DMSGM_ERR_CUDA, "cuTensorMapEncodeTiled (3-D) failed (%d)", int(r));
    h->seqmap.ptr = frames;
    h->seqmap.frames = T;
    h->seqmap.rows = rows;
    h->seqmap.map = *out;
    return DMSGM_OK;
}

int launch_seq(dmsgm_ctx* h, const uint8_t* frames_dev, int T, const double* Hs,
               uint32_t* masks_dev, cudaStream_t stream, int* flags) {
    int sms = 0;
    DMSGM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    const SeqShape sh = pick_shape(h, sms);
    if (!sh.nw) return DMSGM_ERR_UNSUPPORTED;   // caller falls back to one launch per frame
    const int th = sh.nw * sh.rpt * h->B;
    const int tiles_x = (h->W + kTileW - 1) / kTileW, tiles_y = (h->H + th - 1) / th;
    const int tiles = tiles_x * tiles_y;
    const size_t fbytes = size_t(h->W) * h->H;
    const long long fwords = (long long)h->H * ((h->W + 31) / 32);
    static thread_local SeqParams p;
    for (int c0 = 0; c0 < T; c0 += kSeqMaxFrames) {
        const int n = std::min(kSeqMaxFrames, T - c0);
        double ex = 0, ey = 0;
        bool bounded = true;
        for (int k = 0; k < n && bounded; ++k) {
            double fx, fy;
            if (!displacement_bound(Hs + 9 * size_t(c0 + k), h->W, h->H, h->B, &fx, &fy)) bounded = false;
            ex = std::max(ex, fx);
            ey = std::max(ey, fy);
        }
        int rx = tiles_x, ry = tiles_y;
        if (bounded) {
            // a source block lies within ceil(|e|) + 1 blocks, one more for
            // the kernel's FP32 rounding of the floor
            rx = std::min<double>(tiles_x, std::ceil((std::ceil(ex) + 2.0) / (kTileW / h->B)));
            ry = std::min<double>(tiles_y, std::ceil((std::ceil(ey) + 2.0) / (th / h->B)));
        }
        for (int k = 0; k < n; ++k) {
            int affine = 0;
            if (!make_coef(Hs + 9 * size_t(c0 + k), h->B, &p.coef[k], &affine))
                return fail(DMSGM_ERR_INVALID_ARG, "homography %d is not finite in FP32", c0 + k);
            p.affine[k] = uint8_t(affine);
        }
        p.buf[0] = h->buf[0];
        p.buf[1] = h->buf[1];
        p.masks = masks_dev + size_t(c0) * fwords;
        p.flags = flags;
        p.status = h->status_dev;
        p.frame_words = fwords;
        p.W = h->W;
        p.H = h->H;
        p.Gx = h->Gx;
        p.Gy = h->Gy;
        p.mask_words = (h->W + 31) / 32;
        p.T = n;
        p.p0 = h->parity;
        p.first = h->initialized ? 0 : 1;
        p.age_max = h->age_max;
        p.theta_s = h->theta_s;
        p.theta_d = h->theta_d;
        p.spread = h->mix_spread;
        p.tiles_x = tiles_x;
        p.tiles_y = tiles_y;
        p.rx = rx;
        p.ry = ry;
        CUtensorMap tm;
        int rc = seq_map(h, frames_dev + size_t(c0) * fbytes, n, th, &tm);
        if (rc) return rc;
        DMSGM_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int) * size_t(tiles), stream));
        cudaError_t e;
        if (h->B == 4)
            e = h->prec == DMSGM_STATE_FP16 ? seq_launch<4, __half>(sh.nw, sh.rpt, tm, p, tiles, stream)
                                            : seq_launch<4, float>(sh.nw, sh.rpt, tm, p, tiles, stream);
        else
            e = h->prec == DMSGM_STATE_FP16 ? seq_launch<8, __half>(sh.nw, sh.rpt, tm, p, tiles, stream)
                                            : seq_launch<8, float>(sh.nw, sh.rpt, tm, p, tiles, stream);
        if (e != cudaSuccess)
            return fail(DMSGM_ERR_CUDA, "multi-frame kernel launch failed: %s", cudaGetErrorString(e));
        h->parity = (h->parity + n) & 1;
        h->initialized = true;
        h->frames += n;
    }
    return DMSGM_OK;
}

}  // namespace dmsgm

// ============================================================ no allocation
// dmsgm_process_seq_noalloc: the multi-frame kernel for callers that may not
// allocate device memory.  Its only scratch -- the per-tile progress
// counters -- lives in this file-scope array instead of a handle's memory.
// Every GPU that loads the library holds the array (16 KB) until the process
// exits, and every call on a device shares it.
namespace dmsgm {

constexpr int kNoAllocCounters = 4096;
static __device__ __align__(256) int g_noalloc_counters[kNoAllocCounters];

// Device address of the array in the current CUDA context.  Host code must
// not hand the symbol itself to a kernel (on the host it only stands in for
// the device object), and an address is valid only in the context where it
// was looked up, so it is looked up once per context -- keyed by the
// context's unique ID, which is never reused, not even after a device reset
// -- with that context current, and cached.
static int noalloc_counters(int** out) {
    using GetCurrent = CUresult (*)(CUcontext*);
    using GetId = CUresult (*)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(p);
    });
    // make the device's primary context current if no context is yet
    DMSGM_CUDA_TRY(cudaFree(nullptr));
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx ||
        get_id(ctx, &id) != CUDA_SUCCESS)
        return fail(DMSGM_ERR_CUDA, "cannot identify the current CUDA context");
    struct Entry {
        unsigned long long id;
        int* addr;
    };
    static std::mutex mu;
    static Entry cache[16] = {};
    static int next = 0;
    std::lock_guard<std::mutex> g(mu);
    for (const Entry& e : cache)
        if (e.addr && e.id == id) {
            *out = e.addr;
            return DMSGM_OK;
        }
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_counters);
    if (e != cudaSuccess || !p)
        return fail(DMSGM_ERR_CUDA, "cudaGetSymbolAddress of the counter array failed: %s",
                    cudaGetErrorString(e));
    cache[next] = Entry{id, static_cast<int*>(p)};
    next = (next + 1) % 16;
    *out = static_cast<int*>(p);
    return DMSGM_OK;
}

}  // namespace dmsgm

using namespace dmsgm;

extern "C" int dmsgm_process_seq_noalloc(int W, int H, int B, int precision, float theta_s,
                                         float theta_d, int age_max, void* state_dev,
                                         size_t state_bytes, int* parity, int first,
                                         const uint8_t* frames_dev, int n, const double* Hs,
                                         uint32_t* masks_dev, void* stream) {
    clear_error();
    const size_t need = dmsgm_state_bytes(W, H, B, precision);
    if (!need) return fail(DMSGM_ERR_INVALID_ARG, "invalid size %dx%d block %d or precision %d", W, H, B, precision);
    if (!(std::isfinite(theta_s) && theta_s > 0) || !(std::isfinite(theta_d) && theta_d > 0))
        return fail(DMSGM_ERR_INVALID_ARG, "theta_s and theta_d must be finite and > 0");
    if (age_max < 1 || age_max > 255) return fail(DMSGM_ERR_INVALID_ARG, "age_max must be in [1, 255]");
    if (!state_dev || state_bytes < need)
        return fail(DMSGM_ERR_INVALID_ARG, "state_dev must hold %zu bytes", need);
    if (reinterpret_cast<uintptr_t>(state_dev) % 256)
        return fail(DMSGM_ERR_INVALID_ARG, "state_dev must be 256-byte aligned");
    if (!parity || (*parity != 0 && *parity != 1)) return fail(DMSGM_ERR_INVALID_ARG, "parity must point to 0 or 1");
    if (n < 0 || (n > 0 && (!frames_dev || !Hs || !masks_dev))) return fail(DMSGM_ERR_INVALID_ARG, "invalid argument");
    if (reinterpret_cast<uintptr_t>(frames_dev) % 16 || reinterpret_cast<uintptr_t>(masks_dev) % 4)
        return fail(DMSGM_ERR_INVALID_ARG, "frames must be 16-byte and masks 4-byte aligned");
    for (long i = 0; i < 9L * n; ++i)
        if (!std::isfinite(Hs[i])) return fail(DMSGM_ERR_INVALID_ARG, "homography %ld is not finite", i / 9);
    if (!((B == 4 || B == 8) && H % B == 0))
        return fail(DMSGM_ERR_UNSUPPORTED, "the multi-frame kernel takes blocks 4 and 8 on whole block rows");
    {
        // even the tallest tile (256 rows) needs more counters than the array holds
        const long least = long((W + kTileW - 1) / kTileW) * ((H + 255) / 256);
        if (least > kNoAllocCounters)
            return fail(DMSGM_ERR_INVALID_ARG, "a %dx%d frame needs at least %ld progress counters, "
                        "the array holds %d", W, H, least, kNoAllocCounters);
    }
    if (n == 0) return DMSGM_OK;
    int dev = 0;
    DMSGM_CUDA_TRY(cudaGetDevice(&dev));
    int* counters = nullptr;
    int rc = noalloc_counters(&counters);
    if (rc) return rc;
    // a handle description on the stack over the caller's memory
    dmsgm_ctx h{};
    h.W = W; h.H = H; h.B = B; h.Gx = W / B; h.Gy = grid_rows(H, B);
    h.prec = precision; h.age_max = age_max;
    h.theta_s = theta_s; h.theta_d = theta_d;
    h.device = dev;
    h.tile_rows = 32;
    h.mem = state_dev;
    h.owns_mem = false;
    h.state_bytes = need;
    const int s = precision == DMSGM_STATE_FP16 ? 2 : 4;
    h.status_dev = static_cast<int*>(state_dev);
    for (int b = 0; b < 2; ++b) h.buf[b] = state_buf(static_cast<char*>(state_dev), W, H, B, s, b);
    h.parity = *parity;
    h.initialized = !first;
    // the counters this launch needs must fit the array
    int sms = 0;
    DMSGM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const SeqShape sh = pick_shape(&h, sms);
    if (!sh.nw)
        return fail(DMSGM_ERR_UNSUPPORTED, "the %dx%d frame's tiles cannot all be resident on this GPU", W, H);
    const int th = sh.nw * sh.rpt * B;
    const long tiles = long((W + kTileW - 1) / kTileW) * ((H + th - 1) / th);
    if (tiles > kNoAllocCounters)
        return fail(DMSGM_ERR_INVALID_ARG, "the frame needs %ld progress counters, the array holds %d",
                    tiles, kNoAllocCounters);
    rc = launch_seq(&h, frames_dev, n, Hs, masks_dev, static_cast<cudaStream_t>(stream), counters);
    if (rc) return rc;
    *parity = h.parity;
    return DMSGM_OK;
}

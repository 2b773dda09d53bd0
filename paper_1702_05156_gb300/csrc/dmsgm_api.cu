// dmsgm_api.cu -- the single-stream fused kernel and the C ABI of dmsgm.h.
//
// One launch per frame: a CTA loads its 256 x TILE_H pixel tile with one
// 2-D TMA copy (cp.async.bulk.tensor) into shared memory, compensates its
// blocks' models from the previous state buffer while the copy is in flight
// (Sec. 2.4), then reduces the pixels, runs the dual-mode update (Sec.
// 2.2-2.3), writes the next state buffer and the bit-packed mask.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <cstdlib>

#include "dmsgm_internal.h"

namespace dmsgm {

// NVTX range over an entry point (free when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

// Fault injection for failure-handling tests: the n-th frame launch
// ("launch:n") or the n-th handle allocation ("alloc:n") of the process fails
// with DMSGM_ERR_CUDA / DMSGM_ERR_OOM before anything reaches the GPU.  Set
// by dmsgm_fault_inject or, at the first use, the DMSGM_FAULT_INJECT
// environment variable; off by default.
struct FaultPlan {
    std::atomic<long> launch_at{0}, alloc_at{0}, launches{0}, allocs{0};
};
static FaultPlan g_fault;

static void fault_parse(const char* spec) {
    g_fault.launch_at = 0;
    g_fault.alloc_at = 0;
    g_fault.launches = 0;
    g_fault.allocs = 0;
    if (!spec) return;
    const char* p = spec;
    while (*p) {
        const char* colon = std::strchr(p, ':');
        if (!colon) break;
        const long v = std::strtol(colon + 1, nullptr, 10);
        if (!std::strncmp(p, "launch", colon - p)) g_fault.launch_at = v;
        if (!std::strncmp(p, "alloc", colon - p)) g_fault.alloc_at = v;
        const char* comma = std::strchr(colon, ',');
        if (!comma) break;
        p = comma + 1;
    }
}

static void fault_init() {
    static std::once_flag once;
    std::call_once(once, [] { fault_parse(std::getenv("DMSGM_FAULT_INJECT")); });
}

static bool fault_launch() {
    fault_init();
    const long at = g_fault.launch_at.load();
    return at > 0 && ++g_fault.launches == at;
}

static bool fault_alloc() {
    fault_init();
    const long at = g_fault.alloc_at.load();
    return at > 0 && ++g_fault.allocs == at;
}

static thread_local char g_err[512];

int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}
void clear_error() { g_err[0] = 0; }

// ------------------------------------------------------------------ kernel
// Diagnostic kernel: waits on a barrier that nothing completes, so the
// bounded wait must give up after timeout_ns and report it.
__global__ void dmsgm_selftest_wait_kernel(int* status, unsigned long long timeout_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0, timeout_ns);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(status, kStatusWaitTimeout);
}

// The per-tile kernel of the handle's block size (dmsgm_step.cuh).
static cudaError_t launch_step(dmsgm_ctx* h, const CUtensorMap& tmap, const StreamArgs& a,
                               const Coef& k, cudaStream_t s, bool pdl) {
    switch (h->B) {
        case 1: return launch_step_block<1>(h, tmap, a, k, s, pdl);
        case 2: return launch_step_block<2>(h, tmap, a, k, s, pdl);
        case 4: return launch_step_block<4>(h, tmap, a, k, s, pdl);
        case 8: return launch_step_block<8>(h, tmap, a, k, s, pdl);
        case 16: return launch_step_block<16>(h, tmap, a, k, s, pdl);
        default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------------ helpers
// Block 1, 2, 4, 8 or 16; W a multiple of 16 (TMA row pitch; so also of
// the block); any H (a bottom block row may be cut by the frame edge).
static bool valid_dims(int W, int H, int B) {
    return W > 0 && H > 0 && (B == 1 || B == 2 || B == 4 || B == 8 || B == 16) && W % 16 == 0 &&
           W <= (1 << 20) && H <= (1 << 20);
}

// Tile height when dmsgm_opts.tile_rows is 0.
// 4 B rows (one strip row per warp, 4 warps) for blocks 1, 2 and 16: their
// lanes hold many models, and the higher occupancy of the small tile wins
// (3840x2160 B = 1: 152 us per frame against 179 us with 8-row tiles; B = 2:
// 30.4 against 35.3 us); 32 rows for blocks 4 and 8.
static int default_tile_rows(int B) { return B == 1 ? 4 : B == 2 ? 8 : B == 16 ? 64 : 32; }

static size_t buf_bytes(size_t N, int prec) {
    return state_buf_bytes(N, prec == DMSGM_STATE_FP16 ? 2 : 4);
}

static void carve(dmsgm_ctx* h) {
    const int s = h->prec == DMSGM_STATE_FP16 ? 2 : 4;
    h->status_dev = reinterpret_cast<int*>(h->mem);
    h->flags_dev = reinterpret_cast<int*>(static_cast<char*>(h->mem) + 256);
    for (int b = 0; b < 2; ++b)
        h->buf[b] = state_buf(static_cast<char*>(h->mem), h->W, h->H, h->B, s, b);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// Tensor map of a W x H uint8 frame with a kTileW x rows box (rows 0: the
// handle's tile_rows).
static int encode_frame_map(const dmsgm_ctx* h, const void* frame, CUtensorMap* out, int rows = 0) {
    auto enc = encode_fn();
    if (!enc) return fail(DMSGM_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    cuuint64_t dims[2] = {cuuint64_t(h->W), cuuint64_t(h->H)};
    cuuint64_t strides[1] = {cuuint64_t(h->W)};
    cuuint32_t box[2] = {cuuint32_t(kTileW), cuuint32_t(rows ? rows : h->tile_rows)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(out, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(frame), dims,
                     strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(DMSGM_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", int(r));
    return DMSGM_OK;
}

static int frame_map(dmsgm_ctx* h, const void* frame, const CUtensorMap** out) {
    for (int i = 0; i < kTmapCache; ++i)
        if (h->tmap[i].ptr == frame) { *out = &h->tmap[i].map; return DMSGM_OK; }
    const int slot = h->tmap_next;
    h->tmap_next = (h->tmap_next + 1) % kTmapCache;
    h->tmap[slot].ptr = nullptr;
    int rc = encode_frame_map(h, frame, &h->tmap[slot].map);
    if (rc) return rc;
    h->tmap[slot].ptr = frame;
    *out = &h->tmap[slot].map;
    return DMSGM_OK;
}

int batch_frame_map(dmsgm_ctx* h, const void* frame, int rows, CUtensorMap* out) {
    for (int i = 0; i < 4; ++i)
        if (h->bmap[i].ptr == frame && h->bmap[i].rows == rows) { *out = h->bmap[i].map; return DMSGM_OK; }
    const int slot = h->bmap_next;
    h->bmap_next = (h->bmap_next + 1) % 4;
    h->bmap[slot].ptr = nullptr;
    h->bmap[slot].rows = rows;
    int rc = encode_frame_map(h, frame, &h->bmap[slot].map, rows);
    if (rc) return rc;
    h->bmap[slot].ptr = frame;
    *out = h->bmap[slot].map;
    return DMSGM_OK;
}

bool make_coef(const double m[9], int B, Coef* c, int* affine) {
    for (int i = 0; i < 9; ++i)
        if (!std::isfinite(m[i])) return false;
    double v[9];
    *affine = 0;
    if (m[6] == 0.0 && m[7] == 0.0 && m[8] > 0.0) {
        // affine: block-unit displacement ex = ax*bx + bx_*by + cx (and ey)
        const double ax = m[0] / m[8] - 1.0, bxx = m[1] / m[8];
        const double ay = m[3] / m[8], byy = m[4] / m[8] - 1.0;
        const double cx = 0.5 * ax + 0.5 * bxx + m[2] / (m[8] * B);
        const double cy = 0.5 * ay + 0.5 * byy + m[5] / (m[8] * B);
        const double lim = 1.0 / 31.0;   // per-lane step rounding below 4.8e-7 blocks (affine_origin)
        const double far = 1.0e6;
        if (std::fabs(ax) <= lim && std::fabs(ay) <= lim && std::fabs(bxx) < far &&
            std::fabs(byy) < far && std::fabs(cx) < far && std::fabs(cy) < far) {
            const double a[6] = {ax, bxx, cx, ay, byy, cy};
            for (int i = 0; i < 6; ++i) {
                const float hi = float(a[i]);
                c->c[2 * i] = hi;
                c->c[2 * i + 1] = float(a[i] - double(hi));
            }
            for (int i = 12; i < 18; ++i) c->c[i] = 0.f;
            *affine = 1;
            return true;
        }
    }
    // general: pixel-space displacement form
    const double g[9] = {m[0] - m[8], m[1], m[2], m[3], m[4] - m[8], m[5], m[6], m[7], m[8]};
    for (int i = 0; i < 9; ++i) v[i] = g[i];
    for (int i = 0; i < 9; ++i) {
        const float hi = float(v[i]);
        const float lo = float(v[i] - double(hi));
        if (!std::isfinite(hi) || !std::isfinite(lo)) return false;
        c->c[2 * i] = hi;
        c->c[2 * i + 1] = lo;
    }
    return true;
}

void fill_args(const dmsgm_ctx* h, int affine, uint32_t* mask_dev, StreamArgs* a) {
    a->prev = h->buf[h->parity];
    a->next = h->buf[h->parity ^ 1];
    a->mask = mask_dev;
    a->W = h->W;
    a->H = h->H;
    a->Gx = h->Gx;
    a->Gy = h->Gy;
    a->mask_words = (h->W + 31) / 32;
    a->first = h->initialized ? 0 : 1;
    a->affine = affine;
    a->age_max = h->age_max;
    a->theta_s = h->theta_s;
    a->theta_d = h->theta_d;
    a->spread = h->mix_spread;
}

void advance(dmsgm_ctx* h) {
    h->parity ^= 1;
    h->initialized = true;
    h->frames++;
}

bool displacement_bound(const double m[9], int W, int H, int B, double* ex, double* ey) {
    // Block centres fill the rectangle [x0, x1] x [y0, y1].  The
    // displacement of a centre (x, y) is (N_x / Z, N_y / Z) with
    //   Z   = h20 x + h21 y + h22,
    //   N_x = (h00 - h22) x + h01 y + h02 - (h20 x + h21 y) x,
    //   N_y = h10 x + (h11 - h22) y + h12 - (h20 x + h21 y) y.
    // Z and the linear parts reach their extremes at the corners; with
    // x, y >= 0 the quadratic parts are at most |h20| x1^2 + |h21| x1 y1
    // (and |h20| x1 y1 + |h21| y1^2) in magnitude.  For an affine map this is
    // the exact maximum.
    const double x0 = 0.5 * B, x1 = (W / B - 0.5) * B;
    const double y0 = 0.5 * B, y1 = (grid_rows(H, B) - 0.5) * B;
    const double cx[4] = {x0, x1, x0, x1}, cy[4] = {y0, y0, y1, y1};
    double zmin = HUGE_VAL, lx = 0.0, ly = 0.0;
    for (int i = 0; i < 4; ++i) {
        const double z = m[6] * cx[i] + m[7] * cy[i] + m[8];
        zmin = std::min(zmin, z);
        lx = std::max(lx, std::fabs((m[0] - m[8]) * cx[i] + m[1] * cy[i] + m[2]));
        ly = std::max(ly, std::fabs(m[3] * cx[i] + (m[4] - m[8]) * cy[i] + m[5]));
    }
    if (!(zmin > 0.0)) return false;
    const double qx = std::fabs(m[6]) * x1 * x1 + std::fabs(m[7]) * x1 * y1;
    const double qy = std::fabs(m[6]) * x1 * y1 + std::fabs(m[7]) * y1 * y1;
    *ex = (lx + qx) / zmin / B;
    *ey = (ly + qy) / zmin / B;
    return std::isfinite(*ex) && std::isfinite(*ey);
}

static int process_one(dmsgm_ctx* h, const uint8_t* frame_dev, const double* H3x3,
                       uint32_t* mask_dev, cudaStream_t s) {
    Coef c;
    int affine = 0;
    if (!make_coef(H3x3, h->B, &c, &affine))
        return fail(DMSGM_ERR_INVALID_ARG, "homography is not finite in FP32");
    if (fault_launch()) return fail(DMSGM_ERR_CUDA, "injected launch failure (DMSGM_FAULT_INJECT)");
    int rc;
    bool pdl = h->use_pdl != 0;
    if (h->pre_fused) {
        // the step kernel filters its own tile (Sec. 2.1 preprocessing)
        StreamArgs a;
        fill_args(h, affine, mask_dev, &a);
        const cudaError_t e = h->B == 4 ? launch_step_pre_block<4>(h, frame_dev, a, c, s, pdl)
                                        : launch_step_pre_block<8>(h, frame_dev, a, c, s, pdl);
        if (e != cudaSuccess)
            return fail(DMSGM_ERR_CUDA, "kernel launch failed: %s", cudaGetErrorString(e));
        h->last_kernel = DMSGM_KERNEL_TILE;
        advance(h);
        return DMSGM_OK;
    }
    if (h->pre_buf) {
        // Sec. 2.1 preprocessing into the handle's scratch frame (two of
        // them, alternating, so a frame's filter never overwrites the pixels
        // the previous frame's kernel may still read); the step then waits
        // for the filter in plain stream order
        uint8_t* dst = h->pre_buf + size_t(h->frames & 1) * h->W * h->H;
        rc = launch_prefilter(frame_dev, dst, h->W, h->H, h->pre_gauss, h->pre_sigma,
                              h->pre_median, s);
        if (rc) return rc;
        frame_dev = dst;
        pdl = false;
    }
    const CUtensorMap* tm = nullptr;
    rc = frame_map(h, frame_dev, &tm);
    if (rc) return rc;
    StreamArgs a;
    fill_args(h, affine, mask_dev, &a);
    cudaError_t e = launch_step(h, *tm, a, c, s, pdl);
    if (e != cudaSuccess)
        return fail(DMSGM_ERR_CUDA, "kernel launch failed: %s", cudaGetErrorString(e));
    h->last_kernel = DMSGM_KERNEL_TILE;
    advance(h);
    return DMSGM_OK;
}

static void free_stage(dmsgm_ctx* h) {
    HostStage& st = h->stage;
    for (int i = 0; i < 2; ++i) {
        if (st.frames[i]) cudaFree(st.frames[i]);
        if (st.masks[i]) cudaFree(st.masks[i]);
        if (st.ev_in[i]) cudaEventDestroy(st.ev_in[i]);
        if (st.ev_k[i]) cudaEventDestroy(st.ev_k[i]);
        if (st.ev_out[i]) cudaEventDestroy(st.ev_out[i]);
    }
    if (st.ev_start) cudaEventDestroy(st.ev_start);
    if (st.h2d) cudaStreamDestroy(st.h2d);
    if (st.d2h) cudaStreamDestroy(st.d2h);
    st = HostStage();
}

static int ensure_stage(dmsgm_ctx* h) {
    HostStage& st = h->stage;
    if (st.slots) return DMSGM_OK;
    const size_t fbytes = size_t(h->W) * h->H;
    const size_t mbytes = size_t(h->H) * ((h->W + 31) / 32) * 4;
    // chunks of ~16 MB of frames, 1..32 frames
    int chunk = int(std::max<size_t>(1, std::min<size_t>(32, (16u << 20) / fbytes)));
    st.chunk = chunk;
    auto bad = [&](cudaError_t e) {
        free_stage(h);
        return fail(e == cudaErrorMemoryAllocation ? DMSGM_ERR_OOM : DMSGM_ERR_CUDA,
                    "staging setup failed: %s", cudaGetErrorString(e));
    };
    cudaError_t e;
    for (int i = 0; i < 2; ++i) {
        if ((e = cudaMalloc(&st.frames[i], fbytes * chunk)) != cudaSuccess) return bad(e);
        if ((e = cudaMalloc(&st.masks[i], mbytes * chunk)) != cudaSuccess) return bad(e);
        if ((e = cudaEventCreateWithFlags(&st.ev_in[i], cudaEventDisableTiming)) != cudaSuccess) return bad(e);
        if ((e = cudaEventCreateWithFlags(&st.ev_k[i], cudaEventDisableTiming)) != cudaSuccess) return bad(e);
        if ((e = cudaEventCreateWithFlags(&st.ev_out[i], cudaEventDisableTiming)) != cudaSuccess) return bad(e);
    }
    if ((e = cudaEventCreateWithFlags(&st.ev_start, cudaEventDisableTiming)) != cudaSuccess) return bad(e);
    if ((e = cudaStreamCreateWithFlags(&st.h2d, cudaStreamNonBlocking)) != cudaSuccess) return bad(e);
    if ((e = cudaStreamCreateWithFlags(&st.d2h, cudaStreamNonBlocking)) != cudaSuccess) return bad(e);
    st.slots = 2;
    return DMSGM_OK;
}

}  // namespace dmsgm

using namespace dmsgm;

// ================================================================== C ABI
extern "C" {

const char* dmsgm_last_error(void) { return g_err; }

const char* dmsgm_version(void) { return "dmsgm-gb300 0.1 (sm_103a)"; }

void dmsgm_fault_inject(const char* spec) {
    fault_init();
    fault_parse(spec);
}

size_t dmsgm_state_bytes(int W, int H, int B, int prec) {
    if (!valid_dims(W, H, B) || (prec != DMSGM_STATE_FP32 && prec != DMSGM_STATE_FP16)) return 0;
    const size_t N = size_t(W / B) * grid_rows(H, B);
    return 256 + seq_flags_bytes(W, H, B) + 2 * buf_bytes(N, prec);
}

size_t dmsgm_host_state_bytes(int W, int H, int B, int prec) {
    if (!valid_dims(W, H, B) || (prec != DMSGM_STATE_FP32 && prec != DMSGM_STATE_FP16)) return 0;
    const size_t N = size_t(W / B) * grid_rows(H, B);
    return N * (4 * (prec == DMSGM_STATE_FP16 ? 2 : 4) + 2);
}

int dmsgm_create(int W, int H, int B, float ts, float td, int age_max, dmsgm_t* out) {
    return dmsgm_create_ex(W, H, B, ts, td, age_max, nullptr, out);
}

int dmsgm_create_ex(int W, int H, int B, float ts, float td, int age_max, const dmsgm_opts* o,
                    dmsgm_t* out) {
    clear_error();
    NvtxRange nvtx("dmsgm_create");
    if (!out) return fail(DMSGM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!valid_dims(W, H, B))
        return fail(DMSGM_ERR_INVALID_ARG,
                    "invalid size %dx%d block %d (need block 1, 2, 4, 8 or 16, W%%16==0, "
                    "W and H <= 2^20)", W, H, B);
    if (!(std::isfinite(ts) && ts > 0) || !(std::isfinite(td) && td > 0))
        return fail(DMSGM_ERR_INVALID_ARG, "theta_s and theta_d must be finite and > 0");
    if (age_max < 1 || age_max > 255) return fail(DMSGM_ERR_INVALID_ARG, "age_max must be in [1, 255]");
    dmsgm_opts opts = {};
    if (o) opts = *o;
    if (opts.precision != DMSGM_STATE_FP32 && opts.precision != DMSGM_STATE_FP16)
        return fail(DMSGM_ERR_INVALID_ARG, "unknown precision %d", opts.precision);
    const int tile_rows = opts.tile_rows ? opts.tile_rows : default_tile_rows(B);
    if (!(tile_rows == 4 * B || tile_rows == 8 * B || tile_rows == 16 * B) || tile_rows > 256)
        return fail(DMSGM_ERR_INVALID_ARG, "tile_rows %d must be 4, 8 or 16 times the block and <= 256",
                    tile_rows);
    if (fault_alloc()) return fail(DMSGM_ERR_OOM, "injected allocation failure (DMSGM_FAULT_INJECT)");
    const size_t need = dmsgm_state_bytes(W, H, B, opts.precision);
    if (opts.state_mem) {
        if (opts.state_bytes < need)
            return fail(DMSGM_ERR_INVALID_ARG, "state_mem holds %zu bytes, need %zu", opts.state_bytes, need);
        if (reinterpret_cast<uintptr_t>(opts.state_mem) % 256)
            return fail(DMSGM_ERR_INVALID_ARG, "state_mem must be 256-byte aligned");
    }
    int dev = 0;
    DMSGM_CUDA_TRY(cudaGetDevice(&dev));
    dmsgm_ctx* h = new (std::nothrow) dmsgm_ctx();
    if (!h) return fail(DMSGM_ERR_OOM, "host allocation failed");
    h->W = W; h->H = H; h->B = B; h->Gx = W / B; h->Gy = grid_rows(H, B);
    h->prec = opts.precision;
    h->age_max = age_max;
    h->theta_s = ts; h->theta_d = td;
    h->device = dev;
    h->tile_rows = tile_rows;
    h->use_pdl = opts.use_pdl > 0 ? 1 : 0;
    if (opts.seq_tile_rows && !(opts.seq_tile_rows % (8 * B) == 0 && opts.seq_tile_rows <= 256 &&
                                ((opts.seq_tile_rows / (8 * B)) & (opts.seq_tile_rows / (8 * B) - 1)) == 0)) {
        delete h;
        return fail(DMSGM_ERR_INVALID_ARG, "seq_tile_rows %d invalid", opts.seq_tile_rows);
    }
    h->seq_tile_rows = opts.seq_tile_rows;
    if (opts.kernel < DMSGM_KERNEL_AUTO || opts.kernel > DMSGM_KERNEL_TILE) {
        delete h;
        return fail(DMSGM_ERR_INVALID_ARG, "unknown kernel %d", opts.kernel);
    }
    h->kernel = opts.kernel;
    h->mix_spread = opts.mix_spread ? 1 : 0;
    if (opts.checked != 0 && opts.checked != 1) {
        delete h;
        return fail(DMSGM_ERR_INVALID_ARG, "checked must be 0 or 1");
    }
    h->checked = opts.checked;
    if (h->checked && (h->mix_spread || opts.pre_gauss || opts.pre_median)) {
        delete h;
        return fail(DMSGM_ERR_INVALID_ARG, "the checked build covers the plain frame step "
                    "(no mixture option, no preprocessing)");
    }
    if ((opts.pre_gauss && (opts.pre_gauss < 3 || opts.pre_gauss > 15 || opts.pre_gauss % 2 == 0 ||
                            !(opts.pre_sigma > 0.0) || !std::isfinite(opts.pre_sigma))) ||
        (opts.pre_median != 0 && opts.pre_median != 1) ||
        (opts.pre_separate != 0 && opts.pre_separate != 1)) {
        delete h;
        return fail(DMSGM_ERR_INVALID_ARG, "preprocessing: Gaussian size 0 or odd 3..15 with sigma > 0, "
                    "median 0 or 1");
    }
    h->pre_gauss = opts.pre_gauss;
    h->pre_sigma = opts.pre_sigma;
    h->pre_median = opts.pre_median;
    if (h->pre_gauss || h->pre_median) {
        if (!make_filt_args(h->pre_gauss, h->pre_sigma, h->pre_median, &h->filt, &h->pre_half)) {
            delete h;
            return fail(DMSGM_ERR_INVALID_ARG, "preprocessing: invalid Gaussian");
        }
        h->pre_fused = !opts.pre_separate && (B == 4 || B == 8) && tile_rows == 32 &&
                       !h->mix_spread && h->pre_half <= 3;
    }
    h->state_bytes = need;
    if (opts.state_mem) {
        h->mem = opts.state_mem;
        h->owns_mem = false;
    } else {
        cudaError_t e = cudaMalloc(&h->mem, need);
        if (e != cudaSuccess) {
            delete h;
            return fail(e == cudaErrorMemoryAllocation ? DMSGM_ERR_OOM : DMSGM_ERR_CUDA,
                        "cudaMalloc(%zu) failed: %s", need, cudaGetErrorString(e));
        }
        h->owns_mem = true;
    }
    if ((h->pre_gauss || h->pre_median) && !h->pre_fused) {   // two scratch frames for the separate pass
        cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&h->pre_buf), 2 * size_t(W) * H);
        if (e != cudaSuccess) {
            if (h->owns_mem) cudaFree(h->mem);
            delete h;
            return fail(e == cudaErrorMemoryAllocation ? DMSGM_ERR_OOM : DMSGM_ERR_CUDA,
                        "cudaMalloc of the preprocessing frames failed: %s", cudaGetErrorString(e));
        }
    }
    carve(h);
    // Only the control block needs a defined value (the status word); the
    // state buffers are written by the first process() or set_state().  A
    // synchronous copy from the host orders it without a device-wide sync.
    static const unsigned char zeros[256] = {0};
    cudaError_t e = cudaMemcpy(h->mem, zeros, sizeof zeros, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        if (h->owns_mem) cudaFree(h->mem);
        delete h;
        return fail(DMSGM_ERR_CUDA, "state init failed: %s", cudaGetErrorString(e));
    }
    h->parity = 0;
    h->initialized = false;
    h->frames = 0;
    h->tmap_next = 0;
    *out = h;
    return DMSGM_OK;
}

int dmsgm_destroy(dmsgm_t h) {
    clear_error();
    if (!h) return DMSGM_OK;
    DeviceGuard g(h->device);
    // Memory the handle owns may still be in use by queued work; memory the
    // caller lent it is the caller's to order.
    cudaError_t e = cudaSuccess;
    if (h->owns_mem || h->stage.slots || h->pre_buf) e = cudaDeviceSynchronize();
    free_stage(h);
    if (h->owns_mem && h->mem) cudaFree(h->mem);
    if (h->pre_buf) cudaFree(h->pre_buf);
    delete h;
    if (e != cudaSuccess) return fail(DMSGM_ERR_CUDA, "synchronize failed: %s", cudaGetErrorString(e));
    return DMSGM_OK;
}

int dmsgm_process(dmsgm_t h, const uint8_t* frame_dev, const double H3x3[9], uint32_t* mask_dev,
                  void* stream) {
    clear_error();
    NvtxRange nvtx("dmsgm_process");
    if (!h || !frame_dev || !H3x3 || !mask_dev) return fail(DMSGM_ERR_INVALID_ARG, "NULL argument");
    if (reinterpret_cast<uintptr_t>(frame_dev) % 16)
        return fail(DMSGM_ERR_INVALID_ARG, "frame must be 16-byte aligned");
    if (reinterpret_cast<uintptr_t>(mask_dev) % 4)
        return fail(DMSGM_ERR_INVALID_ARG, "mask must be 4-byte aligned");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(DMSGM_ERR_CUDA, "cannot select device %d", h->device);
    return process_one(h, frame_dev, H3x3, mask_dev, static_cast<cudaStream_t>(stream));
}

int dmsgm_process_seq(dmsgm_t h, const uint8_t* frames_dev, int n, const double* Hs,
                      uint32_t* masks_dev, void* stream) {
    clear_error();
    NvtxRange nvtx("dmsgm_process_seq");
    if (!h || n < 0 || (n > 0 && (!frames_dev || !Hs || !masks_dev)))
        return fail(DMSGM_ERR_INVALID_ARG, "invalid argument");
    if (reinterpret_cast<uintptr_t>(frames_dev) % 16)
        return fail(DMSGM_ERR_INVALID_ARG, "frames must be 16-byte aligned");
    if (reinterpret_cast<uintptr_t>(masks_dev) % 4)
        return fail(DMSGM_ERR_INVALID_ARG, "masks must be 4-byte aligned");
    for (long i = 0; i < 9L * n; ++i)
        if (!std::isfinite(Hs[i])) return fail(DMSGM_ERR_INVALID_ARG, "homography %ld is not finite", i / 9);
    if (n == 0) return DMSGM_OK;
    DeviceGuard g(h->device);
    if (!g.ok) return fail(DMSGM_ERR_CUDA, "cannot select device %d", h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = launch_seq(h, frames_dev, n, Hs, masks_dev, s, h->flags_dev);
    if (rc != DMSGM_ERR_UNSUPPORTED) return rc;
    // the tiles do not fit the GPU at once: one launch per frame instead
    clear_error();
    const size_t fbytes = size_t(h->W) * h->H, mwords = size_t(h->H) * ((h->W + 31) / 32);
    for (int t = 0; t < n; ++t) {
        rc = process_one(h, frames_dev + t * fbytes, Hs + 9 * size_t(t), masks_dev + t * mwords, s);
        if (rc) return rc;
    }
    return DMSGM_OK;
}

int dmsgm_process_host(dmsgm_t h, const uint8_t* frames_host, int n, const double* Hs,
                       uint32_t* masks_host, void* stream) {
    clear_error();
    NvtxRange nvtx("dmsgm_process_host");
    if (!h || n < 0 || (n > 0 && (!frames_host || !Hs || !masks_host)))
        return fail(DMSGM_ERR_INVALID_ARG, "invalid argument");
    for (long i = 0; i < 9L * n; ++i)
        if (!std::isfinite(Hs[i])) return fail(DMSGM_ERR_INVALID_ARG, "homography %ld is not finite", i / 9);
    if (n == 0) return DMSGM_OK;
    DeviceGuard g(h->device);
    if (!g.ok) return fail(DMSGM_ERR_CUDA, "cannot select device %d", h->device);
    int rc = ensure_stage(h);
    if (rc) return rc;
    HostStage& st = h->stage;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t fbytes = size_t(h->W) * h->H;
    const size_t mwords = size_t(h->H) * ((h->W + 31) / 32);
    DMSGM_CUDA_TRY(cudaEventRecord(st.ev_start, s));
    DMSGM_CUDA_TRY(cudaStreamWaitEvent(st.h2d, st.ev_start, 0));
    for (int c0 = 0, ci = 0; c0 < n; c0 += st.chunk, ++ci) {
        const int cnt = std::min(st.chunk, n - c0);
        const int sl = ci & 1;
        // frames of this chunk -> slot sl, once the kernels that read the
        // slot two chunks ago are done
        DMSGM_CUDA_TRY(cudaStreamWaitEvent(st.h2d, st.ev_k[sl], 0));
        DMSGM_CUDA_TRY(cudaMemcpyAsync(st.frames[sl], frames_host + size_t(c0) * fbytes,
                                       size_t(cnt) * fbytes, cudaMemcpyHostToDevice, st.h2d));
        DMSGM_CUDA_TRY(cudaEventRecord(st.ev_in[sl], st.h2d));
        DMSGM_CUDA_TRY(cudaStreamWaitEvent(s, st.ev_in[sl], 0));
        DMSGM_CUDA_TRY(cudaStreamWaitEvent(s, st.ev_out[sl], 0));
        for (int f = 0; f < cnt; ++f) {
            rc = process_one(h, st.frames[sl] + size_t(f) * fbytes, Hs + 9 * size_t(c0 + f),
                             st.masks[sl] + size_t(f) * mwords, s);
            if (rc) return rc;
        }
        DMSGM_CUDA_TRY(cudaEventRecord(st.ev_k[sl], s));
        DMSGM_CUDA_TRY(cudaStreamWaitEvent(st.d2h, st.ev_k[sl], 0));
        DMSGM_CUDA_TRY(cudaMemcpyAsync(masks_host + size_t(c0) * mwords, st.masks[sl],
                                       size_t(cnt) * mwords * 4, cudaMemcpyDeviceToHost, st.d2h));
        DMSGM_CUDA_TRY(cudaEventRecord(st.ev_out[sl], st.d2h));
    }
    DMSGM_CUDA_TRY(cudaStreamWaitEvent(s, st.ev_out[0], 0));
    DMSGM_CUDA_TRY(cudaStreamWaitEvent(s, st.ev_out[1], 0));
    return DMSGM_OK;
}

int dmsgm_process_batch(int n, const dmsgm_t* hs, const uint8_t* const* frames_dev,
                        const double* Hs, uint32_t* const* masks_dev, void* stream) {
    return dmsgm_process_batch_ex(n, hs, frames_dev, Hs, masks_dev, nullptr, stream);
}

int dmsgm_process_batch_ex(int n, const dmsgm_t* hs, const uint8_t* const* frames_dev,
                           const double* Hs, uint32_t* const* masks_dev,
                           const dmsgm_batch_opts* opts, void* stream) {
    clear_error();
    NvtxRange nvtx("dmsgm_process_batch");
    if (n < 0 || n > DMSGM_MAX_BATCH) return fail(DMSGM_ERR_INVALID_ARG, "n=%d out of range", n);
    if (n == 0) return DMSGM_OK;
    if (!hs || !frames_dev || !Hs || !masks_dev) return fail(DMSGM_ERR_INVALID_ARG, "NULL argument");
    for (int i = 0; i < n; ++i) {
        if (!hs[i] || !frames_dev[i] || !masks_dev[i])
            return fail(DMSGM_ERR_INVALID_ARG, "NULL entry %d", i);
        if (reinterpret_cast<uintptr_t>(frames_dev[i]) % 16 || reinterpret_cast<uintptr_t>(masks_dev[i]) % 4)
            return fail(DMSGM_ERR_INVALID_ARG, "entry %d misaligned", i);
        if (hs[i]->device != hs[0]->device)
            return fail(DMSGM_ERR_INVALID_ARG, "handles on different devices");
        for (int j = 0; j < i; ++j)
            if (hs[j] == hs[i]) return fail(DMSGM_ERR_INVALID_ARG, "handle %d appears twice", i);
        Coef c;
        int affine = 0;
        if (!make_coef(Hs + 9 * size_t(i), hs[i]->B, &c, &affine))
            return fail(DMSGM_ERR_INVALID_ARG, "homography %d is not finite in FP32", i);
    }
    DeviceGuard g(hs[0]->device);
    if (!g.ok) return fail(DMSGM_ERR_CUDA, "cannot select device %d", hs[0]->device);
    dmsgm_batch_opts o = {};
    if (opts) o = *opts;
    if (fault_launch()) return fail(DMSGM_ERR_CUDA, "injected launch failure (DMSGM_FAULT_INJECT)");
    return launch_batch(n, hs, frames_dev, Hs, masks_dev, o, static_cast<cudaStream_t>(stream));
}

int dmsgm_process_batch_host(int n, const dmsgm_t* hs, const uint8_t* const* frames_host,
                             uint8_t* const* frames_dev, const double* Hs,
                             uint32_t* const* masks_dev, uint32_t* const* masks_host,
                             const dmsgm_batch_opts* opts, void* h2d, void* compute, void* d2h) {
    clear_error();
    NvtxRange nvtx("dmsgm_process_batch_host");
    if (n < 0 || n > DMSGM_MAX_BATCH) return fail(DMSGM_ERR_INVALID_ARG, "n=%d out of range", n);
    if (n == 0) return DMSGM_OK;
    if (!hs || !frames_host || !frames_dev || !masks_dev || !masks_host)
        return fail(DMSGM_ERR_INVALID_ARG, "NULL argument");
    if (h2d == compute || compute == d2h || h2d == d2h)
        return fail(DMSGM_ERR_INVALID_ARG, "the three streams must differ");
    for (int i = 0; i < n; ++i)
        if (!hs[i] || !frames_host[i] || !masks_host[i])
            return fail(DMSGM_ERR_INVALID_ARG, "NULL entry %d", i);
    DeviceGuard g(hs[0]->device);
    if (!g.ok) return fail(DMSGM_ERR_CUDA, "cannot select device %d", hs[0]->device);
    // per-thread events, reused across calls (a re-record only moves the
    // point later waits refer to; waits already enqueued keep theirs)
    static thread_local cudaEvent_t ev_in = nullptr, ev_k = nullptr;
    if (!ev_in) {
        DMSGM_CUDA_TRY(cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming));
        DMSGM_CUDA_TRY(cudaEventCreateWithFlags(&ev_k, cudaEventDisableTiming));
    }
    cudaStream_t sh = static_cast<cudaStream_t>(h2d), sc = static_cast<cudaStream_t>(compute),
                 sd = static_cast<cudaStream_t>(d2h);
    for (int i = 0; i < n; ++i)
        DMSGM_CUDA_TRY(cudaMemcpyAsync(frames_dev[i], frames_host[i], size_t(hs[i]->W) * hs[i]->H,
                                       cudaMemcpyHostToDevice, sh));
    DMSGM_CUDA_TRY(cudaEventRecord(ev_in, sh));
    DMSGM_CUDA_TRY(cudaStreamWaitEvent(sc, ev_in, 0));
    int rc = dmsgm_process_batch_ex(n, hs, frames_dev, Hs, masks_dev, opts, compute);
    if (rc) return rc;
    DMSGM_CUDA_TRY(cudaEventRecord(ev_k, sc));
    DMSGM_CUDA_TRY(cudaStreamWaitEvent(sd, ev_k, 0));
    for (int i = 0; i < n; ++i)
        DMSGM_CUDA_TRY(cudaMemcpyAsync(masks_host[i], masks_dev[i],
                                       size_t(hs[i]->H) * ((hs[i]->W + 31) / 32) * 4,
                                       cudaMemcpyDeviceToHost, sd));
    return DMSGM_OK;
}

int dmsgm_selftest_wait(dmsgm_t h, unsigned long long timeout_ns, void* stream) {
    clear_error();
    if (!h) return fail(DMSGM_ERR_INVALID_ARG, "NULL handle");
    if (timeout_ns > 1000000000ull) return fail(DMSGM_ERR_INVALID_ARG, "timeout above 1 s");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(DMSGM_ERR_CUDA, "cannot select device %d", h->device);
    dmsgm_selftest_wait_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(h->status_dev,
                                                                              timeout_ns);
    DMSGM_CUDA_TRY(cudaGetLastError());
    return DMSGM_OK;
}

int dmsgm_get_state(dmsgm_t h, void* host_buf, size_t bytes) {
    clear_error();
    if (!h || !host_buf) return fail(DMSGM_ERR_INVALID_ARG, "NULL argument");
    const size_t need = dmsgm_host_state_bytes(h->W, h->H, h->B, h->prec);
    if (bytes < need) return fail(DMSGM_ERR_INVALID_ARG, "buffer holds %zu bytes, need %zu", bytes, need);
    DeviceGuard g(h->device);
    DMSGM_CUDA_TRY(cudaDeviceSynchronize());
    const size_t N = size_t(h->Gx) * h->Gy, s = h->prec == DMSGM_STATE_FP16 ? 2 : 4;
    const StateBuf& sb = h->buf[h->parity];
    char* p = static_cast<char*>(host_buf);
    const void* src[3] = {sb.mu, sb.var, sb.age};
    const size_t len[3] = {2 * N * s, 2 * N * s, 2 * N};
    for (int i = 0; i < 3; ++i) {
        DMSGM_CUDA_TRY(cudaMemcpy(p, src[i], len[i], cudaMemcpyDeviceToHost));
        p += len[i];
    }
    return DMSGM_OK;
}

int dmsgm_set_state(dmsgm_t h, const void* host_buf, size_t bytes) {
    clear_error();
    if (!h || !host_buf) return fail(DMSGM_ERR_INVALID_ARG, "NULL argument");
    const size_t need = dmsgm_host_state_bytes(h->W, h->H, h->B, h->prec);
    if (bytes < need) return fail(DMSGM_ERR_INVALID_ARG, "buffer holds %zu bytes, need %zu", bytes, need);
    DeviceGuard g(h->device);
    DMSGM_CUDA_TRY(cudaDeviceSynchronize());
    const size_t N = size_t(h->Gx) * h->Gy, s = h->prec == DMSGM_STATE_FP16 ? 2 : 4;
    const StateBuf& sb = h->buf[h->parity];
    const char* p = static_cast<const char*>(host_buf);
    void* dst[3] = {sb.mu, sb.var, sb.age};
    const size_t len[3] = {2 * N * s, 2 * N * s, 2 * N};
    for (int i = 0; i < 3; ++i) {
        DMSGM_CUDA_TRY(cudaMemcpy(dst[i], p, len[i], cudaMemcpyHostToDevice));
        p += len[i];
    }
    DMSGM_CUDA_TRY(cudaDeviceSynchronize());
    h->initialized = true;
    return DMSGM_OK;
}

int dmsgm_reset(dmsgm_t h) {
    clear_error();
    if (!h) return fail(DMSGM_ERR_INVALID_ARG, "NULL handle");
    h->initialized = false;
    h->frames = 0;
    return DMSGM_OK;
}

int dmsgm_get_info(dmsgm_t h, dmsgm_info* o) {
    clear_error();
    if (!h || !o) return fail(DMSGM_ERR_INVALID_ARG, "NULL argument");
    o->width = h->W; o->height = h->H; o->block = h->B;
    o->grid_w = h->Gx; o->grid_h = h->Gy;
    o->precision = h->prec; o->age_max = h->age_max;
    o->theta_s = h->theta_s; o->theta_d = h->theta_d;
    o->initialized = h->initialized ? 1 : 0;
    o->parity = h->parity;
    o->frames = h->frames;
    o->state_bytes = h->state_bytes;
    o->host_state_bytes = dmsgm_host_state_bytes(h->W, h->H, h->B, h->prec);
    o->tile_rows = h->tile_rows;
    o->device = h->device;
    o->kernel = h->kernel;
    o->last_kernel = h->last_kernel;
    o->mix_spread = h->mix_spread;
    o->pre_fused = h->pre_fused;
    o->checked = h->checked;
    return DMSGM_OK;
}

int dmsgm_status(dmsgm_t h) {
    clear_error();
    if (!h) return fail(DMSGM_ERR_INVALID_ARG, "NULL handle");
    DeviceGuard g(h->device);
    DMSGM_CUDA_TRY(cudaDeviceSynchronize());
    int word = 0;
    DMSGM_CUDA_TRY(cudaMemcpy(&word, h->status_dev, sizeof word, cudaMemcpyDeviceToHost));
    if (word) {
        DMSGM_CUDA_TRY(cudaMemset(h->status_dev, 0, sizeof word));
        DMSGM_CUDA_TRY(cudaDeviceSynchronize());
        if (word & kStatusBounds)
            return fail(DMSGM_ERR_DEVICE_STATUS,
                        "a checked kernel met an index out of range and skipped it (status 0x%x)", word);
        return fail(DMSGM_ERR_TIMEOUT, "a kernel gave up waiting for its pixel tile (status 0x%x)", word);
    }
    return DMSGM_OK;
}

}  // extern "C"

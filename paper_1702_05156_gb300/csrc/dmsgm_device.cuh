// dmsgm_device.cuh -- device-side building blocks of the fused DMSGM step.
//
// A CTA of NW warps owns a tile of kTileW x (NW * B * RPT) pixels whose
// pixels arrive in shared memory by TMA.  Warp w takes strip rows w, w + NW,
// ...; lane l owns the 8 pixel columns [8l, 8l + 8) of its strip row, that is
// two 4x4 blocks (B = 4) or one 8x8 block (B = 8).  Per block the lane
//   (a) compensates the previous models for camera motion (Sec. 2.4):
//       projects the block centre through the homography and mixes the <= 4
//       overlapped previous blocks by overlap area;
//   (b) reduces sum / min / max of the block's pixels (Sec. 2.2, M_i and
//       V_i) and runs match -> update -> reset -> swap (Sec. 2.2 and 2.3);
//   (c) tests each pixel against the final apparent model (appendix code,
//       threshold theta_d * var_A) and writes one mask byte per pixel row.

#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dmsgm {

constexpr float kVarInit = 255.0f;   // Sec. 2.3: reset variance
constexpr float kVarFloor = 0.1f;    // appendix code: max(var, .1) in the match tests
constexpr float kMinWeight = 1e-3f;  // in-grid weight below this: no source
constexpr int kTileW = 256;          // pixels per tile row (one TMA box row)
constexpr int kLanePx = 8;           // pixel columns a lane owns for B >= 4 (one mask byte per row)

// Blocks a lane owns: 8 / B for B <= 8; for B = 16 a pair of lanes shares one.
template <int B>
constexpr int kLaneBlocks = B <= 8 ? 8 / B : 1;

// Grid rows: ceil(H / B); a bottom block row cut by the frame edge holds
// H - (Gy - 1) * B pixel rows.
__host__ __device__ __forceinline__ int grid_rows(int H, int B) { return (H + B - 1) / B; }
// Adding kMagic = 1.5 * 2^23 to a float x with |x| < 2^22 leaves an integer
// in the low mantissa bits (the ulp there is 1); with a directed rounding
// mode the sum is kMagic + floor(x) or kMagic + ceil(x), exactly.
constexpr float kMagic = 12582912.0f;
constexpr int kMagicBits = 0x4B400000;

// device status word bits
constexpr int kStatusWaitTimeout = 1;
constexpr int kStatusBounds = 2;   // a checked kernel met an index out of range (and skipped it)

// The frame's homography, reduced on the host from FP64 to pairs of floats
// (hi + lo, "double-float") in one of two forms:
//  * affine (h20 = h21 = 0, h22 > 0, displacements bounded): the block-unit
//    displacement of block (bx, by) is linear,
//        ex = c0*bx + c2*by + c4,   ey = c6*bx + c8*by + c10
//    (pair (c[2k], c[2k+1]) is one coefficient); ex, ey is where the block's
//    back-projected square starts relative to (bx, by), in blocks;
//  * general: the pixel-space displacement form.  For a centre (x, y):
//        Z  = c12*x + c14*y + c16
//        dx = (c0*x + c2*y + c4 - (c12*x + c14*y)*x) / Z       (= X/Z - x)
//        dy = (c6*x + c8*y + c10 - (c12*x + c14*y)*y) / Z      (= Y/Z - y)
//    with c0 = h00 - h22, c2 = h01, c4 = h02, c6 = h10, c8 = h11 - h22,
//    c10 = h12, (c12, c14, c16) = (h20, h21, h22).
// Evaluating displacements (not absolute positions) in double-float keeps the
// fractional block position that sets the mixing weights exact to ~1e-7 even
// for 150 px shifts at 4K, with FP32 instructions only.
struct Coef {
    float c[18];
};

// One ping-pong buffer of model state, a structure of arrays over the
// blocks; in each array the apparent (A) and candidate (C) values of a block
// sit side by side, so one 8-byte (FP32) or 4-byte (FP16) load fetches both:
//   mu[k]  = (mu_A, mu_C)     float2 or __half2
//   var[k] = (var_A, var_C)   float2 or __half2
//   age[k] = age_A | age_C << 8
struct StateBuf {
    void* mu;
    void* var;
    uint16_t* age;
};

// Device-memory layout of a handle: a 256-byte control block (status word
// first), the per-tile progress counters of the multi-frame kernel (one int
// per 256 x 8B tile, the smallest tile it uses), then the two state buffers;
// every array 256-byte aligned.  s is the size of one stored value (4: FP32,
// 2: FP16).
__host__ __device__ __forceinline__ size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
__host__ __device__ __forceinline__ size_t state_buf_bytes(size_t N, int s) {
    return 2 * align256(N * 2 * s) + align256(N * 2);
}
__host__ __device__ __forceinline__ size_t seq_flag_count(int W, int H, int B) {
    return size_t((W + kTileW - 1) / kTileW) * size_t((H + 8 * B - 1) / (8 * B));
}
__host__ __device__ __forceinline__ size_t seq_flags_bytes(int W, int H, int B) {
    return align256(4 * seq_flag_count(W, H, B));
}
__host__ __device__ __forceinline__ StateBuf state_buf(char* mem, int W, int H, int B, int s,
                                                      int which) {
    const size_t N = size_t(W / B) * grid_rows(H, B);
    char* p = mem + 256 + seq_flags_bytes(W, H, B) + size_t(which) * state_buf_bytes(N, s);
    StateBuf b;
    b.mu = p; p += align256(N * 2 * s);
    b.var = p; p += align256(N * 2 * s);
    b.age = reinterpret_cast<uint16_t*>(p);
    return b;
}

// Everything one stream's frame step needs besides its pixels.
struct StreamArgs {
    StateBuf prev, next;
    uint32_t* mask;
    int W, H, Gx, Gy;
    int mask_words;     // uint32 words per mask row = ceil(W / 32)
    int first;          // 1: no previous state (first frame after create/reset)
    int affine;         // 1: coef holds the affine block-unit form
    int age_max;
    float theta_s, theta_d;
    int spread;         // 1: the mixed variance carries the spread of the mixed means
};

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

// Make the mbarrier initialisation visible to the async (TMA) proxy.
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// One bounded wait for phase `parity`: the thread is suspended until the
// phase completes or about kSuspendHintNs have passed (a hint to the
// hardware), so a waiting warp issues almost nothing.
constexpr uint32_t kSuspendHintNs = 20000;

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(kSuspendHintNs)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of the barrier, giving up after ~timeout_ns.
// Returns false on timeout (the caller reports it and abandons the tile).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint64_t timeout_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_timer_ns() - t0 > timeout_ns) return false;
    }
}

// 2-D tiled TMA load of box (x, y) of `tmap` into shared memory, completing
// on `bar` (transaction bytes).  x * 1 byte must be a multiple of 16.
__device__ __forceinline__ void tma_load_2d(void* smem_dst, const CUtensorMap* tmap, int x,
                                            int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

// 3-D tiled TMA load (x, y, z) -- z selects the frame of a sequence.
__device__ __forceinline__ void tma_load_3d(void* smem_dst, const CUtensorMap* tmap, int x, int y,
                                            int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

// Progress counters of the multi-frame kernel: release store / acquire load
// at GPU scope.
__device__ __forceinline__ void st_release_gpu(int* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// 1-D bulk copy global -> shared (TMA engine, no tensor map).  Both addresses
// 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_load_1d(void* smem_dst, const void* gsrc, uint32_t bytes,
                                             uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(gsrc)), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap* tmap) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tmap)) : "memory");
}

// Programmatic dependent launch: wait for the previous grid in the stream
// (no-op when the launch has no programmatic dependency) / allow the next
// grid to start launching.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}


// ------------------------------------------------------------------ state I/O
// Both models of a block, as (A, C) float pairs.  COH = false: read-only
// cache path (the previous buffer is not written during the launch);
// COH = true: L2 only, for state that other CTAs of the same launch write.
template <bool COH>
__device__ __forceinline__ float2 ld2(const void* base, int k, float*) {
    const float2* p = static_cast<const float2*>(base) + k;
    return COH ? __ldcg(p) : __ldg(p);
}
template <bool COH>
__device__ __forceinline__ float2 ld2(const void* base, int k, __half*) {
    const __half2* p = static_cast<const __half2*>(base) + k;
    return __half22float2(COH ? __ldcg(p) : __ldg(p));
}
template <bool COH>
__device__ __forceinline__ uint32_t ld_age(const uint16_t* base, int k) {
    return COH ? __ldcg(base + k) : __ldg(base + k);
}
__device__ __forceinline__ void st2(void* base, int k, float2 v, float*) {
    static_cast<float2*>(base)[k] = v;
}
__device__ __forceinline__ void st2(void* base, int k, float2 v, __half*) {
    static_cast<__half2*>(base)[k] = __float22half2_rn(v);
}

// (age_A, age_C) bytes -> exact floats, no conversion instruction: each byte
// becomes the low mantissa byte of 2^23 + byte, then 2^23 is subtracted.
__device__ __forceinline__ float2 age2f(uint32_t a) {
    const float2 m = make_float2(__int_as_float(__byte_perm(a, 0x4B000000u, 0x7540)),
                                 __int_as_float(__byte_perm(a, 0x4B000000u, 0x7541)));
    return __fadd2_rn(m, make_float2(-8388608.0f, -8388608.0f));
}

__device__ __forceinline__ float2 dup2(float w) { return make_float2(w, w); }

// One Gaussian model.  The age is kept as a float holding a small exact
// integer (0 .. 255), so the learning rate and the comparisons need no
// int <-> float conversions.
struct Model {
    float mu, var, age;
};

// Compensated (tilde) models of one block.  src == false: no source.
struct Comp {
    Model A, C;
    bool src;
};


// ---------------------------------------------------- double-float helpers
// A value is hi + lo with |lo| <= ulp(hi)/2.  Only additions, subtractions
// and explicit fmaf are used, so contraction cannot change the results.
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_quick(float a, float b) {   // |a| >= |b|
    const float s = a + b;
    return DF{s, b - (s - a)};
}
__device__ __forceinline__ DF df_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return DF{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
    DF s = df_two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return df_quick(s.hi, s.lo);
}
__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }
// (hi + lo) * x for a float x (exact product of hi and x via fmaf)
__device__ __forceinline__ DF df_mul(float hi, float lo, float x) {
    const float p = hi * x;
    const float e = fmaf(hi, x, -p);
    return df_quick(p, fmaf(lo, x, e));
}
__device__ __forceinline__ DF df_mulv(DF a, float x) { return df_mul(a.hi, a.lo, x); }
// a / b, one Newton correction of the float quotient
__device__ __forceinline__ DF df_div(DF a, DF b) {
    const float q1 = a.hi / b.hi;
    const DF p = df_mul(b.hi, b.lo, q1);
    const DF r = df_add(a, df_neg(p));
    const float q2 = r.hi / b.hi;
    return df_quick(q1, q2);
}

// floor and fraction of hi + lo: fl integer-valued, f in [0, 1]
__device__ __forceinline__ void df_floor_frac(DF v, float& fl, float& f) {
    fl = floorf(v.hi);
    if (v.hi == fl && v.lo < 0.f) fl -= 1.f;
    f = (v.hi - fl) + v.lo;
    f = fminf(fmaxf(f, 0.f), 1.f);
}

// General form: block-unit displacement (ex, ey) of the centre (x, y); false
// if Z <= 0.
__device__ __forceinline__ bool project_general(const Coef& k, float x, float y, DF& ex, DF& ey,
                                                float inv_b) {
    const float* c = k.c;
    const DF t = df_add(df_mul(c[12], c[13], x), df_mul(c[14], c[15], y));   // h20 x + h21 y
    const DF Z = df_add(t, DF{c[16], c[17]});
    if (!(Z.hi > 0.f)) return false;
    DF nx = df_add(df_add(df_mul(c[0], c[1], x), df_mul(c[2], c[3], y)), DF{c[4], c[5]});
    DF ny = df_add(df_add(df_mul(c[6], c[7], x), df_mul(c[8], c[9], y)), DF{c[10], c[11]});
    nx = df_add(nx, df_neg(df_mulv(t, x)));
    ny = df_add(ny, df_neg(df_mulv(t, y)));
    ex = df_div(nx, Z);
    ey = df_div(ny, Z);
    ex.hi *= inv_b; ex.lo *= inv_b;   // exact: B is a power of two
    ey.hi *= inv_b; ey.lo *= inv_b;
    return true;
}


// ------------------------------------------------------------------ (a)
// Affine form: the displacement at the first block bx0 of a half-warp's
// strip (by), split into integer parts and fractions.  One thread per
// origin computes it in double-float and publishes it in shared memory; a
// lane then steps from bx0 to its own block (at most 128 / B - 1 blocks
// away: 31 for B = 4, 127 for B = 1) with two FMAs.  The host admits the
// affine form only when |d ex / d bx| <= 1/31, so the stepped value stays
// below 2 (B >= 4), 3.1 (B = 2) or 5.1 (B = 1) in magnitude and its rounding
// below 1.2e-7, 2.4e-7 or 4.8e-7 blocks.
struct Origin {
    int nx, ny;
    float fx, fy;
};

__device__ __forceinline__ Origin affine_origin(const Coef& k, int bx0, int by) {
    const float* c = k.c;
    const DF ux = df_add(df_add(df_mul(c[0], c[1], float(bx0)), df_mul(c[2], c[3], float(by))),
                         DF{c[4], c[5]});
    const DF uy = df_add(df_add(df_mul(c[6], c[7], float(bx0)), df_mul(c[8], c[9], float(by))),
                         DF{c[10], c[11]});
    float nx, ny;
    Origin o;
    df_floor_frac(ux, nx, o.fx);
    df_floor_frac(uy, ny, o.fy);
    o.nx = int(nx);
    o.ny = int(ny);
    return o;
}

// Origins of a tile with `strips` strip rows: entry (s << 1) | h belongs to
// strip row s, half-warp h, whose first block is (tx0 + 128 h) / B.  Threads
// 0 .. 2*strips-1 fill one entry each.
template <int B>
__device__ __forceinline__ void fill_origins(const StreamArgs& a, const Coef& k, int tx0, int ty0,
                                             int strips, Origin* orig) {
    const int t = threadIdx.x;
    if (a.affine && !a.first && t < 2 * strips)
        orig[t] = affine_origin(k, (tx0 + 128 * (t & 1)) / B, ty0 / B + (t >> 1));
}

// Back-projection of one block (Sec. 2.4): the previous-grid block (i0, j0)
// at the top left of the overlapped 2x2 group and the fractional position
// (fx, fy) of the back-projected square inside it.  ok == false: no source
// (first frame, or the general form put the centre behind the camera or
// far off the grid).  Depends on the homography only, not on the state.
struct Proj {
    int i0, j0;
    float fx, fy;
    bool ok;
};

__device__ __forceinline__ Proj no_proj() { return Proj{0, 0, 0.f, 0.f, false}; }

// For the affine form, o is the origin of the lane's half-warp and bx0 its
// first block.
template <int B>
__device__ __forceinline__ Proj project(const StreamArgs& a, const Coef& k, int bx, int by,
                                        int bx0, const Origin& o) {
    if (a.first) return no_proj();
    const float* c = k.c;
    Proj p;
    if (a.affine) {
        // (x, y) side by side: w = o.f + (c_hi + c_lo) * dl, its floor and fraction
        const float2 dl = dup2(float(bx - bx0));
        const float2 w = __ffma2_rn(make_float2(c[1], c[7]), dl,
                                    __ffma2_rn(make_float2(c[0], c[6]), dl, make_float2(o.fx, o.fy)));
        const float2 m = __fadd2_rd(w, dup2(kMagic));                  // kMagic + floor(w)
        const float2 f = __ffma2_rn(__fadd2_rn(m, dup2(-kMagic)), dup2(-1.0f), w);
        p.fx = f.x;
        p.fy = f.y;
        p.i0 = bx + o.nx + (__float_as_int(m.x) - kMagicBits);
        p.j0 = by + o.ny + (__float_as_int(m.y) - kMagicBits);
    } else {
        DF ex, ey;
        if (!project_general(k, (bx + 0.5f) * B, (by + 0.5f) * B, ex, ey, 1.0f / B))
            return no_proj();
        if (!(fabsf(ex.hi) < 1.0e7f) || !(fabsf(ey.hi) < 1.0e7f)) return no_proj();
        float flx, fly;
        df_floor_frac(ex, flx, p.fx);
        df_floor_frac(ey, fly, p.fy);
        p.i0 = bx + int(flx);
        p.j0 = by + int(fly);
    }
    p.ok = true;
    return p;
}

// Bilinear overlap areas of the four blocks (i0, j0), (i0+1, j0), (i0, j0+1),
// (i0+1, j0+1).
struct Weights {
    float w00, w10, w01, w11;
};
__device__ __forceinline__ Weights overlap(const Proj& p) {
    const float2 g = __ffma2_rn(make_float2(p.fx, p.fy), dup2(-1.0f), dup2(1.0f));   // 1 - f
    const float2 top = __fmul2_rn(make_float2(g.x, p.fx), dup2(g.y));
    const float2 bot = __fmul2_rn(make_float2(g.x, p.fx), dup2(p.fy));
    return Weights{top.x, top.y, bot.x, bot.y};
}

// Compensated models from the mixed (A, C) pairs; the mixed age is rounded
// half up: floor(age + 0.5).
__device__ __forceinline__ Comp comp_from(float2 mu, float2 var, float2 ag) {
    Comp r;
    r.src = true;
    r.A.mu = mu.x;
    r.C.mu = mu.y;
    r.A.var = var.x;
    r.C.var = var.y;
    const float2 age = __fadd2_rn(__fadd2_rd(__fadd2_rn(ag, dup2(0.5f)), dup2(kMagic)), dup2(-kMagic));
    r.A.age = age.x;
    r.C.age = age.y;
    return r;
}

__device__ __forceinline__ Comp no_source() {
    Comp r;
    r.src = false;
    r.A = Model{0.f, 0.f, 0.f};
    r.C = r.A;
    return r;
}

// Where a gather reads the previous state.  at(i, j) is the index of grid
// block (i, j), pitch the index step from one grid row to the next.
// GlobalSrc: the previous state buffer in global memory.
template <typename T, bool COH>
struct GlobalSrc {
    const void* mu;
    const void* var;
    const uint16_t* age;
    int pitch;
    __device__ __forceinline__ int at(int i, int j) const { return j * pitch + i; }
    __device__ __forceinline__ float2 ld_mu(int k) const { return ld2<COH>(mu, k, (T*)nullptr); }
    __device__ __forceinline__ float2 ld_var(int k) const { return ld2<COH>(var, k, (T*)nullptr); }
    __device__ __forceinline__ uint32_t ld_ag(int k) const { return ld_age<COH>(age, k); }
};
template <typename T, bool COH>
__device__ __forceinline__ GlobalSrc<T, COH> global_src(const StreamArgs& a) {
    return GlobalSrc<T, COH>{a.prev.mu, a.prev.var, a.prev.age, a.Gx};
}

// CheckedSrc: GlobalSrc whose loads check the block index against the grid
// (n blocks); an index out of range sets kStatusBounds and reads zeros.
template <typename T, bool COH>
struct CheckedSrc {
    GlobalSrc<T, COH> g;
    int n;
    int* status;
    int pitch;
    __device__ __forceinline__ int at(int i, int j) const { return g.at(i, j); }
    __device__ __forceinline__ bool ok(int k) const {
        if (k >= 0 && k < n) return true;
        atomicOr(status, kStatusBounds);
        return false;
    }
    __device__ __forceinline__ float2 ld_mu(int k) const { return ok(k) ? g.ld_mu(k) : make_float2(0.f, 0.f); }
    __device__ __forceinline__ float2 ld_var(int k) const { return ok(k) ? g.ld_var(k) : make_float2(0.f, 0.f); }
    __device__ __forceinline__ uint32_t ld_ag(int k) const { return ok(k) ? g.ld_ag(k) : 0u; }
};

// Area-weighted mix of the four overlapped blocks whose top-left one is k0
// (all four on the grid; the weights sum to 1).
// With spread, Yi et al.'s mixture variance: the spread of the four means
// about their mix, sum w (mu_k - mu~)^2, is added to the mixed variance.
template <typename Src>
__device__ __forceinline__ Comp mix4(const Src& src, int k0, const Weights& w, bool spread) {
    const int k1 = k0 + src.pitch;
    const float2 W00 = dup2(w.w00), W10 = dup2(w.w10), W01 = dup2(w.w01), W11 = dup2(w.w11);
    const float2 m00 = src.ld_mu(k0), m10 = src.ld_mu(k0 + 1);
    const float2 m01 = src.ld_mu(k1), m11 = src.ld_mu(k1 + 1);
    float2 mu, var, ag;
    mu = __fmul2_rn(W00, m00);
    mu = __ffma2_rn(W10, m10, mu);
    mu = __ffma2_rn(W01, m01, mu);
    mu = __ffma2_rn(W11, m11, mu);
    var = __fmul2_rn(W00, src.ld_var(k0));
    var = __ffma2_rn(W10, src.ld_var(k0 + 1), var);
    var = __ffma2_rn(W01, src.ld_var(k1), var);
    var = __ffma2_rn(W11, src.ld_var(k1 + 1), var);
    if (spread) {
        const float2 nm = make_float2(-mu.x, -mu.y);
        float2 d = __fadd2_rn(m00, nm);
        var = __ffma2_rn(__fmul2_rn(W00, d), d, var);
        d = __fadd2_rn(m10, nm);
        var = __ffma2_rn(__fmul2_rn(W10, d), d, var);
        d = __fadd2_rn(m01, nm);
        var = __ffma2_rn(__fmul2_rn(W01, d), d, var);
        d = __fadd2_rn(m11, nm);
        var = __ffma2_rn(__fmul2_rn(W11, d), d, var);
    }
    ag = __fmul2_rn(W00, age2f(src.ld_ag(k0)));
    ag = __ffma2_rn(W10, age2f(src.ld_ag(k0 + 1)), ag);
    ag = __ffma2_rn(W01, age2f(src.ld_ag(k1)), ag);
    ag = __ffma2_rn(W11, age2f(src.ld_ag(k1 + 1)), ag);
    return comp_from(mu, var, ag);
}

// Motion compensation of one block (Sec. 2.4) from its projection: the
// area-weighted mix of the previous blocks its back-projected square
// overlaps.  At the grid border the blocks off the grid are dropped and the
// remaining weights renormalised.  src must hold the blocks (i0 .. i0+1,
// j0 .. j0+1) that lie on the grid.  SPREAD: the kernel is built to honour
// a.spread (the mixture-variance option); without it the option's code is
// compiled out, and with it the register demand grows.
template <bool SPREAD, typename Src>
__device__ __forceinline__ Comp gather(const StreamArgs& a, const Proj& p, const Src& src) {
    if (!p.ok) return no_source();
    const Weights w = overlap(p);
    const bool spread = SPREAD && a.spread != 0;
    if (p.i0 >= 0 && p.i0 + 1 < a.Gx && p.j0 >= 0 && p.j0 + 1 < a.Gy)
        return mix4(src, src.at(p.i0, p.j0), w, spread);
    float wsum = 0.f;
    float2 mu = make_float2(0.f, 0.f), var = mu, ag = mu;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = p.i0 + (q & 1), j = p.j0 + (q >> 1);
        const float wq = q == 0 ? w.w00 : q == 1 ? w.w10 : q == 2 ? w.w01 : w.w11;
        if (i >= 0 && i < a.Gx && j >= 0 && j < a.Gy) {
            const int kk = src.at(i, j);
            const float2 W = dup2(wq);
            wsum += wq;
            mu = __ffma2_rn(W, src.ld_mu(kk), mu);
            var = __ffma2_rn(W, src.ld_var(kk), var);
            ag = __ffma2_rn(W, age2f(src.ld_ag(kk)), ag);
        }
    }
    if (!(wsum >= kMinWeight)) return no_source();
    const float2 mt = make_float2(mu.x / wsum, mu.y / wsum);
    if (spread) {   // second pass: the spread of the in-grid means about their mix
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = p.i0 + (q & 1), j = p.j0 + (q >> 1);
            const float wq = q == 0 ? w.w00 : q == 1 ? w.w10 : q == 2 ? w.w01 : w.w11;
            if (i >= 0 && i < a.Gx && j >= 0 && j < a.Gy) {
                const float2 d = __fadd2_rn(src.ld_mu(src.at(i, j)), make_float2(-mt.x, -mt.y));
                var = __ffma2_rn(__fmul2_rn(dup2(wq), d), d, var);
            }
        }
    }
    return comp_from(mt, make_float2(var.x / wsum, var.y / wsum),
                     make_float2(ag.x / wsum, ag.y / wsum));
}
template <typename T, bool COH, bool SPREAD>
__device__ __forceinline__ Comp gather(const StreamArgs& a, const Proj& p) {
    return gather<SPREAD>(a, p, global_src<T, COH>(a));
}

// ------------------------------------------------------------------ (b)
// Block statistics: mean M_i and the extremes that give V_i (Sec. 2.2).
struct Stats {
    float M, mn, mx;
};

// Sec. 2.2 update with learning rate 1/(age~ + 1), written incrementally:
// mu = mu~ + (M - mu~)/(age~+1), V = max_j (mu - I_j)^2 = max((mu-min)^2,
// (max-mu)^2), var = var~ + (V - var~)/(age~+1), age + 1 below the cap.
__device__ __forceinline__ void sgm_update(Model& m, const Stats& st, float age_max) {
    const float rcp = __fdividef(1.0f, m.age + 1.0f);   // ~2 ulp
    const float mu = fmaf(st.M - m.mu, rcp, m.mu);
    const float d0 = mu - st.mn, d1 = st.mx - mu;
    const float V = fmaxf(d0 * d0, d1 * d1);
    m.var = fmaf(V - m.var, rcp, m.var);
    m.mu = mu;
    m.age = (m.age < age_max) ? m.age + 1.0f : m.age;
}

// Match -> update -> reset -> swap (Sec. 2.3) from the compensated models.
// PACKED = false: branches on the tests, one scalar update.  PACKED = true:
// both models' tests and updates run side by side in packed FP32 pairs (each
// lane of a pair rounded exactly like its scalar form, so the results are
// the same bits), and selects keep the update of the model that matched --
// the apparent one if it does, else the candidate, else the candidate
// restarts -- so a warp runs one path whatever its blocks decide.  Measured
// (graph replays): 1920x1080 block 4 FP32 3.45 instead of 3.59 us per frame;
// 3840x2160 block 4 FP32 unchanged, block 4 FP16 and block 8 1-2 % slower,
// where they keep the branches.
template <bool PACKED>
__device__ __forceinline__ void dual_mode_step(Comp& c, const Stats& st, const StreamArgs& a) {
    if constexpr (!PACKED) {
        const Model reset{st.M, kVarInit, 1.0f};
        if (!c.src) {
            c.A = reset;
            c.C = reset;
            return;
        }
        const float age_max = static_cast<float>(a.age_max);
        const float dA = st.M - c.A.mu, dC = st.M - c.C.mu;
        if (dA * dA < a.theta_s * fmaxf(c.A.var, kVarFloor)) {
            sgm_update(c.A, st, age_max);
        } else if (dC * dC < a.theta_s * fmaxf(c.C.var, kVarFloor)) {
            sgm_update(c.C, st, age_max);
        } else {
            c.C = reset;
        }
        if (c.C.age > c.A.age) {
            c.A = c.C;
            c.C = reset;
        }
        return;
    }
    const Model reset{st.M, kVarInit, 1.0f};
    if (!c.src) {
        c.A = reset;
        c.C = reset;
        return;
    }
    const float age_max = static_cast<float>(a.age_max);
    const float2 mu = make_float2(c.A.mu, c.C.mu);
    const float2 var = make_float2(c.A.var, c.C.var);
    const float2 age = make_float2(c.A.age, c.C.age);
    // match tests (M - mu~)^2 < theta_s * max(var~, 0.1)
    const float2 d = __fadd2_rn(dup2(st.M), make_float2(-mu.x, -mu.y));
    const float2 lhs = __fmul2_rn(d, d);
    const float2 rhs = __fmul2_rn(dup2(a.theta_s), make_float2(fmaxf(var.x, kVarFloor),
                                                               fmaxf(var.y, kVarFloor)));
    const bool mA = lhs.x < rhs.x;
    const bool mC = !mA && lhs.y < rhs.y;
    // the Sec. 2.2 update of both (as sgm_update)
    const float2 rcp = make_float2(__fdividef(1.0f, age.x + 1.0f), __fdividef(1.0f, age.y + 1.0f));
    const float2 nmu = __ffma2_rn(d, rcp, mu);
    const float2 d0 = __fadd2_rn(nmu, dup2(-st.mn));
    const float2 d1 = __fadd2_rn(dup2(st.mx), make_float2(-nmu.x, -nmu.y));
    const float2 q0 = __fmul2_rn(d0, d0), q1 = __fmul2_rn(d1, d1);
    const float2 V = make_float2(fmaxf(q0.x, q1.x), fmaxf(q0.y, q1.y));
    const float2 nvar = __ffma2_rn(__fadd2_rn(V, make_float2(-var.x, -var.y)), rcp, var);
    // one more year below the cap (a compensated age never exceeds it)
    const float2 nage = make_float2(age.x < age_max ? age.x + 1.0f : age.x,
                                    age.y < age_max ? age.y + 1.0f : age.y);
    Model A = mA ? Model{nmu.x, nvar.x, nage.x} : c.A;
    Model C = mC ? Model{nmu.y, nvar.y, nage.y} : (mA ? c.C : reset);
    if (C.age > A.age) {   // swap: selects
        A = C;
        C = reset;
    }
    c.A = A;
    c.C = C;
}

// Byte statistics of a block given as N words (4 pixels each): the sum by
// 4-way dot products, min and max on 16-bit lanes (bytes 0/2 and 1/3 of each
// word) with the 3-input DPX min/max instructions.
template <int N>
__device__ __forceinline__ Stats block_stats(const uint32_t* w) {
    uint32_t s = 0, lo2 = 0x00FF00FFu, hi2 = 0u;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        s = __dp4a(w[i], 0x01010101u, s);
        const uint32_t e = w[i] & 0x00FF00FFu, o = (w[i] >> 8) & 0x00FF00FFu;
        lo2 = __vimin3_u16x2(lo2, e, o);
        hi2 = __vimax3_u16x2(hi2, e, o);
    }
    Stats st;
    // (2^23 + s) / (4N) - 2^23 / (4N): both steps exact (4N is a power of two)
    st.M = fmaf(__int_as_float(0x4B000000 | s), 1.0f / (4 * N), -8388608.0f / (4 * N));
    const uint32_t mn = __vimin3_u16x2(lo2, lo2 >> 16, lo2) & 0xFFFFu;
    const uint32_t mx = __vimax3_u16x2(hi2, hi2 >> 16, hi2) & 0xFFFFu;
    const float2 e = __fadd2_rn(make_float2(__int_as_float(0x4B000000 | mn), __int_as_float(0x4B000000 | mx)),
                                dup2(-8388608.0f));   // exact small integers
    st.mn = e.x;
    st.mx = e.y;
    return st;
}

// Statistics from an exact byte sum over n pixels and 16-bit-lane min / max
// words; nfull is the pixel count of an unclipped block (a power of two).
// NFULL > 0: a whole block of NFULL pixels (a power of two), whose mean
// (2^23 + s) / NFULL - 2^23 / NFULL is exact in both steps; NFULL = 0: a
// block cut by the frame edge, n pixels, approximate divide (within 2 ulp).
template <int NFULL>
__device__ __forceinline__ Stats stats_from(uint32_t s, uint32_t lo2, uint32_t hi2, int n = 0) {
    Stats st;
    const float m = __int_as_float(0x4B000000 | s);   // 2^23 + s, exact: s < 2^23
    if constexpr (NFULL > 0) st.M = fmaf(m, 1.0f / NFULL, -8388608.0f / NFULL);
    else st.M = __fdividef(m - 8388608.0f, float(max(n, 1)));
    const uint32_t mn = __vimin3_u16x2(lo2, lo2 >> 16, lo2) & 0xFFFFu;
    const uint32_t mx = __vimax3_u16x2(hi2, hi2 >> 16, hi2) & 0xFFFFu;
    const float2 e = __fadd2_rn(make_float2(__int_as_float(0x4B000000 | mn), __int_as_float(0x4B000000 | mx)),
                                dup2(-8388608.0f));
    st.mn = e.x;
    st.mx = e.y;
    return st;
}

// Exact byte sum and 16-bit-lane min / max of words w[0 .. nv) of N; the
// words from nv on (rows below a cut frame edge) are left out.  With nv = N
// known at the call the selects fold away.
template <int N>
__device__ __forceinline__ void raw_stats(const uint32_t* w, int nv, uint32_t& s, uint32_t& lo,
                                          uint32_t& hi) {
    s = 0;
    lo = 0x00FF00FFu;
    hi = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const bool in = i < nv;
        const uint32_t x = in ? w[i] : 0u;
        s = __dp4a(x, 0x01010101u, s);
        const uint32_t e = x & 0x00FF00FFu, o = (x >> 8) & 0x00FF00FFu;
        lo = __vimin3_u16x2(lo, in ? e : 0x00FF00FFu, in ? o : 0x00FF00FFu);
        hi = __vimax3_u16x2(hi, e, o);   // a left-out word is 0 and never raises the max
    }
}

// Byte j of w as an exact float (the byte becomes the low mantissa byte of 2^23 + j).
__device__ __forceinline__ float byte_f(uint32_t w, int j) {
    return __int_as_float(__byte_perm(w, 0x4B000000u, 0x7540 + j)) - 8388608.0f;
}

// ------------------------------------------------------------------ (c)
// The per-pixel test (I - mu)^2 > thr, evaluated in FP32, is monotone in
// |I - mu|, so its background set is an interval [lo, hi] of intensities.
// bg_interval finds that interval exactly (the FP32 test itself decides the
// boundary integers) and fg_bits then tests 4 pixels at once on bytes:
// x > hi  <=>  x + (255 - hi) carries out of the byte, and
// x < lo  <=>  (255 - x) + lo carries out of the byte.
struct Thresh {
    uint32_t c_gt;   // 255 - hi in every byte
    uint32_t c_lt;   // lo in every byte
};

__device__ __forceinline__ Thresh thresh_of(int ih, int il) {
    const int hi = min(ih, 255), lo = max(il, 0);
    Thresh t;
    if (lo > hi) {   // no intensity is background: both tests fire on every byte
        t.c_gt = t.c_lt = 0xFFFFFFFFu;
    } else {
        t.c_gt = __byte_perm(uint32_t(255 - hi), 0u, 0x0000);
        t.c_lt = __byte_perm(uint32_t(lo), 0u, 0x0000);
    }
    return t;
}

// Two models side by side (x and y lanes of the packed operations, each
// rounded exactly like its scalar form).  s is slightly below sqrt(thr) (the
// approximate rsqrt is within 3e-7), so every integer within s of mu is
// background and the true ends of the interval lie at most one step beyond
// floor(mu + s) / ceil(mu - s); s is capped where the interval already covers
// every intensity.
__device__ __forceinline__ void bg_interval2(float2 mu, float2 thr, Thresh& tx, Thresh& ty) {
    const float2 rs = make_float2(rsqrtf(fmaxf(thr.x, 1.0e-30f)), rsqrtf(fmaxf(thr.y, 1.0e-30f)));
    float2 s = __fmul2_rn(__fmul2_rn(thr, rs), dup2(1.0f - 1.0e-6f));
    s = make_float2(fminf(s.x, 1024.0f), fminf(s.y, 1024.0f));
    const float2 hm = __fadd2_rd(__fadd2_rn(mu, s), dup2(kMagic));                 // kMagic + floor(mu + s)
    const float2 lm = __fadd2_ru(__ffma2_rn(s, dup2(-1.0f), mu), dup2(kMagic));    // kMagic + ceil(mu - s)
    const float2 dh = __ffma2_rn(mu, dup2(-1.0f), __fadd2_rn(hm, dup2(-(kMagic - 1.0f))));  // (hi + 1) - mu
    const float2 dl = __ffma2_rn(mu, dup2(-1.0f), __fadd2_rn(lm, dup2(-(kMagic + 1.0f))));  // (lo - 1) - mu
    const float2 qh = __fmul2_rn(dh, dh), ql = __fmul2_rn(dl, dl);
    tx = thresh_of(__float_as_int(hm.x) - kMagicBits + (qh.x <= thr.x ? 1 : 0),
                   __float_as_int(lm.x) - kMagicBits - (ql.x <= thr.x ? 1 : 0));
    ty = thresh_of(__float_as_int(hm.y) - kMagicBits + (qh.y <= thr.y ? 1 : 0),
                   __float_as_int(lm.y) - kMagicBits - (ql.y <= thr.y ? 1 : 0));
}

__device__ __forceinline__ Thresh bg_interval(float mu, float thr) {
    Thresh t, u;
    bg_interval2(make_float2(mu, mu), make_float2(thr, thr), t, u);
    return t;
}

// Foreground flags of the 4 pixels of w: bit 7 of byte j <=> pixel j is
// foreground.  A byte's carry out of x + c is the majority of the two top
// bits and the carry into bit 7 (bit 7 of the 7-bit sum); ~x's low 7 bits
// are 0x7f - (x & 0x7f), so both sums share x & 0x7f7f7f7f.
__device__ __forceinline__ uint32_t fg_bits(uint32_t w, const Thresh& t) {
    const uint32_t xm = w & 0x7f7f7f7fu;
    const uint32_t s1 = xm + (t.c_gt & 0x7f7f7f7fu);
    const uint32_t s2 = (0x7f7f7f7fu + (t.c_lt & 0x7f7f7f7fu)) - xm;
    const uint32_t m1 = (w & t.c_gt) | ((w | t.c_gt) & s1);
    const uint32_t m2 = (~w & t.c_lt) | ((~w | t.c_lt) & s2);
    return (m1 | m2) & 0x80808080u;
}

// One mask byte from the flags of the left and right 4 pixels: the high word
// of each product gathers the four flags (bits 7, 15, 23, 31) into bits
// 0..3 (left) or 4..7 (right); every other partial product lands on its own
// bit outside bits 32..39, so nothing carries into the byte.
__device__ __forceinline__ uint32_t mask_byte(uint32_t fl, uint32_t fr) {
    return __umulhi(fr, 0x20408100u) + __umulhi(fl, 0x02040810u);
}

// Store a block's next state (both models).  Ages are <= 255.
__device__ __forceinline__ uint32_t age_pair(const Comp& c) {
    // kMagic + age has the age in its low byte and a zero in byte 1
    return __byte_perm(__float_as_uint(c.A.age + kMagic), __float_as_uint(c.C.age + kMagic),
                       0x1140);
}
template <typename T>
__device__ __forceinline__ void store_block(const StreamArgs& a, int k, const Comp& c) {
    st2(a.next.mu, k, make_float2(c.A.mu, c.C.mu), (T*)nullptr);
    st2(a.next.var, k, make_float2(c.A.var, c.C.var), (T*)nullptr);
    a.next.age[k] = static_cast<uint16_t>(age_pair(c));
}
// Blocks k and k + 1 with k even: one 16-byte (FP32) or 8-byte (FP16) store
// per array and one 4-byte store of the ages.
__device__ __forceinline__ void st4(void* base, int k, float4 v, float*) {
    reinterpret_cast<float4*>(base)[k >> 1] = v;
}
__device__ __forceinline__ void st4(void* base, int k, float4 v, __half*) {
    const __half2 lo = __float22half2_rn(make_float2(v.x, v.y));
    const __half2 hi = __float22half2_rn(make_float2(v.z, v.w));
    reinterpret_cast<uint2*>(base)[k >> 1] =
        make_uint2(*reinterpret_cast<const uint32_t*>(&lo), *reinterpret_cast<const uint32_t*>(&hi));
}
template <typename T>
__device__ __forceinline__ void store_pair(const StreamArgs& a, int k, const Comp& c0,
                                           const Comp& c1) {
    st4(a.next.mu, k, make_float4(c0.A.mu, c0.C.mu, c1.A.mu, c1.C.mu), (T*)nullptr);
    st4(a.next.var, k, make_float4(c0.A.var, c0.C.var, c1.A.var, c1.C.var), (T*)nullptr);
    reinterpret_cast<uint32_t*>(a.next.age)[k >> 1] = __byte_perm(age_pair(c0), age_pair(c1), 0x5410);
}

// ------------------------------------------------------------------ tiles
// Lane layout: warp w of the CTA takes strip rows w, w + NW, ...; lane l owns
// pixel columns [tx0 + 8l, tx0 + 8l + 8) of its strip row, i.e. two 4x4
// blocks (B = 4) or one 8x8 block (B = 8), and writes one mask byte per row.
// B = 1 and 2 interleave instead: lane l owns blocks tx0 / B + l + 32 j
// (j < 8 / B), so that a warp's gathers and stores of block j touch 32
// consecutive blocks, and the mask words of a row come from ballots.
// A tile is kTileW x (NW * B * RPT) pixels, its pixels in shared memory with
// row pitch kTileW.  A step runs tile_stats and tile_project (frame and
// homography only), then tile_update (reads the previous state, writes the
// next) and tile_mask.
template <int B>
__device__ __forceinline__ uint2 tile_words(const uint8_t* tile, int row, int lane) {
    return *reinterpret_cast<const uint2*>(tile + row * kTileW + kLanePx * lane);
}

// Pixel rows of the lane's strip row s that lie inside the frame (B unless
// the frame's bottom edge cuts the block row; 0 past the grid).
template <int B>
__device__ __forceinline__ int strip_rows(const StreamArgs& a, int ty0, int s) {
    return max(0, min(B, a.H - ty0 - B * s));
}

// Block statistics of the lane's blocks (Sec. 2.2 M_i, and the extremes for
// V_i), over the pixels inside the frame.  Lanes past the frame's right edge
// read whatever the staged tile holds there: their statistics are never used
// (no state store, no mask bit, no vote).
template <int B, int NW, int RPT>
__device__ __forceinline__ void tile_stats(const StreamArgs& a, const uint8_t* tile, int ty0,
                                           bool xin, Stats (&st)[RPT][kLaneBlocks<B>]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int s = warp + NW * r;
        const int vr = strip_rows<B>(a, ty0, s);
        if constexpr (B == 1) {
            // one pixel per block: M = min = max = the pixel (interleaved lanes)
            const uint8_t* row = tile + s * kTileW + lane;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float f = float(row[32 * j]);
                st[r][j] = Stats{f, f, f};
            }
        } else if constexpr (B == 2) {
            // block j of the lane: bytes 2 (lane + 32 j), +1 of the strip's rows
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                uint32_t sum = 0, mn = 255, mx = 0;
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    if (i >= vr) break;
                    const uint32_t v = *reinterpret_cast<const uint16_t*>(
                        tile + (B * s + i) * kTileW + 2 * (lane + 32 * j));
                    const uint32_t p0 = v & 0xFFu, p1 = v >> 8;
                    sum += p0 + p1;
                    mn = min(mn, min(p0, p1));
                    mx = max(mx, max(p0, p1));
                }
                st[r][j] = vr == 2 ? stats_from<4>(sum, mn | 0x00FF0000u, mx)
                                   : stats_from<0>(sum, mn | 0x00FF0000u, mx, 2 * vr);
            }
        } else {
            uint32_t lw[B], rw[B];
#pragma unroll
            for (int i = 0; i < B; ++i) {
                const uint2 v = tile_words<B>(tile, B * s + i, lane);
                lw[i] = v.x;
                rw[i] = v.y;
            }
            if constexpr (B == 4) {
                uint32_t sl, ll, hl, sr, lr, hr;
                if (vr == B) {
                    raw_stats<4>(lw, 4, sl, ll, hl);
                    raw_stats<4>(rw, 4, sr, lr, hr);
                    st[r][0] = stats_from<16>(sl, ll, hl);
                    st[r][1] = stats_from<16>(sr, lr, hr);
                } else {   // the bottom block row, cut by the frame edge
                    raw_stats<4>(lw, vr, sl, ll, hl);
                    raw_stats<4>(rw, vr, sr, lr, hr);
                    st[r][0] = stats_from<0>(sl, ll, hl, 4 * vr);
                    st[r][1] = stats_from<0>(sr, lr, hr, 4 * vr);
                }
            } else {
                // B = 8: the lane's 8 columns are the whole block; B = 16: half
                // of it, and the lane pair (l, l ^ 1) combines its halves
                uint32_t all[2 * B];
#pragma unroll
                for (int i = 0; i < B; ++i) {
                    all[2 * i] = lw[i];
                    all[2 * i + 1] = rw[i];
                }
                uint32_t sm, lo, hi;
                const bool whole = vr == B;   // warp-uniform
                if (whole) raw_stats<2 * B>(all, 2 * B, sm, lo, hi);
                else raw_stats<2 * B>(all, 2 * vr, sm, lo, hi);
                if constexpr (B == 16) {
                    sm += __shfl_xor_sync(0xffffffffu, sm, 1);
                    lo = __vimin3_u16x2(lo, __shfl_xor_sync(0xffffffffu, lo, 1), lo);
                    hi = __vimax3_u16x2(hi, __shfl_xor_sync(0xffffffffu, hi, 1), hi);
                }
                st[r][0] = whole ? stats_from<B * B>(sm, lo, hi) : stats_from<0>(sm, lo, hi, B * vr);
            }
        }
    }
}

template <int B, int NW, int RPT>
__device__ __forceinline__ void tile_project(const StreamArgs& a, const Coef& k, int tx0,
                                             int ty0, const Origin* orig,
                                             Proj (&pj)[RPT][kLaneBlocks<B>]) {
    constexpr int BPL = kLaneBlocks<B>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if constexpr (B <= 2) {
        // block j of the lane is tx0 / B + lane + 32 j, in half-warp strip
        // j / (4 / B): the same origin and distance from it as in the blocked
        // layout
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            const int s = warp + NW * r;
            const int by = ty0 / B + s;
#pragma unroll
            for (int j = 0; j < BPL; ++j) {
                const int bx = tx0 / B + lane + 32 * j, half = j / (4 / B);
                pj[r][j] = bx < a.Gx && by < a.Gy
                               ? project<B>(a, k, bx, by, (tx0 + 128 * half) / B, orig[(s << 1) | half])
                               : no_proj();
            }
        }
        return;
    }
    const int x = tx0 + kLanePx * lane;
    const int bx = x / B;
    const int half = lane >> 4;
    const int bx0 = (tx0 + 128 * half) / B;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int s = warp + NW * r;
        const int by = ty0 / B + s;
        const bool in = x < a.W && by < a.Gy;
#pragma unroll
        for (int j = 0; j < BPL; ++j)
            pj[r][j] = in ? project<B>(a, k, bx + j, by, bx0, orig[(s << 1) | half]) : no_proj();
    }
}

// Gather (gather_fn: Proj -> Comp), update and store the state of the lane's
// blocks; returns per block the final apparent mean and the mask threshold
// theta_d * var_A.
// CHECK: the state stores check their block index (status: kStatusBounds).
template <int B, typename T, int NW, int RPT, typename GatherFn, bool CHECK = false>
__device__ __forceinline__ void tile_update_with(const StreamArgs& a, int tx0, int ty0,
                                                 const Proj (&pj)[RPT][kLaneBlocks<B>],
                                                 const Stats (&st)[RPT][kLaneBlocks<B>],
                                                 float (&muA)[RPT][kLaneBlocks<B>],
                                                 float (&thr)[RPT][kLaneBlocks<B>],
                                                 const GatherFn& gather_fn,
                                                 int* status = nullptr) {
    constexpr int BPL = kLaneBlocks<B>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int x = tx0 + kLanePx * lane;
    const bool xin = x < a.W;
    const int bx = x / B;
    // all strip rows' gathers first: the loads of a later row cannot move
    // above an earlier row's state stores on their own (the compiler does not
    // know that the two buffers are distinct)
    Comp cc[RPT][BPL];
#pragma unroll
    for (int r = 0; r < RPT; ++r)
#pragma unroll
        for (int j = 0; j < BPL; ++j) cc[r][j] = gather_fn(pj[r][j]);
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int s = warp + NW * r;
        const int by = ty0 / B + s;
        Comp (&c)[BPL] = cc[r];
#pragma unroll
        for (int j = 0; j < BPL; ++j)
            dual_mode_step<B == 4 && sizeof(T) == 4>(c[j], st[r][j], a);
        if constexpr (B <= 2) {
            // interleaved blocks: one store per block, 32 consecutive per warp
#pragma unroll
            for (int j = 0; j < BPL; ++j) {
                const int bj = tx0 / B + lane + 32 * j;
                bool sj = bj < a.Gx && by < a.Gy;
                const int kj = by * a.Gx + bj;
                if constexpr (CHECK) {
                    if (sj && !(kj >= 0 && kj < a.Gx * a.Gy && bj < a.Gx)) {
                        atomicOr(status, kStatusBounds);
                        sj = false;
                    }
                }
                if (sj) store_block<T>(a, kj, c[j]);
                muA[r][j] = c[j].A.mu;
                thr[r][j] = a.theta_d * c[j].A.var;
            }
            continue;
        }
        bool store = xin && by < a.Gy;
        if constexpr (CHECK) {
            const int k = by * a.Gx + bx;
            if (store && !(k >= 0 && k + BPL <= a.Gx * a.Gy && bx + BPL <= a.Gx)) {
                atomicOr(status, kStatusBounds);
                store = false;
            }
        }
        if (store) {
            const int k = by * a.Gx + bx;   // even for B <= 4: pairs are 16-byte aligned
            if constexpr (B <= 4) {
#pragma unroll
                for (int j = 0; j < BPL; j += 2) store_pair<T>(a, k + j, c[j], c[j + 1]);
            } else if constexpr (B == 8) {
                store_block<T>(a, k, c[0]);
            } else {
                if ((lane & 1) == 0) store_block<T>(a, k, c[0]);   // one lane of the pair
            }
        }
#pragma unroll
        for (int j = 0; j < BPL; ++j) {
            muA[r][j] = c[j].A.mu;
            thr[r][j] = a.theta_d * c[j].A.var;
        }
    }
}

template <int B, typename T, int NW, int RPT, bool COH, bool SPREAD>
__device__ __forceinline__ void tile_update(const StreamArgs& a, int tx0, int ty0,
                                            const Proj (&pj)[RPT][kLaneBlocks<B>],
                                            const Stats (&st)[RPT][kLaneBlocks<B>],
                                            float (&muA)[RPT][kLaneBlocks<B>],
                                            float (&thr)[RPT][kLaneBlocks<B>]) {
    const GlobalSrc<T, COH> src = global_src<T, COH>(a);
    tile_update_with<B, T, NW, RPT>(a, tx0, ty0, pj, st, muA, thr,
                                    [&](const Proj& p) { return gather<SPREAD>(a, p, src); });
}

// Both extremes of a block's pixels pass the background test: then every
// pixel does, since the background set of the FP32 test is an interval of
// intensities containing [mn, mx].  Same operations as the per-pixel test.
__device__ __forceinline__ bool block_all_bg(const Stats& st, float mu, float thr) {
    const float2 d = __fadd2_rn(make_float2(st.mn, st.mx), dup2(-mu));
    const float2 q = __fmul2_rn(d, d);
    return q.x <= thr && q.y <= thr;
}

// Bit k of a 16-bit value to bit 2 k.
__device__ __forceinline__ uint32_t spread_bits16(uint32_t x) {
    x = (x | (x << 8)) & 0x00FF00FFu;
    x = (x | (x << 4)) & 0x0F0F0F0Fu;
    x = (x | (x << 2)) & 0x33333333u;
    return (x | (x << 1)) & 0x55555555u;
}

// Mask bytes of the lane's pixel rows from the final apparent models.  A
// warp whose blocks are all background writes zero bytes without the
// per-pixel test.  Lanes past the frame's right edge but inside the last
// mask word write zeros, so the padding bits are defined; rows past the
// frame's bottom edge are not written.  Blocks 1 and 2 (interleaved lanes)
// run the per-pixel test and store whole words instead: ballots of the
// lanes' pixels, lanes 0..7 writing the tile row's 8 words.
// CHECK: every mask byte's row and column are checked (status: kStatusBounds).
template <int B, int NW, int RPT, bool CHECK = false>
__device__ __forceinline__ void tile_mask(const StreamArgs& a, const uint8_t* tile, int tx0,
                                          int ty0, const Stats (&st)[RPT][kLaneBlocks<B>],
                                          const float (&muA)[RPT][kLaneBlocks<B>],
                                          const float (&thr)[RPT][kLaneBlocks<B>],
                                          int* status = nullptr) {
    constexpr int BPL = kLaneBlocks<B>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int x = tx0 + kLanePx * lane;
    const bool active = x < a.mask_words * 32;      // owns a byte of the mask row
    const bool xin = x < a.W;
    const size_t mrow = size_t(a.mask_words) * 4;   // mask bytes per row
    uint8_t* mcol = reinterpret_cast<uint8_t*>(a.mask) + (x >> 3);
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int s = warp + NW * r;
        if (ty0 / B + s >= a.Gy) break;   // warp-uniform
        if constexpr (B == 1) {
            // interleaved pixels: the per-pixel FP32 test, then mask word j of
            // the tile's row is the ballot of the lanes' pixel j
            const int y = ty0 + s, w0 = tx0 >> 5;
            const uint8_t* row = tile + s * kTileW + lane;
            uint32_t mine = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float d = __fadd_rn(float(row[32 * j]), -muA[r][j]);
                const bool fg = tx0 + lane + 32 * j < a.W && __fmul_rn(d, d) > thr[r][j];
                const uint32_t wv = __ballot_sync(0xffffffffu, fg);
                if (lane == j) mine = wv;
            }
            if (lane < 8 && w0 + lane < a.mask_words) {
                if constexpr (CHECK) {
                    if (y < 0 || y >= a.H) {
                        atomicOr(status, kStatusBounds);
                        continue;
                    }
                }
                a.mask[size_t(y) * a.mask_words + w0 + lane] = mine;
            }
            continue;
        }
        if constexpr (B == 2) {
            // interleaved blocks: per pixel row, ballots of the blocks' left
            // and right pixels; mask word 2 j + h holds lanes 16 h .. 16 h + 15
            // of block j, their bits interleaved (left, right)
            const int vr2 = strip_rows<B>(a, ty0, s), w0 = tx0 >> 5;
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                if (i >= vr2) break;
                const int y = ty0 + B * s + i;
                uint32_t bl[4], br[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint32_t v = *reinterpret_cast<const uint16_t*>(
                        tile + (B * s + i) * kTileW + 2 * (lane + 32 * j));
                    const bool in = tx0 / B + lane + 32 * j < a.Gx;
                    const float d0 = __fadd_rn(float(v & 0xFFu), -muA[r][j]);
                    const float d1 = __fadd_rn(float(v >> 8), -muA[r][j]);
                    bl[j] = __ballot_sync(0xffffffffu, in && __fmul_rn(d0, d0) > thr[r][j]);
                    br[j] = __ballot_sync(0xffffffffu, in && __fmul_rn(d1, d1) > thr[r][j]);
                }
                if (lane < 8 && w0 + lane < a.mask_words) {
                    if constexpr (CHECK) {
                        if (y < 0 || y >= a.H) {
                            atomicOr(status, kStatusBounds);
                            continue;
                        }
                    }
                    const int j = lane >> 1, sh = 16 * (lane & 1);
                    const uint32_t L = ((j == 0 ? bl[0] : j == 1 ? bl[1] : j == 2 ? bl[2] : bl[3]) >> sh) & 0xFFFFu;
                    const uint32_t R = ((j == 0 ? br[0] : j == 1 ? br[1] : j == 2 ? br[2] : br[3]) >> sh) & 0xFFFFu;
                    a.mask[size_t(y) * a.mask_words + w0 + lane] = spread_bits16(L) | (spread_bits16(R) << 1);
                }
            }
            continue;
        }
        const int vr = strip_rows<B>(a, ty0, s);
        uint8_t* m = mcol + size_t(ty0 + B * s) * mrow;
        if constexpr (CHECK) {
            // the rows written are ty0 + B s + i, i < vr; the column byte x / 8
            const bool bad = active && (ty0 + B * s < 0 || ty0 + B * s + vr > a.H ||
                                        size_t(x >> 3) >= mrow || vr < 0);
            if (bad) {
                atomicOr(status, kStatusBounds);
                continue;
            }
        }
        bool flat = true;   // lanes outside the frame count as flat
        if (xin) {
#pragma unroll
            for (int j = 0; j < BPL; ++j) flat = flat && block_all_bg(st[r][j], muA[r][j], thr[r][j]);
        }
        // rows of this strip to write: all B (the loops unroll without a
        // guard), or the rows above a frame edge that cuts the block row
        auto rows = [&](auto body) {
            if (vr == B) {
#pragma unroll
                for (int i = 0; i < B; ++i) body(i);
            } else {
#pragma unroll
                for (int i = 0; i < B; ++i)
                    if (i < vr) body(i);
            }
        };
        if (__all_sync(0xffffffffu, flat) || !xin || flat) {
            if (active) rows([&](int i) { m[i * mrow] = 0; });
            continue;
        }
        if constexpr (B <= 2) {
            // small blocks: the per-pixel FP32 test itself, two pixels per
            // packed operation; pixel p belongs to block p / B
            rows([&](int i) {
                const uint2 v = tile_words<B>(tile, B * s + i, lane);
                uint32_t byte = 0;
#pragma unroll
                for (int p = 0; p < 8; p += 2) {
                    const uint32_t w = p < 4 ? v.x : v.y;
                    const int j0 = p / B, j1 = (p + 1) / B;
                    const float2 d = __fadd2_rn(make_float2(byte_f(w, p & 3), byte_f(w, (p + 1) & 3)),
                                                make_float2(-muA[r][j0], -muA[r][j1]));
                    const float2 q = __fmul2_rn(d, d);
                    byte |= (q.x > thr[r][j0] ? 1u : 0u) << p;
                    byte |= (q.y > thr[r][j1] ? 1u : 0u) << (p + 1);
                }
                m[i * mrow] = uint8_t(byte);
            });
        } else {
            Thresh tl, tr;
            if (BPL == 1) {
                tl = tr = bg_interval(muA[r][0], thr[r][0]);
            } else {
                bg_interval2(make_float2(muA[r][0], muA[r][BPL - 1]),
                             make_float2(thr[r][0], thr[r][BPL - 1]), tl, tr);
            }
            rows([&](int i) {
                const uint2 v = tile_words<B>(tile, B * s + i, lane);
                m[i * mrow] = uint8_t(mask_byte(fg_bits(v.x, tl), fg_bits(v.y, tr)));
            });
        }
    }
}

}  // namespace dmsgm

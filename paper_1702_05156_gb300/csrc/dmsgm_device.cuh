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
constexpr int kLanePx = 8;           // pixel columns a lane owns (one mask byte per row)

// device status word bits
constexpr int kStatusWaitTimeout = 1;

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
    const size_t N = size_t(W / B) * (H / B);
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

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
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
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 63u && global_timer_ns() - t0 > timeout_ns) return false;
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

struct Model {
    float mu, var;
    int age;
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
// lane then steps from bx0 to its own block (at most 31 blocks away) with
// one FMA, whose rounding stays below 1.2e-7 blocks because the host admits
// the affine form only when |d ex / d bx| * 31 <= 2.
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

// Motion compensation of block (bx, by): area-weighted mix of the previous
// blocks that the back-projected BxB square overlaps (Sec. 2.4).  For the
// affine form, o is the origin of the lane's half-warp, bx0 its first block.
template <int B, typename T, bool COH = false>
__device__ __forceinline__ Comp compensate(const StreamArgs& a, const Coef& k, int bx, int by,
                                           int bx0, const Origin& o) {
    Comp r;
    r.src = false;
    r.A = Model{0.f, 0.f, 0};
    r.C = r.A;
    if (a.first) return r;
    const float* c = k.c;
    float fx, fy;
    int i0, j0;
    if (a.affine) {
        const float dl = float(bx - bx0);
        const float wx = fmaf(c[1], dl, fmaf(c[0], dl, o.fx));
        const float wy = fmaf(c[7], dl, fmaf(c[6], dl, o.fy));
        const float flx = floorf(wx), fly = floorf(wy);
        fx = wx - flx;
        fy = wy - fly;
        i0 = bx + o.nx + int(flx);
        j0 = by + o.ny + int(fly);
    } else {
        DF ex, ey;
        if (!project_general(k, (bx + 0.5f) * B, (by + 0.5f) * B, ex, ey, 1.0f / B)) return r;
        if (!(fabsf(ex.hi) < 1.0e7f) || !(fabsf(ey.hi) < 1.0e7f)) return r;  // NaN/inf/far: off grid
        float flx, fly;
        df_floor_frac(ex, flx, fx);
        df_floor_frac(ey, fly, fy);
        i0 = bx + int(flx);
        j0 = by + int(fly);
    }
    const float w00 = (1.f - fx) * (1.f - fy), w10 = fx * (1.f - fy);
    const float w01 = (1.f - fx) * fy, w11 = fx * fy;
    float2 mu, var, ag;
    if (i0 >= 0 && i0 + 1 < a.Gx && j0 >= 0 && j0 + 1 < a.Gy) {
        // interior: all four overlapped blocks exist and the weights sum to 1
        const int k0 = j0 * a.Gx + i0, k1 = k0 + a.Gx;
        const float2 W00 = dup2(w00), W10 = dup2(w10), W01 = dup2(w01), W11 = dup2(w11);
        mu = __fmul2_rn(W00, ld2<COH>(a.prev.mu, k0, (T*)nullptr));
        mu = __ffma2_rn(W10, ld2<COH>(a.prev.mu, k0 + 1, (T*)nullptr), mu);
        mu = __ffma2_rn(W01, ld2<COH>(a.prev.mu, k1, (T*)nullptr), mu);
        mu = __ffma2_rn(W11, ld2<COH>(a.prev.mu, k1 + 1, (T*)nullptr), mu);
        var = __fmul2_rn(W00, ld2<COH>(a.prev.var, k0, (T*)nullptr));
        var = __ffma2_rn(W10, ld2<COH>(a.prev.var, k0 + 1, (T*)nullptr), var);
        var = __ffma2_rn(W01, ld2<COH>(a.prev.var, k1, (T*)nullptr), var);
        var = __ffma2_rn(W11, ld2<COH>(a.prev.var, k1 + 1, (T*)nullptr), var);
        ag = __fmul2_rn(W00, age2f(ld_age<COH>(a.prev.age, k0)));
        ag = __ffma2_rn(W10, age2f(ld_age<COH>(a.prev.age, k0 + 1)), ag);
        ag = __ffma2_rn(W01, age2f(ld_age<COH>(a.prev.age, k1)), ag);
        ag = __ffma2_rn(W11, age2f(ld_age<COH>(a.prev.age, k1 + 1)), ag);
    } else {
        // border: drop out-of-grid blocks and renormalise the rest
        float wsum = 0.f;
        mu = var = ag = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + (q & 1), j = j0 + (q >> 1);
            const float w = q == 0 ? w00 : q == 1 ? w10 : q == 2 ? w01 : w11;
            if (i >= 0 && i < a.Gx && j >= 0 && j < a.Gy) {
                const int k = j * a.Gx + i;
                const float2 W = dup2(w);
                wsum += w;
                mu = __ffma2_rn(W, ld2<COH>(a.prev.mu, k, (T*)nullptr), mu);
                var = __ffma2_rn(W, ld2<COH>(a.prev.var, k, (T*)nullptr), var);
                ag = __ffma2_rn(W, age2f(ld_age<COH>(a.prev.age, k)), ag);
            }
        }
        if (!(wsum >= kMinWeight)) return r;
        mu = make_float2(mu.x / wsum, mu.y / wsum);
        var = make_float2(var.x / wsum, var.y / wsum);
        ag = make_float2(ag.x / wsum, ag.y / wsum);
    }
    r.src = true;
    r.A.mu = mu.x;
    r.C.mu = mu.y;
    r.A.var = var.x;
    r.C.var = var.y;
    r.A.age = __float2int_rd(ag.x + 0.5f);   // mixed age, rounded half up
    r.C.age = __float2int_rd(ag.y + 0.5f);
    return r;
}

// ------------------------------------------------------------------ (b)
// Sec. 2.2 update with learning rate 1/(age~ + 1), written incrementally:
// mu = mu~ + (M - mu~)/(age~+1), V = max_j (mu - I_j)^2 = max((mu-min)^2,
// (max-mu)^2), var = var~ + (V - var~)/(age~+1), age + 1 below the cap.
__device__ __forceinline__ void sgm_update(Model& m, float M, float mn, float mx, int age_max) {
    const float rcp = __fdividef(1.0f, static_cast<float>(m.age) + 1.0f);   // ~2 ulp
    const float mu = fmaf(M - m.mu, rcp, m.mu);
    const float d0 = mu - mn, d1 = mx - mu;
    const float V = fmaxf(d0 * d0, d1 * d1);
    m.var = fmaf(V - m.var, rcp, m.var);
    m.mu = mu;
    m.age = (m.age < age_max) ? m.age + 1 : m.age;
}

// Match -> update -> reset -> swap (Sec. 2.3) from the compensated models.
__device__ __forceinline__ void dual_mode_step(Comp& c, float M, float mn, float mx,
                                               const StreamArgs& a) {
    const Model reset{M, kVarInit, 1};
    if (!c.src) {
        c.A = reset;
        c.C = reset;
        return;
    }
    const float dA = M - c.A.mu, dC = M - c.C.mu;
    if (dA * dA < a.theta_s * fmaxf(c.A.var, kVarFloor)) {
        sgm_update(c.A, M, mn, mx, a.age_max);
    } else if (dC * dC < a.theta_s * fmaxf(c.C.var, kVarFloor)) {
        sgm_update(c.C, M, mn, mx, a.age_max);
    } else {
        c.C = reset;
    }
    if (c.C.age > c.A.age) {
        c.A = c.C;
        c.C = reset;
    }
}

// Byte statistics of a block given as N words (4 pixels each): the sum by
// 4-way dot products, min and max on 16-bit lanes (bytes 0/2 and 1/3 of each
// word) with the 3-input DPX min/max instructions.
template <int N>
__device__ __forceinline__ void block_stats(const uint32_t* w, float& M, float& mn, float& mx) {
    uint32_t s = 0, lo2 = 0x00FF00FFu, hi2 = 0u;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        s = __dp4a(w[i], 0x01010101u, s);
        const uint32_t e = w[i] & 0x00FF00FFu, o = (w[i] >> 8) & 0x00FF00FFu;
        lo2 = __vimin3_u16x2(lo2, e, o);
        hi2 = __vimax3_u16x2(hi2, e, o);
    }
    M = static_cast<float>(s) * (1.0f / (4 * N));   // exact: 4N is a power of two
    mn = static_cast<float>(min(lo2 & 0xFFFFu, lo2 >> 16));
    mx = static_cast<float>(max(hi2 & 0xFFFFu, hi2 >> 16));
}

// ------------------------------------------------------------------ (c)
// The per-pixel test (I - mu)^2 > thr, evaluated in FP32, is monotone in
// |I - mu|, so its background set is an interval [lo, hi] of intensities.
// bg_interval finds that interval exactly (the FP32 test itself decides the
// boundary integers) and fg_nibble then tests 4 pixels at once on bytes.
__device__ __forceinline__ bool is_bg(float I, float mu, float thr) {
    const float d = I - mu;
    return d * d <= thr;
}

struct Thresh {
    uint32_t c_gt;   // 255 - hi in every byte: x > hi  <=>  x + c_gt carries
    uint32_t c_lt;   // lo in every byte:       x < lo  <=>  ~x + c_lt carries
    uint32_t all;    // 0x80808080 when no intensity is background
};

__device__ __forceinline__ Thresh bg_interval(float mu, float thr) {
    // s slightly below sqrt(thr) (the approximate rsqrt is within 3e-7), so
    // every integer within s of mu is background and the true ends of the
    // interval lie at most one step beyond floor(mu + s) / ceil(mu - s)
    const float s = thr * rsqrtf(fmaxf(thr, 1.0e-30f)) * (1.0f - 1.0e-6f);
    float hi = floorf(mu + s);
    float lo = ceilf(mu - s);
    hi += is_bg(hi + 1.f, mu, thr) ? 1.f : 0.f;
    lo -= is_bg(lo - 1.f, mu, thr) ? 1.f : 0.f;
    const int ih = min(max(__float2int_rd(hi), -1), 255);
    const int il = min(max(__float2int_rd(lo), 0), 256);
    Thresh t;
    t.all = il > ih ? 0x80808080u : 0u;
    t.c_gt = uint32_t(255 - max(ih, 0)) * 0x01010101u;
    t.c_lt = uint32_t(min(il, 255)) * 0x01010101u;
    return t;
}

// Per-byte carry out of x + c (bit 7 of every byte), no carries between bytes:
// the majority of the two top bits and the carry into bit 7.
__device__ __forceinline__ uint32_t carry8(uint32_t x, uint32_t c) {
    const uint32_t s = (x & 0x7f7f7f7fu) + (c & 0x7f7f7f7fu);
    return ((x & c) | ((x | c) & s)) & 0x80808080u;
}

// Foreground bits of the 4 pixels of w (byte j -> bit j), at bits 28..31.
__device__ __forceinline__ uint32_t fg_nibble_hi(uint32_t w, const Thresh& t) {
    const uint32_t f = carry8(w, t.c_gt) | carry8(~w, t.c_lt) | t.all;
    // byte j's flag -> bit 28 + j; the cross terms of the product all land
    // below bit 28 (on distinct bits, so nothing carries) and are masked off
    return (((f >> 7) & 0x01010101u) * 0x10204080u) & 0xF0000000u;
}

// Store a block's next state (both models).
template <typename T>
__device__ __forceinline__ void store_block(const StreamArgs& a, int k, const Comp& c) {
    st2(a.next.mu, k, make_float2(c.A.mu, c.C.mu), (T*)nullptr);
    st2(a.next.var, k, make_float2(c.A.var, c.C.var), (T*)nullptr);
    a.next.age[k] = static_cast<uint16_t>(min(c.A.age, 255) | (min(c.C.age, 255) << 8));
}

// ------------------------------------------------------------------ tiles
// Lane layout: warp w of the CTA takes strip rows w, w + NW, ...; lane l owns
// pixel columns [tx0 + 8l, tx0 + 8l + 8) of its strip row, i.e. two 4x4
// blocks (B = 4) or one 8x8 block (B = 8), and writes one mask byte per row.
// A tile is kTileW x (NW * B * RPT) pixels.
template <int B, typename T, int NW, int RPT>
__device__ __forceinline__ void compensate_tile(const StreamArgs& a, const Coef& k, int tx0,
                                                int ty0, const Origin* orig,
                                                Comp (&comp)[RPT][kLanePx / B]) {
    constexpr int BPL = kLanePx / B;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
        for (int j = 0; j < BPL; ++j) {
            if (in) comp[r][j] = compensate<B, T>(a, k, bx + j, by, bx0, orig[(s << 1) | half]);
            else comp[r][j].src = false;
        }
    }
}

// Finish a tile whose pixels are in shared memory (row pitch kTileW): block
// statistics, the dual-mode update, the next state and the mask bytes.
template <int B, typename T, int NW, int RPT>
__device__ __forceinline__ void finish_tile(const StreamArgs& a, const uint8_t* tile, int tx0,
                                            int ty0, Comp (&comp)[RPT][kLanePx / B]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int x = tx0 + kLanePx * lane;
    const bool xin = x < a.W;
    const bool xpad = !xin && x < a.mask_words * 32;         // padding bits of the last word
    const int bx = x / B;
    const size_t mrow = size_t(a.mask_words) * 4;            // mask bytes per row
    uint8_t* mcol = reinterpret_cast<uint8_t*>(a.mask) + (x >> 3);
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int s = warp + NW * r;
        const int by = ty0 / B + s;
        if (by >= a.Gy) break;                                 // warp-uniform
        uint32_t lw[B], rw[B];                                 // left / right 4 pixels per row
#pragma unroll
        for (int i = 0; i < B; ++i) {
            const uint2 v = xin ? *reinterpret_cast<const uint2*>(tile + (B * s + i) * kTileW +
                                                                  kLanePx * lane)
                                : make_uint2(0u, 0u);
            lw[i] = v.x;
            rw[i] = v.y;
        }
        uint8_t* m = mcol + size_t(ty0 + B * s) * mrow;
        const int k = by * a.Gx + bx;
        if (B == 4) {
            float M, mn, mx;
            Comp cl = comp[r][0], cr = comp[r][kLanePx / B - 1];
            block_stats<4>(lw, M, mn, mx);
            dual_mode_step(cl, M, mn, mx, a);
            block_stats<4>(rw, M, mn, mx);
            dual_mode_step(cr, M, mn, mx, a);
            if (xin) {
                store_block<T>(a, k, cl);
                store_block<T>(a, k + 1, cr);
            }
            const Thresh tl = bg_interval(cl.A.mu, a.theta_d * cl.A.var);
            const Thresh tr = bg_interval(cr.A.mu, a.theta_d * cr.A.var);
            if (xin) {
#pragma unroll
                for (int i = 0; i < B; ++i)
                    m[i * mrow] = uint8_t((fg_nibble_hi(lw[i], tl) >> 28) |
                                          (fg_nibble_hi(rw[i], tr) >> 24));
            } else if (xpad) {
#pragma unroll
                for (int i = 0; i < B; ++i) m[i * mrow] = 0;
            }
        } else {
            uint32_t all[2 * B];
#pragma unroll
            for (int i = 0; i < B; ++i) {
                all[2 * i] = lw[i];
                all[2 * i + 1] = rw[i];
            }
            float M, mn, mx;
            Comp c = comp[r][0];
            block_stats<2 * B>(all, M, mn, mx);
            dual_mode_step(c, M, mn, mx, a);
            if (xin) store_block<T>(a, k, c);
            const Thresh t = bg_interval(c.A.mu, a.theta_d * c.A.var);
            if (xin) {
#pragma unroll
                for (int i = 0; i < B; ++i)
                    m[i * mrow] = uint8_t((fg_nibble_hi(lw[i], t) >> 28) |
                                          (fg_nibble_hi(rw[i], t) >> 24));
            } else if (xpad) {
#pragma unroll
                for (int i = 0; i < B; ++i) m[i * mrow] = 0;
            }
        }
    }
}

}  // namespace dmsgm

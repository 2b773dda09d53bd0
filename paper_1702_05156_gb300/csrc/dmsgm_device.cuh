// dmsgm_device.cuh -- device-side building blocks of the fused DMSGM step.
//
// One CTA owns a tile of kTileW x TILE_H pixels (TILE_H = 4 * B * RPT).  Its
// pixels arrive in shared memory by TMA; every thread owns a "strip" of 4
// pixel columns x B rows, i.e. one 4x4 block (B = 4) or half of an 8x8 block
// (B = 8, two adjacent lanes per block).  Per strip the thread
//   (a) compensates the block's previous models (Sec. 2.4): projects the
//       block centre through the homography, mixes the <= 4 overlapped
//       previous blocks by overlap area;
//   (b) reduces sum / min / max of the block's pixels (Sec. 2.2, M_i and
//       V_i) and runs match -> update -> reset -> swap (Sec. 2.2 and 2.3);
//   (c) tests each pixel against the final apparent model and assembles
//       the bit-packed mask with warp shuffles (appendix code, threshold
//       theta_d * var_A).
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
constexpr int kThreads = 256;        // threads per CTA
constexpr int kStripCols = kTileW / 4;                     // 64 strips across a tile
constexpr int kStripRowsPerPass = kThreads / kStripCols;   // 4 strip rows per pass

// device status word bits
constexpr int kStatusWaitTimeout = 1;

// Displacement form of the homography.  For a block centre (x, y):
//   Z  = hz0*x + hz1*y + hz2
//   dx = (ax0*x + ax1*y + ax2 - (hz0*x + hz1*y)*x) / Z      (= X/Z - x)
//   dy = (ay0*x + ay1*y + ay2 - (hz0*x + hz1*y)*y) / Z      (= Y/Z - y)
// with ax0 = h00 - h22, ax1 = h01, ax2 = h02, ay0 = h10, ay1 = h11 - h22,
// ay2 = h12, (hz0, hz1, hz2) = (h20, h21, h22).  Each coefficient arrives as
// an unevaluated sum of two floats (hi + lo) rounded once from FP64 on the
// host, and the displacement is evaluated in double-float arithmetic (error-
// free products and sums, Dekker/Knuth), so the fractional block position
// that sets the mixing weights is exact to ~1e-7 even for 150 px shifts at
// 4K -- all in FP32 instructions, no FP64 on the GPU.
struct Coef {
    float ax0, ax1, ax2, ay0, ay1, ay2, hz0, hz1, hz2;            // hi parts
    float ax0l, ax1l, ax2l, ay0l, ay1l, ay2l, hz0l, hz1l, hz2l;   // lo parts
};

// One ping-pong buffer of model state (structure of arrays over the blocks).
struct StateBuf {
    void* muA;
    void* varA;
    void* muC;
    void* varC;
    uint8_t* ageA;
    uint8_t* ageC;
};

// Everything one stream's frame step needs besides its pixels.
struct StreamArgs {
    StateBuf prev, next;
    uint32_t* mask;
    int W, H, Gx, Gy;
    int mask_words;     // uint32 words per mask row = ceil(W / 32)
    int first;          // 1: no previous state (first frame after create/reset)
    int age_max;
    float theta_s, theta_d;
    Coef coef;
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
__device__ __forceinline__ float ld_state(const void* base, int i, float*) {
    return __ldg(static_cast<const float*>(base) + i);
}
__device__ __forceinline__ float ld_state(const void* base, int i, __half*) {
    return __half2float(__ldg(static_cast<const __half*>(base) + i));
}
__device__ __forceinline__ void st_state(void* base, int i, float v, float*) {
    static_cast<float*>(base)[i] = v;
}
__device__ __forceinline__ void st_state(void* base, int i, float v, __half*) {
    static_cast<__half*>(base)[i] = __float2half_rn(v);
}

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

// Block-unit displacement (ex, ey) of the centre (x, y); false if Z <= 0.
__device__ __forceinline__ bool project_df(const Coef& c, float x, float y, DF& ex, DF& ey,
                                           float inv_b) {
    const DF t = df_add(df_mul(c.hz0, c.hz0l, x), df_mul(c.hz1, c.hz1l, y));   // h20 x + h21 y
    const DF Z = df_add(t, DF{c.hz2, c.hz2l});
    if (!(Z.hi > 0.f)) return false;
    DF nx = df_add(df_add(df_mul(c.ax0, c.ax0l, x), df_mul(c.ax1, c.ax1l, y)), DF{c.ax2, c.ax2l});
    DF ny = df_add(df_add(df_mul(c.ay0, c.ay0l, x), df_mul(c.ay1, c.ay1l, y)), DF{c.ay2, c.ay2l});
    nx = df_add(nx, df_neg(df_mulv(t, x)));
    ny = df_add(ny, df_neg(df_mulv(t, y)));
    ex = df_div(nx, Z);
    ey = df_div(ny, Z);
    ex.hi *= inv_b; ex.lo *= inv_b;   // exact: B is a power of two
    ey.hi *= inv_b; ey.lo *= inv_b;
    return true;
}

// floor and fraction of hi + lo: fl integer-valued, f in [0, 1]
__device__ __forceinline__ void df_floor_frac(DF v, float& fl, float& f) {
    fl = floorf(v.hi);
    if (v.hi == fl && v.lo < 0.f) fl -= 1.f;
    f = (v.hi - fl) + v.lo;
    f = fminf(fmaxf(f, 0.f), 1.f);
}

// (a) motion compensation of block (bx, by): area-weighted mix of the
// previous blocks that the back-projected BxB square overlaps (Sec. 2.4).
template <int B, typename T>
__device__ __forceinline__ Comp compensate(const StreamArgs& a, int bx, int by) {
    Comp r;
    r.src = false;
    r.A = Model{0.f, 0.f, 0};
    r.C = r.A;
    if (a.first) return r;
    const float x = (bx + 0.5f) * B, y = (by + 0.5f) * B;
    DF ex, ey;
    if (!project_df(a.coef, x, y, ex, ey, 1.0f / B)) return r;
    // the back-projected square's top-left corner sits at (bx + ex, by + ey)
    if (!(fabsf(ex.hi) < 1.0e7f) || !(fabsf(ey.hi) < 1.0e7f)) return r;  // NaN/inf/far: off grid
    float flx, fly, fx, fy;
    df_floor_frac(ex, flx, fx);
    df_floor_frac(ey, fly, fy);
    const int i0 = bx + static_cast<int>(flx);
    const int j0 = by + static_cast<int>(fly);
    float wsum = 0.f, sAm = 0.f, sAv = 0.f, sAa = 0.f, sCm = 0.f, sCv = 0.f, sCa = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int di = q & 1, dj = q >> 1;
        const int i = i0 + di, j = j0 + dj;
        const float w = (di ? fx : 1.f - fx) * (dj ? fy : 1.f - fy);
        if (i >= 0 && i < a.Gx && j >= 0 && j < a.Gy) {
            const int k = j * a.Gx + i;
            wsum += w;
            sAm = fmaf(w, ld_state(a.prev.muA, k, (T*)nullptr), sAm);
            sAv = fmaf(w, ld_state(a.prev.varA, k, (T*)nullptr), sAv);
            sAa = fmaf(w, static_cast<float>(__ldg(a.prev.ageA + k)), sAa);
            sCm = fmaf(w, ld_state(a.prev.muC, k, (T*)nullptr), sCm);
            sCv = fmaf(w, ld_state(a.prev.varC, k, (T*)nullptr), sCv);
            sCa = fmaf(w, static_cast<float>(__ldg(a.prev.ageC + k)), sCa);
        }
    }
    if (!(wsum >= kMinWeight)) return r;
    r.src = true;
    r.A.mu = sAm / wsum;
    r.A.var = sAv / wsum;
    r.A.age = static_cast<int>(floorf(sAa / wsum + 0.5f));   // mixed age, half up
    r.C.mu = sCm / wsum;
    r.C.var = sCv / wsum;
    r.C.age = static_cast<int>(floorf(sCa / wsum + 0.5f));
    return r;
}

// Sec. 2.2 update with learning rate 1/(age~ + 1), written incrementally:
// mu = mu~ + (M - mu~)/(age~+1), V = max_j (mu - I_j)^2 = max((mu-min)^2,
// (max-mu)^2), var = var~ + (V - var~)/(age~+1), age + 1 below the cap.
__device__ __forceinline__ void sgm_update(Model& m, float M, float mn, float mx, int age_max) {
    const float a1 = static_cast<float>(m.age) + 1.0f;
    const float mu = m.mu + (M - m.mu) / a1;
    const float d0 = mu - mn, d1 = mx - mu;
    const float V = fmaxf(d0 * d0, d1 * d1);
    m.var = m.var + (V - m.var) / a1;
    m.mu = mu;
    m.age = (m.age < age_max) ? m.age + 1 : m.age;
}

// (b) match -> update -> reset -> swap (Sec. 2.3) from the compensated models.
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

// Foreground bits of 4 pixels packed in a little-endian word.
__device__ __forceinline__ uint32_t fg_nibble(uint32_t px4, float mu, float thr) {
    uint32_t nib = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float d = static_cast<float>((px4 >> (8 * j)) & 0xffu) - mu;
        nib |= (d * d > thr) ? (1u << j) : 0u;
    }
    return nib;
}

// Sum / min / max of the 4 bytes of a word, accumulated.
__device__ __forceinline__ void stats4(uint32_t w, uint32_t& sum, uint32_t& mn4, uint32_t& mx4) {
    sum = __dp4a(w, 0x01010101u, sum);
    mn4 = __vminu4(mn4, w);
    mx4 = __vmaxu4(mx4, w);
}

__device__ __forceinline__ uint32_t min_byte(uint32_t v) {
    v = __vminu4(v, v >> 16);
    v = __vminu4(v, v >> 8);
    return v & 0xffu;
}
__device__ __forceinline__ uint32_t max_byte(uint32_t v) {
    v = __vmaxu4(v, v >> 16);
    v = __vmaxu4(v, v >> 8);
    return v & 0xffu;
}

// Process one tile whose pixels are in shared memory (row pitch kTileW).
// tx0 / ty0: pixel origin of the tile.  The caller has compensated every
// strip of the thread into comp[] (before waiting for the pixels).
template <int B, typename T, int RPT>
__device__ __forceinline__ void finish_tile(const StreamArgs& a, const uint8_t* tile, int tx0,
                                            int ty0, Comp (&comp)[RPT]) {
    const int sc = threadIdx.x % kStripCols;
    const int sr = threadIdx.x / kStripCols;
    const int lane = threadIdx.x & 31;
    const int x = tx0 + 4 * sc;
    const bool xin = x < a.W;
    const int bx = x / B;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int s = sr + kStripRowsPerPass * r;        // strip row inside the tile
        const int by = ty0 / B + s;
        if (by >= a.Gy) break;                           // warp-uniform
        uint32_t px[B];
        uint32_t sum = 0, mn4 = 0xffffffffu, mx4 = 0u;
#pragma unroll
        for (int i = 0; i < B; ++i) {
            px[i] = xin ? *reinterpret_cast<const uint32_t*>(tile + (B * s + i) * kTileW + 4 * sc)
                        : 0u;
            stats4(px[i], sum, mn4, mx4);
        }
        uint32_t mn = min_byte(mn4), mx = max_byte(mx4);
        if (B == 8) {  // the other half of the block sits in the neighbour lane
            sum += __shfl_xor_sync(0xffffffffu, sum, 1);
            mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, 1));
            mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
        }
        const float M = static_cast<float>(sum) * (1.0f / (B * B));   // exact
        Comp c = comp[r];
        dual_mode_step(c, M, static_cast<float>(mn), static_cast<float>(mx), a);
        const int k = by * a.Gx + bx;
        if (xin && (B == 4 || (lane & 1) == 0)) {
            st_state(a.next.muA, k, c.A.mu, (T*)nullptr);
            st_state(a.next.varA, k, c.A.var, (T*)nullptr);
            st_state(a.next.muC, k, c.C.mu, (T*)nullptr);
            st_state(a.next.varC, k, c.C.var, (T*)nullptr);
            a.next.ageA[k] = static_cast<uint8_t>(min(c.A.age, 255));
            a.next.ageC[k] = static_cast<uint8_t>(min(c.C.age, 255));
        }
        // (c) the mask, with the final apparent model
        const float thr = a.theta_d * c.A.var;
        const int y0 = ty0 + B * s;
#pragma unroll
        for (int i = 0; i < B; ++i) {
            uint32_t v = xin ? (fg_nibble(px[i], c.A.mu, thr) << (4 * (lane & 7))) : 0u;
            v |= __shfl_xor_sync(0xffffffffu, v, 1);
            v |= __shfl_xor_sync(0xffffffffu, v, 2);
            v |= __shfl_xor_sync(0xffffffffu, v, 4);
            if ((lane & 7) == 0 && xin)
                a.mask[static_cast<size_t>(y0 + i) * a.mask_words + (x >> 5)] = v;
        }
    }
}

// Compensation of every strip the thread owns in a tile.
template <int B, typename T, int RPT>
__device__ __forceinline__ void compensate_tile(const StreamArgs& a, int tx0, int ty0,
                                                Comp (&comp)[RPT]) {
    const int sc = threadIdx.x % kStripCols;
    const int sr = threadIdx.x / kStripCols;
    const int x = tx0 + 4 * sc;
    const int bx = x / B;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int by = ty0 / B + sr + kStripRowsPerPass * r;
        if (x < a.W && by < a.Gy) comp[r] = compensate<B, T>(a, bx, by);
        else comp[r].src = false;
    }
}

}  // namespace dmsgm

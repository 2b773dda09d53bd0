// dmsgm_filter.cuh -- the preprocessing of the paper's Sec. 2.1 (an N x N
// Gaussian blur, then a 3 x 3 median, both clamping coordinates to the frame)
// on one kTileW x TH tile, in shared memory.  The standalone filter kernel
// writes the tile to a frame; the step kernel with preprocessing filters its
// own tile before the block statistics.
//
// Exactness.  The blur is the fixed-point form of the paper's sum: 8-bit 1-D
// weights q_t (sum 256), the 2-D kernel their outer product (sum 65536) and
// the blurred pixel floor(sum q_s q_t I / 65536).  Evaluated separably, the
// row sums h = sum_t q_t I are integers <= 255 * 256, formed exactly by dp4a;
// the column sum sum_s (q_s / 65536) h_s has at most 8 integer and 16
// fractional bits at every partial step, so FP32 (24-bit significand) holds
// it exactly, and floor is an add rounded down onto 1.5 * 2^23.  The median
// is the 5th of the 9 clamped neighbours of the blurred frame.
//
// Layout.  The staged source box holds rows ty0 - R .. ty0 + TH + R
// (R = HALF + 1: the blur's half-size plus the median's ring) and columns
// tx0 - 16 .. tx0 + kTileW + 15, coordinates clamped to the frame.  Blurred
// rows -1 .. TH and columns -1 .. kTileW are kept as row pairs: word (e, j)
// holds blurred (e, j) in its low 16 bits and (e + 1, j) in its high 16 bits,
// so one column sort of three words serves two output rows.
#pragma once

#include "dmsgm_device.cuh"

namespace dmsgm {

constexpr int kFiltHalo = 16;                          // staged columns each side
constexpr int kFiltSrcPitch = kTileW + 2 * kFiltHalo;  // bytes per staged row
constexpr int kFiltRpOff = 4;                          // row-pair column j at word j + 4
constexpr int kFiltRpPitch = kTileW + 8;               // words per row-pair row
constexpr int kFiltMaxHalf = 7;                        // Gaussian sizes up to 15

// The filter of a handle or call: the 1-D weights as dp4a operands and as
// FP32 column weights, and whether the median follows.
struct FiltArgs {
    uint32_t qb[4];     // q_0 .. q_2h, four per word (byte i = tap 4u + i), zero padded
    float qf[2 * kFiltMaxHalf + 1];   // q_t / 65536
    int median;         // 1: 3 x 3 median after the blur
};

template <int HALF, int TH>
constexpr int filt_src_rows() { return TH + 2 * (HALF + 1) + 1; }
template <int HALF, int TH>
constexpr int filt_src_bytes() { return filt_src_rows<HALF, TH>() * kFiltSrcPitch; }
template <int TH>
constexpr int filt_rp_words() { return (TH + 1) * kFiltRpPitch; }

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(smem_dst)),
                 "l"(gsrc)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// Stage the source box of the tile at (tx0, ty0).  W % 16 == 0, so every
// 16-byte chunk lies wholly inside or wholly outside the frame's columns:
// inside chunks are copied (from the clamped row), outside ones repeat the
// row's edge pixel.  Returns after this thread's copies have landed.
template <int HALF, int TH, int NT>
__device__ __forceinline__ void filt_stage(const uint8_t* __restrict__ frame, int W, int H, int tx0,
                                           int ty0, uint8_t* src) {
    constexpr int R = HALF + 1, ROWS = filt_src_rows<HALF, TH>(), CH = kFiltSrcPitch / 16;
    for (int i = threadIdx.x; i < ROWS * CH; i += NT) {
        const int r = i / CH, ch = i - r * CH;
        const int gy = min(max(ty0 - R + r, 0), H - 1);
        const int gx = tx0 - kFiltHalo + 16 * ch;
        const uint8_t* row = frame + size_t(gy) * W;
        uint8_t* dst = src + r * kFiltSrcPitch + 16 * ch;
        if (gx >= 0 && gx < W) {
            cp_async16(dst, row + gx);
        } else {
            const uint32_t v = uint32_t(row[gx < 0 ? 0 : W - 1]) * 0x01010101u;
            *reinterpret_cast<uint4*>(dst) = make_uint4(v, v, v, v);
        }
    }
    cp_async_wait_all();
}

// byte_perm selector of the 4 bytes starting at byte d (0..4) of a word pair
__device__ __forceinline__ uint32_t filt_sel(int d) {
    return uint32_t(d) | uint32_t(d + 1) << 4 | uint32_t(d + 2) << 8 | uint32_t(d + 3) << 12;
}

// The row sum of the Gaussian at one column, as dp4a operands: the tap
// weights shifted by the column's byte offset `a` (0..4) within its first
// staged word, so that word u of the row pairs with weight word u:
// w[u] byte i = q_{4u + i - a} (0 outside 0 .. 2 HALF).
template <int HALF>
struct FiltTaps {
    static constexpr int U = (2 * HALF + 4) / 4;   // dp4a chunks of the 2 HALF + 1 taps
    uint32_t w[U + 1];
    __device__ __forceinline__ FiltTaps(const FiltArgs& f, int a) {
#pragma unroll
        for (int u = 0; u <= U; ++u) {
            const uint32_t lo = u > 0 ? f.qb[u - 1] : 0u, hi = u < U ? f.qb[u] : 0u;
            w[u] = __byte_perm(lo, hi, filt_sel(4 - a));
        }
    }
};

// Row sums of the Gaussian at two columns of one staged row, as exact floats:
// word wb of the row onwards, weights t0 and t1.  The dp4a chain starts from
// the bits of 2^23, so its result is the float 2^23 + sum; one subtraction
// leaves the sum.
template <int HALF>
__device__ __forceinline__ float2 filt_hsum(const uint8_t* row, int wb, const FiltTaps<HALF>& t0,
                                            const FiltTaps<HALF>& t1) {
    constexpr int U = FiltTaps<HALF>::U;
    const uint32_t* w = reinterpret_cast<const uint32_t*>(row) + wb;
    uint32_t s0 = 0x4B000000u, s1 = 0x4B000000u;
#pragma unroll
    for (int u = 0; u <= U; ++u) {
        const uint32_t v = w[u];
        s0 = __dp4a(v, t0.w[u], s0);
        s1 = __dp4a(v, t1.w[u], s1);
    }
    return __fadd2_rn(make_float2(__uint_as_float(s0), __uint_as_float(s1)), dup2(-8388608.0f));
}

// Blur (or, with HALF == 0, copy) the tile into the row-pair array.
//
// Main items: the column pairs (c, c + 1), c = 0, 2, .., kTileW - 2, times
// NR = NT / 128 runs of LEN row-pair entries; a run walks its source rows
// once, each row sum feeding the 2 HALF + 1 blurred rows it belongs to.
// Edge items: blurred columns -1 and kTileW, one pixel per thread, directly.
template <int HALF, int TH, int NT>
__device__ __forceinline__ void filt_blur(const FiltArgs& f, const uint8_t* src, uint32_t* rp) {
    static_assert(NT % 128 == 0, "a run per 128 threads");
    constexpr int NR = NT / 128;
    constexpr int LEN = (TH + 1 + NR - 1) / NR;   // entries -1 .. TH - 1 over the runs
    const int p = threadIdx.x & 127, run = threadIdx.x >> 7;
    const int c = 2 * p;
    const int e0 = -1 + run * LEN;
    // blurred row k, tap t reads staged row k + t + 1
    if constexpr (HALF == 0) {
        uint32_t prev = 0;
#pragma unroll
        for (int j = 0; j <= LEN; ++j) {
            const int k = e0 + j;
            const uint32_t cur = *reinterpret_cast<const uint16_t*>(src + (k + 1) * kFiltSrcPitch +
                                                                    kFiltHalo + c);
            if (j > 0 && k - 1 < TH) {
                uint32_t* d = rp + k * kFiltRpPitch + kFiltRpOff + c;   // entry k - 1
                *reinterpret_cast<uint2*>(d) =
                    make_uint2(__byte_perm(prev, cur, 0x2420), __byte_perm(prev, cur, 0x2521));
            }
            prev = cur;
        }
    } else {
        const int b0 = c - HALF + kFiltHalo;   // staged byte of column c - HALF
        const int wb = b0 >> 2;
        const FiltTaps<HALF> t0(f, b0 & 3), t1(f, (b0 & 3) + 1);
        float2 acc[LEN + 1];
#pragma unroll
        for (int j = 0; j <= LEN; ++j) acc[j] = make_float2(0.f, 0.f);
        float2 prev = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i <= LEN + 2 * HALF; ++i) {
            const float2 h = filt_hsum<HALF>(src + (e0 + 1 + i) * kFiltSrcPitch, wb, t0, t1);
#pragma unroll
            for (int t = 0; t <= 2 * HALF; ++t)
                if (i - t >= 0 && i - t <= LEN) acc[i - t] = __ffma2_rn(dup2(f.qf[t]), h, acc[i - t]);
            const int j = i - 2 * HALF;   // blurred row e0 + j is complete
            if (j >= 0) {
                const float2 m = __fadd2_rd(acc[j], dup2(kMagic));   // bits 0..7: floor
                const int k = e0 + j;
                if (j > 0 && k - 1 < TH) {
                    uint32_t* d = rp + k * kFiltRpPitch + kFiltRpOff + c;   // entry k - 1
                    *reinterpret_cast<uint2*>(d) =
                        make_uint2(__byte_perm(__float_as_uint(prev.x), __float_as_uint(m.x), 0x5410),
                                   __byte_perm(__float_as_uint(prev.y), __float_as_uint(m.y), 0x5410));
                }
                prev = m;
            }
        }
    }
    // edge columns -1 and kTileW of blurred rows -1 .. TH
    for (int i = threadIdx.x; i < 2 * (TH + 2); i += NT) {
        const int ce = (i & 1) ? kTileW : -1, k = (i >> 1) - 1;
        uint32_t b;
        if constexpr (HALF == 0) {
            b = src[(k + 1) * kFiltSrcPitch + kFiltHalo + ce];
        } else {
            const int b0 = ce - HALF + kFiltHalo;
            const FiltTaps<HALF> tc(f, b0 & 3);
            float acc = 0.f;
#pragma unroll
            for (int t = 0; t <= 2 * HALF; ++t)
                acc = __fmaf_rn(f.qf[t],
                                filt_hsum<HALF>(src + (k + t + 1) * kFiltSrcPitch, b0 >> 2, tc, tc).x,
                                acc);
            b = __float_as_uint(__fadd_rd(acc, kMagic)) & 0xFFu;
        }
        uint16_t* d = reinterpret_cast<uint16_t*>(rp + kFiltRpOff + ce);
        if (k >= 0) d[2 * (k * kFiltRpPitch) + 1] = uint16_t(b);             // entry k - 1, high
        if (k < TH) d[2 * ((k + 1) * kFiltRpPitch)] = uint16_t(b);           // entry k, low
    }
}

// The median clamps its window on the blurred frame: past an edge of the
// frame it repeats the blurred edge row or column (not the blur evaluated
// outside).  Tiles on the frame's edges overwrite their halo accordingly,
// columns first so that corners take the corner pixel.  CTA-uniform branches.
template <int TH, int NT>
__device__ __forceinline__ void filt_clamp_edges(uint32_t* rp, int tx0, int ty0, int W, int H) {
    const int wl = W - tx0, hl = H - ty0;   // frame columns / rows inside the tile
    const bool left = tx0 == 0, right = wl <= kTileW, top = ty0 == 0, bottom = hl <= TH;
    if (left || right) {
        for (int e = threadIdx.x; e <= TH; e += NT) {   // entries -1 .. TH - 1
            uint32_t* row = rp + e * kFiltRpPitch + kFiltRpOff;
            if (left) row[-1] = row[0];
            if (right) row[wl] = row[wl - 1];
        }
        __syncthreads();
    }
    if (top || bottom) {
        for (int j = int(threadIdx.x) - 1; j <= kTileW; j += NT) {   // columns -1 .. kTileW
            if (top) {   // entry -1: row -1 takes row 0
                uint32_t& w = rp[kFiltRpOff + j];
                w = (w >> 16) | (w & 0xFFFF0000u);
            }
            if (bottom) {   // row hl takes row hl - 1, in entries hl - 1 and hl
                uint32_t& a = rp[hl * kFiltRpPitch + kFiltRpOff + j];
                a = (a & 0xFFFFu) | (a << 16);
                if (hl < TH) {
                    uint32_t& b = rp[(hl + 1) * kFiltRpPitch + kFiltRpOff + j];
                    b = (b & 0xFFFF0000u) | (a & 0xFFFFu);
                }
            }
        }
        __syncthreads();
    }
}

// Median of three packed 16-bit lanes each.
__device__ __forceinline__ uint32_t med3_u16x2(uint32_t x, uint32_t y, uint32_t z) {
    return __vmaxu2(__vminu2(x, y), __vminu2(__vmaxu2(x, y), z));
}

// The 3 x 3 median of output rows r, r + 1 (r even) and columns c .. c + 3
// (c % 4 == 0): returns the two rows' 4 bytes each.
__device__ __forceinline__ uint2 filt_median8(const uint32_t* rp, int r, int c) {
    // sorted columns c - 1 .. c + 4; the lanes are the windows of rows r and r + 1
    uint32_t lo[6], mid[6], hi[6];
    uint32_t x[3][6];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const uint32_t* row = rp + (r + e) * kFiltRpPitch + kFiltRpOff;   // entry r - 1 + e
        const uint4 q = *reinterpret_cast<const uint4*>(row + c);
        x[e][0] = row[c - 1];
        x[e][1] = q.x; x[e][2] = q.y; x[e][3] = q.z; x[e][4] = q.w;
        x[e][5] = row[c + 4];
    }
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        lo[j] = __vimin3_u16x2(x[0][j], x[1][j], x[2][j]);
        hi[j] = __vimax3_u16x2(x[0][j], x[1][j], x[2][j]);
        mid[j] = x[0][j] + x[1][j] + x[2][j] - lo[j] - hi[j];   // lanes never borrow
    }
    // the middle middles: windows i and i + 1 share the sorted pair of
    // mid[i + 1], mid[i + 2]; med3(x, p, q) = max(min p q, min(max p q, x))
    uint32_t mm[4];
#pragma unroll
    for (int i = 0; i < 4; i += 2) {
        const uint32_t pn = __vminu2(mid[i + 1], mid[i + 2]), px = __vmaxu2(mid[i + 1], mid[i + 2]);
        mm[i] = __vmaxu2(pn, __vminu2(px, mid[i]));
        mm[i + 1] = __vmaxu2(pn, __vminu2(px, mid[i + 3]));
    }
    uint32_t res[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        // the median of 9 from sorted columns: med3 of the largest minimum,
        // the middle middle and the smallest maximum
        const uint32_t a = __vimax3_u16x2(lo[i], lo[i + 1], lo[i + 2]);
        const uint32_t d = __vimin3_u16x2(hi[i], hi[i + 1], hi[i + 2]);
        res[i] = med3_u16x2(a, mm[i], d);
    }
    const uint32_t t01 = __byte_perm(res[0], res[1], 0x6240);   // r: c, c+1; r+1: c, c+1
    const uint32_t t23 = __byte_perm(res[2], res[3], 0x6240);
    return make_uint2(__byte_perm(t01, t23, 0x5410), __byte_perm(t01, t23, 0x7632));
}

// Row r (0 .. TH - 1), columns c .. c + 3 of the blurred tile, unmedianed.
__device__ __forceinline__ uint32_t filt_plain4(const uint32_t* rp, int r, int c) {
    const uint4 q = *reinterpret_cast<const uint4*>(rp + (r + 1) * kFiltRpPitch + kFiltRpOff + c);
    return __byte_perm(__byte_perm(q.x, q.y, 0x0040), __byte_perm(q.z, q.w, 0x0040), 0x5410);
}

// Write the filtered tile at (tx0, ty0) of a W x H frame: `out` points at its
// pixel (0, 0), row pitch `pitch`; rows at or past `rows` and columns at or
// past `cols` are skipped.  Starts and ends with the CTA in step.
template <int TH, int NT>
__device__ __forceinline__ void filt_write(const FiltArgs& f, uint32_t* rp, int tx0, int ty0,
                                           int W, int H, uint8_t* out, int pitch, int rows,
                                           int cols) {
    constexpr int G = kTileW / 4;
    if (f.median) {
        filt_clamp_edges<TH, NT>(rp, tx0, ty0, W, H);
#pragma unroll
        for (int i = threadIdx.x; i < G * (TH / 2); i += NT) {
            const int c = 4 * (i % G), r = 2 * (i / G);
            if (c >= cols || r >= rows) continue;
            const uint2 v = filt_median8(rp, r, c);
            *reinterpret_cast<uint32_t*>(out + size_t(r) * pitch + c) = v.x;
            if (r + 1 < rows) *reinterpret_cast<uint32_t*>(out + size_t(r + 1) * pitch + c) = v.y;
        }
    } else {
        for (int i = threadIdx.x; i < G * TH; i += NT) {
            const int c = 4 * (i % G), r = i / G;
            if (c >= cols || r >= rows) continue;
            *reinterpret_cast<uint32_t*>(out + size_t(r) * pitch + c) = filt_plain4(rp, r, c);
        }
    }
}

}  // namespace dmsgm

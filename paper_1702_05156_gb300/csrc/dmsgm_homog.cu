// dmsgm_homog.cu -- the motion-estimation front end on the GPU: Shi-Tomasi
// corners of the previous frame, Bouguet's pyramidal Lucas-Kanade into the
// current one (Sec. 2.4, Sec. 3.1.3 and the motion-compensation appendix of
// arXiv:1702.05156), and the C ABI of dmsgm_homog.h.  The RANSAC that turns
// the tracked pairs into the homography is in dmsgm_homog_ransac.cu.
//
// Corners, one pass per step, all on the device (counts and cuts pass through
// a control block, no host round trip):
//   score    tiled: the frame tile with its halo and the Sobel gradients in
//            shared memory, the structure tensor summed over the window, the
//            score in FP32 in the fixed order of IEEE operations the method
//            defines for the tile and a one-pixel ring, the frame maximum
//            (atomicMax on the float bits, scores being >= 0), and the
//            tile's local maxima listed with their scores (the score map
//            itself is never stored);
//   select   the strongest 8192 candidates (listed maxima above the cut)
//            exactly, without sorting them all: a histogram of the scores'
//            high 16 bits finds the bucket of the cut, a second one of the
//            low 16 bits inside it the cut value; candidates above it are
//            kept, those at it (ties) are ordered by index;
//   sort     rank by counting over the GPU (keys are distinct: a key's rank
//            is the number of smaller ones), then a scatter;
//   spacing  one warp takes the sorted candidates 32 at a time: each lane
//            checks the kept corners of the 3 x 3 cells around it (linked
//            lists per cell of at least ceil(min_distance) pixels, in shared
//            memory) and the earlier lanes of its group, and the group is
//            resolved in order with warp shuffles.
// Tracking: one CTA per point; per level the window's previous-frame samples
// (intensity and both gradients, bilinear) stay in shared memory for the
// iterations, which sample a staged patch of the current frame (restaged only
// when the update leaves it) and reduce across the CTA in a fixed order.
#include <cmath>
#include <cstring>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "dmsgm_homog.cuh"

namespace dmsgm {

__device__ __forceinline__ int clampi_d(int v, int lo, int hi) { return min(max(v, lo), hi); }

// ---------------------------------------------------------------- scores
constexpr int kScTX = 64, kScTY = 32;   // 256 threads, 8 pixels each

// Scores of a kScTX x kScTY tile and the ring of pixels around it (the
// neighbours of the local-maximum test), from the clamped frame tile and its
// Sobel gradients in shared memory; the tile's maximum goes to the frame's
// maximum (one atomicMax per CTA), and the tile's interior local maxima with
// a positive score are listed as keys (~score bits << 32 | index), one
// global atomic per CTA for their slots.  A candidate (Sec. 2.4 corners:
// a local maximum above quality x the frame's maximum) is a listed key above
// the cut, so the later passes read the list, not the frame.
template <int BS>
__global__ void __launch_bounds__(256) ho_score_kernel(const uint8_t* const* __restrict__ frames,
                                                       int W, int H,
                                                       unsigned long long* __restrict__ lmax,
                                                       uint32_t* __restrict__ ctrl) {
    const uint8_t* __restrict__ img = frames[0];
    constexpr int r = BS / 2;
    constexpr int SW = kScTX + 2, SH = kScTY + 2;     // scores: the tile and a 1-pixel ring
    constexpr int GW = SW + 2 * r, GH = SH + 2 * r;   // gradients of their window positions
    constexpr int IW = GW + 2, IH = GH + 2;           // staged pixels (clamped)
    constexpr int ROWS = kScTY / (256 / kScTX);
    __shared__ uint8_t px[IH][IW];
    __shared__ short gx[GH][GW], gy[GH][GW];
    __shared__ float sc[SH][SW];
    __shared__ uint32_t wmax[8], wcnt[8], base;
    const int x0 = blockIdx.x * kScTX, y0 = blockIdx.y * kScTY;
    const int px0 = x0 - 2 - r, py0 = y0 - 2 - r;     // frame position of px[0][0]
    for (int i = threadIdx.x; i < IW * IH; i += 256) {
        const int yy = i / IW, xx = i - yy * IW;
        px[yy][xx] = img[size_t(clampi_d(py0 + yy, 0, H - 1)) * W + clampi_d(px0 + xx, 0, W - 1)];
    }
    __syncthreads();
    // the gradient of a window position is that of the clamped position
    for (int i = threadIdx.x; i < GW * GH; i += 256) {
        const int yy = i / GW, xx = i - yy * GW;
        const int cx = clampi_d(x0 - 1 - r + xx, 0, W - 1) - px0;
        const int cy = clampi_d(y0 - 1 - r + yy, 0, H - 1) - py0;
        gx[yy][xx] = short((px[cy - 1][cx + 1] + 2 * px[cy][cx + 1] + px[cy + 1][cx + 1]) -
                           (px[cy - 1][cx - 1] + 2 * px[cy][cx - 1] + px[cy + 1][cx - 1]));
        gy[yy][xx] = short((px[cy + 1][cx - 1] + 2 * px[cy + 1][cx] + px[cy + 1][cx + 1]) -
                           (px[cy - 1][cx - 1] + 2 * px[cy - 1][cx] + px[cy - 1][cx + 1]));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < SW * SH; i += 256) {
        const int yy = i / SW, xx = i - yy * SW;
        int A = 0, B = 0, C = 0;
#pragma unroll
        for (int j = 0; j < BS; ++j)
#pragma unroll
            for (int q = 0; q < BS; ++q) {
                const int a = gx[yy + j][xx + q], b = gy[yy + j][xx + q];
                A += a * a;
                B += a * b;
                C += b * b;
            }
        const float fa = __int2float_rn(A), fb = __int2float_rn(B), fc = __int2float_rn(C);
        const float t = __fadd_rn(fa, fc);
        const float d = __fsub_rn(fa, fc);
        const float e = __fmul_rn(d, d);
        const float f = __fmul_rn(fb, fb);
        const float g = __fmul_rn(4.0f, f);
        const float rr = __fsqrt_rn(__fadd_rn(e, g));
        const float v = __fmul_rn(0.5f, __fsub_rn(t, rr));
        sc[yy][xx] = v > 0.0f ? v : 0.0f;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tx = threadIdx.x % kScTX, ty0 = threadIdx.x / kScTX;
    const int x = x0 + tx;
    uint32_t bits = 0, nl = 0;
    unsigned long long kk[ROWS];
#pragma unroll
    for (int q = 0; q < ROWS; ++q) {
        const int ty = ty0 + q * (256 / kScTX), y = y0 + ty;
        kk[q] = 0ull;
        if (x >= W || y >= H) continue;
        const float v = sc[ty + 1][tx + 1];
        bits = max(bits, __float_as_uint(v));
        if (x < 1 || y < 1 || x > W - 2 || y > H - 2 || !(v > 0.0f)) continue;
        bool lm = true;
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i)
                if ((i != 1 || j != 1) && sc[ty + j][tx + i] > v) lm = false;
        if (!lm) continue;
        kk[q] = (static_cast<unsigned long long>(~__float_as_uint(v)) << 32) | uint32_t(y * W + x);
        ++nl;
    }
    bits = __reduce_max_sync(0xffffffffu, bits);
    const uint32_t wn = __reduce_add_sync(0xffffffffu, nl);
    uint32_t pre = nl;   // inclusive prefix in the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, pre, o);
        if (lane >= o) pre += y;
    }
    if (lane == 0) {
        wmax[warp] = bits;
        wcnt[warp] = wn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t m = 0, tot = 0;
        for (int w = 0; w < 8; ++w) {
            m = max(m, wmax[w]);
            const uint32_t c = wcnt[w];
            wcnt[w] = tot;   // exclusive prefix over warps
            tot += c;
        }
        if (m) atomicMax(&ctrl[kCtrlMaxBits], m);
        base = tot ? atomicAdd(&ctrl[kCtrlLocalMax], tot) : 0u;
    }
    __syncthreads();
    uint32_t slot = base + wcnt[warp] + pre - nl;
#pragma unroll
    for (int q = 0; q < ROWS; ++q)
        if (kk[q]) lmax[slot++] = kk[q];
}

// ---------------------------------------------------------------- candidates
// Passes over the listed local maxima (grid-stride, 2048 keys per CTA and
// round).  A candidate is a listed key whose score is above the cut
// quality x max (FP32 product).  mode 0: histogram of the candidates' high 16
// score bits and their count; 1: histogram of the low 16 bits inside the
// cut's bucket; 2: collect the keys above / at the cut.  Counts and key slots
// are aggregated per CTA (one global atomic per CTA, round and counter);
// histogram buckets take one atomic per distinct bucket in a warp.
// The high-bits histogram of mode 0 is gathered in shared memory when the
// candidates' high 16 bits (those of the cut up to those of the maximum) span
// at most kCandSpan buckets, and added to the global one once per CTA and
// bucket: the busiest buckets would otherwise take one global atomic per
// warp from every CTA.
constexpr int kCandPer = 8;
constexpr int kCandSpan = 8192;

__global__ void __launch_bounds__(256) ho_cand_kernel(const unsigned long long* __restrict__ lmax,
                                                      double quality, int mode, uint32_t* ctrl,
                                                      uint32_t* hist_hi, uint32_t* hist_lo,
                                                      unsigned long long* keys) {
    __shared__ uint32_t cnt[2], base[2];
    __shared__ uint32_t shist[kCandSpan];
    if (mode == 1 && ctrl[kCtrlTakeAll]) return;
    const uint32_t n = ctrl[kCtrlLocalMax];
    const uint32_t maxbits = ctrl[kCtrlMaxBits];
    const float thr = __fmul_rn(__double2float_rn(quality), __uint_as_float(maxbits));
    const int lane = threadIdx.x & 31;
    const uint32_t below = (1u << lane) - 1u;
    const bool take_all = ctrl[kCtrlTakeAll] != 0;
    const uint32_t hi_cut = ctrl[kCtrlHiCut], cut = ctrl[kCtrlCut];
    // candidates have bits > thr's, so their high 16 bits lie in [lo, maxbits >> 16]
    const uint32_t lo = __float_as_uint(thr) >> 16;
    const uint32_t span = (maxbits >> 16) - lo + 1u;
    const bool local = mode == 0 && span <= uint32_t(kCandSpan) && uint32_t(blockIdx.x) * 256u * kCandPer < n;
    if (local)
        for (uint32_t b = threadIdx.x; b < span; b += 256) shist[b] = 0;
    for (uint32_t c0 = blockIdx.x * 256u * kCandPer; c0 < n; c0 += gridDim.x * 256u * kCandPer) {
        if (threadIdx.x < 2) cnt[threadIdx.x] = 0;
        __syncthreads();
        unsigned long long kq[kCandPer];
        uint32_t ng = 0, ne = 0;   // this thread's keys above / at the cut
#pragma unroll
        for (int q = 0; q < kCandPer; ++q) {
            const uint32_t k = c0 + q * 256u + threadIdx.x;
            const unsigned long long key = k < n ? lmax[k] : 0ull;
            const uint32_t bits = ~uint32_t(key >> 32);
            const bool cand = k < n && __uint_as_float(bits) > thr;
            kq[q] = cand ? key : 0ull;
            if (mode == 0) {
                const uint32_t peers = __match_any_sync(0xffffffffu, cand ? (bits >> 16) : 0xFFFFFFFFu);
                if (cand && (peers & below) == 0u) {
                    if (local) atomicAdd(&shist[(bits >> 16) - lo], uint32_t(__popc(peers)));
                    else atomicAdd(&hist_hi[bits >> 16], uint32_t(__popc(peers)));
                }
                ng += cand;
            } else if (mode == 1) {
                const bool in = cand && (bits >> 16) == hi_cut;
                const uint32_t peers = __match_any_sync(0xffffffffu, in ? (bits & 0xFFFFu) : 0xFFFFFFFFu);
                if (in && (peers & below) == 0u) atomicAdd(&hist_lo[bits & 0xFFFFu], uint32_t(__popc(peers)));
            } else {
                ng += cand && (take_all || bits > cut);
                ne += cand && !take_all && bits == cut;
            }
        }
        if (mode == 1) continue;
        const uint32_t wg = __reduce_add_sync(0xffffffffu, ng), we = __reduce_add_sync(0xffffffffu, ne);
        uint32_t pg = ng, pe = ne;   // inclusive prefixes in the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t a1 = __shfl_up_sync(0xffffffffu, pg, o), a2 = __shfl_up_sync(0xffffffffu, pe, o);
            if (lane >= o) {
                pg += a1;
                pe += a2;
            }
        }
        pg -= ng;
        pe -= ne;
        uint32_t wbase_g = 0, wbase_e = 0;
        if (lane == 0) {
            wbase_g = atomicAdd(&cnt[0], wg);
            wbase_e = atomicAdd(&cnt[1], we);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (mode == 0) {
                if (cnt[0]) atomicAdd(&ctrl[kCtrlCand], cnt[0]);
            } else {
                base[0] = cnt[0] ? atomicAdd(&ctrl[kCtrlNGt], cnt[0]) : 0u;
                base[1] = cnt[1] ? atomicAdd(&ctrl[kCtrlNEq], cnt[1]) : 0u;
            }
        }
        __syncthreads();
        if (mode == 0) continue;
        uint32_t kg = base[0] + __shfl_sync(0xffffffffu, wbase_g, 0) + pg;
        uint32_t ke = base[1] + __shfl_sync(0xffffffffu, wbase_e, 0) + pe;
#pragma unroll
        for (int q = 0; q < kCandPer; ++q) {
            const unsigned long long key = kq[q];
            if (!key) continue;
            const uint32_t bits = ~uint32_t(key >> 32);
            if (take_all || bits > cut) {
                if (kg < uint32_t(kHoKmax)) keys[kg] = key;   // < kHoKmax by the cut
                else ctrl[kCtrlOverflow] = 1;
                ++kg;
            } else if (bits == cut) {
                if (ke < uint32_t(kHoTieCap)) keys[kHoKmax + ke] = key;
                else ctrl[kCtrlOverflow] = 1;
                ++ke;
            }
        }
    }
    if (local) {
        __syncthreads();
        for (uint32_t b = threadIdx.x; b < span; b += 256)
            if (shist[b]) atomicAdd(&hist_hi[lo + b], shist[b]);
    }
}

// Inclusive-from-the-top scan of a 65536-bucket histogram by one CTA of 1024
// threads: the bucket b where the count of buckets above b is < need and
// that count plus hist[b] reaches it; *above = that count.
__device__ void ho_find_cut(const uint32_t* hist, uint32_t need, uint32_t* cut, uint32_t* above) {
    __shared__ uint32_t warp_sum[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int top = 65535 - 64 * t;   // this thread's buckets: top, top - 1, .., top - 63
    uint32_t local = 0;
    const uint4* h4 = reinterpret_cast<const uint4*>(hist + (top - 63));
    uint4 v4[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) v4[q] = h4[q];
#pragma unroll
    for (int q = 0; q < 16; ++q) local += v4[q].x + v4[q].y + v4[q].z + v4[q].w;
    // exclusive prefix over threads (thread 0 holds the highest buckets)
    uint32_t v = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t n = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += n;
    }
    if (lane == 31) warp_sum[warp] = v;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = warp_sum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t n = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += n;
        }
        warp_sum[lane] = w;
    }
    __syncthreads();
    const uint32_t before = (warp ? warp_sum[warp - 1] : 0u) + v - local;
    if (before < need && before + local >= need) {
        // this thread's buckets again (16 independent loads), then from the top
        uint4 r4[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) r4[q] = h4[q];
        uint32_t cum = before;
        bool found = false;
#pragma unroll
        for (int b = 0; b < 64; ++b) {
            const uint4 q4 = r4[15 - b / 4];
            const int e = 3 - b % 4;
            const uint32_t h = e == 0 ? q4.x : e == 1 ? q4.y : e == 2 ? q4.z : q4.w;
            if (!found && cum + h >= need) {
                *cut = uint32_t(top - b);
                *above = cum;
                found = true;
            }
            cum += h;
        }
    }
}

// stage 0: after the high histogram; stage 1: after the low one
__global__ void __launch_bounds__(1024) ho_select_kernel(int stage, uint32_t* ctrl,
                                                         const uint32_t* hist_hi,
                                                         const uint32_t* hist_lo) {
    __shared__ uint32_t cut, above;
    if (threadIdx.x == 0) {
        cut = 0;
        above = 0;
    }
    __syncthreads();
    if (stage == 0) {
        if (ctrl[kCtrlCand] <= uint32_t(kHoKmax)) {
            if (threadIdx.x == 0) ctrl[kCtrlTakeAll] = 1;
            return;
        }
        ho_find_cut(hist_hi, kHoKmax, &cut, &above);
        __syncthreads();
        if (threadIdx.x == 0) {
            ctrl[kCtrlHiCut] = cut;
            ctrl[kCtrlAboveHi] = above;
        }
    } else {
        if (ctrl[kCtrlTakeAll]) return;
        const uint32_t a = ctrl[kCtrlAboveHi];
        ho_find_cut(hist_lo, kHoKmax - a, &cut, &above);
        __syncthreads();
        if (threadIdx.x == 0) ctrl[kCtrlCut] = (ctrl[kCtrlHiCut] << 16) | cut;
    }
}

// The collected keys in ascending order (score descending, index ascending)
// by counting: keys are distinct, so a key's rank is the number of smaller
// keys.  Every key above the cut is smaller than every key at it, so the
// two regions rank separately (the ties after the ngt keys above).  rank:
// CTA (x, y) counts, for its 256 keys of a region, the smaller keys in the
// y-th of kHoRankSplit ranges of that region (staged in shared memory);
// scatter: the partial counts add up to the rank, and keys ranked below
// kHoKmax are written to it.
constexpr int kRankCtasGt = kHoKmax / 256, kRankCtasEq = kHoTieCap / 256;
constexpr int kRankChunk = (kHoKmax + kHoRankSplit - 1) / kHoRankSplit;

__device__ __forceinline__ void ho_regions(const uint32_t* ctrl, int& ngt, int& neq) {
    ngt = int(min(ctrl[kCtrlNGt], uint32_t(kHoKmax)));
    neq = int(min(ctrl[kCtrlNEq], uint32_t(kHoTieCap)));
}

__global__ void __launch_bounds__(256) ho_rank_kernel(const uint32_t* ctrl,
                                                      const unsigned long long* __restrict__ keys,
                                                      uint32_t* __restrict__ part) {
    __shared__ __align__(16) unsigned long long sk[kRankChunk];
    int ngt, neq;
    ho_regions(ctrl, ngt, neq);
    const bool tie = blockIdx.x >= kRankCtasGt;
    const int off = tie ? kHoKmax : 0, nreg = tie ? neq : ngt;
    const int i0 = (int(blockIdx.x) - (tie ? kRankCtasGt : 0)) * 256;
    if (i0 >= nreg) return;   // the whole CTA
    const int chunk = (nreg + kHoRankSplit - 1) / kHoRankSplit;
    const int j0 = int(blockIdx.y) * chunk, nj = max(0, min(nreg, j0 + chunk) - j0);
    for (int j = threadIdx.x; j < nj; j += 256) sk[j] = keys[off + j0 + j];
    if ((nj & 1) && threadIdx.x == 0) sk[nj] = ~0ull;   // pads the last pair (counted as larger)
    __syncthreads();
    const int i = i0 + int(threadIdx.x);
    if (i >= nreg) return;
    const unsigned long long ki = keys[off + i];
    uint32_t c0 = 0, c1 = 0;
    const ulonglong2* s2 = reinterpret_cast<const ulonglong2*>(sk);
#pragma unroll 8
    for (int j = 0; j < (nj + 1) / 2; ++j) {
        const ulonglong2 v = s2[j];
        c0 += v.x < ki;
        c1 += v.y < ki;
    }
    part[size_t(blockIdx.y) * kHoSortCap + off + i] = c0 + c1;
}

__global__ void __launch_bounds__(256) ho_scatter_kernel(uint32_t* ctrl,
                                                         const unsigned long long* __restrict__ keys,
                                                         const uint32_t* __restrict__ part,
                                                         unsigned long long* __restrict__ sel) {
    int ngt, neq;
    ho_regions(ctrl, ngt, neq);
    const int slot = int(blockIdx.x) * 256 + int(threadIdx.x);
    const bool tie = slot >= kHoKmax;
    const int i = slot - (tie ? kHoKmax : 0);
    if (i < (tie ? neq : ngt)) {
        uint32_t r = tie ? uint32_t(ngt) : 0u;
#pragma unroll
        for (int y = 0; y < kHoRankSplit; ++y) r += part[size_t(y) * kHoSortCap + slot];
        if (r < uint32_t(kHoKmax)) sel[r] = keys[slot];
    }
    if (slot == 0) ctrl[kCtrlNSel] = uint32_t(min(ngt + neq, kHoKmax));
}

// One warp.  Dynamic shared memory (when min_distance > 1): the kept
// corners as linked lists per cell -- head[gw * gh], next[max_corners],
// position[max_corners] -- with cells of `cell` >= ceil(min_distance) pixels,
// so that any corner closer than min_distance lies in the 3 x 3 cells around.
// Distances are compared as integers: for an integer d2, d2 < md2 (md2 =
// min_distance^2 in FP64) exactly when d2 < ceil(md2) = t2, which the host
// computes.  A group of 32 candidates is resolved in order: a lane that is
// not blocked by a kept corner and has no earlier conflicting lane in its
// group is kept outright, and the lanes with such conflicts are visited in
// lane order, each kept when none of the lanes kept before it conflicts.
__global__ void __launch_bounds__(32) ho_spacing_kernel(uint32_t* ctrl,
                                                        const unsigned long long* __restrict__ sel,
                                                        int W, int t2, int max_corners, int gw,
                                                        int gh, int cell, int* corners,
                                                        float* cscore, float2* pts) {
    extern __shared__ int ssm[];
    const int lane = threadIdx.x;
    const uint32_t below = (1u << lane) - 1u;
    const int n = int(ctrl[kCtrlNSel]);
    const bool spaced = t2 > 1;   // distinct pixels are >= 1 apart
    int* head = ssm;
    int* nxt = head + gw * gh;
    int* pos = nxt + max_corners;
    if (spaced) {
        for (int i = lane; i < gw * gh; i += 32) head[i] = -1;
        __syncwarp();
    }
    int count = 0;
    for (int g = 0; g < n && count < max_corners; g += 32) {
        const int k = g + lane;
        const bool valid = k < n;
        const unsigned long long key = valid ? sel[k] : 0ull;
        const int idx = int(uint32_t(key));
        const int x = idx % W, y = idx / W;
        bool blocked = !valid;
        uint32_t conf = 0;
        if (spaced) {
            if (valid) {
                const int cx = x / cell, cy = y / cell;
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int qx = cx + dx, qy = cy + dy;
                        if (qx < 0 || qy < 0 || qx >= gw || qy >= gh) continue;
                        for (int e = head[qy * gw + qx]; e >= 0; e = nxt[e]) {
                            const int ddx = x - (pos[e] & 0xFFFF), ddy = y - (pos[e] >> 16);
                            if (ddx * ddx + ddy * ddy < t2) blocked = true;
                        }
                    }
            }
#pragma unroll 8
            for (int j = 0; j < 32; ++j) {
                const int xj = __shfl_sync(0xffffffffu, x, j), yj = __shfl_sync(0xffffffffu, y, j);
                const int ddx = x - xj, ddy = y - yj;
                if (j < lane && g + j < n && ddx * ddx + ddy * ddy < t2) conf |= 1u << j;
            }
        }
        const uint32_t cl = __ballot_sync(0xffffffffu, !blocked && conf != 0u);
        uint32_t acc = __ballot_sync(0xffffffffu, !blocked) & ~cl;
        for (uint32_t rem = cl; rem; rem &= rem - 1u) {
            const int i = __ffs(rem) - 1;
            if ((__shfl_sync(0xffffffffu, conf, i) & acc) == 0u) acc |= 1u << i;
        }
        // the count cap keeps the first kept lanes
        while (__popc(acc) > max_corners - count) acc &= ~(1u << (31 - __clz(acc)));
        if ((acc >> lane) & 1u) {
            const int p = count + __popc(acc & below);
            corners[2 * p] = x;
            corners[2 * p + 1] = y;
            cscore[p] = __uint_as_float(~uint32_t(key >> 32));
            pts[p] = make_float2(float(x), float(y));
            if (spaced) {
                pos[p] = x | (y << 16);
                nxt[p] = atomicExch(&head[(y / cell) * gw + x / cell], p);
            }
        }
        __syncwarp();
        count += __popc(acc);
    }
    if (lane == 0) {
        ctrl[kCtrlNCorners] = uint32_t(count);
        ctrl[kCtrlNPts] = uint32_t(count);
    }
}

// ---------------------------------------------------------------- pyramid
// 4 horizontally adjacent outputs per thread: a CTA covers 128 x 8 outputs.
// in0 / in1 NULL: the level below is the frame pair itself (the slot).
__global__ void __launch_bounds__(256) ho_pyr_kernel(const uint8_t* in0, const uint8_t* in1,
                                                     const uint8_t* const* frames, int w, int h,
                                                     uint8_t* __restrict__ out0,
                                                     uint8_t* __restrict__ out1, int w2, int h2) {
    const uint8_t* __restrict__ in = in0 ? (blockIdx.z ? in1 : in0) : frames[blockIdx.z];
    uint8_t* out = blockIdx.z ? out1 : out0;
    const int xb = blockIdx.x * 128 + 4 * (threadIdx.x & 31), y = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (xb >= w2 || y >= h2) return;
    const int k[5] = {1, 4, 6, 4, 1};
    int cs[11];   // vertical sums of input columns 2 xb - 2 .. 2 xb + 8
#pragma unroll
    for (int c = 0; c < 11; ++c) cs[c] = 0;
#pragma unroll
    for (int j = -2; j <= 2; ++j) {
        const uint8_t* row = in + size_t(clampi_d(2 * y + j, 0, h - 1)) * w;
#pragma unroll
        for (int c = 0; c < 11; ++c) cs[c] += k[j + 2] * row[clampi_d(2 * xb - 2 + c, 0, w - 1)];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (xb + q >= w2) break;
        int v = 0;
#pragma unroll
        for (int i = 0; i < 5; ++i) v += k[i] * cs[2 * q + i];
        out[size_t(y) * w2 + xb + q] = uint8_t((v + 128) >> 8);
    }
}

// ---------------------------------------------------------------- tracking
struct HoTrackArgs {
    HoPyr P, Q;                     // levels 1..; level 0 is the frame pair (the slot)
    const uint8_t* const* frames;
    int levels, wh, max_iters, n_fixed;
    float eps2, min_eig;
    const float2* pts;
    const uint32_t* npts;   // device count (NULL: n_fixed)
    float2* out;
    uint8_t* status;
};

constexpr int kTrackThreads = 128;   // one CTA per point
constexpr size_t kHoSpaceMax = 200 * 1024;  // shared memory of the spacing kernel

static size_t ho_spacing_smem(int gw, int gh, int max_corners) {
    return sizeof(int) * (size_t(gw) * gh + 2 * size_t(max_corners));
}

__device__ __forceinline__ float ho_px(const uint8_t* p, int w, int h, int x, int y) {
    return float(p[size_t(clampi_d(y, 0, h - 1)) * w + clampi_d(x, 0, w - 1)]);
}

__device__ __forceinline__ float ho_bil(float v00, float v10, float v01, float v11, float fx,
                                        float fy) {
    return (1.0f - fx) * (1.0f - fy) * v00 + fx * (1.0f - fy) * v10 + (1.0f - fx) * fy * v01 +
           fx * fy * v11;
}

__device__ __forceinline__ float ho_wsum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// CTA sums of N <= 3 values, the same on every thread (a fixed order: warp
// trees, then warps 0..3).  red is one of two alternating 12-float slots:
// consecutive calls use different slots, so one barrier per call suffices
// (a slot is rewritten two calls later, after every thread has passed the
// barrier of the call in between).
template <int N>
__device__ __forceinline__ void ho_csum(float (&v)[3], float* red) {
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = ho_wsum(v[i]);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int i = 0; i < N; ++i) red[3 * w + i] = v[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = ((red[i] + red[3 + i]) + red[6 + i]) + red[9 + i];
}

constexpr int kTrackMargin = 4;   // pixels staged around the current frame's window
constexpr int kTrackQ = (31 * 31 + kTrackThreads - 1) / kTrackThreads;   // samples per thread (win_half <= 15)

// shared floats per tracking CTA: a pixel patch (the previous frame's, side
// ws + 3; the current frame's, side ws + 1 + 2 margins, reused while the
// iterations stay inside it)
__host__ __device__ constexpr int ho_track_floats(int wh) {
    return (2 * wh + 2 + 2 * kTrackMargin) * (2 * wh + 2 + 2 * kTrackMargin);
}

// One CTA per point.  Thread t owns the window samples s = t + 128 q: their
// offsets and, per level, the previous frame's intensity and gradients stay
// in its registers; the iterations sum the mismatch over them in the order
// of s, then across the CTA.
__global__ void __launch_bounds__(kTrackThreads) ho_track_kernel(const HoTrackArgs a) {
    extern __shared__ float pt[];
    __shared__ float red[2][12];
    const int tid = threadIdx.x;
    const int k = blockIdx.x;
    const int n = a.npts ? int(*a.npts) : a.n_fixed;
    if (k >= n) return;   // the whole CTA
    const int wh = a.wh, ws = 2 * wh + 1, NS = ws * ws;
    const int PS = ws + 3, QS = ws + 1 + 2 * kTrackMargin;
    int sij[kTrackQ];   // (j << 16) | i of sample t + 128 q, -1 past the window
#pragma unroll
    for (int q = 0; q < kTrackQ; ++q) {
        const int s = tid + kTrackThreads * q;
        const int j = s / ws;
        sij[q] = s < NS ? (j << 16) | (s - j * ws) : -1;
    }
    float sI[kTrackQ], sX[kTrackQ], sY[kTrackQ];
    int rb = 0;
    const float2 u = a.pts[k];
    float gx = 0.f, gy = 0.f, dx = 0.f, dy = 0.f;
    bool ok = true;
    for (int l = a.levels; l >= 0 && ok; --l) {
        const float sc = ldexpf(1.0f, -l);
        const float ux = u.x * sc, uy = u.y * sc;
        const uint8_t* P = l ? a.P.p[l] : a.frames[0];
        const int w = a.P.w[l], h = a.P.h[l];
        const float fx0 = floorf(ux), fy0 = floorf(uy);
        const int ix = int(fx0), iy = int(fy0);
        const float fx = ux - fx0, fy = uy - fy0;
        // the previous frame's pixels ix - wh - 1 .. ix + wh + 2 (and rows)
        for (int q = tid; q < PS * PS; q += kTrackThreads) {
            const int r = q / PS, c = q - r * PS;
            pt[q] = ho_px(P, w, h, ix - wh - 1 + c, iy - wh - 1 + r);
        }
        __syncthreads();
        float G[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int q = 0; q < kTrackQ; ++q) {
            sI[q] = sX[q] = sY[q] = 0.f;
            if (sij[q] < 0) continue;
            const float* b = pt + (sij[q] >> 16) * PS + (sij[q] & 0xFFFF);   // pixel (x0 - 1, y0 - 1)
            const float v11 = b[PS + 1], v12 = b[PS + 2], v21 = b[2 * PS + 1], v22 = b[2 * PS + 2];
            const float I = ho_bil(v11, v12, v21, v22, fx, fy);
            const float Ix = ho_bil(0.5f * (v12 - b[PS]), 0.5f * (b[PS + 3] - v11),
                                    0.5f * (v22 - b[2 * PS]), 0.5f * (b[2 * PS + 3] - v21), fx, fy);
            const float Iy = ho_bil(0.5f * (v21 - b[1]), 0.5f * (v22 - b[2]),
                                    0.5f * (b[3 * PS + 1] - v11), 0.5f * (b[3 * PS + 2] - v12), fx, fy);
            sI[q] = I;
            sX[q] = Ix;
            sY[q] = Iy;
            G[0] += Ix * Ix;
            G[1] += Ix * Iy;
            G[2] += Iy * Iy;
        }
        ho_csum<3>(G, red[rb]);   // also: every thread is done with the patch
        rb ^= 1;
        const float ga = G[0], gb = G[1], gc = G[2];
        const float det = ga * gc - gb * gb;
        const float lmin = 0.5f * ((ga + gc) - sqrtf((ga - gc) * (ga - gc) + 4.0f * gb * gb));
        if (lmin / float(NS) < a.min_eig || det == 0.0f) {
            ok = false;
            break;
        }
        const uint8_t* Qp = l ? a.Q.p[l] : a.frames[1];
        float vx = 0.f, vy = 0.f;
        int sx0 = 0, sy0 = 0;
        bool staged = false;
        for (int it = 0; it < a.max_iters; ++it) {
            const float qx = ux + gx + vx, qy = uy + gy + vy;
            const float qx0 = floorf(qx), qy0 = floorf(qy);
            const int jx = int(qx0), jy = int(qy0);
            const float qfx = qx - qx0, qfy = qy - qy0;
            // the window needs columns jx - wh .. jx + wh + 1 (and rows)
            const int ox = jx - wh - sx0, oy = jy - wh - sy0;
            if (!staged || ox < 0 || oy < 0 || ox > 2 * kTrackMargin || oy > 2 * kTrackMargin) {
                sx0 = jx - wh - kTrackMargin;
                sy0 = jy - wh - kTrackMargin;
                for (int q = tid; q < QS * QS; q += kTrackThreads) {
                    const int r = q / QS, c = q - r * QS;
                    pt[q] = ho_px(Qp, w, h, sx0 + c, sy0 + r);
                }
                __syncthreads();
                staged = true;
            }
            const float* pw = pt + (jy - wh - sy0) * QS + (jx - wh - sx0);
            float bb[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int q = 0; q < kTrackQ; ++q) {
                if (sij[q] < 0) continue;
                const float* b = pw + (sij[q] >> 16) * QS + (sij[q] & 0xFFFF);
                const float J = ho_bil(b[0], b[1], b[QS], b[QS + 1], qfx, qfy);
                const float d = sI[q] - J;
                bb[0] += d * sX[q];
                bb[1] += d * sY[q];
            }
            ho_csum<2>(bb, red[rb]);   // also: every thread is done with the patch
            rb ^= 1;
            const float ex = (gc * bb[0] - gb * bb[1]) / det;
            const float ey = (ga * bb[1] - gb * bb[0]) / det;
            vx += ex;
            vy += ey;
            if (ex * ex + ey * ey < a.eps2) break;
        }
        dx = vx;
        dy = vy;
        if (l > 0) {
            gx = 2.0f * (gx + dx);
            gy = 2.0f * (gy + dy);
        }
    }
    const float px = u.x + gx + dx, py = u.y + gy + dy;
    if (ok && !(px >= 0.0f && px <= float(a.P.w[0] - 1) && py >= 0.0f && py <= float(a.P.h[0] - 1)))
        ok = false;
    if (tid == 0) {
        a.out[k] = make_float2(px, py);
        a.status[k] = ok ? 1 : 0;
    }
}

// ---------------------------------------------------------------- launches
static int ho_check(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return DMSGM_OK;
    return fail(e == cudaErrorMemoryAllocation ? DMSGM_ERR_OOM : DMSGM_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

// The corners of the frame in slot 0.
static int ho_corner_launches(dmsgm_homog_ctx* h, cudaStream_t s) {
    const int W = h->W, H = h->H;
    const dim3 grid((W + kScTX - 1) / kScTX, (H + kScTY - 1) / kScTY);
    switch (h->p.block_size) {
        case 1: ho_score_kernel<1><<<grid, 256, 0, s>>>(h->fdev, W, H, h->lmax, h->ctrl); break;
        case 3: ho_score_kernel<3><<<grid, 256, 0, s>>>(h->fdev, W, H, h->lmax, h->ctrl); break;
        case 5: ho_score_kernel<5><<<grid, 256, 0, s>>>(h->fdev, W, H, h->lmax, h->ctrl); break;
        default: ho_score_kernel<7><<<grid, 256, 0, s>>>(h->fdev, W, H, h->lmax, h->ctrl); break;
    }
    for (int mode = 0; mode < 3; ++mode) {
        ho_cand_kernel<<<h->cand_ctas, 256, 0, s>>>(h->lmax, h->p.quality, mode, h->ctrl,
                                                    h->hist_hi, h->hist_lo, h->keys);
        if (mode < 2) ho_select_kernel<<<1, 1024, 0, s>>>(mode, h->ctrl, h->hist_hi, h->hist_lo);
    }
    ho_rank_kernel<<<dim3(kRankCtasGt + kRankCtasEq, kHoRankSplit), 256, 0, s>>>(h->ctrl, h->keys,
                                                                                  h->rank);
    ho_scatter_kernel<<<kHoSortCap / 256, 256, 0, s>>>(h->ctrl, h->keys, h->rank, h->sel);
    // d2 < min_distance^2 (FP64) <=> d2 < ceil(min_distance^2) for integer d2
    const double md2 = h->p.min_distance * h->p.min_distance;
    const int t2 = int(std::ceil(md2));
    ho_spacing_kernel<<<1, 32, ho_spacing_smem(h->gw, h->gh, h->p.max_corners), s>>>(
        h->ctrl, h->sel, W, t2, h->p.max_corners, h->gw, h->gh, h->cell, h->corners, h->cscore,
        h->pts_in);
    return ho_check(cudaGetLastError(), "corner kernels");
}

static void ho_pyramids(const dmsgm_homog_ctx* h, HoPyr* P, HoPyr* Q) {
    for (int l = 0; l <= h->p.levels; ++l) {
        P->w[l] = Q->w[l] = h->lw[l];
        P->h[l] = Q->h[l] = h->lh[l];
        P->p[l] = l ? h->pyr[0][l] : nullptr;   // level 0: the slot's frames
        Q->p[l] = l ? h->pyr[1][l] : nullptr;
    }
}

// Pyramids of the frame pair in the slot and the tracking of h->pts_in.
static int ho_track_launches(dmsgm_homog_ctx* h, int n_fixed, bool device_count, cudaStream_t s) {
    for (int l = 1; l <= h->p.levels; ++l) {
        const dim3 grid((h->lw[l] + 127) / 128, (h->lh[l] + 7) / 8, 2);
        ho_pyr_kernel<<<grid, 256, 0, s>>>(l > 1 ? h->pyr[0][l - 1] : nullptr,
                                           l > 1 ? h->pyr[1][l - 1] : nullptr, h->fdev,
                                           h->lw[l - 1], h->lh[l - 1], h->pyr[0][l], h->pyr[1][l],
                                           h->lw[l], h->lh[l]);
    }
    HoTrackArgs a;
    ho_pyramids(h, &a.P, &a.Q);
    a.frames = h->fdev;
    a.levels = h->p.levels;
    a.wh = h->p.win_half;
    a.max_iters = h->p.max_iters;
    a.n_fixed = n_fixed;
    a.eps2 = float(h->p.eps * h->p.eps);
    a.min_eig = float(h->p.min_eig);
    a.pts = h->pts_in;
    a.npts = device_count ? h->ctrl + kCtrlNPts : nullptr;
    a.out = h->pts_out;
    a.status = h->status;
    const size_t smem = size_t(ho_track_floats(a.wh)) * sizeof(float);
    const int n = device_count ? h->p.max_corners : n_fixed;
    if (n > 0)
        ho_track_kernel<<<n, kTrackThreads, smem, s>>>(a);
    return ho_check(cudaGetLastError(), "tracking kernels");
}

}  // namespace dmsgm

using namespace dmsgm;

// ---------------------------------------------------------------- C ABI
extern "C" {

void dmsgm_homog_default_params(dmsgm_homog_params* p) {
    if (!p) return;
    p->block_size = 3;
    p->quality = 0.01;
    p->min_distance = 10.0;
    p->max_corners = 500;
    p->levels = 5;
    p->win_half = 10;
    p->max_iters = 30;
    p->eps = 0.01;
    p->min_eig = 1e-3;
    p->ransac_iters = 2000;
    p->thresh = 3.0;
    p->seed = 0;
}

int dmsgm_homog_destroy(dmsgm_homog_t h) {
    if (!h) return DMSGM_OK;
    cudaStreamSynchronize(0);
    void* bufs[] = {h->lmax, h->zeroed, h->keys, h->sel, h->rank, h->corners, h->cscore,
                    h->pts_in, h->pts_out, h->status, h->src, h->dst, h->pf, h->inl, h->hyp, h->hypf,
                    h->hcount, h->fitpart, h->rout};
    for (void* b : bufs)
        if (b) cudaFree(b);
    for (int i = 0; i < 2; ++i)
        for (int l = 0; l <= kHoMaxLevels; ++l)
            if (h->pyr[i][l]) cudaFree(h->pyr[i][l]);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    if (h->fdev) cudaFree(h->fdev);
    if (h->host) cudaFreeHost(h->host);
    if (h->fhost) cudaFreeHost(h->fhost);
    delete h;
    return DMSGM_OK;
}

static cudaError_t ho_capture(dmsgm_homog_ctx* h);

int dmsgm_homog_create(int W, int H, const dmsgm_homog_params* pin, dmsgm_homog_t* out) {
    clear_error();
    if (!out) return fail(DMSGM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    dmsgm_homog_params p;
    dmsgm_homog_default_params(&p);
    if (pin) p = *pin;
    if (W < 16 || H < 16 || W > 16384 || H > 16384 || W % 16)
        return fail(DMSGM_ERR_INVALID_ARG, "frame %dx%d: need 16 <= W, H <= 16384 and W %% 16 == 0", W, H);
    if (p.block_size < 1 || p.block_size > 7 || p.block_size % 2 == 0 || !(p.quality > 0.0) ||
        !std::isfinite(p.quality) || !(p.min_distance >= 0.0) || !std::isfinite(p.min_distance) ||
        p.min_distance > 4096.0 || p.max_corners < 1 || p.max_corners > kHoMaxPts ||
        p.levels < 0 || p.levels > kHoMaxLevels || p.win_half < 1 || p.win_half > 15 ||
        p.max_iters < 1 || !(p.eps >= 0.0) || !std::isfinite(p.eps) || !(p.min_eig >= 0.0) ||
        !std::isfinite(p.min_eig) || p.ransac_iters < 1 || p.ransac_iters > 65536 ||
        !(p.thresh > 0.0) || !std::isfinite(p.thresh))
        return fail(DMSGM_ERR_INVALID_ARG, "invalid homography parameters");
    dmsgm_homog_ctx* h = new (std::nothrow) dmsgm_homog_ctx();
    if (!h) return fail(DMSGM_ERR_OOM, "out of host memory");
    h->W = W;
    h->H = H;
    h->p = p;
    cudaGetDevice(&h->device);
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess || sms < 1)
        sms = 1;
    h->cand_ctas = 2 * sms;   // the list passes' grid-stride CTAs
    // spacing cells: at least ceil(min_distance) pixels, widened until the
    // per-cell lists fit the spacing kernel's shared memory
    const int c0 = p.min_distance > 1.0 ? int(std::ceil(p.min_distance)) : 1;
    for (int f = 1;; ++f) {
        h->cell = c0 * f;
        h->gw = (W + h->cell - 1) / h->cell;
        h->gh = (H + h->cell - 1) / h->cell;
        if (p.min_distance <= 1.0) {
            h->gw = h->gh = 0;   // no spacing rule: no grid
            break;
        }
        if (ho_spacing_smem(h->gw, h->gh, p.max_corners) <= kHoSpaceMax) break;
    }
    h->lw[0] = W;
    h->lh[0] = H;
    for (int l = 1; l <= p.levels; ++l) {
        h->lw[l] = (h->lw[l - 1] + 1) / 2;
        h->lh[l] = (h->lh[l - 1] + 1) / 2;
    }
    const size_t zwords = kCtrlWords + 2 * 65536;
    cudaError_t e = cudaSuccess;
    auto al = [&](void** ptr, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
    };
    al(reinterpret_cast<void**>(&h->lmax), sizeof(unsigned long long) * size_t(W) * H);
    al(reinterpret_cast<void**>(&h->zeroed), sizeof(uint32_t) * zwords);
    al(reinterpret_cast<void**>(&h->keys), sizeof(unsigned long long) * kHoSortCap);
    al(reinterpret_cast<void**>(&h->sel), sizeof(unsigned long long) * kHoKmax);
    al(reinterpret_cast<void**>(&h->rank), sizeof(uint32_t) * kHoRankSplit * kHoSortCap);
    al(reinterpret_cast<void**>(&h->corners), sizeof(int) * 2 * kHoMaxPts);
    al(reinterpret_cast<void**>(&h->cscore), sizeof(float) * kHoMaxPts);
    al(reinterpret_cast<void**>(&h->pts_in), sizeof(float2) * kHoMaxPts);
    al(reinterpret_cast<void**>(&h->pts_out), sizeof(float2) * kHoMaxPts);
    al(reinterpret_cast<void**>(&h->status), kHoMaxPts);
    al(reinterpret_cast<void**>(&h->src), sizeof(double) * 2 * kHoMaxPts);
    al(reinterpret_cast<void**>(&h->dst), sizeof(double) * 2 * kHoMaxPts);
    al(reinterpret_cast<void**>(&h->pf), sizeof(float4) * kHoMaxPts);
    al(reinterpret_cast<void**>(&h->inl), kHoMaxPts);
    al(reinterpret_cast<void**>(&h->hyp), sizeof(double) * 9 * size_t(p.ransac_iters));
    al(reinterpret_cast<void**>(&h->hcount), sizeof(int) * size_t(p.ransac_iters));
    al(reinterpret_cast<void**>(&h->hypf), sizeof(float) * 10 * size_t(p.ransac_iters));
    al(reinterpret_cast<void**>(&h->fitpart), sizeof(double) * kHoFitCtas * kHoFitTerms);
    al(reinterpret_cast<void**>(&h->rout), sizeof(HoRansacOut));
    for (int i = 0; i < 2; ++i)
        for (int l = 1; l <= p.levels; ++l)
            al(reinterpret_cast<void**>(&h->pyr[i][l]), size_t(h->lw[l]) * h->lh[l]);
    al(reinterpret_cast<void**>(&h->fdev), 2 * sizeof(const uint8_t*));
    if (e == cudaSuccess) e = cudaMallocHost(&h->host, 256 * 1024);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&h->fhost), 2 * sizeof(const uint8_t*));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(ho_spacing_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   int(kHoSpaceMax));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(ho_track_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   int(ho_track_floats(15) * sizeof(float)));
    if (e == cudaSuccess) {
        h->ctrl = h->zeroed;
        h->hist_hi = h->zeroed + kCtrlWords;
        h->hist_lo = h->hist_hi + 65536;
        e = ho_capture(h);
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        dmsgm_homog_destroy(h);
        return fail(e == cudaErrorMemoryAllocation ? DMSGM_ERR_OOM : DMSGM_ERR_CUDA,
                    "homography handle: %s", cudaGetErrorString(e));
    }
    *out = h;
    return DMSGM_OK;
}

static int ho_frame_ok(const dmsgm_homog_ctx* h, const uint8_t* f) {
    return f && reinterpret_cast<uintptr_t>(f) % 16 == 0;
}

// The frame pair into the device slot that the kernels read (a copy from
// pinned staging, so that a captured graph serves any pair; every entry
// point synchronises before it returns, so the staging is free again).
static int ho_set_frames(dmsgm_homog_ctx* h, const uint8_t* prev, const uint8_t* cur,
                         cudaStream_t s) {
    h->fhost[0] = prev;
    h->fhost[1] = cur;
    return ho_check(cudaMemcpyAsync(h->fdev, h->fhost, 2 * sizeof(const uint8_t*),
                                    cudaMemcpyHostToDevice, s), "frame slot");
}

// corners of the slot's first frame into the handle's buffers; counts in ctrl
static int ho_corners_dev(dmsgm_homog_ctx* h, cudaStream_t s) {
    const size_t zbytes = sizeof(uint32_t) * (kCtrlWords + 2 * 65536);
    int rc = ho_check(cudaMemsetAsync(h->zeroed, 0, zbytes, s), "clear");
    if (rc) return rc;
    return ho_corner_launches(h, s);
}

// The whole estimate after the frame slot is set: corners, tracking, RANSAC
// and the copies of the control words and the result into pinned memory.
// Captured once per handle into a CUDA graph.
static int ho_estimate_launches(dmsgm_homog_ctx* h, cudaStream_t s) {
    int rc = ho_check(cudaMemcpyAsync(h->fdev, h->fhost, 2 * sizeof(const uint8_t*),
                                      cudaMemcpyHostToDevice, s), "frame slot");
    if (!rc) rc = ho_corners_dev(h, s);
    if (!rc) rc = ho_track_launches(h, 0, true, s);
    if (!rc) rc = ho_launch_ransac(h, true, s);
    uint32_t* hc = static_cast<uint32_t*>(h->host);
    HoRansacOut* ho = reinterpret_cast<HoRansacOut*>(hc + kCtrlWords);
    if (!rc) rc = ho_check(cudaMemcpyAsync(hc, h->ctrl, sizeof(uint32_t) * kCtrlWords, cudaMemcpyDeviceToHost, s), "copy");
    if (!rc) rc = ho_check(cudaMemcpyAsync(ho, h->rout, sizeof(HoRansacOut), cudaMemcpyDeviceToHost, s), "copy");
    return rc;
}

static cudaError_t ho_capture(dmsgm_homog_ctx* h) {
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        const int rc = ho_estimate_launches(h, cs);
        e = cudaStreamEndCapture(cs, &g);
        if (e == cudaSuccess && rc) e = cudaErrorUnknown;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&h->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    return e;
}

int dmsgm_homog_corners(dmsgm_homog_t h, const uint8_t* img_dev, int* xy, float* scores, int* n,
                        int* n_cand, void* stream) {
    clear_error();
    if (!h || !ho_frame_ok(h, img_dev) || !xy || !n)
        return fail(DMSGM_ERR_INVALID_ARG, "NULL handle, output or misaligned frame");
    DeviceGuard dg(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = ho_set_frames(h, img_dev, img_dev, s);
    if (!rc) rc = ho_corners_dev(h, s);
    if (rc) return rc;
    uint32_t* hc = static_cast<uint32_t*>(h->host);
    int* hxy = reinterpret_cast<int*>(hc + kCtrlWords);
    float* hs = reinterpret_cast<float*>(hxy + 2 * kHoMaxPts);
    rc = ho_check(cudaMemcpyAsync(hc, h->ctrl, sizeof(uint32_t) * kCtrlWords, cudaMemcpyDeviceToHost, s), "copy");
    if (!rc) rc = ho_check(cudaMemcpyAsync(hxy, h->corners, sizeof(int) * 2 * h->p.max_corners, cudaMemcpyDeviceToHost, s), "copy");
    if (!rc) rc = ho_check(cudaMemcpyAsync(hs, h->cscore, sizeof(float) * h->p.max_corners, cudaMemcpyDeviceToHost, s), "copy");
    if (!rc) rc = ho_check(cudaStreamSynchronize(s), "corners");
    if (rc) return rc;
    if (hc[kCtrlOverflow])
        return fail(DMSGM_ERR_UNSUPPORTED, "more than %d candidates tied at the selection cut", kHoTieCap);
    const int m = int(hc[kCtrlNCorners]);
    memcpy(xy, hxy, sizeof(int) * 2 * m);
    if (scores) memcpy(scores, hs, sizeof(float) * m);
    *n = m;
    if (n_cand) *n_cand = int(hc[kCtrlCand]);
    return DMSGM_OK;
}

int dmsgm_homog_track(dmsgm_homog_t h, const uint8_t* prev_dev, const uint8_t* cur_dev,
                      const float* pts, int n, float* out, uint8_t* status, void* stream) {
    clear_error();
    if (!h || !ho_frame_ok(h, prev_dev) || !ho_frame_ok(h, cur_dev) || n < 0 || n > kHoMaxPts ||
        (n > 0 && (!pts || !out || !status)))
        return fail(DMSGM_ERR_INVALID_ARG, "invalid tracking arguments (n <= %d)", kHoMaxPts);
    if (n == 0) return DMSGM_OK;
    DeviceGuard dg(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float* hp = static_cast<float*>(h->host);
    memcpy(hp, pts, sizeof(float) * 2 * n);
    int rc = ho_check(cudaMemcpyAsync(h->pts_in, hp, sizeof(float) * 2 * n, cudaMemcpyHostToDevice, s), "copy");
    if (!rc) rc = ho_set_frames(h, prev_dev, cur_dev, s);
    if (!rc) rc = ho_track_launches(h, n, false, s);
    uint8_t* hs = reinterpret_cast<uint8_t*>(hp + 2 * kHoMaxPts);
    if (!rc) rc = ho_check(cudaMemcpyAsync(hp, h->pts_out, sizeof(float) * 2 * n, cudaMemcpyDeviceToHost, s), "copy");
    if (!rc) rc = ho_check(cudaMemcpyAsync(hs, h->status, n, cudaMemcpyDeviceToHost, s), "copy");
    if (!rc) rc = ho_check(cudaStreamSynchronize(s), "tracking");
    if (rc) return rc;
    memcpy(out, hp, sizeof(float) * 2 * n);
    memcpy(status, hs, n);
    return DMSGM_OK;
}

static void ho_result(const HoRansacOut& r, double* H3x3, dmsgm_homog_result* res) {
    if (r.inliers < 0) {
        for (int i = 0; i < 9; ++i) H3x3[i] = (i % 4 == 0) ? 1.0 : 0.0;
    } else {
        memcpy(H3x3, r.H, sizeof r.H);
    }
    if (res) {
        res->inliers = r.inliers;
        res->best = r.best;
    }
}

int dmsgm_homog_ransac(dmsgm_homog_t h, const double* src, const double* dst, int n,
                       double H3x3[9], uint8_t* inliers, dmsgm_homog_result* res, void* stream) {
    clear_error();
    if (!h || !H3x3 || n < 0 || n > kHoMaxPts || (n > 0 && (!src || !dst)))
        return fail(DMSGM_ERR_INVALID_ARG, "invalid RANSAC arguments (n <= %d)", kHoMaxPts);
    DeviceGuard dg(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* hd = static_cast<double*>(h->host);
    memcpy(hd, src, sizeof(double) * 2 * n);
    memcpy(hd + 2 * kHoMaxPts, dst, sizeof(double) * 2 * n);
    uint32_t* hn = reinterpret_cast<uint32_t*>(hd + 4 * kHoMaxPts);
    *hn = uint32_t(n);
    int rc = ho_check(cudaMemcpyAsync(h->src, hd, sizeof(double) * 2 * n, cudaMemcpyHostToDevice, s), "copy");
    if (!rc) rc = ho_check(cudaMemcpyAsync(h->dst, hd + 2 * kHoMaxPts, sizeof(double) * 2 * n, cudaMemcpyHostToDevice, s), "copy");
    if (!rc) rc = ho_check(cudaMemcpyAsync(h->ctrl + kCtrlNPairs, hn, sizeof(uint32_t), cudaMemcpyHostToDevice, s), "copy");
    if (!rc) rc = ho_launch_ransac(h, false, s);
    HoRansacOut* ho = reinterpret_cast<HoRansacOut*>(hn + 4);
    uint8_t* hi = reinterpret_cast<uint8_t*>(ho + 1);
    if (!rc) rc = ho_check(cudaMemcpyAsync(ho, h->rout, sizeof(HoRansacOut), cudaMemcpyDeviceToHost, s), "copy");
    if (!rc && n) rc = ho_check(cudaMemcpyAsync(hi, h->inl, n, cudaMemcpyDeviceToHost, s), "copy");
    if (!rc) rc = ho_check(cudaStreamSynchronize(s), "RANSAC");
    if (rc) return rc;
    ho_result(*ho, H3x3, res);
    if (inliers && n) memcpy(inliers, hi, n);
    return DMSGM_OK;
}

static int ho_estimate(dmsgm_homog_t h, const uint8_t* prev_dev, const uint8_t* cur_dev,
                       double H3x3[9], dmsgm_homog_result* res, void* stream);

int dmsgm_homog_estimate(dmsgm_homog_t h, const uint8_t* prev_dev, const uint8_t* cur_dev,
                         double H3x3[9], dmsgm_homog_result* res, void* stream) {
    clear_error();
    nvtxRangePushA("dmsgm_homog_estimate");
    const int rc = ho_estimate(h, prev_dev, cur_dev, H3x3, res, stream);
    nvtxRangePop();
    return rc;
}

static int ho_estimate(dmsgm_homog_t h, const uint8_t* prev_dev, const uint8_t* cur_dev,
                       double H3x3[9], dmsgm_homog_result* res, void* stream) {
    if (!h || !H3x3 || !ho_frame_ok(h, prev_dev) || !ho_frame_ok(h, cur_dev))
        return fail(DMSGM_ERR_INVALID_ARG, "NULL handle or output, or misaligned frame");
    DeviceGuard dg(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    h->fhost[0] = prev_dev;
    h->fhost[1] = cur_dev;
    int rc = ho_check(cudaGraphLaunch(h->graph, s), "homography graph");
    const uint32_t* hc = static_cast<const uint32_t*>(h->host);
    const HoRansacOut* ho = reinterpret_cast<const HoRansacOut*>(hc + kCtrlWords);
    if (!rc) rc = ho_check(cudaStreamSynchronize(s), "homography");
    if (rc) return rc;
    if (hc[kCtrlOverflow])
        return fail(DMSGM_ERR_UNSUPPORTED, "more than %d candidates tied at the selection cut", kHoTieCap);
    ho_result(*ho, H3x3, res);
    if (res) {
        res->corners = int(hc[kCtrlNCorners]);
        res->candidates = int(hc[kCtrlCand]);
        res->tracked = int(hc[kCtrlNPairs]);
    }
    return DMSGM_OK;
}

}  // extern "C"

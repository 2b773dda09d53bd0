// dmsgm_prefilter.cu -- the preprocessing of the paper's Sec. 2.1: an N x N
// Gaussian blur, then a 3 x 3 median, both clamping coordinates to the frame.
//
// The blur is exact integer arithmetic: 8-bit fixed-point 1-D weights q
// (sum 256) whose outer product is the 2-D kernel (sum 65536); the blurred
// pixel is floor(sum q_i q_j I / 65536), the paper's float sum cast to an
// 8-bit value made exact, so every result is reproducible bit for bit.  The
// 2-D sum is evaluated separably (rows, then columns), which is the same
// integer because clamping acts on each coordinate alone.  The median is the
// 5th of the 9 clamped neighbours of the blurred frame.
//
// One CTA filters a 128 x 32 output tile: it stages the clamped source
// region with its halo in shared memory, runs the horizontal pass into 16-bit
// sums (at most 255 * 256), the vertical pass into the blurred tile plus a
// one-pixel ring, and the median, 4 output pixels per thread and store.
#include <cmath>

#include "dmsgm_internal.h"

namespace dmsgm {

constexpr int kPfTW = 128, kPfTH = 32;   // output tile
constexpr int kPfMaxHalf = 7;            // Gaussian sizes up to 15
constexpr int kPfMaxR = kPfMaxHalf + 1;  // halo: blur half-size + median ring

struct PfArgs {
    int half;     // Gaussian half-size h (0: no blur)
    int median;   // 1: 3 x 3 median after the blur
    int q[2 * kPfMaxHalf + 1];
};

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

// Sorted (lo, mid, hi) of three values.
__device__ __forceinline__ void sort3(int a, int b, int c, int& lo, int& mid, int& hi) {
    const int x = min(a, b), y = max(a, b);
    lo = min(x, c);
    hi = max(y, c);
    mid = max(x, min(y, c));
}
__device__ __forceinline__ int med3(int a, int b, int c) { return max(min(a, b), min(max(a, b), c)); }

// HALF: the Gaussian half-size (0: no blur), so the tap loops unroll.
template <int HALF>
__global__ void __launch_bounds__(256) dmsgm_prefilter_kernel(const uint8_t* __restrict__ in,
                                                              uint8_t* __restrict__ out, int W,
                                                              int H, const PfArgs p) {
    constexpr int SW = kPfTW + 2 * kPfMaxR, SH = kPfTH + 2 * kPfMaxR, BW = kPfTW + 2;
    __shared__ uint8_t src[SH * SW];          // clamped source region
    __shared__ uint16_t hs[SH * BW];          // horizontal sums
    __shared__ uint8_t bl[(kPfTH + 2) * BW];  // blurred tile and its one-pixel ring
    const int tx0 = blockIdx.x * kPfTW, ty0 = blockIdx.y * kPfTH;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;   // 8 warps
    const int m = p.median ? 1 : 0, R = HALF + m;
    const int sw = kPfTW + 2 * R, sh = kPfTH + 2 * R;   // used source region
    const int bw = kPfTW + 2 * m, bh = kPfTH + 2 * m;   // used blurred region
    // warps take rows, lanes take columns (consecutive bytes: no bank conflicts)
    for (int i = warp; i < sh; i += 8) {
        const uint8_t* row = in + size_t(clampi(ty0 - R + i, 0, H - 1)) * W;
        for (int j = lane; j < sw; j += 32) src[i * SW + j] = row[clampi(tx0 - R + j, 0, W - 1)];
    }
    __syncthreads();
    // blurred pixel (bi, bj) of the tile, at (ty0 - m + bi, tx0 - m + bj),
    // reads source rows bi .. bi + 2 HALF and columns bj .. bj + 2 HALF
    if constexpr (HALF > 0) {
        for (int i = warp; i < sh; i += 8)
            for (int j = lane; j < bw; j += 32) {
                int s = 0;
#pragma unroll
                for (int t = 0; t <= 2 * HALF; ++t) s += p.q[t] * src[i * SW + j + t];
                hs[i * BW + j] = uint16_t(s);   // at most 255 * 256
            }
        __syncthreads();
        for (int i = warp; i < bh; i += 8)
            for (int j = lane; j < bw; j += 32) {
                int s = 0;
#pragma unroll
                for (int t = 0; t <= 2 * HALF; ++t) s += p.q[t] * hs[(i + t) * BW + j];
                bl[i * BW + j] = uint8_t(s >> 16);
            }
    } else {
        for (int i = warp; i < bh; i += 8)
            for (int j = lane; j < bw; j += 32) bl[i * BW + j] = src[i * SW + j];
    }
    __syncthreads();
    // output: each thread 4 consecutive pixels of one row (W % 16 == 0, so a
    // group never straddles the right edge)
    for (int g = threadIdx.x; g < kPfTH * (kPfTW / 4); g += blockDim.x) {
        const int oy = g / (kPfTW / 4), ox = 4 * (g % (kPfTW / 4));
        const int gy = ty0 + oy, gx = tx0 + ox;
        if (gy >= H || gx >= W) continue;
        uint32_t word = 0;
        if (m) {
            // the median's window clamps on the blurred frame: the rows and
            // columns of each neighbour, clamped, mapped into the tile's
            // blurred region; the 4 pixels share 6 sorted columns
            const int r0 = clampi(gy - 1, 0, H - 1) - (ty0 - 1), r1 = gy - (ty0 - 1);
            const int r2 = clampi(gy + 1, 0, H - 1) - (ty0 - 1);
            int lo[6], mid[6], hi[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                const int bj = clampi(gx - 1 + c, 0, W - 1) - (tx0 - 1);
                sort3(bl[r0 * BW + bj], bl[r1 * BW + bj], bl[r2 * BW + bj], lo[c], mid[c], hi[c]);
            }
            // sorted columns: the median of the 9 is the median of the
            // largest column minimum, the middle middle and the smallest maximum
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int v = med3(max(max(lo[k], lo[k + 1]), lo[k + 2]),
                                   med3(mid[k], mid[k + 1], mid[k + 2]),
                                   min(min(hi[k], hi[k + 1]), hi[k + 2]));
                word |= uint32_t(v) << (8 * k);
            }
        } else {
            const uint8_t* b = bl + oy * BW + ox;   // row pitch 130: bytes, not a word load
            word = uint32_t(b[0]) | uint32_t(b[1]) << 8 | uint32_t(b[2]) << 16 | uint32_t(b[3]) << 24;
        }
        *reinterpret_cast<uint32_t*>(out + size_t(gy) * W + gx) = word;
    }
}

// The 1-D weights: the normalised Gaussian rounded to 1/256 off the centre,
// the centre taking up the remainder so that the weights sum to 256.
static bool gauss_weights(int size, double sigma, int* q) {
    if (size < 3 || size % 2 == 0 || size > 2 * kPfMaxHalf + 1 || !(sigma > 0.0) ||
        !std::isfinite(sigma))
        return false;
    const int h = size / 2;
    double g[2 * kPfMaxHalf + 1], sum = 0.0;
    for (int x = -h; x <= h; ++x) {
        g[x + h] = std::exp(-double(x) * x / (2.0 * sigma * sigma));
        sum += g[x + h];
    }
    int rest = 0;
    for (int x = -h; x <= h; ++x)
        if (x != 0) {
            q[x + h] = int(std::floor(256.0 * g[x + h] / sum + 0.5));
            rest += q[x + h];
        }
    q[h] = 256 - rest;
    return true;
}

int launch_prefilter(const uint8_t* in_dev, uint8_t* out_dev, int W, int H, int gauss_size,
                     double sigma, int median, cudaStream_t s) {
    PfArgs p = {};
    p.median = median ? 1 : 0;
    if (gauss_size) {
        if (!gauss_weights(gauss_size, sigma, p.q))
            return fail(DMSGM_ERR_INVALID_ARG, "Gaussian size %d (odd, 3..15) or sigma %g invalid",
                        gauss_size, sigma);
        p.half = gauss_size / 2;
    }
    const dim3 grid((W + kPfTW - 1) / kPfTW, (H + kPfTH - 1) / kPfTH);
    switch (p.half) {
        case 0: dmsgm_prefilter_kernel<0><<<grid, 256, 0, s>>>(in_dev, out_dev, W, H, p); break;
        case 1: dmsgm_prefilter_kernel<1><<<grid, 256, 0, s>>>(in_dev, out_dev, W, H, p); break;
        case 2: dmsgm_prefilter_kernel<2><<<grid, 256, 0, s>>>(in_dev, out_dev, W, H, p); break;
        case 3: dmsgm_prefilter_kernel<3><<<grid, 256, 0, s>>>(in_dev, out_dev, W, H, p); break;
        case 4: dmsgm_prefilter_kernel<4><<<grid, 256, 0, s>>>(in_dev, out_dev, W, H, p); break;
        case 5: dmsgm_prefilter_kernel<5><<<grid, 256, 0, s>>>(in_dev, out_dev, W, H, p); break;
        case 6: dmsgm_prefilter_kernel<6><<<grid, 256, 0, s>>>(in_dev, out_dev, W, H, p); break;
        default: dmsgm_prefilter_kernel<7><<<grid, 256, 0, s>>>(in_dev, out_dev, W, H, p); break;
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(DMSGM_ERR_CUDA, "prefilter launch failed: %s", cudaGetErrorString(e));
    return DMSGM_OK;
}

}  // namespace dmsgm

using namespace dmsgm;

extern "C" int dmsgm_prefilter(const uint8_t* in_dev, uint8_t* out_dev, int W, int H,
                               int gauss_size, double sigma, int median, void* stream) {
    clear_error();
    if (!in_dev || !out_dev || W <= 0 || H <= 0 || W % 16 || W > (1 << 20) || H > (1 << 20))
        return fail(DMSGM_ERR_INVALID_ARG, "invalid frame %dx%d (W %% 16 == 0) or NULL buffer", W, H);
    if (reinterpret_cast<uintptr_t>(in_dev) % 16 || reinterpret_cast<uintptr_t>(out_dev) % 16)
        return fail(DMSGM_ERR_INVALID_ARG, "frames must be 16-byte aligned");
    const size_t n = size_t(W) * H;
    const uintptr_t a = reinterpret_cast<uintptr_t>(in_dev), b = reinterpret_cast<uintptr_t>(out_dev);
    if (a < b + n && b < a + n) return fail(DMSGM_ERR_INVALID_ARG, "in and out must not overlap");
    if (!gauss_size && !median) return fail(DMSGM_ERR_INVALID_ARG, "no filter selected");
    return launch_prefilter(in_dev, out_dev, W, H, gauss_size, sigma, median,
                            static_cast<cudaStream_t>(stream));
}

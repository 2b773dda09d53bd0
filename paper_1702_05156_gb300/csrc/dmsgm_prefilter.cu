// dmsgm_prefilter.cu -- the preprocessing of the paper's Sec. 2.1 as its own
// pass over a frame: an N x N Gaussian blur, then a 3 x 3 median, both
// clamping coordinates to the frame.  One CTA filters a kTileW x 32 tile with
// the shared-memory routines of dmsgm_filter.cuh (exact fixed-point blur,
// row-paired median) and writes it out.  Also here: the filter's weights.
#include <cmath>

#include "dmsgm_filter.cuh"
#include "dmsgm_internal.h"

namespace dmsgm {

constexpr int kPfTH = 32;   // tile rows of the standalone pass

// HALF: the Gaussian half-size (0: no blur), so the tap loops unroll.
template <int HALF>
__global__ void __launch_bounds__(256) dmsgm_prefilter_kernel(const uint8_t* __restrict__ in,
                                                              uint8_t* __restrict__ out, int W,
                                                              int H, const FiltArgs f) {
    __shared__ __align__(16) uint8_t src[filt_src_bytes<HALF, kPfTH>()];
    __shared__ __align__(16) uint32_t rp[filt_rp_words<kPfTH>()];
    const int tx0 = blockIdx.x * kTileW, ty0 = blockIdx.y * kPfTH;
    filt_stage<HALF, kPfTH, 256>(in, W, H, tx0, ty0, src);
    __syncthreads();
    filt_blur<HALF, kPfTH, 256>(f, src, rp);
    __syncthreads();
    filt_write<kPfTH, 256>(f, rp, tx0, ty0, W, H, out + size_t(ty0) * W + tx0, W,
                           min(kPfTH, H - ty0), min(kTileW, W - tx0));
}

// The 1-D weights: the normalised Gaussian rounded to 1/256 off the centre,
// the centre taking up the remainder so that the weights sum to 256.
static bool gauss_weights(int size, double sigma, int* q) {
    if (size < 3 || size % 2 == 0 || size > 2 * kFiltMaxHalf + 1 || !(sigma > 0.0) ||
        !std::isfinite(sigma))
        return false;
    const int h = size / 2;
    double g[2 * kFiltMaxHalf + 1], sum = 0.0;
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

bool make_filt_args(int gauss_size, double sigma, int median, FiltArgs* f, int* half) {
    *f = FiltArgs();
    f->median = median ? 1 : 0;
    *half = 0;
    if (!gauss_size) return true;
    int q[2 * kFiltMaxHalf + 1] = {0};
    if (!gauss_weights(gauss_size, sigma, q)) return false;
    const int h = gauss_size / 2;
    if (q[h] == 256) return true;   // every other weight is 0: the blur is the identity
    for (int t = 0; t <= 2 * h; ++t) {
        f->qb[t / 4] |= uint32_t(q[t]) << (8 * (t % 4));   // q_t <= 255 here
        f->qf[t] = float(q[t]) / 65536.0f;                 // exact: a power-of-2 scaling
    }
    *half = h;
    return true;
}

int launch_prefilter(const uint8_t* in_dev, uint8_t* out_dev, int W, int H, int gauss_size,
                     double sigma, int median, cudaStream_t s) {
    FiltArgs f;
    int half = 0;
    if (!make_filt_args(gauss_size, sigma, median, &f, &half))
        return fail(DMSGM_ERR_INVALID_ARG, "Gaussian size %d (odd, 3..15) or sigma %g invalid",
                    gauss_size, sigma);
    const dim3 grid((W + kTileW - 1) / kTileW, (H + kPfTH - 1) / kPfTH);
    switch (half) {
        case 0: dmsgm_prefilter_kernel<0><<<grid, 256, 0, s>>>(in_dev, out_dev, W, H, f); break;
        case 1: dmsgm_prefilter_kernel<1><<<grid, 256, 0, s>>>(in_dev, out_dev, W, H, f); break;
        case 2: dmsgm_prefilter_kernel<2><<<grid, 256, 0, s>>>(in_dev, out_dev, W, H, f); break;
        case 3: dmsgm_prefilter_kernel<3><<<grid, 256, 0, s>>>(in_dev, out_dev, W, H, f); break;
        case 4: dmsgm_prefilter_kernel<4><<<grid, 256, 0, s>>>(in_dev, out_dev, W, H, f); break;
        case 5: dmsgm_prefilter_kernel<5><<<grid, 256, 0, s>>>(in_dev, out_dev, W, H, f); break;
        case 6: dmsgm_prefilter_kernel<6><<<grid, 256, 0, s>>>(in_dev, out_dev, W, H, f); break;
        default: dmsgm_prefilter_kernel<7><<<grid, 256, 0, s>>>(in_dev, out_dev, W, H, f); break;
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

// dmsgm_homog_ransac.cu -- the RANSAC homography of the motion-estimation
// front end (Sec. 2.4 of arXiv:1702.05156 names RANSAC; Fischler & Bolles'
// method with a 4-point DLT model), in FP64.
//
// This unit is compiled with -fmad=false: every expression is evaluated as
// written, one IEEE operation at a time, so a model and its inlier count are
// the exact values of the method's operations (a hypothesis' count decides
// which model wins).  FP64 runs at a small fraction of the FP32 rate on this
// part, so the FP64 work is spread over as many threads as it allows.
//   pairs       one CTA: the tracked points, in corner order, become pairs
//               (current pixel centre -> previous pixel centre);
//   hypotheses  one thread per hypothesis: 4 indices from SplitMix64 on the
//               counter seed + (1 + 64 m + j) * golden gamma, the 8 x 8 DLT
//               system in frame-normalised coordinates, Gaussian elimination
//               with partial pivoting, back to pixel coordinates;
//   counts      one CTA per hypothesis, threads over the pairs;
//   best        one CTA: most inliers, lowest index; its inlier mask; the
//               least-squares refit, its normal equations summed by the CTA (a
//               fixed order, not the index order: the refit agrees with the
//               sequential sum to rounding), solved by one thread.
#include "dmsgm_homog.cuh"

namespace dmsgm {

__device__ __forceinline__ uint64_t ho_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// 4 distinct indices of hypothesis m (at most 64 draws)
__device__ bool ho_draw4(uint64_t seed, int m, int n, int* idx) {
    int got = 0;
    for (int j = 0; j < 64 && got < 4; ++j) {
        const uint64_t z = ho_mix64(seed + 0x9E3779B97F4A7C15ull * uint64_t(1 + 64 * int64_t(m) + j));
        const int v = int(uint32_t(z >> 32) % uint32_t(n));
        bool dup = false;
        for (int a = 0; a < got; ++a) dup |= idx[a] == v;
        if (!dup) idx[got++] = v;
    }
    return got == 4;
}

struct HoNorm {
    double ox, oy, s;   // x' = (x - ox) * s
};

__device__ __forceinline__ HoNorm ho_norm(int W, int H) {
    HoNorm t;
    t.ox = W / 2.0;
    t.oy = H / 2.0;
    t.s = 2.0 / (W > H ? W : H);
    return t;
}

__device__ __forceinline__ void ho_rows(double x, double y, double X, double Y, double* r0,
                                        double* r1, double* b) {
    r0[0] = x; r0[1] = y; r0[2] = 1.0; r0[3] = 0.0; r0[4] = 0.0; r0[5] = 0.0;
    r0[6] = -x * X; r0[7] = -y * X;
    r1[0] = 0.0; r1[1] = 0.0; r1[2] = 0.0; r1[3] = x; r1[4] = y; r1[5] = 1.0;
    r1[6] = -x * Y; r1[7] = -y * Y;
    b[0] = X;
    b[1] = Y;
}

// Gaussian elimination with partial pivoting on [M | r] (8 x 8, row-major)
__device__ bool ho_solve8(double* M, double* r, double* x) {
    constexpr int n = 8;
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int i = c + 1; i < n; ++i)
            if (fabs(M[i * n + c]) > fabs(M[p * n + c])) p = i;
        if (fabs(M[p * n + c]) < 1e-12) return false;
        if (p != c) {
            for (int j = 0; j < n; ++j) {
                const double t = M[c * n + j];
                M[c * n + j] = M[p * n + j];
                M[p * n + j] = t;
            }
            const double t = r[c];
            r[c] = r[p];
            r[p] = t;
        }
        for (int i = c + 1; i < n; ++i) {
            const double f = M[i * n + c] / M[c * n + c];
            for (int j = c; j < n; ++j) M[i * n + j] = M[i * n + j] - f * M[c * n + j];
            r[i] = r[i] - f * r[c];
        }
    }
    for (int c = n - 1; c >= 0; --c) {
        double s = r[c];
        for (int j = c + 1; j < n; ++j) s = s - M[c * n + j] * x[j];
        x[c] = s / M[c * n + c];
    }
    return true;
}

// pixel-coordinate homography Tinv * Hn * T of the normalised model h
__device__ void ho_denorm(const double* h, HoNorm t, double* Hp) {
    const double Hn[9] = {h[0], h[1], h[2], h[3], h[4], h[5], h[6], h[7], 1.0};
    const double T[9] = {t.s, 0.0, -t.s * t.ox, 0.0, t.s, -t.s * t.oy, 0.0, 0.0, 1.0};
    const double Ti[9] = {1.0 / t.s, 0.0, t.ox, 0.0, 1.0 / t.s, t.oy, 0.0, 0.0, 1.0};
    double M[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s = s + Hn[i * 3 + k] * T[k * 3 + j];
            M[i * 3 + j] = s;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s = s + Ti[i * 3 + k] * M[k * 3 + j];
            Hp[i * 3 + j] = s;
        }
    const double z = Hp[8];
    for (int i = 0; i < 9; ++i) Hp[i] = Hp[i] / z;
}

// pair k is an inlier of Hp: it projects in front (Z > 0) and within thr,
// |(X, Y) - Z dst|^2 < thr^2 Z^2 (the reprojection error without a division)
__device__ __forceinline__ bool ho_inlier(const double* Hp, const double* src, const double* dst,
                                          int k, double t2) {
    const double x = src[2 * k], y = src[2 * k + 1];
    const double X = Hp[0] * x + Hp[1] * y + Hp[2];
    const double Y = Hp[3] * x + Hp[4] * y + Hp[5];
    const double Z = Hp[6] * x + Hp[7] * y + Hp[8];
    if (!(Z > 0.0)) return false;
    const double ex = X - dst[2 * k] * Z, ey = Y - dst[2 * k + 1] * Z;
    return ex * ex + ey * ey < t2 * Z * Z;
}

__global__ void __launch_bounds__(1024) ho_pairs_kernel(uint32_t* ctrl, const float2* pin,
                                                        const float2* pout, const uint8_t* st,
                                                        double* src, double* dst) {
    __shared__ int wsum[32];
    const int n = int(ctrl[kCtrlNPts]);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    bool f[4];
    int c = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int k = 4 * t + q;
        f[q] = k < n && st[k];
        c += f[q];
    }
    int v = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) wsum[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int w = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    int pos = (warp ? wsum[warp - 1] : 0) + v - c;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int k = 4 * t + q;
        if (!f[q]) continue;
        src[2 * pos] = double(pout[k].x) + 0.5;
        src[2 * pos + 1] = double(pout[k].y) + 0.5;
        dst[2 * pos] = double(pin[k].x) + 0.5;
        dst[2 * pos + 1] = double(pin[k].y) + 0.5;
        ++pos;
    }
    if (t == 1023) ctrl[kCtrlNPairs] = uint32_t(wsum[31]);
}

__global__ void __launch_bounds__(128) ho_hyp_kernel(const uint32_t* ctrl, const double* src,
                                                     const double* dst, int W, int H, int iters,
                                                     uint64_t seed, double* hyp, int* hcount) {
    const int m = blockIdx.x * 128 + threadIdx.x;
    if (m >= iters) return;
    const int n = int(ctrl[kCtrlNPairs]);
    int idx[4];
    bool ok = n >= 4 && ho_draw4(seed, m, n, idx);
    if (ok) {
        const HoNorm t = ho_norm(W, H);
        double M[64], r[8], h[8];
        for (int a = 0; a < 4; ++a) {
            const int k = idx[a];
            ho_rows((src[2 * k] - t.ox) * t.s, (src[2 * k + 1] - t.oy) * t.s,
                    (dst[2 * k] - t.ox) * t.s, (dst[2 * k + 1] - t.oy) * t.s, M + 16 * a,
                    M + 16 * a + 8, r + 2 * a);
        }
        ok = ho_solve8(M, r, h);
        if (ok) ho_denorm(h, t, hyp + 9 * size_t(m));
    }
    hcount[m] = ok ? 0 : -1;
}

__global__ void __launch_bounds__(128) ho_count_kernel(const uint32_t* ctrl, const double* src,
                                                       const double* dst, double thr,
                                                       const double* hyp, int* hcount) {
    __shared__ int ws[4];
    const int m = blockIdx.x;
    if (hcount[m] < 0) return;   // the whole CTA
    const int n = int(ctrl[kCtrlNPairs]);
    double Hp[9];
    for (int i = 0; i < 9; ++i) Hp[i] = hyp[9 * size_t(m) + i];
    const double t2 = thr * thr;
    int c = 0;
    for (int k = threadIdx.x; k < n; k += 128) c += ho_inlier(Hp, src, dst, k, t2);
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) hcount[m] = ws[0] + ws[1] + ws[2] + ws[3];
}

__global__ void __launch_bounds__(256) ho_best_kernel(const uint32_t* ctrl, const double* src,
                                                      const double* dst, int W, int H, int iters,
                                                      double thr, const double* hyp,
                                                      const int* hcount, uint8_t* inl,
                                                      HoRansacOut* out) {
    __shared__ unsigned long long wbest[8];
    __shared__ double N[72];
    __shared__ double Hb[9];
    __shared__ int bm, bc;
    const int t = threadIdx.x;
    unsigned long long key = 0;
    for (int m = t; m < iters; m += 256) {
        const int c = hcount[m];
        if (c >= 0) {
            const unsigned long long k = (static_cast<unsigned long long>(c) << 32) | (0xFFFFFFFFu - uint32_t(m));
            key = k > key ? k : key;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, key, o);
        key = y > key ? y : key;
    }
    if ((t & 31) == 0) wbest[t >> 5] = key;
    __syncthreads();
    if (t == 0) {
        unsigned long long k = 0;
        for (int w = 0; w < 8; ++w) k = wbest[w] > k ? wbest[w] : k;
        bm = k ? int(0xFFFFFFFFu - uint32_t(k)) : -1;
        bc = k ? int(k >> 32) : -1;
        if (bm >= 0)
            for (int i = 0; i < 9; ++i) Hb[i] = hyp[9 * size_t(bm) + i];
    }
    __syncthreads();
    const int n = int(ctrl[kCtrlNPairs]);
    if (bm < 0) {
        if (t == 0) {
            out->inliers = -1;
            out->best = -1;
        }
        return;
    }
    const double t2 = thr * thr;
    for (int k = t; k < n; k += 256) inl[k] = ho_inlier(Hb, src, dst, k, t2) ? 1 : 0;
    __syncthreads();
    // normal equations over the inliers: each thread sums the upper triangle
    // (36) and the right side (8) over inliers k = t, t + 256, ..; a fixed
    // tree of warp shuffles and one pass over the 8 warps adds the partials
    const HoNorm tn = ho_norm(W, H);
    double acc[44];
#pragma unroll
    for (int e = 0; e < 44; ++e) acc[e] = 0.0;
    for (int k = t; k < n; k += 256) {
        if (!inl[k]) continue;
        double r0[8], r1[8], b[2];
        ho_rows((src[2 * k] - tn.ox) * tn.s, (src[2 * k + 1] - tn.oy) * tn.s,
                (dst[2 * k] - tn.ox) * tn.s, (dst[2 * k + 1] - tn.oy) * tn.s, r0, r1, b);
        int e = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = i; j < 8; ++j) acc[e++] += r0[i] * r0[j] + r1[i] * r1[j];
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[36 + i] += r0[i] * b[0] + r1[i] * b[1];
    }
#pragma unroll
    for (int e = 0; e < 44; ++e) {
        double v = acc[e];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        acc[e] = v;
    }
    __shared__ double part[8][44];
    if ((t & 31) == 0)
#pragma unroll
        for (int e = 0; e < 44; ++e) part[t >> 5][e] = acc[e];
    __syncthreads();
    if (t < 44) {
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v += part[w][t];
        int i = 0, e = t;   // entry t of the upper triangle -> (i, j)
        if (t < 36) {
            while (e >= 8 - i) {
                e -= 8 - i;
                ++i;
            }
            const int j = i + e;
            N[i * 8 + j] = v;
            N[j * 8 + i] = v;
        } else {
            N[64 + (t - 36)] = v;
        }
    }
    __syncthreads();
    if (t == 0) {
        double M[64], r[8], h[8], Hr[9];
        for (int i = 0; i < 64; ++i) M[i] = N[i];
        for (int i = 0; i < 8; ++i) r[i] = N[64 + i];
        const bool ok = bc >= 4 && ho_solve8(M, r, h);
        if (ok) ho_denorm(h, tn, Hr);
        for (int i = 0; i < 9; ++i) out->H[i] = ok ? Hr[i] : Hb[i];
        out->inliers = bc;
        out->best = bm;
    }
}

int ho_launch_ransac(dmsgm_homog_ctx* h, bool pairs_from_track, cudaStream_t s) {
    if (pairs_from_track)
        ho_pairs_kernel<<<1, 1024, 0, s>>>(h->ctrl, h->pts_in, h->pts_out, h->status, h->src, h->dst);
    const int it = h->p.ransac_iters;
    ho_hyp_kernel<<<(it + 127) / 128, 128, 0, s>>>(h->ctrl, h->src, h->dst, h->W, h->H, it,
                                                   h->p.seed, h->hyp, h->hcount);
    ho_count_kernel<<<it, 128, 0, s>>>(h->ctrl, h->src, h->dst, h->p.thresh, h->hyp, h->hcount);
    ho_best_kernel<<<1, 256, 0, s>>>(h->ctrl, h->src, h->dst, h->W, h->H, it, h->p.thresh, h->hyp,
                                     h->hcount, h->inl, h->rout);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(DMSGM_ERR_CUDA, "RANSAC kernels: %s", cudaGetErrorString(e));
    return DMSGM_OK;
}

}  // namespace dmsgm

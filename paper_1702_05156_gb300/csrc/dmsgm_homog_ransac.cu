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
//   hypotheses  eight lanes per hypothesis (rows of the system spread over
//               the lanes, FP64 latency being the bound): 4 indices from SplitMix64 on the
//               counter seed + (1 + 64 m + j) * golden gamma, the 8 x 8 DLT
//               system in frame-normalised coordinates, Gaussian elimination
//               with partial pivoting, back to pixel coordinates;
//   counts      one CTA per hypothesis, threads over the pairs: an FP32
//               pre-test with a rigorous error bound decides almost every
//               pair, the rest are tested in FP64 (the counts are exact);
//   refit       one warp per 32 pairs: the best hypothesis (most inliers,
//               lowest index), its inlier mask, the least-squares refit's
//               normal equations summed per warp; then one warp adds the
//               warps' sums (a fixed order, not the index order: the refit
//               agrees with the sequential sum to rounding) and solves.
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

// Gaussian elimination with partial pivoting on the 8 x 8 system [M | r],
// by 8 lanes of a warp (lane l & 7 holds row l: m[0..7], rr).  For column c
// the pivot is the first row i >= c of largest |M[i][c]| (every lane of the
// group reads the column and scans it in row order); a pivot below 1e-12
// rejects the system.  Rows c and p are swapped and the pivot row broadcast
// by shuffles; row i > c becomes M[i][j] - f M[c][j] for j >= c and
// r[i] - f r[c], f = M[i][c] / M[c][c]; back substitution takes
// x[c] = (r[c] - sum_{j > c} M[c][j] x[j]) / M[c][c], the sum in order of j.
// All 32 lanes call it (four independent groups); every lane of a group ends
// with x and the group's verdict.
__device__ bool ho_solve8_group(double (&m)[8], double& rr, double (&x)[8]) {
    const int l = threadIdx.x & 7;
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        int p = c;
        double pv = __shfl_sync(0xffffffffu, m[c], c, 8);
#pragma unroll
        for (int i = c + 1; i < 8; ++i) {
            const double v = __shfl_sync(0xffffffffu, m[c], i, 8);
            if (fabs(v) > fabs(pv)) {
                p = i;
                pv = v;
            }
        }
        ok = ok && !(fabs(pv) < 1e-12);
        const int partner = l == c ? p : (l == p ? c : l);
#pragma unroll
        for (int j = 0; j < 8; ++j) m[j] = __shfl_sync(0xffffffffu, m[j], partner, 8);
        rr = __shfl_sync(0xffffffffu, rr, partner, 8);
        double pr[8];
#pragma unroll
        for (int j = c; j < 8; ++j) pr[j] = __shfl_sync(0xffffffffu, m[j], c, 8);
        const double prr = __shfl_sync(0xffffffffu, rr, c, 8);
        if (l > c) {
            const double f = m[c] / pr[c];
#pragma unroll
            for (int j = c; j < 8; ++j) m[j] = m[j] - f * pr[j];
            rr = rr - f * prr;
        }
    }
#pragma unroll
    for (int c = 7; c >= 0; --c) {
        double s = rr;
#pragma unroll
        for (int j = c + 1; j < 8; ++j) s = s - m[j] * x[j];
        x[c] = __shfl_sync(0xffffffffu, s / m[c], c, 8);
    }
    return ok;
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

// FP32 pre-test of ho_inlier.  The decision is taken in FP32 only where a
// bound on the distance between the FP32 and the FP64 evaluations shows
// that both fall on the same side of it; the rest go to FP64, so a count
// equals the FP64 count exactly.  With u = 2^-24 and inputs rounded to FP32
// (each a normal float, or exactly 0; the products of such inputs stay
// normal), the FP32 values differ from the FP64 ones by at most
//   X, Y, Z:   5.02 u M        M = |h0 x| + |h1 y| + |h2| (per row),
//   ex, ey:    8.1 u (M_X + |dx| M_Z)   (and the same with Y, dy),
//   lhs:       2 |ex| e_x + e_x^2 + 2 |ey| e_y + e_y^2 + 2.01 u lhs,
//   rhs:       t2 (2 |Z| e_Z + e_Z^2) + 3.02 u rhs
// (forward error analysis of each rounded operation; the FP64 rounding is
// below 1e-15 u).  The bounds used below are at least 2.4 times these, so
// that the rounding of the final FP32 comparisons stays inside the margin.
struct HoF32H {
    float h[9], t2;
    bool ok;   // every coefficient and t2 in the range the bounds assume
};

__device__ __forceinline__ bool ho_f32_range(double d, float& f) {
    f = __double2float_rn(d);
    const float a = fabsf(f);
    return ((__double_as_longlong(d) << 1) == 0) || (a >= 1e-15f && a <= 1e15f);
}

// The coefficients' FP32 copy (t2 is set by the caller).
__device__ __forceinline__ HoF32H ho_f32_model(const double* Hp, double t2) {
    HoF32H m;
    m.ok = true;
    m.t2 = 0.0f;
#pragma unroll
    for (int i = 0; i < 9; ++i) m.ok = ho_f32_range(Hp[i], m.h[i]) && m.ok;
    return m;
}

// (x, y, dx, dy) of pair k in FP32, x = NaN when one of them is out of range
__device__ __forceinline__ float4 ho_f32_pair(const double* src, const double* dst, int k) {
    float4 v;
    bool ok = ho_f32_range(src[2 * k], v.x);
    ok = ho_f32_range(src[2 * k + 1], v.y) && ok;
    ok = ho_f32_range(dst[2 * k], v.z) && ok;
    ok = ho_f32_range(dst[2 * k + 1], v.w) && ok;
    if (!ok) v.x = __int_as_float(0x7fc00000);
    return v;
}

// 1: an inlier, 0: not, 2: too close to call in FP32
__device__ __forceinline__ int ho_inlier_f32(const HoF32H& m, float4 p) {
    constexpr float u = 5.9604645e-8f;   // 2^-24
    const float* h = m.h;
    const float a0 = h[0] * p.x, a1 = h[1] * p.y;
    const float b0 = h[3] * p.x, b1 = h[4] * p.y;
    const float c0 = h[6] * p.x, c1 = h[7] * p.y;
    const float X = (a0 + a1) + h[2], Y = (b0 + b1) + h[5], Z = (c0 + c1) + h[8];
    const float MX = (fabsf(a0) + fabsf(a1)) + fabsf(h[2]);
    const float MY = (fabsf(b0) + fabsf(b1)) + fabsf(h[5]);
    const float MZ = (fabsf(c0) + fabsf(c1)) + fabsf(h[8]);
    const float eZ = (16.0f * u) * MZ + 1e-30f;
    if (!(Z > eZ)) return (Z < -eZ && eZ < 3.0e38f) ? 0 : 2;
    const float ex = X - p.z * Z, ey = Y - p.w * Z;
    const float ax = (20.0f * u) * (MX + fabsf(p.z) * MZ) + 1e-30f;
    const float ay = (20.0f * u) * (MY + fabsf(p.w) * MZ) + 1e-30f;
    const float lhs = ex * ex + ey * ey;
    const float rhs = (m.t2 * Z) * Z;
    const float el = ((2.0f * fabsf(ex) * ax + ax * ax) + (2.0f * fabsf(ey) * ay + ay * ay)) +
                     ((8.0f * u) * lhs + 1e-36f);
    const float er = m.t2 * (2.0f * Z * eZ + eZ * eZ) + ((16.0f * u) * rhs + 1e-36f);
    if (!(fabsf(lhs) < 3.0e38f && rhs < 3.0e38f && el < 3.0e38f && er < 3.0e38f && rhs >= 1e-30f))
        return 2;
    if ((lhs + el) + er < rhs) return 1;
    if (lhs > rhs + (el + er)) return 0;
    return 2;
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

// Four hypotheses per warp, eight lanes each: lane l of a group builds row
// l of the hypothesis' DLT system (point l / 2, its x or y row), the group
// solves it (ho_solve8_group), every lane of the group forms the
// pixel-coordinate model and lane l stores its entry l (lane 0 also entry 8).  The FP32 copy of the model
// for the counts' pre-test is made here once.  The threads also round the
// pairs to FP32.
constexpr int kHypWarps = 4;   // per CTA

__global__ void __launch_bounds__(32 * kHypWarps) ho_hyp_kernel(uint32_t* ctrl, const double* src,
                                                               const double* dst, int W, int H,
                                                               int iters, uint64_t seed, double* hyp,
                                                               float* hypf, int* hcount, float4* pf) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = int(ctrl[kCtrlNPairs]);
    for (int k = tid; k < n; k += gridDim.x * blockDim.x) pf[k] = ho_f32_pair(src, dst, k);
    const int m = tid >> 3, l = tid & 7;
    if (int(blockIdx.x * blockDim.x + (threadIdx.x & ~31u)) >= 8 * iters) return;   // the whole warp
    const bool live = m < iters;
    int idx[4];
    bool ok = live && n >= 4 && ho_draw4(seed, m, n, idx);
    const HoNorm t = ho_norm(W, H);
    double mr[8], rr = 0.0, x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) mr[j] = 0.0;
    if (ok) {
        const int k = idx[l >> 1];
        double r0[8], r1[8], b[2];
        ho_rows((src[2 * k] - t.ox) * t.s, (src[2 * k + 1] - t.oy) * t.s,
                (dst[2 * k] - t.ox) * t.s, (dst[2 * k + 1] - t.oy) * t.s, r0, r1, b);
#pragma unroll
        for (int j = 0; j < 8; ++j) mr[j] = (l & 1) ? r1[j] : r0[j];
        rr = (l & 1) ? b[1] : b[0];
    }
    ok = ho_solve8_group(mr, rr, x) && ok;
    if (!live) return;
    double Hp[9];
    if (ok) {
        ho_denorm(x, t, Hp);
        double v = Hp[0];
#pragma unroll
        for (int i = 1; i < 8; ++i) v = l == i ? Hp[i] : v;
        hyp[9 * size_t(m) + l] = v;
        if (l == 0) hyp[9 * size_t(m) + 8] = Hp[8];
    }
    if (l == 0) {
        hcount[m] = ok ? 0 : -1;
        if (ok) {
            const HoF32H f = ho_f32_model(Hp, 0.0);
            for (int i = 0; i < 9; ++i) hypf[10 * size_t(m) + i] = f.h[i];
            hypf[10 * size_t(m) + 9] = f.ok ? 1.0f : 0.0f;
        }
    }
}

// One CTA per hypothesis: the FP32 pre-test over the pairs, then the pairs
// it could not decide in FP64 (shared-memory list; the count is a sum, so
// the list's order does not matter).
__global__ void __launch_bounds__(128) ho_count_kernel(const uint32_t* ctrl, const double* src,
                                                       const double* dst, const float4* pf,
                                                       double thr, const double* hyp,
                                                       const float* hypf, int* hcount) {
    __shared__ int ws[4];
    __shared__ uint16_t q[kHoMaxPts];
    __shared__ int nq;
    const int m = blockIdx.x;
    if (hcount[m] < 0) return;   // the whole CTA
    const int n = int(ctrl[kCtrlNPairs]);
    const double t2 = thr * thr;
    HoF32H fm;
#pragma unroll
    for (int i = 0; i < 9; ++i) fm.h[i] = hypf[10 * size_t(m) + i];
    fm.ok = ho_f32_range(t2, fm.t2) && fm.t2 > 0.0f && hypf[10 * size_t(m) + 9] != 0.0f;
    if (threadIdx.x == 0) nq = 0;
    __syncthreads();
    int c = 0;
    for (int k = threadIdx.x; k < n; k += 128) {
        const int d = fm.ok ? ho_inlier_f32(fm, pf[k]) : 2;
        if (d == 2) q[atomicAdd(&nq, 1)] = uint16_t(k);
        else c += d;
    }
    __syncthreads();
    const int nqs = nq;
    if (nqs) {
        double Hp[9];
        for (int i = 0; i < 9; ++i) Hp[i] = hyp[9 * size_t(m) + i];
        for (int i = threadIdx.x; i < nqs; i += 128) c += ho_inlier(Hp, src, dst, q[i], t2);
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) hcount[m] = ws[0] + ws[1] + ws[2] + ws[3];
}

// The refit (two kernels).  ho_refit_kernel, one warp per kFitPts pairs:
// every CTA finds the best hypothesis (most inliers, lowest index; CTA 0
// records it), marks its pairs' inliers and sums their normal-equation terms
// (the upper triangle, 36, and the right side, 8) over its lanes in lane
// order.  ho_fit_kernel, one warp: the CTAs' partial sums in CTA order, the
// 8 x 8 solve and the pixel-coordinate model.  The sums' order is fixed, so
// the refit is deterministic; it agrees with the sequential sum to rounding.
constexpr int kFitPts = kHoMaxPts / kHoFitCtas;
constexpr int kFitTerms = kHoFitTerms;
static_assert(kFitPts == 32, "one warp per refit CTA");

__global__ void __launch_bounds__(kFitPts) ho_refit_kernel(uint32_t* ctrl, const double* src,
                                                           const double* dst, int W, int H,
                                                           int iters, double thr, const double* hyp,
                                                           const int* hcount, uint8_t* inl,
                                                           double* part) {
    __shared__ double sh[kFitPts][kFitTerms + 1];
    const int lane = threadIdx.x;
    unsigned long long key = 0;
    for (int m0 = lane; m0 < iters; m0 += 8 * kFitPts) {
        int cs[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) cs[q] = m0 + q * kFitPts < iters ? hcount[m0 + q * kFitPts] : -1;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int m = m0 + q * kFitPts;
            if (cs[q] >= 0) {
                const unsigned long long k = (static_cast<unsigned long long>(cs[q]) << 32) | (0xFFFFFFFFu - uint32_t(m));
                key = k > key ? k : key;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, key, o);
        key = y > key ? y : key;
    }
    const int bm = key ? int(0xFFFFFFFFu - uint32_t(key)) : -1;
    const int bc = key ? int(key >> 32) : -1;
    if (blockIdx.x == 0 && lane == 0) {
        ctrl[kCtrlBestM] = uint32_t(bm);
        ctrl[kCtrlBestC] = uint32_t(bc);
    }
    if (bm < 0) return;
    const int n = int(ctrl[kCtrlNPairs]);
    if (int(blockIdx.x) * kFitPts >= n) return;   // the whole CTA
    double Hb[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) Hb[i] = hyp[9 * size_t(bm) + i];
    const HoNorm tn = ho_norm(W, H);
    double acc[kFitTerms];
#pragma unroll
    for (int e = 0; e < kFitTerms; ++e) acc[e] = 0.0;
    const int k = blockIdx.x * kFitPts + lane;
    if (k < n) {
        const bool f = ho_inlier(Hb, src, dst, k, thr * thr);
        inl[k] = f ? 1 : 0;
        if (f) {
            double r0[8], r1[8], b[2];
            ho_rows((src[2 * k] - tn.ox) * tn.s, (src[2 * k + 1] - tn.oy) * tn.s,
                    (dst[2 * k] - tn.ox) * tn.s, (dst[2 * k + 1] - tn.oy) * tn.s, r0, r1, b);
            int e = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = i; j < 8; ++j) acc[e++] = r0[i] * r0[j] + r1[i] * r1[j];
#pragma unroll
            for (int i = 0; i < 8; ++i) acc[36 + i] = r0[i] * b[0] + r1[i] * b[1];
        }
    }
#pragma unroll
    for (int e = 0; e < kFitTerms; ++e) sh[lane][e] = acc[e];
    __syncwarp();
    for (int e = lane; e < kFitTerms; e += kFitPts) {
        double v = 0.0;
        for (int i = 0; i < kFitPts; ++i) v = v + sh[i][e];
        part[size_t(blockIdx.x) * kFitTerms + e] = v;
    }
}

__global__ void __launch_bounds__(32) ho_fit_kernel(const uint32_t* ctrl, int W, int H,
                                                    const double* hyp, const double* part,
                                                    HoRansacOut* out) {
    __shared__ double N[kFitTerms];
    const int lane = threadIdx.x;
    const int bm = int(ctrl[kCtrlBestM]), bc = int(ctrl[kCtrlBestC]);
    if (bm < 0) {
        if (lane == 0) {
            out->inliers = -1;
            out->best = -1;
        }
        return;
    }
    const int nct = (int(ctrl[kCtrlNPairs]) + kFitPts - 1) / kFitPts;
    for (int e = lane; e < kFitTerms; e += 32) {
        double v = 0.0;
        for (int c = 0; c < nct; ++c) v = v + part[size_t(c) * kFitTerms + e];
        N[e] = v;
    }
    __syncwarp();
    // the 8 x 8 system by lanes 0..7 (the other groups solve the same copy)
    const int row = lane & 7;
    double mrow[8], x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int a = row < j ? row : j, b = row < j ? j : row;   // upper-triangle entry (a, b)
        mrow[j] = N[a * 8 - a * (a - 1) / 2 + (b - a)];
    }
    double rrow = N[36 + row];
    const bool solved = ho_solve8_group(mrow, rrow, x);
    if (lane == 0) {
        const HoNorm tn = ho_norm(W, H);
        double Hr[9];
        const bool ok = bc >= 4 && solved;
        if (ok) ho_denorm(x, tn, Hr);
        for (int i = 0; i < 9; ++i) out->H[i] = ok ? Hr[i] : hyp[9 * size_t(bm) + i];
        out->inliers = bc;
        out->best = bm;
    }
}

int ho_launch_ransac(dmsgm_homog_ctx* h, bool pairs_from_track, cudaStream_t s) {
    if (pairs_from_track)
        ho_pairs_kernel<<<1, 1024, 0, s>>>(h->ctrl, h->pts_in, h->pts_out, h->status, h->src, h->dst);
    const int it = h->p.ransac_iters;
    const int hyp_ctas = (8 * it + 32 * kHypWarps - 1) / (32 * kHypWarps);
    ho_hyp_kernel<<<hyp_ctas, 32 * kHypWarps, 0, s>>>(h->ctrl, h->src, h->dst, h->W, h->H, it,
                                                      h->p.seed, h->hyp, h->hypf, h->hcount, h->pf);
    ho_count_kernel<<<it, 128, 0, s>>>(h->ctrl, h->src, h->dst, h->pf, h->p.thresh, h->hyp,
                                       h->hypf, h->hcount);
    ho_refit_kernel<<<kHoFitCtas, kFitPts, 0, s>>>(h->ctrl, h->src, h->dst, h->W, h->H, it,
                                                   h->p.thresh, h->hyp, h->hcount, h->inl,
                                                   h->fitpart);
    ho_fit_kernel<<<1, 32, 0, s>>>(h->ctrl, h->W, h->H, h->hyp, h->fitpart, h->rout);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(DMSGM_ERR_CUDA, "RANSAC kernels: %s", cudaGetErrorString(e));
    return DMSGM_OK;
}

}  // namespace dmsgm

/*
 * homog_oracle.c -- plain CPU oracle of the motion-estimation front end that
 * produces the homography the DMSGM step consumes (arXiv:1702.05156,
 * Sec. 2.4 "Motion Compensation" and Sec. 3.1.3; the appendix "Motion
 * Compensation Code Snippets": good features to track, pyramidal
 * Lucas-Kanade with a 20 x 20 window and 5 pyramid levels, RANSAC
 * homography).  The paper names these methods and the library calls that
 * run them; the steps below are the published methods (Shi & Tomasi 1994,
 * Bouguet's pyramidal Lucas-Kanade, Fischler & Bolles' RANSAC with a DLT
 * model), written out plainly.
 *
 * TEST INFRASTRUCTURE ONLY.  Tests, the smoke check and the benchmark's CPU
 * baseline use it to check and time the CUDA library; product code never
 * links, loads or calls it, and it shares no code with the CUDA library.
 *
 * Readings (each listed in the design notes):
 *   M1 corner score: Shi-Tomasi's smaller eigenvalue of the structure tensor
 *      [A B; B C] summed over a bs x bs window of 3 x 3 Sobel gradients
 *      (integers, so A, B, C are exact), coordinates clamped to the frame.
 *      The eigenvalues of a symmetric 2 x 2 matrix are
 *      ((A + C) -+ sqrt((A - C)^2 + 4 B^2)) / 2; the score is the smaller
 *      one, evaluated in FP64 and clamped to >= 0 (the tensor is positive
 *      semi-definite; rounding can only push the value below 0).
 *   M2 candidates: pixels with 1 <= x <= W-2, 1 <= y <= H-2, s > q * max s
 *      (max over all pixels) and s >= each of the 8 neighbours' scores.
 *   M3 order: score descending, then row-major index ascending; at most the
 *      first 8192 candidates in that order are considered.
 *   M4 greedy spacing: a candidate is accepted when every accepted corner
 *      lies at squared distance >= min_distance^2; at most max_corners.
 *   M5 pyramid: level l+1 is the 5 x 5 binomial ([1 4 6 4 1] / 16 in each
 *      direction) of level l, rounded ((sum + 128) >> 8), sampled at even
 *      pixels, coordinates clamped; sizes ((w + 1) / 2, (h + 1) / 2).
 *   M6 tracking (Bouguet): window half-width wh (the paper's 20 x 20 read as
 *      21 x 21 samples, wh = 10); gradients are central differences of the
 *      previous level, (I(x+1) - I(x-1)) / 2, coordinates clamped; samples
 *      are bilinear with clamped coordinates; per level from the coarsest,
 *      G = sum [Ix^2 IxIy; IxIy Iy^2], and up to max_iters updates
 *      eta = G^-1 sum (I - J(. + g + nu)) [Ix; Iy], stopping once
 *      |eta| < eps; the guess doubles to the next level.  A point fails when
 *      G's smaller eigenvalue over the window's sample count is below
 *      min_eig at any level, or its final position leaves the frame.
 *   M7 RANSAC: correspondences map current pixel centres (tracked point
 *      + 0.5) to previous ones (corner + 0.5), the direction the DMSGM step
 *      takes.  Hypothesis m draws 4 distinct indices with SplitMix64 on the
 *      counter seed + (1 + 64 m + j) * golden-gamma, index = (z >> 32) % n,
 *      j = 0, 1, ... (at most 64 draws); its model solves the 8 x 8 DLT
 *      system (h33 = 1) in coordinates normalised by the frame,
 *      x' = (x - W/2) * 2/max(W,H), by Gaussian elimination with partial
 *      pivoting (a pivot below 1e-12 rejects the hypothesis).  A pair is an
 *      inlier when it projects in front (w > 0) with reprojection error below
 *      thr: with (X, Y, w) = Hp (x, y, 1), the pair is an inlier when
 *      w > 0 and (X / w - dx)^2 + (Y / w - dy)^2 < thr^2.
 *      Best model: most inliers, ties to the lower index.  All of this in
 *      FP64.
 *   M8 refit: least squares of the same DLT equations over the best model's
 *      inliers (normal equations, same elimination); the result has
 *      h33 = 1.
 *
 * Build: part of liboracle.so (gcc -O2 -std=c11 -ffp-contract=off: no fused
 * multiply-add, so x86 and Arm hosts compute the same FP64 values).
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define HO_KMAX 8192

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* ---------------------------------------------------------------- corners */

/* M1: the structure tensor of every pixel: A = sum gx^2, B = sum gx gy,
 * C = sum gy^2 over the bs x bs window (exact integers, returned as
 * doubles; any of the outputs may be NULL). */
void ho_tensor_map(const uint8_t* img, int W, int H, int bs, double* outA, double* outB,
                   double* outC) {
    int* gx = (int*)malloc(sizeof(int) * (size_t)W * H);
    int* gy = (int*)malloc(sizeof(int) * (size_t)W * H);
#define P(xx, yy) ((int)img[(size_t)clampi(yy, 0, H - 1) * W + clampi(xx, 0, W - 1)])
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            gx[(size_t)y * W + x] = (P(x + 1, y - 1) + 2 * P(x + 1, y) + P(x + 1, y + 1)) -
                                    (P(x - 1, y - 1) + 2 * P(x - 1, y) + P(x - 1, y + 1));
            gy[(size_t)y * W + x] = (P(x - 1, y + 1) + 2 * P(x, y + 1) + P(x + 1, y + 1)) -
                                    (P(x - 1, y - 1) + 2 * P(x, y - 1) + P(x + 1, y - 1));
        }
#undef P
    const int r = bs / 2;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            long long A = 0, B = 0, C = 0;
            for (int j = -r; j <= r; ++j)
                for (int i = -r; i <= r; ++i) {
                    const size_t k = (size_t)clampi(y + j, 0, H - 1) * W + clampi(x + i, 0, W - 1);
                    A += (long long)gx[k] * gx[k];
                    B += (long long)gx[k] * gy[k];
                    C += (long long)gy[k] * gy[k];
                }
            const size_t o = (size_t)y * W + x;
            if (outA) outA[o] = (double)A;
            if (outB) outB[o] = (double)B;
            if (outC) outC[o] = (double)C;
        }
    free(gx);
    free(gy);
}

/* M1: the score of every pixel, the smaller eigenvalue of its tensor. */
void ho_score_map(const uint8_t* img, int W, int H, int bs, double* score) {
    const size_t n = (size_t)W * H;
    double* A = (double*)malloc(sizeof(double) * n);
    double* B = (double*)malloc(sizeof(double) * n);
    double* C = (double*)malloc(sizeof(double) * n);
    ho_tensor_map(img, W, H, bs, A, B, C);
    for (size_t k = 0; k < n; ++k) {
        const double lmin = ((A[k] + C[k]) - sqrt((A[k] - C[k]) * (A[k] - C[k]) + 4.0 * B[k] * B[k])) / 2.0;
        score[k] = lmin > 0.0 ? lmin : 0.0;
    }
    free(A);
    free(B);
    free(C);
}

typedef struct {
    double s;
    int idx;
} Cand;

static int cand_cmp(const void* a, const void* b) {
    const Cand* p = (const Cand*)a;
    const Cand* q = (const Cand*)b;
    if (p->s != q->s) return p->s > q->s ? -1 : 1;
    return p->idx < q->idx ? -1 : (p->idx > q->idx ? 1 : 0);
}

/* M2-M4: the corners (pixel indices), strongest first.  Returns their
 * number; *n_cand receives the number of candidates (before the cap). */
int ho_corners(const uint8_t* img, int W, int H, int bs, double quality, double min_dist,
               int max_corners, int* xy, double* sc, int* n_cand) {
    if (W < 3 || H < 3 || bs < 1 || bs % 2 == 0 || max_corners < 1) return -1;
    double* s = (double*)malloc(sizeof(double) * (size_t)W * H);
    ho_score_map(img, W, H, bs, s);
    double mx = 0.0;
    for (size_t k = 0; k < (size_t)W * H; ++k) mx = s[k] > mx ? s[k] : mx;
    const double thr = quality * mx;
    size_t cap = 1024, n = 0;
    Cand* c = (Cand*)malloc(sizeof(Cand) * cap);
    for (int y = 1; y <= H - 2; ++y)
        for (int x = 1; x <= W - 2; ++x) {
            const double v = s[(size_t)y * W + x];
            if (!(v > thr)) continue;
            int peak = 1;
            for (int j = -1; j <= 1 && peak; ++j)
                for (int i = -1; i <= 1; ++i)
                    if ((i || j) && s[(size_t)(y + j) * W + x + i] > v) { peak = 0; break; }
            if (!peak) continue;
            if (n == cap) {
                cap *= 2;
                c = (Cand*)realloc(c, sizeof(Cand) * cap);
            }
            c[n].s = v;
            c[n].idx = y * W + x;
            ++n;
        }
    *n_cand = (int)n;
    qsort(c, n, sizeof(Cand), cand_cmp);
    if (n > HO_KMAX) n = HO_KMAX;
    const double md2 = min_dist * min_dist;
    int m = 0;
    for (size_t k = 0; k < n && m < max_corners; ++k) {
        const int x = c[k].idx % W, y = c[k].idx / W;
        int ok = 1;
        for (int a = 0; a < m && ok; ++a) {
            const long long dx = x - xy[2 * a], dy = y - xy[2 * a + 1];
            if ((double)(dx * dx + dy * dy) < md2) ok = 0;
        }
        if (!ok) continue;
        xy[2 * m] = x;
        xy[2 * m + 1] = y;
        sc[m] = c[k].s;
        ++m;
    }
    free(c);
    free(s);
    return m;
}

/* ---------------------------------------------------------------- pyramid */

/* M5: one pyramid step. */
void ho_pyr_down(const uint8_t* in, int w, int h, uint8_t* out) {
    static const int k[5] = {1, 4, 6, 4, 1};
    const int w2 = (w + 1) / 2, h2 = (h + 1) / 2;
    for (int y = 0; y < h2; ++y)
        for (int x = 0; x < w2; ++x) {
            int s = 0;
            for (int j = -2; j <= 2; ++j)
                for (int i = -2; i <= 2; ++i)
                    s += k[j + 2] * k[i + 2] *
                         in[(size_t)clampi(2 * y + j, 0, h - 1) * w + clampi(2 * x + i, 0, w - 1)];
            out[(size_t)y * w2 + x] = (uint8_t)((s + 128) >> 8);
        }
}

/* ---------------------------------------------------------------- tracking */

typedef struct {
    const uint8_t* p;
    int w, h;
} Img;

static double px(Img a, int x, int y) {
    return (double)a.p[(size_t)clampi(y, 0, a.h - 1) * a.w + clampi(x, 0, a.w - 1)];
}

/* bilinear sample of the image (which = 0), its x gradient (1) or y gradient (2) */
static double sample(Img a, double x, double y, int which) {
    const double fx0 = floor(x), fy0 = floor(y);
    const int x0 = (int)fx0, y0 = (int)fy0;
    const double fx = x - fx0, fy = y - fy0;
    double v[2][2];
    for (int j = 0; j < 2; ++j)
        for (int i = 0; i < 2; ++i) {
            const int xi = x0 + i, yj = y0 + j;
            if (which == 0) v[j][i] = px(a, xi, yj);
            else if (which == 1) v[j][i] = (px(a, xi + 1, yj) - px(a, xi - 1, yj)) / 2.0;
            else v[j][i] = (px(a, xi, yj + 1) - px(a, xi, yj - 1)) / 2.0;
        }
    /* clamped coordinates: the clamp acts on the integer sample positions */
    return (1.0 - fx) * (1.0 - fy) * v[0][0] + fx * (1.0 - fy) * v[0][1] +
           (1.0 - fx) * fy * v[1][0] + fx * fy * v[1][1];
}

/* M6: track n points (pixel indices, x y pairs) from prev to cur.  Returns 0
 * or -1 on bad arguments; status[i] = 1 for a tracked point. */
int ho_track(const uint8_t* prev, const uint8_t* cur, int W, int H, int levels, int wh,
             int max_iters, double eps, double min_eig, const double* in, int n, double* out,
             uint8_t* status) {
    if (levels < 0 || levels > 12 || wh < 1 || max_iters < 1) return -1;
    Img P[13], Q[13];
    uint8_t* bufs[26] = {0};
    P[0].p = prev; P[0].w = W; P[0].h = H;
    Q[0].p = cur;  Q[0].w = W; Q[0].h = H;
    for (int l = 1; l <= levels; ++l) {
        const int w2 = (P[l - 1].w + 1) / 2, h2 = (P[l - 1].h + 1) / 2;
        bufs[2 * l] = (uint8_t*)malloc((size_t)w2 * h2);
        bufs[2 * l + 1] = (uint8_t*)malloc((size_t)w2 * h2);
        ho_pyr_down(P[l - 1].p, P[l - 1].w, P[l - 1].h, bufs[2 * l]);
        ho_pyr_down(Q[l - 1].p, Q[l - 1].w, Q[l - 1].h, bufs[2 * l + 1]);
        P[l].p = bufs[2 * l]; P[l].w = w2; P[l].h = h2;
        Q[l].p = bufs[2 * l + 1]; Q[l].w = w2; Q[l].h = h2;
    }
    const double nsamp = (double)(2 * wh + 1) * (2 * wh + 1);
    for (int k = 0; k < n; ++k) {
        int ok = 1;
        double gx = 0.0, gy = 0.0, dx = 0.0, dy = 0.0;
        for (int l = levels; l >= 0; --l) {
            const double sc = ldexp(1.0, -l);
            const double ux = in[2 * k] * sc, uy = in[2 * k + 1] * sc;
            double a = 0.0, b = 0.0, c = 0.0;
            for (int j = -wh; j <= wh; ++j)
                for (int i = -wh; i <= wh; ++i) {
                    const double ix = sample(P[l], ux + i, uy + j, 1);
                    const double iy = sample(P[l], ux + i, uy + j, 2);
                    a += ix * ix;
                    b += ix * iy;
                    c += iy * iy;
                }
            const double det = a * c - b * b;
            const double lmin = ((a + c) - sqrt((a - c) * (a - c) + 4.0 * b * b)) / 2.0;
            if (lmin / nsamp < min_eig || det == 0.0) { ok = 0; break; }
            double vx = 0.0, vy = 0.0;
            for (int it = 0; it < max_iters; ++it) {
                double bx = 0.0, by = 0.0;
                for (int j = -wh; j <= wh; ++j)
                    for (int i = -wh; i <= wh; ++i) {
                        const double x = ux + i, y = uy + j;
                        const double d = sample(P[l], x, y, 0) - sample(Q[l], x + gx + vx, y + gy + vy, 0);
                        bx += d * sample(P[l], x, y, 1);
                        by += d * sample(P[l], x, y, 2);
                    }
                const double ex = (c * bx - b * by) / det;
                const double ey = (a * by - b * bx) / det;
                vx += ex;
                vy += ey;
                if (ex * ex + ey * ey < eps * eps) break;
            }
            dx = vx;
            dy = vy;
            if (l > 0) {
                gx = 2.0 * (gx + dx);
                gy = 2.0 * (gy + dy);
            }
        }
        const double fx = in[2 * k] + gx + dx, fy = in[2 * k + 1] + gy + dy;
        if (ok && !(fx >= 0.0 && fx <= W - 1 && fy >= 0.0 && fy <= H - 1)) ok = 0;
        out[2 * k] = fx;
        out[2 * k + 1] = fy;
        status[k] = (uint8_t)ok;
    }
    for (int i = 0; i < 26; ++i) free(bufs[i]);
    return 0;
}

/* ---------------------------------------------------------------- RANSAC */

/* SplitMix64 (Steele, Lea & Flood 2014; the finaliser of Vigna's
 * splitmix64.c): the z-th output of the counter z. */
uint64_t ho_splitmix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* The 4 sample indices of hypothesis m (0 if drawn, -1 if 64 draws did not
 * give 4 distinct indices). */
int ho_sample4(uint64_t seed, int m, int n, int* idx) {
    int got = 0;
    for (int j = 0; j < 64 && got < 4; ++j) {
        const uint64_t z = ho_splitmix64(seed + 0x9E3779B97F4A7C15ull * (uint64_t)(1 + 64 * (int64_t)m + j));
        const int v = (int)((uint32_t)(z >> 32) % (uint32_t)n);
        int dup = 0;
        for (int a = 0; a < got; ++a) dup |= idx[a] == v;
        if (!dup) idx[got++] = v;
    }
    return got == 4 ? 0 : -1;
}

/* Gaussian elimination with partial pivoting on the n x n system [M | r]
 * (row-major, M overwritten); 0 or -1 if a pivot's magnitude is < 1e-12. */
static int solve(double* M, double* r, int n, double* x) {
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int i = c + 1; i < n; ++i)
            if (fabs(M[i * n + c]) > fabs(M[p * n + c])) p = i;
        if (fabs(M[p * n + c]) < 1e-12) return -1;
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
    return 0;
}

typedef struct {
    double ox, oy, s;   /* x' = (x - ox) * s */
} Norm;

static Norm norm_of(int W, int H) {
    Norm t;
    t.ox = W / 2.0;
    t.oy = H / 2.0;
    t.s = 2.0 / (W > H ? W : H);
    return t;
}

/* the two DLT rows of the pair (x, y) -> (X, Y), normalised coordinates */
static void dlt_rows(double x, double y, double X, double Y, double* r0, double* r1, double* b) {
    r0[0] = x; r0[1] = y; r0[2] = 1.0; r0[3] = 0.0; r0[4] = 0.0; r0[5] = 0.0;
    r0[6] = -x * X; r0[7] = -y * X;
    r1[0] = 0.0; r1[1] = 0.0; r1[2] = 0.0; r1[3] = x; r1[4] = y; r1[5] = 1.0;
    r1[6] = -x * Y; r1[7] = -y * Y;
    b[0] = X;
    b[1] = Y;
}

/* the pixel-coordinate homography of normalised model h (8 values) */
static void denorm(const double* h, Norm t, double* Hp) {
    /* Hp = T^-1 Hn T with T = [s 0 -s ox; 0 s -s oy; 0 0 1] */
    double Hn[9] = {h[0], h[1], h[2], h[3], h[4], h[5], h[6], h[7], 1.0};
    double T[9] = {t.s, 0.0, -t.s * t.ox, 0.0, t.s, -t.s * t.oy, 0.0, 0.0, 1.0};
    double Ti[9] = {1.0 / t.s, 0.0, t.ox, 0.0, 1.0 / t.s, t.oy, 0.0, 0.0, 1.0};
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

/* the model of 4 pairs (src -> dst, pixel coordinates); 0 or -1 */
static int model4(const double* src, const double* dst, const int* idx, Norm t, double* Hp) {
    double M[64], r[8], h[8];
    for (int a = 0; a < 4; ++a) {
        const int k = idx[a];
        dlt_rows((src[2 * k] - t.ox) * t.s, (src[2 * k + 1] - t.oy) * t.s,
                 (dst[2 * k] - t.ox) * t.s, (dst[2 * k + 1] - t.oy) * t.s,
                 M + 16 * a, M + 16 * a + 8, r + 2 * a);
    }
    if (solve(M, r, 8, h)) return -1;
    denorm(h, t, Hp);
    return 0;
}

/* pair k is an inlier of Hp (M7): it projects in front (w > 0) and its
 * reprojection lands within thr of its partner,
 * (X / w - dx)^2 + (Y / w - dy)^2 < thr^2 */
static double reproj_err2(const double* Hp, const double* src, const double* dst, int k, int* front) {
    const double x = src[2 * k], y = src[2 * k + 1];
    const double X = Hp[0] * x + Hp[1] * y + Hp[2];
    const double Y = Hp[3] * x + Hp[4] * y + Hp[5];
    const double w = Hp[6] * x + Hp[7] * y + Hp[8];
    *front = w > 0.0;
    if (!*front) return 0.0;
    const double ex = X / w - dst[2 * k], ey = Y / w - dst[2 * k + 1];
    return ex * ex + ey * ey;
}

static int inlier(const double* Hp, const double* src, const double* dst, int k, double t2) {
    int front;
    const double e2 = reproj_err2(Hp, src, dst, k, &front);
    return front && e2 < t2;
}

/* The inlier decisions of model Hp (M7) over n pairs: inl[k] = 1 for an
 * inlier; near[k] = 1 when the pair is in front of the model and its squared
 * reprojection error lies within band * thr^2 of thr^2 (either may be NULL).
 * Returns the inlier count. */
int ho_inliers(const double* Hp, const double* src, const double* dst, int n, double thr,
               double band, uint8_t* inl, uint8_t* near) {
    const double t2 = thr * thr;
    int cnt = 0;
    for (int k = 0; k < n; ++k) {
        int front;
        const double e2 = reproj_err2(Hp, src, dst, k, &front);
        const int in = front && e2 < t2;
        cnt += in;
        if (inl) inl[k] = (uint8_t)in;
        if (near) near[k] = (uint8_t)(front && fabs(e2 - t2) <= band * t2);
    }
    return cnt;
}

/* The model of hypothesis m over the pairs src -> dst (M7): 0, or -1 when
 * its sample or its DLT system gives none. */
int ho_hypothesis(const double* src, const double* dst, int n, int W, int H, uint64_t seed, int m,
                  double* Hp) {
    if (n < 4 || m < 0) return -1;
    int idx[4];
    if (ho_sample4(seed, m, n, idx)) return -1;
    return model4(src, dst, idx, norm_of(W, H), Hp);
}

/* Per hypothesis m < iters: counts[m] = its inlier count (-1: no model) and
 * near[m] = how many of the pairs in front of it have a squared
 * reprojection error within band * thr^2 of thr^2 (the decisions that a
 * computation rounding differently may take the other way). */
int ho_ransac_counts(const double* src, const double* dst, int n, int W, int H, int iters,
                     double thr, uint64_t seed, double band, int* counts, int* near) {
    if (n < 4 || iters < 1) return -1;
    const double t2 = thr * thr;
    for (int m = 0; m < iters; ++m) {
        double Hp[9];
        counts[m] = -1;
        near[m] = 0;
        if (ho_hypothesis(src, dst, n, W, H, seed, m, Hp)) continue;
        int cnt = 0, nb = 0;
        for (int k = 0; k < n; ++k) {
            int front;
            const double e2 = reproj_err2(Hp, src, dst, k, &front);
            if (!front) continue;
            cnt += e2 < t2;
            nb += fabs(e2 - t2) <= band * t2;
        }
        counts[m] = cnt;
        near[m] = nb;
    }
    return 0;
}

/* M8: the least-squares fit of the DLT equations of the pairs with inl[k]
 * set (normal equations, the same elimination); 0, or -1 when fewer than 4
 * pairs are marked or the system is singular. */
int ho_refit(const double* src, const double* dst, const uint8_t* inl, int n, int W, int H,
             double* Hout) {
    const Norm t = norm_of(W, H);
    double N[64] = {0}, r[8] = {0}, h[8];
    int m = 0;
    for (int k = 0; k < n; ++k) {
        if (!inl[k]) continue;
        ++m;
        double r0[8], r1[8], b[2];
        dlt_rows((src[2 * k] - t.ox) * t.s, (src[2 * k + 1] - t.oy) * t.s,
                 (dst[2 * k] - t.ox) * t.s, (dst[2 * k + 1] - t.oy) * t.s, r0, r1, b);
        for (int i = 0; i < 8; ++i) {
            for (int j = 0; j < 8; ++j) N[i * 8 + j] += r0[i] * r0[j] + r1[i] * r1[j];
            r[i] += r0[i] * b[0] + r1[i] * b[1];
        }
    }
    if (m < 4 || solve(N, r, 8, h)) return -1;
    denorm(h, t, Hout);
    return 0;
}

/* M7-M8: the homography src -> dst (both n x 2, pixel coordinates of a W x H
 * frame).  Returns the inlier count of the best hypothesis (inl[k] = 1 for
 * its inliers) or -1 when no hypothesis gives a model; *best = its index. */
int ho_ransac(const double* src, const double* dst, int n, int W, int H, int iters, double thr,
              uint64_t seed, double* Hout, uint8_t* inl, int* best) {
    if (n < 4 || iters < 1) return -1;
    const Norm t = norm_of(W, H);
    const double t2 = thr * thr;
    int bestc = -1, bm = -1;
    double Hb[9];
    for (int m = 0; m < iters; ++m) {
        double Hp[9];
        if (ho_hypothesis(src, dst, n, W, H, seed, m, Hp)) continue;
        int cnt = 0;
        for (int k = 0; k < n; ++k) cnt += inlier(Hp, src, dst, k, t2);
        if (cnt > bestc) {
            bestc = cnt;
            bm = m;
            memcpy(Hb, Hp, sizeof Hb);
        }
    }
    if (bm < 0) return -1;
    *best = bm;
    for (int k = 0; k < n; ++k) inl[k] = (uint8_t)inlier(Hb, src, dst, k, t2);
    /* M8: the least-squares refit over the inliers */
    if (bestc < 4 || ho_refit(src, dst, inl, n, W, H, Hout)) memcpy(Hout, Hb, sizeof Hb);
    return bestc;
}

/* The whole front end: corners of prev, tracked into cur, RANSAC; H maps
 * cur pixel centres to prev ones.  Returns the inlier count or -1. */
int ho_estimate(const uint8_t* prev, const uint8_t* cur, int W, int H, int bs, double quality,
                double min_dist, int max_corners, int levels, int wh, int max_iters, double eps,
                double min_eig, int iters, double thr, uint64_t seed, double* Hout,
                int* n_corners, int* n_tracked) {
    int* xy = (int*)malloc(sizeof(int) * 2 * (size_t)max_corners);
    double* sc = (double*)malloc(sizeof(double) * (size_t)max_corners);
    int ncand = 0;
    const int m = ho_corners(prev, W, H, bs, quality, min_dist, max_corners, xy, sc, &ncand);
    *n_corners = m < 0 ? 0 : m;
    int res = -1;
    if (m >= 4) {
        double* in = (double*)malloc(sizeof(double) * 2 * m);
        double* out = (double*)malloc(sizeof(double) * 2 * m);
        uint8_t* st = (uint8_t*)malloc((size_t)m);
        for (int k = 0; k < 2 * m; ++k) in[k] = xy[k];
        ho_track(prev, cur, W, H, levels, wh, max_iters, eps, min_eig, in, m, out, st);
        double* src = (double*)malloc(sizeof(double) * 2 * m);
        double* dst = (double*)malloc(sizeof(double) * 2 * m);
        int nt = 0;
        for (int k = 0; k < m; ++k)
            if (st[k]) {
                src[2 * nt] = out[2 * k] + 0.5;
                src[2 * nt + 1] = out[2 * k + 1] + 0.5;
                dst[2 * nt] = in[2 * k] + 0.5;
                dst[2 * nt + 1] = in[2 * k + 1] + 0.5;
                ++nt;
            }
        *n_tracked = nt;
        uint8_t* inl = (uint8_t*)malloc(nt > 0 ? (size_t)nt : 1);
        int best = -1;
        res = ho_ransac(src, dst, nt, W, H, iters, thr, seed, Hout, inl, &best);
        free(inl);
        free(src);
        free(dst);
        free(in);
        free(out);
        free(st);
    } else {
        *n_tracked = 0;
    }
    free(xy);
    free(sc);
    return res;
}

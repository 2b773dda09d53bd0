/*
 * dmsgm_oracle.c -- plain FP64 CPU oracle of one DMSGM block-grid step.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of what the GPU path computes; it exists so that tests, the
 * smoke check and the CPU-baseline leg of the benchmark can compare the CUDA
 * library against it.  Product code never links, loads or calls it, and it
 * shares no code, header or constant with the CUDA library.
 *
 * The method is Yi et al.'s Dual-Mode Single Gaussian Model as restated by
 * Henderson & Vertescher (arXiv:1702.05156):
 *   - block mean M_i                          Sec. 2.2, eq. for M_i
 *   - mean update                             Sec. 2.2, eq. for mu_i^(t)
 *   - variance sample V_i (max over block)    Sec. 2.2, eq. for V_i
 *   - variance update                         Sec. 2.2, eq. for sigma_i^(t)
 *   - age update, cap 30                      Sec. 2.2, age eq. and text
 *   - apparent / candidate match tests        Sec. 2.3, the two match inequalities
 *   - candidate reset (VAR_INIT = 255)        Sec. 2.3, text after the match tests
 *   - swap when the candidate is older        Sec. 2.3, age inequality
 *   - motion compensation by block mixing     Sec. 2.4 (words only)
 *   - the per-pixel foreground test           Appendix "Dual-mode SGM Inner
 *                                             Update Code Snippet", with the
 *                                             threshold theta_d * sigma_A
 *
 * Readings where the paper is silent or inconsistent (each listed in the
 * design notes):
 *   R1 learning rate 1/(age~ + 1) as in the equations of Sec. 2.2;
 *   R2 variance floor 0.1 inside the two match tests only (appendix code);
 *   R3 mask threshold theta_d * var_A (the appendix's max(0.25, I) is a slip);
 *   R4 no quantisation of the state (the paper stores uchar);
 *   R5 the match tests use the compensated values mu~, var~;
 *   R6 mixing: area-weighted over the <= 4 previous blocks that the
 *      back-projected, axis-aligned BxB square overlaps; weights of
 *      out-of-grid blocks are dropped and the rest renormalised;
 *   R7 a mixed age is rounded half up to an integer;
 *   R8 H maps CURRENT pixel-centre coordinates to PREVIOUS ones;
 *   R9 strict '<' in the match tests, strict '>' in the swap and the mask;
 *   R10 a block with no source (first frame, Z <= 0, non-finite projection,
 *      or in-grid weight below 1e-3) resets both models to (M, 255, 1) and
 *      skips the match step;
 *   R11 sides that are not multiples of B: the grid has ceil(W/B) x ceil(H/B)
 *      blocks with the nominal geometry (centres, back-projected squares,
 *      mixing); a block cut by the right or bottom edge takes M_i, its
 *      extremes and V_i over its pixels inside the frame, and only those
 *      pixels get mask values;
 *   R12 (option, off by default) Yi et al.'s mixture variance: the mixed
 *      variance also carries the spread of the mixed means,
 *      var~ = sum_k w_k (var_k + (mu_k - mu~)^2) / sum_k w_k.
 *
 * Pixel (x, y) has its centre at (x + 0.5, y + 0.5).  Block (bx, by) covers
 * pixels [bx*B, (bx+1)*B) x [by*B, (by+1)*B) clipped to the frame; its centre
 * is ((bx + 0.5) * B, (by + 0.5) * B).
 *
 * Build:  gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared [-fopenmp] -o liboracle.so
 *         dmsgm_oracle.c homog_oracle.c -lm
 * (-ffp-contract=off so that x86 and Arm hosts round identically.)
 */
#include <math.h>
#include <stddef.h>
#include <string.h>

/* Constants fixed by the paper. */
static const double VAR_INIT = 255.0;     /* Sec. 2.3: reset variance          */
static const double VAR_FLOOR = 0.1;      /* appendix code: max(var, .1)        */
static const double MIN_WEIGHT = 1e-3;    /* R10: below this, no source         */

/* Per-block diagnostics written when diag != NULL (ORACLE_DIAG doubles per
 * block).  Tests use them to locate decisions that sit on a threshold. */
enum {
    DG_M = 0,        /* block mean M                                         */
    DG_NOSRC,        /* 1 if the block had no source this frame               */
    DG_WSUM,         /* in-grid weight sum before normalisation               */
    DG_MU_A,         /* compensated apparent mean  mu~_A                      */
    DG_VAR_A,        /* compensated apparent var   var~_A                     */
    DG_XAGE_A,       /* unrounded mixed apparent age                          */
    DG_MU_C,         /* compensated candidate mean mu~_C                      */
    DG_VAR_C,        /* compensated candidate var  var~_C                     */
    DG_XAGE_C,       /* unrounded mixed candidate age                         */
    DG_BRANCH,       /* 0: A matched, 1: C matched, 2: C reset, 3: no source  */
    DG_SWAP,         /* 1 if the models were swapped                          */
    DG_MIN,          /* min pixel of the block                                */
    DG_MAX,          /* max pixel of the block                                */
    ORACLE_DIAG
};

int oracle_diag_stride(void) { return ORACLE_DIAG; }

/* One Gaussian model of one block. */
typedef struct { double mu, var; int age; } model_t;

/* Sec. 2.2: update of one SGM from its compensated value (mu~, var~, age~)
 * with the block's pixels.  The equations are applied as printed:
 *   mu    = age~/(age~+1) * mu~  + 1/(age~+1) * M
 *   V     = max_j (mu - I_j)^2          (uses the UPDATED mean)
 *   var   = age~/(age~+1) * var~ + 1/(age~+1) * V
 *   age   = age~ + 1, not beyond age_max (appendix: increment only below cap)
 */
static model_t sgm_update(model_t m, double M, const unsigned char* frame, int W,
                          int x0, int y0, int x1, int y1, int age_max)
{
    model_t out;
    double a = (double)m.age;
    out.mu = a / (a + 1.0) * m.mu + 1.0 / (a + 1.0) * M;
    double V = 0.0;
    for (int y = y0; y < y1; ++y)
        for (int x = x0; x < x1; ++x) {
            double d = out.mu - (double)frame[(size_t)y * W + x];
            if (d * d > V) V = d * d;
        }
    out.var = a / (a + 1.0) * m.var + 1.0 / (a + 1.0) * V;
    out.age = (m.age < age_max) ? m.age + 1 : m.age;
    return out;
}

/* Sec. 2.3: the reset model (M, VAR_INIT, 1). */
static model_t sgm_reset(double M)
{
    model_t r = { M, VAR_INIT, 1 };
    return r;
}

/*
 * oracle_step -- one frame of the DMSGM block-grid method.
 *
 * frame     W*H bytes, row-major, pitch W.
 * Hm        3x3 row-major homography, CURRENT -> PREVIOUS coordinates (R8).
 * first     nonzero on the first frame of a stream (no previous state).
 * *_in      previous state, Gx*Gy entries each (ignored when first != 0).
 * *_out     next state (apparent A, candidate C).
 * mask_out  W*H bytes, 1 = foreground, 0 = background.
 * diag      NULL or Gx*Gy*ORACLE_DIAG doubles.
 *
 * Returns 0, or -1 on invalid sizes.  Inputs and outputs must not alias.
 * The grid is Gx x Gy = ceil(W/B) x ceil(H/B) blocks (R11).  mix_spread
 * (oracle_step_ex only) switches on R12.
 */
int oracle_step_ex(int W, int H, int B, double theta_s, double theta_d, int age_max,
                   int mix_spread, int first, const unsigned char* frame, const double* Hm,
                const double* muA_in, const double* varA_in, const int* ageA_in,
                const double* muC_in, const double* varC_in, const int* ageC_in,
                double* muA_out, double* varA_out, int* ageA_out,
                double* muC_out, double* varC_out, int* ageC_out,
                unsigned char* mask_out, double* diag)
{
    if (W <= 0 || H <= 0 || B <= 0) return -1;
    const int Gx = (W + B - 1) / B, Gy = (H + B - 1) / B;

    /* Every block reads only the frame and the previous state and writes only
     * its own state, mask pixels and diagnostics: the block rows may run on
     * several threads (OpenMP when built with it, as the paper's CPU version
     * splits rows over TBB tasks) without changing any result. */
#pragma omp parallel for schedule(static)
    for (int by = 0; by < Gy; ++by) {
        for (int bx = 0; bx < Gx; ++bx) {
            const size_t k = (size_t)by * Gx + bx;
            const int x0 = bx * B, y0 = by * B;
            const int x1 = x0 + B < W ? x0 + B : W;    /* R11: clipped to the frame */
            const int y1 = y0 + B < H ? y0 + B : H;

            /* Sec. 2.2 eq. for M_i: mean of the block's pixels. */
            double S = 0.0, mn = 255.0, mx = 0.0;
            for (int y = y0; y < y1; ++y)
                for (int x = x0; x < x1; ++x) {
                    double I = (double)frame[(size_t)y * W + x];
                    S += I;
                    if (I < mn) mn = I;
                    if (I > mx) mx = I;
                }
            const double M = S / ((double)(x1 - x0) * (double)(y1 - y0));

            /* Sec. 2.4 + R6/R8/R10: compensate the previous models by mixing
             * the blocks that the back-projected square overlaps. */
            int nosrc = first ? 1 : 0;
            double wsum = 0.0, xageA = 0.0, xageC = 0.0;
            model_t A = { 0, 0, 0 }, C = { 0, 0, 0 };
            if (!nosrc) {
                const double cx = (bx + 0.5) * B, cy = (by + 0.5) * B;
                const double X = Hm[0] * cx + Hm[1] * cy + Hm[2];
                const double Y = Hm[3] * cx + Hm[4] * cy + Hm[5];
                const double Z = Hm[6] * cx + Hm[7] * cy + Hm[8];
                double px = 0, py = 0;
                if (!(Z > 0.0)) nosrc = 1;
                else {
                    px = X / Z;
                    py = Y / Z;
                    if (!isfinite(px) || !isfinite(py)) nosrc = 1;
                }
                if (!nosrc) {
                    /* Top-left corner of the back-projected square, in block
                     * units; the square spans [u, u+1) x [w, w+1). */
                    const double u = (px - 0.5 * B) / B;
                    const double w = (py - 0.5 * B) / B;
                    const double i0 = floor(u), j0 = floor(w);
                    const double fx = u - i0, fy = w - j0;
                    double sA_mu = 0, sA_var = 0, sA_age = 0;
                    double sC_mu = 0, sC_var = 0, sC_age = 0;
                    for (int dj = 0; dj < 2; ++dj)
                        for (int di = 0; di < 2; ++di) {
                            const double ii = i0 + di, jj = j0 + dj;
                            /* overlap area of the square with cell (ii, jj) */
                            const double wgt = (di ? fx : 1.0 - fx) * (dj ? fy : 1.0 - fy);
                            if (ii < 0 || ii >= Gx || jj < 0 || jj >= Gy) continue;
                            const size_t n = (size_t)jj * Gx + (size_t)ii;
                            wsum += wgt;
                            sA_mu += wgt * muA_in[n];
                            sA_var += wgt * varA_in[n];
                            sA_age += wgt * ageA_in[n];
                            sC_mu += wgt * muC_in[n];
                            sC_var += wgt * varC_in[n];
                            sC_age += wgt * ageC_in[n];
                        }
                    if (!(wsum >= MIN_WEIGHT)) nosrc = 1;
                    else if (mix_spread) {
                        /* R12: second pass, the spread of the mixed means */
                        const double mA = sA_mu / wsum, mC = sC_mu / wsum;
                        for (int dj = 0; dj < 2; ++dj)
                            for (int di = 0; di < 2; ++di) {
                                const double ii = i0 + di, jj = j0 + dj;
                                const double wgt = (di ? fx : 1.0 - fx) * (dj ? fy : 1.0 - fy);
                                if (ii < 0 || ii >= Gx || jj < 0 || jj >= Gy) continue;
                                const size_t n = (size_t)jj * Gx + (size_t)ii;
                                sA_var += wgt * (muA_in[n] - mA) * (muA_in[n] - mA);
                                sC_var += wgt * (muC_in[n] - mC) * (muC_in[n] - mC);
                            }
                    }
                    if (!nosrc) {
                        A.mu = sA_mu / wsum;
                        A.var = sA_var / wsum;
                        xageA = sA_age / wsum;
                        A.age = (int)floor(xageA + 0.5);     /* R7 */
                        C.mu = sC_mu / wsum;
                        C.var = sC_var / wsum;
                        xageC = sC_age / wsum;
                        C.age = (int)floor(xageC + 0.5);
                    }
                }
            }
            if (diag) {
                double* d = diag + k * ORACLE_DIAG;
                d[DG_WSUM] = wsum;
                d[DG_MU_A] = A.mu; d[DG_VAR_A] = A.var; d[DG_XAGE_A] = xageA;
                d[DG_MU_C] = C.mu; d[DG_VAR_C] = C.var; d[DG_XAGE_C] = xageC;
            }

            /* Sec. 2.3: match -> update -> reset -> swap. */
            int branch, swapped = 0;
            if (nosrc) {
                A = sgm_reset(M);
                C = sgm_reset(M);
                branch = 3;
            } else {
                const double dA = M - A.mu, dC = M - C.mu;
                if (dA * dA < theta_s * fmax(A.var, VAR_FLOOR)) {
                    A = sgm_update(A, M, frame, W, x0, y0, x1, y1, age_max);
                    branch = 0;
                } else if (dC * dC < theta_s * fmax(C.var, VAR_FLOOR)) {
                    C = sgm_update(C, M, frame, W, x0, y0, x1, y1, age_max);
                    branch = 1;
                } else {
                    C = sgm_reset(M);
                    branch = 2;
                }
                if (C.age > A.age) {
                    A = C;
                    C = sgm_reset(M);
                    swapped = 1;
                }
            }
            muA_out[k] = A.mu; varA_out[k] = A.var; ageA_out[k] = A.age;
            muC_out[k] = C.mu; varC_out[k] = C.var; ageC_out[k] = C.age;

            /* Per-pixel foreground test with the final apparent model. */
            for (int y = y0; y < y1; ++y)
                for (int x = x0; x < x1; ++x) {
                    double d = (double)frame[(size_t)y * W + x] - A.mu;
                    mask_out[(size_t)y * W + x] = (d * d > theta_d * A.var) ? 1 : 0;
                }

            if (diag) {
                double* d = diag + k * ORACLE_DIAG;
                d[DG_M] = M;
                d[DG_NOSRC] = nosrc;
                d[DG_BRANCH] = branch;
                d[DG_SWAP] = swapped;
                d[DG_MIN] = mn;
                d[DG_MAX] = mx;
            }
        }
    }
    return 0;
}

int oracle_step(int W, int H, int B, double theta_s, double theta_d, int age_max,
                int first, const unsigned char* frame, const double* Hm,
                const double* muA_in, const double* varA_in, const int* ageA_in,
                const double* muC_in, const double* varC_in, const int* ageC_in,
                double* muA_out, double* varA_out, int* ageA_out,
                double* muC_out, double* varC_out, int* ageC_out,
                unsigned char* mask_out, double* diag)
{
    return oracle_step_ex(W, H, B, theta_s, theta_d, age_max, 0, first, frame, Hm,
                          muA_in, varA_in, ageA_in, muC_in, varC_in, ageC_in,
                          muA_out, varA_out, ageA_out, muC_out, varC_out, ageC_out,
                          mask_out, diag);
}

/* Threads of the block-row loop (n <= 0: all available); returns the count in
 * use, 1 when the library was built without OpenMP. */
#ifdef _OPENMP
#include <omp.h>
#endif
int oracle_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    else omp_set_num_threads(omp_get_num_procs());
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/*
 * oracle_run -- T frames in a row, free-running, from an empty state.
 * frames: T*W*H bytes; Hs: T*9 doubles (Hs[0] is ignored: first frame).
 * The state after the last frame is left in the *_out arrays and the masks
 * of every frame in masks (T*W*H bytes).  Scratch: 6 arrays of Gx*Gy that
 * the caller passes in (st_* ping buffers) so that this file allocates
 * nothing.
 */
int oracle_run_ex(int W, int H, int B, double theta_s, double theta_d, int age_max,
                  int mix_spread, int T,
               const unsigned char* frames, const double* Hs,
               double* muA, double* varA, int* ageA,
               double* muC, double* varC, int* ageC,
               double* tmu_A, double* tvar_A, int* tage_A,
               double* tmu_C, double* tvar_C, int* tage_C,
               unsigned char* masks)
{
    if (W <= 0 || H <= 0 || B <= 0 || T < 0) return -1;
    const size_t npx = (size_t)W * H;
    const size_t nb = (size_t)((W + B - 1) / B) * (size_t)((H + B - 1) / B);
    for (int t = 0; t < T; ++t) {
        int rc = oracle_step_ex(W, H, B, theta_s, theta_d, age_max, mix_spread, t == 0,
                             frames + (size_t)t * npx, Hs + (size_t)t * 9,
                             muA, varA, ageA, muC, varC, ageC,
                             tmu_A, tvar_A, tage_A, tmu_C, tvar_C, tage_C,
                             masks + (size_t)t * npx, NULL);
        if (rc) return rc;
        memcpy(muA, tmu_A, nb * sizeof(double));
        memcpy(varA, tvar_A, nb * sizeof(double));
        memcpy(ageA, tage_A, nb * sizeof(int));
        memcpy(muC, tmu_C, nb * sizeof(double));
        memcpy(varC, tvar_C, nb * sizeof(double));
        memcpy(ageC, tage_C, nb * sizeof(int));
    }
    return 0;
}

int oracle_run(int W, int H, int B, double theta_s, double theta_d, int age_max, int T,
               const unsigned char* frames, const double* Hs,
               double* muA, double* varA, int* ageA,
               double* muC, double* varC, int* ageC,
               double* tmu_A, double* tvar_A, int* tage_A,
               double* tmu_C, double* tvar_C, int* tage_C,
               unsigned char* masks)
{
    return oracle_run_ex(W, H, B, theta_s, theta_d, age_max, 0, T, frames, Hs,
                         muA, varA, ageA, muC, varC, ageC,
                         tmu_A, tvar_A, tage_A, tmu_C, tvar_C, tage_C, masks);
}

/*
 * Preprocessing (the paper's Gaussian blur then 3x3 median, both clamping
 * coordinates to the frame; Sec. 2.1 and the appendix filter listings).
 *
 * Readings where the paper leaves the filter open:
 *   P1 the Gaussian comes first, then the median;
 *   P2 the N x N Gaussian (N odd, sigma > 0) is the outer product of the 1-D
 *      weights g(x) = exp(-x^2 / (2 sigma^2)), x = -N/2 .. N/2, normalised
 *      and quantised to 8-bit fixed point: q(x) = round(256 g(x) / sum g)
 *      for x != 0 and q(0) = 256 - sum_{x != 0} q(x), so the 2-D weights
 *      q(i) q(j) sum to exactly 65536;
 *   P3 the blurred pixel is floor(sum_ij q(i) q(j) I(r+i, c+j) / 65536) --
 *      the paper's float sum cast to an 8-bit value, computed exactly;
 *   P4 the median is the 5th smallest of the 9 clamped neighbours.
 * gauss_size 0 skips the blur; median 0 skips the median.
 */
static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

int oracle_gauss_weights(int gauss_size, double sigma, int* q)
{
    if (gauss_size < 1 || gauss_size % 2 == 0 || !(sigma > 0.0)) return -1;
    const int h = gauss_size / 2;
    double g[64], sum = 0.0;
    if (gauss_size > 63) return -1;
    for (int x = -h; x <= h; ++x) {
        g[x + h] = exp(-(double)x * x / (2.0 * sigma * sigma));
        sum += g[x + h];
    }
    int rest = 0;
    for (int x = -h; x <= h; ++x)
        if (x != 0) {
            q[x + h] = (int)floor(256.0 * g[x + h] / sum + 0.5);
            rest += q[x + h];
        }
    q[h] = 256 - rest;
    return 0;
}

int oracle_prefilter(int W, int H, const unsigned char* in, unsigned char* out,
                     int gauss_size, double sigma, int median)
{
    if (W <= 0 || H <= 0) return -1;
    const size_t n = (size_t)W * H;
    /* the blurred frame goes to out; the caller applies the median to it */
    if (gauss_size > 0) {
        int q[64];
        if (oracle_gauss_weights(gauss_size, sigma, q)) return -1;
        const int h = gauss_size / 2;
        for (int r = 0; r < H; ++r)
            for (int c = 0; c < W; ++c) {
                long long s = 0;
                for (int i = -h; i <= h; ++i)
                    for (int j = -h; j <= h; ++j)
                        s += (long long)q[i + h] * q[j + h] *
                             in[(size_t)clampi(r + i, 0, H - 1) * W + clampi(c + j, 0, W - 1)];
                out[(size_t)r * W + c] = (unsigned char)(s >> 16);
            }
    } else {
        memcpy(out, in, n);
    }
    return median ? 1 : 0;   /* the caller applies the median (oracle_median3) */
}

int oracle_median3(int W, int H, const unsigned char* in, unsigned char* out)
{
    if (W <= 0 || H <= 0) return -1;
    for (int r = 0; r < H; ++r)
        for (int c = 0; c < W; ++c) {
            /* P4 (Sec. 2.1): the median of the 9 clamped neighbours is the
             * intensity v of rank 5, i.e. the smallest v with at least 5 of
             * the 9 values <= v.  Count the 9 values per intensity, then
             * accumulate the counts upwards until they reach 5. */
            int count[256] = {0};
            for (int i = -1; i <= 1; ++i)
                for (int j = -1; j <= 1; ++j)
                    ++count[in[(size_t)clampi(r + i, 0, H - 1) * W + clampi(c + j, 0, W - 1)]];
            int v = 0, le = count[0];
            while (le < 5) le += count[++v];
            out[(size_t)r * W + c] = (unsigned char)v;
        }
    return 0;
}

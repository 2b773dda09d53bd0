/*
 * dmsgm_homog.h -- C ABI of the motion-estimation front end: the homography
 * that the DMSGM step (dmsgm.h) consumes, estimated on the GPU from two
 * frames (arXiv:1702.05156, Sec. 2.4 "Motion Compensation", Sec. 3.1.3 and
 * the appendix "Motion Compensation Code Snippets": good features to track,
 * pyramidal Lucas-Kanade with a 20 x 20 window and 5 levels, and a RANSAC
 * homography).
 *
 * Method, per call (the readings are those of the library's design notes):
 *   1. corners of the previous frame: Shi-Tomasi's smaller eigenvalue of the
 *      structure tensor of 3 x 3 Sobel gradients summed over a
 *      block_size^2 window (evaluated in FP32 in a fixed operation order),
 *      local maxima above quality * max score, at most the 8192 strongest
 *      (ties by row-major index), kept greedily when every kept corner is at
 *      least min_distance away, at most max_corners;
 *   2. each corner tracked into the current frame by Bouguet's pyramidal
 *      Lucas-Kanade (binomial pyramid of `levels` halvings, a
 *      (2 win_half + 1)^2 window, up to max_iters updates per level until an
 *      update is shorter than eps; points whose gradient matrix has a
 *      smaller eigenvalue per sample below min_eig, or that leave the frame,
 *      are dropped);
 *   3. RANSAC over the tracked pairs (current pixel centre -> previous pixel
 *      centre): ransac_iters 4-point hypotheses drawn by SplitMix64 from
 *      `seed`, an FP64 DLT model each, inliers within `thresh` pixels, the
 *      best (most inliers, lowest index) refitted by least squares on its
 *      inliers.
 * The result maps CURRENT pixel-centre coordinates to PREVIOUS ones, h33 = 1:
 * exactly the H3x3 argument of dmsgm_process.
 *
 * Conventions: frames are W x H uint8 device buffers, pitch W, 16-byte
 * aligned, W % 16 == 0, 16 <= W, H <= 16384.  Entry points run on the given
 * CUDA stream (0 = legacy) and return when their host outputs are written
 * (they synchronise the stream).  Errors: DMSGM_ERR_INVALID_ARG for bad
 * arguments (nothing launched), DMSGM_ERR_CUDA for launch failures,
 * DMSGM_ERR_OOM, and DMSGM_ERR_UNSUPPORTED when a frame has more tied
 * candidates at the selection cut than the library holds (4096); the
 * message is in dmsgm_last_error().  A handle is not thread-safe.
 */
#ifndef DMSGM_HOMOG_H
#define DMSGM_HOMOG_H

#include <stddef.h>
#include <stdint.h>

#include "dmsgm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dmsgm_homog_ctx* dmsgm_homog_t;

typedef struct {
    int block_size;        /* structure-tensor window, odd 1..7 (3)            */
    double quality;        /* score cut relative to the maximum, > 0 (0.01)    */
    double min_distance;   /* spacing of kept corners in pixels, >= 0 (10)     */
    int max_corners;       /* 1..4096 (500)                                    */
    int levels;            /* pyramid halvings, 0..8 (5, the paper's)          */
    int win_half;          /* window half-width, 1..15 (10: the paper's 20)    */
    int max_iters;         /* updates per level, >= 1 (30)                     */
    double eps;            /* update length that stops a level (0.01 px)       */
    double min_eig;        /* smallest eigenvalue per window sample (1e-3)     */
    int ransac_iters;      /* hypotheses, 1..65536 (2000)                      */
    double thresh;         /* inlier reprojection distance in pixels (3)       */
    unsigned long long seed; /* SplitMix64 counter origin (0)                  */
} dmsgm_homog_params;

typedef struct {
    int corners;     /* corners kept                                          */
    int candidates;  /* local maxima above the cut (before the 8192 cap)      */
    int tracked;     /* corners tracked into the current frame                */
    int inliers;     /* inliers of the best hypothesis (-1: no model)         */
    int best;        /* index of the best hypothesis (-1: none)               */
} dmsgm_homog_result;

/* Fill p with the defaults above. */
void dmsgm_homog_default_params(dmsgm_homog_params* p);

/* A handle for W x H frames; p = NULL takes the defaults.  Allocates the
 * pyramids, the list of local maxima, the selection and RANSAC scratch and
 * a CUDA graph of the whole estimate. */
int dmsgm_homog_create(int W, int H, const dmsgm_homog_params* p, dmsgm_homog_t* out);

/* Steps 1-3: H3x3 (host, row-major) maps cur pixel centres to prev ones.
 * When fewer than 4 points are tracked or no hypothesis gives a model, H3x3
 * is the identity and res->inliers = -1 (the call still returns DMSGM_OK).
 * res may be NULL. */
int dmsgm_homog_estimate(dmsgm_homog_t h, const uint8_t* prev_dev, const uint8_t* cur_dev,
                         double H3x3[9], dmsgm_homog_result* res, void* stream);

/* Step 1 alone: up to max_corners corners of img, strongest first, as pixel
 * indices (xy[2k] = x, xy[2k+1] = y, host) with their scores (host, may be
 * NULL); *n = how many; *n_cand = the candidates before the cap. */
int dmsgm_homog_corners(dmsgm_homog_t h, const uint8_t* img_dev, int* xy, float* scores, int* n,
                        int* n_cand, void* stream);

/* Step 2 alone: n points (host, pixel indices, x y pairs) of prev tracked
 * into cur: positions (host, n x 2) and status (host, 1 = tracked). */
int dmsgm_homog_track(dmsgm_homog_t h, const uint8_t* prev_dev, const uint8_t* cur_dev,
                      const float* pts, int n, float* out, uint8_t* status, void* stream);

/* Step 3 alone: n pairs src -> dst (host, pixel coordinates, x y pairs;
 * n <= 4096).  H3x3 (host) as in dmsgm_homog_estimate; inliers (host, n
 * bytes, may be NULL); res->inliers / res->best as above. */
int dmsgm_homog_ransac(dmsgm_homog_t h, const double* src, const double* dst, int n,
                       double H3x3[9], uint8_t* inliers, dmsgm_homog_result* res, void* stream);

/* NULL-safe. */
int dmsgm_homog_destroy(dmsgm_homog_t h);

#ifdef __cplusplus
}
#endif

#endif /* DMSGM_HOMOG_H */

/*
 * dmsgm.h -- C ABI of the GB300 (sm_103a) DMSGM motion-mask library.
 *
 * The library runs the data-parallel hot path of the Dual-Mode Single
 * Gaussian Model (Yi et al., restated in arXiv:1702.05156) on a block grid:
 * per frame, in ONE fused kernel,
 *   (a) motion-compensate the previous block models by the frame's
 *       homography: each block's back-projected BxB square mixes mean,
 *       variance and age of the <= 4 previous blocks it overlaps, weighted
 *       by overlap area (Sec. 2.4; "tilde" values of Sec. 2.2);
 *   (b) compute each block's mean M (Sec. 2.2, eq. for M_i) and run the
 *       apparent/candidate match -> update -> reset -> swap (Sec. 2.2 mean,
 *       variance and age equations; Sec. 2.3 match tests and swap rule);
 *   (c) write the per-pixel foreground mask (I - mu_A)^2 > theta_d * var_A
 *       (appendix "Dual-mode SGM Inner Update Code Snippet", threshold taken
 *       against the apparent variance).
 *
 * Conventions
 *   - Frames are W x H uint8, row-major, pitch W bytes, device memory,
 *     16-byte aligned base.  W % 16 == 0 (so W is a multiple of every
 *     block size); H is any height.
 *   - block is 1, 2, 4, 8 or 16 (1 is the paper's per-pixel model).  The
 *     grid is Gx x Gy = W/B x ceil(H/B) blocks; block (bx, by) covers pixels
 *     [bx*B, (bx+1)*B) x [by*B, (by+1)*B) clipped to the frame: a bottom
 *     block row cut by the frame edge takes its mean, extremes and variance
 *     sample over its pixels inside the frame, while its centre and
 *     back-projected square keep the nominal B x B geometry.  Pixel (x, y)
 *     has its centre at (x + 0.5, y + 0.5).
 *   - The homography is a host double[9], row-major, and maps CURRENT
 *     pixel-centre coordinates to PREVIOUS ones.  It is reduced on the host
 *     (FP64) to FP32 displacement coefficients; the GPU does no FP64 work.
 *   - The mask is bit-packed: H rows of ceil(W/32) uint32 words; bit j of
 *     word i in row y is pixel x = 32*i + j (LSB = leftmost).  1 = foreground.
 *   - Model state lives on the device in two ping-pong buffers per handle
 *     (read t-1, write t), each a structure of arrays over the Gx*Gy blocks
 *     (row-major, bx fastest): mu, var and age, where entry k of each array
 *     holds the apparent and the candidate value of block k side by side
 *     ((mu_A, mu_C) and (var_A, var_C) as FP32 or FP16 pairs, (age_A, age_C)
 *     as a byte pair).
 *   - The first process() after create/reset (and any block whose
 *     back-projection has no in-grid source) starts both models at
 *     (M, 255, 1), the paper's candidate-reset values (Sec. 2.3).
 *
 * Errors: every call returns DMSGM_OK (0) or a negative code; the message of
 * the last failure on the calling thread is in dmsgm_last_error().  Invalid
 * arguments never touch device state.  Kernels that detect a fault on the
 * device (a TMA wait that ran out) set a status word that dmsgm_status()
 * reports.
 *
 * Threading: a handle must not be used from two host threads or two streams
 * at once.  Different handles are independent.
 */
#ifndef DMSGM_H
#define DMSGM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dmsgm_ctx* dmsgm_t;

enum {
    DMSGM_OK = 0,
    DMSGM_ERR_INVALID_ARG = -1,
    DMSGM_ERR_OOM = -2,
    DMSGM_ERR_CUDA = -3,
    DMSGM_ERR_TIMEOUT = -4,
    DMSGM_ERR_DEVICE_STATUS = -5,
    DMSGM_ERR_UNSUPPORTED = -6
};

enum { DMSGM_STATE_FP32 = 0, DMSGM_STATE_FP16 = 1 };

/* Optional create-time settings; a zero-initialised struct means defaults. */
typedef struct {
    int precision;      /* DMSGM_STATE_FP32 (default) or DMSGM_STATE_FP16:
                           FP16 storage of mu/var, FP32 arithmetic           */
    void* state_mem;    /* optional caller-owned device memory for the state
                           (>= dmsgm_state_bytes(), 256-byte aligned); it must
                           outlive the handle.  NULL: the handle allocates.   */
    size_t state_bytes; /* size of state_mem                                  */
    int tile_rows;      /* rows of pixels per CTA tile: 4, 8 or 16 times the
                           block size, at most 256; 0 = built-in choice (8
                           for block 1, 16 for 2, 32 for 4 and 8, 64 for 16) */
    int use_pdl;        /* 1: programmatic dependent launch -- a frame's
                           pixel load overlaps the previous kernel's tail, so
                           the frame must not be written by the kernel that
                           immediately precedes the call on the stream;
                           0 (default): plain stream order                    */
    int seq_tile_rows;  /* tile height of dmsgm_process_seq: 8, 16, 32 or 64
                           times the block size / 2 (32, 64, 128, 256 rows
                           for block 4; 64, 128, 256 for block 8); 0 = the
                           built-in choice                                    */
    int kernel;         /* frame-step kernel of dmsgm_process and
                           dmsgm_process_host: DMSGM_KERNEL_AUTO (0) or
                           DMSGM_KERNEL_TILE (1), both the per-tile kernel
                           (one CTA per tile); other values are refused.     */
    int mix_spread;     /* 1: Yi et al.'s mixture variance -- the compensated
                           variance also carries the spread of the mixed
                           means, sum_k w_k (var_k + (mu_k - mu~)^2) / sum w;
                           0 (default): the variances alone (Sec. 2.4).  Not
                           available through dmsgm_process_seq_noalloc.      */
    int pre_gauss;      /* preprocessing (Sec. 2.1), applied to every frame
                           before the step, as dmsgm_prefilter: Gaussian size
                           (0: none, or odd 3..15) ...                       */
    double pre_sigma;   /* ... and its sigma (> 0)                            */
    int pre_median;     /* 1: then the 3 x 3 median.  With either filter the
                           batched and multi-frame paths are not available
                           (DMSGM_ERR_UNSUPPORTED / per-frame launches).
                           For block 4 or 8 with the default tile_rows (32),
                           Gaussian size 0, 3, 5 or 7 and mix_spread 0, the
                           step kernel filters its own tile (the filter runs
                           before the wait on the previous frame's kernel);
                           otherwise the handle owns two W*H scratch frames,
                           the filter runs as its own pass and the step
                           without programmatic dependent launch.  Results
                           are identical.                                    */
    int pre_separate;   /* 1: always run the preprocessing as its own pass   */
    int checked;        /* 1: the checked build of the frame step: every state
                           load and store and every mask byte checks its
                           index against the grid and the frame; an index
                           out of range is skipped and sets bit 2 of the
                           device status word (dmsgm_status then returns
                           DMSGM_ERR_DEVICE_STATUS).
                           Slower; for debugging.  Not with mix_spread or the
                           preprocessing (DMSGM_ERR_INVALID_ARG); the
                           multi-frame entry point runs per-frame launches
                           and the batched one refuses such handles
                           (DMSGM_ERR_UNSUPPORTED).                          */
} dmsgm_opts;

enum { DMSGM_KERNEL_AUTO = 0, DMSGM_KERNEL_TILE = 1 };

/* Read-only description of a handle. */
typedef struct {
    int width, height, block, grid_w, grid_h, precision, age_max;
    float theta_s, theta_d;
    int initialized;             /* 0 until the first process()/set_state()  */
    int parity;                  /* index of the buffer holding the state    */
    unsigned long long frames;   /* process() calls since create/reset       */
    size_t state_bytes;          /* device bytes (both buffers + control)    */
    size_t host_state_bytes;     /* bytes of the packed image of get/set_state */
    int tile_rows;               /* rows per CTA tile in use                 */
    int device;                  /* CUDA device of the handle                */
    int kernel;                  /* frame-step kernel setting (DMSGM_KERNEL_*) */
    int last_kernel;             /* kernel of the last dmsgm_process step:
                                    DMSGM_KERNEL_TILE; 0 before the first     */
    int mix_spread;              /* dmsgm_opts.mix_spread in use              */
    int pre_fused;               /* 1: the step kernel filters its own tile   */
    int checked;                 /* dmsgm_opts.checked in use                 */
} dmsgm_info;

/* Device bytes a handle needs for its state: a 256-byte control block, one
 * int per 256 x (8*block) pixel tile (the multi-frame kernel's progress
 * counters), and two buffers of three arrays (Gx*Gy*2*s, Gx*Gy*2*s and
 * Gx*Gy*2 bytes; s = 4 for FP32, 2 for FP16), every part 256-byte aligned.
 * Returns 0 for invalid sizes. */
size_t dmsgm_state_bytes(int width, int height, int block, int precision);

/* Bytes of the packed host image used by dmsgm_get_state/dmsgm_set_state:
 * the three state arrays back to back, no padding -- mu (Gx*Gy pairs
 * (mu_A, mu_C)), var (Gx*Gy pairs (var_A, var_C)), both FP32 or FP16 as
 * stored, then age (Gx*Gy byte pairs (age_A, age_C)). */
size_t dmsgm_host_state_bytes(int width, int height, int block, int precision);

/* Create a handle on the current CUDA device.  The state is undefined until
 * the first process() (which starts every block afresh) or set_state().
 * theta_s is the match
 * threshold of Sec. 2.3, theta_d the foreground threshold, age_max the age
 * cap of Sec. 2.2 (30 in the paper).  Validation: width, height > 0;
 * block in {1, 2, 4, 8, 16}; width % 16 == 0; width and height <= 2^20;
 * theta_s, theta_d finite and > 0; 1 <= age_max <= 255. */
int dmsgm_create(int width, int height, int block, float theta_s, float theta_d,
                 int age_max, dmsgm_t* out);
int dmsgm_create_ex(int width, int height, int block, float theta_s, float theta_d,
                    int age_max, const dmsgm_opts* opts, dmsgm_t* out);

/* Destroy a handle (NULL-safe).  If the handle allocated its own state or
 * staging memory, the device is synchronised before that memory is freed;
 * with caller-owned state memory (dmsgm_opts.state_mem) nothing waits, and
 * the caller keeps the memory alive until its queued work is done. */
int dmsgm_destroy(dmsgm_t h);

/* One frame, asynchronously on cuda_stream (a cudaStream_t; NULL = legacy
 * default stream).  frame_dev: W*H bytes of device memory, 16-byte aligned.
 * H3x3: host, row-major, current -> previous coordinates, finite.
 * mask_dev: device, H*ceil(W/32) uint32 words, 4-byte aligned.  frame_dev
 * and mask_dev must stay valid until the stream reaches this work.  When a
 * stream capture records a sequence of k calls, the handle's host-side
 * buffer parity advances by k at capture time; replays are consistent with
 * it when k is even (or the graph is replayed once). */
int dmsgm_process(dmsgm_t h, const uint8_t* frame_dev, const double H3x3[9],
                  uint32_t* mask_dev, void* cuda_stream);

/* n consecutive frames of the handle's stream from device memory in
 * persistent launches (at most 256 frames each): frames_dev holds frame t at
 * t*W*H (16-byte aligned), masks_dev receives frame t's mask at
 * t*H*ceil(W/32) words, H3x3s holds n host homographies.  Each CTA owns one
 * tile for the whole launch and starts frame t+1 as soon as the tiles within
 * the dependency radius of the frames' homographies have published frame t
 * (per-tile progress counters in the handle's memory, Sec. 2.4 fixes that
 * radius); the launch is cooperative and every wait is bounded (a timeout
 * sets the status word).  Results equal n calls of dmsgm_process.  The
 * kernel is built for blocks 4 and 8 on whole block rows; for other sizes,
 * or if the tiles cannot all be resident at once, the call falls back to
 * one launch per frame.  Asynchronous on cuda_stream. */
int dmsgm_process_seq(dmsgm_t h, const uint8_t* frames_dev, int n, const double* H3x3s,
                      uint32_t* masks_dev, void* cuda_stream);

/* dmsgm_process_seq for callers that may not allocate device memory -- for
 * example an application whose device memory is all handed out by its own
 * allocator or a fixed real-time budget, or one that must avoid the
 * device-wide synchronisation a cudaMalloc or cudaFree can cause.  The paper
 * has no counterpart; this is an integration convenience.
 *
 * Nothing is allocated and no handle is needed.  The caller passes the state
 * memory (state_dev: state_bytes >= dmsgm_state_bytes(width, height, block,
 * precision), 256-byte aligned, laid out as a handle's memory; its first
 * word is the device status word, set nonzero if a wait runs out, never
 * cleared here; its counter region is not used), *parity (0 or 1: the
 * buffer holding the state, updated on return), first (1: start every block
 * afresh, as after create/reset), and the frames, homographies and masks as
 * in dmsgm_process_seq.  The multi-frame kernel's progress counters live in
 * one static array of 4096 ints in the library: a frame needing more tiles
 * is rejected with DMSGM_ERR_INVALID_ARG, and one whose tiles cannot all be
 * resident on the GPU, or whose block is not 4 or 8 or whose height is not
 * a multiple of the block, with DMSGM_ERR_UNSUPPORTED.  Every call on a device
 * shares that array (each launch clears the counters it uses), so calls
 * whose work may overlap on the GPU race: keep them on one stream.  The
 * first call on a device looks up the array's device address; make that
 * first call before any stream capture. */
int dmsgm_process_seq_noalloc(int width, int height, int block, int precision, float theta_s,
                              float theta_d, int age_max, void* state_dev, size_t state_bytes,
                              int* parity, int first, const uint8_t* frames_dev, int n,
                              const double* H3x3s, uint32_t* masks_dev, void* cuda_stream);

/* n frames from HOST memory (frames_host: n*W*H bytes, pinned for overlap)
 * into host masks (masks_host: n*H*ceil(W/32) words), pipelined: host->device
 * copies, kernels and device->host copies of consecutive chunks overlap on
 * internal streams.  H3x3s: n*9 doubles.  Ordered after earlier work on
 * cuda_stream; returns when all work is enqueued, and the results are in
 * masks_host once cuda_stream reaches the end of it (synchronise it).  The
 * first call allocates device staging owned by the handle. */
int dmsgm_process_host(dmsgm_t h, const uint8_t* frames_host, int n,
                       const double* H3x3s, uint32_t* masks_host, void* cuda_stream);

/* n handles, one frame each, in ONE kernel launch over a (stream, tile)
 * work list -- by default one work item per CTA, or a persistent grid that
 * walks the list when dmsgm_batch_opts.ctas asks for fewer CTAs than items
 * (Sec. 2.2-2.4 per item, as dmsgm_process).  Handles may differ in size, block and
 * precision; all on one device; no handle twice; width and height at most
 * 65535; block 4 or 8 with the height a multiple of it, else
 * DMSGM_ERR_UNSUPPORTED.  frames_dev[i], masks_dev[i] and H3x3s[9*i..] are handle i's
 * arguments as in dmsgm_process.  1 <= n <= DMSGM_MAX_BATCH (n == 0 is a
 * no-op).  The per-stream descriptors travel in the launch's parameters:
 * the call allocates nothing and copies nothing to the device, and a stream
 * capture records one kernel node per call. */
#define DMSGM_MAX_BATCH 256
int dmsgm_process_batch(int n, const dmsgm_t* hs, const uint8_t* const* frames_dev,
                        const double* H3x3s, uint32_t* const* masks_dev, void* cuda_stream);

/* Preprocessing of the paper's Sec. 2.1: an N x N Gaussian blur (gauss_size
 * N odd in 3..15 with sigma > 0, or 0 for none), then a 3 x 3 median
 * (median 1, or 0 for none), both clamping coordinates to the frame.  The
 * 1-D weights are the normalised Gaussian rounded to 1/256 off the centre,
 * the centre weight making the sum exactly 256; the 2-D kernel is their
 * outer product and a blurred pixel is floor(sum / 65536) -- the paper's
 * float sum cast to an 8-bit value, computed exactly.  The median is the 5th
 * of the 9 clamped neighbours of the blurred frame.
 * in_dev, out_dev: W*H bytes each, device, 16-byte aligned, not
 * overlapping; W % 16 == 0.  At least one filter.  Asynchronous on
 * cuda_stream. */
int dmsgm_prefilter(const uint8_t* in_dev, uint8_t* out_dev, int width, int height,
                    int gauss_size, double sigma, int median, void* cuda_stream);

/* Launch shape of the batched kernel; zero-initialised = built-in choice.
 * A work item is a 256 x (item_warps * block) pixel tile of one stream, one
 * CTA of item_warps warps. */
typedef struct {
    int reserved;    /* must be 0                                             */
    int ctas;        /* CTAs of the launch: 0, or at least the number of
                        work items = one item per CTA (the single-item
                        kernel, the built-in choice); fewer = a persistent
                        grid, each CTA walking the work list with a stride
                        of ctas                                              */
    int use_pdl;     /* 1: programmatic dependent launch (the first tile's
                        pixels load while the previous kernel drains; frames
                        must not be written by the immediately preceding
                        kernel on the stream); 0: plain stream order          */
    int item_warps;  /* warps, i.e. strip rows of blocks, per work item: 4 or
                        8; 0 = 4.  Other values: DMSGM_ERR_INVALID_ARG       */
} dmsgm_batch_opts;

int dmsgm_process_batch_ex(int n, const dmsgm_t* hs, const uint8_t* const* frames_dev,
                           const double* H3x3s, uint32_t* const* masks_dev,
                           const dmsgm_batch_opts* opts, void* cuda_stream);

/* One serving step: n handles, one frame each, with host buffers.  For
 * every i, frames_host[i] (W_i*H_i bytes, pinned for overlap) is copied to
 * the caller's device slot frames_dev[i] on h2d_stream; one batched launch
 * (as dmsgm_process_batch_ex, opts may be NULL) runs on compute_stream after
 * those copies; then masks_dev[i] is copied to masks_host[i] on d2h_stream
 * after the launch.  All three streams are cudaStream_t and must differ.
 * Returns once everything is enqueued; the masks are in host memory when
 * d2h_stream reaches the end of this call's work.  The caller must not
 * reuse a device slot before the step that last used it has completed. */
int dmsgm_process_batch_host(int n, const dmsgm_t* hs, const uint8_t* const* frames_host,
                             uint8_t* const* frames_dev, const double* H3x3s,
                             uint32_t* const* masks_dev, uint32_t* const* masks_host,
                             const dmsgm_batch_opts* opts, void* h2d_stream,
                             void* compute_stream, void* d2h_stream);

/* Copy the current state to / from a packed host image (layout: see
 * dmsgm_host_state_bytes).  Both synchronise the device.  set_state marks
 * the handle initialised, so the next process() compensates from it. */
int dmsgm_get_state(dmsgm_t h, void* host_buf, size_t bytes);
int dmsgm_set_state(dmsgm_t h, const void* host_buf, size_t bytes);

/* Forget the state: the next process() starts every block afresh. */
int dmsgm_reset(dmsgm_t h);

int dmsgm_get_info(dmsgm_t h, dmsgm_info* out);

/* Synchronise the handle's device and read its device status word:
 * DMSGM_OK; DMSGM_ERR_DEVICE_STATUS if a checked kernel met an index out of
 * range; DMSGM_ERR_TIMEOUT if a kernel gave up on a wait.  A set word is
 * cleared. */
int dmsgm_status(dmsgm_t h);

/* Diagnostic of the device-side failure path: enqueue a kernel that waits on
 * a barrier nothing ever completes, bounded by timeout_ns (at most 1 s).
 * The wait gives up, the kernel sets the handle's status word and returns,
 * and the context stays usable; dmsgm_status() then reports
 * DMSGM_ERR_TIMEOUT.  The paper has no counterpart. */
int dmsgm_selftest_wait(dmsgm_t h, unsigned long long timeout_ns, void* cuda_stream);

/* Message of the last failure on the calling thread ("" if none). */
const char* dmsgm_last_error(void);

/* Failure-handling tests (never needed otherwise).  spec "launch:n" makes the
 * n-th frame launch of the process (dmsgm_process and the per-frame launches
 * of the host and multi-frame entry points; one per dmsgm_process_batch call)
 * return DMSGM_ERR_CUDA before anything is launched; "alloc:n" makes the n-th
 * dmsgm_create/_ex return DMSGM_ERR_OOM before allocating.  Counting restarts
 * at every call; "launch:0,alloc:0" or NULL switch injection off.  The
 * environment variable DMSGM_FAULT_INJECT, read once, sets the same. */
void dmsgm_fault_inject(const char* spec);

/* Library version string. */
const char* dmsgm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DMSGM_H */

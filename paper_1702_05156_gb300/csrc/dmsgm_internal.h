// dmsgm_internal.h -- host-side internals shared by the library's translation
// units (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstddef>
#include <cstdint>

#include "dmsgm.h"
#include "dmsgm_device.cuh"
#include "dmsgm_filter.cuh"

namespace dmsgm {

// Thread-local error message + code helper.
int fail(int code, const char* fmt, ...);
void clear_error();

#define DMSGM_CUDA_TRY(call)                                                           \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return ::dmsgm::fail(DMSGM_ERR_CUDA, "%s failed: %s", #call,               \
                                 cudaGetErrorString(e_));                              \
    } while (0)

constexpr int kTmapCache = 16;

// Makes `dev` current for a scope and restores the previous device.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

struct HostStage {              // device staging of dmsgm_process_host
    int chunk = 0;              // frames per chunk
    int slots = 0;
    uint8_t* frames[2] = {nullptr, nullptr};
    uint32_t* masks[2] = {nullptr, nullptr};
    cudaStream_t h2d = nullptr, d2h = nullptr;
    cudaEvent_t ev_in[2] = {nullptr, nullptr};
    cudaEvent_t ev_k[2] = {nullptr, nullptr};
    cudaEvent_t ev_out[2] = {nullptr, nullptr};
    cudaEvent_t ev_start = nullptr;
};

}  // namespace dmsgm

struct dmsgm_ctx {
    int W, H, B, Gx, Gy, prec, age_max;
    float theta_s, theta_d;
    int device;
    int tile_rows;
    int use_pdl;
    int seq_tile_rows;           // 0: automatic
    int kernel;                  // DMSGM_KERNEL_*
    int mix_spread;              // 1: mixed variance carries the spread of the mixed means
    int checked;                 // 1: the per-tile kernel's checked build
    int pre_gauss;               // preprocessing: Gaussian size (0: none)
    double pre_sigma;            //   its sigma
    int pre_median;              //   1: 3 x 3 median
    int pre_half;                //   Gaussian half-size after weight quantisation (0: no blur)
    int pre_fused;               //   1: the step kernel filters its own tile
    dmsgm::FiltArgs filt;        //   the filter's weights
    uint8_t* pre_buf;            //   two scratch frames of the separate pass (NULL: none)
    int last_kernel;             // kernel of the last dmsgm_process step
    int step_rpt;                // strip rows per warp of the per-tile kernel at tile_rows = 8 B (0: not chosen yet)
    int step_narrow;             // block 4, 32-row tiles: 1 one block per lane, -1 two (0: not chosen yet)
    void* mem;                   // control block + two state buffers
    bool owns_mem;
    size_t state_bytes;
    int* status_dev;             // device status word (inside mem)
    int* flags_dev;              // per-tile progress counters of the multi-frame kernel
    dmsgm::StateBuf buf[2];
    int parity;                  // buffer holding the current state
    bool initialized;
    unsigned long long frames;
    struct {
        const void* ptr;
        CUtensorMap map;
    } tmap[dmsgm::kTmapCache];
    int tmap_next;
    struct {                     // frame tensor maps of the batched kernel (box 256 x rows)
        const void* ptr;
        int rows;
        CUtensorMap map;
    } bmap[4];
    int bmap_next;
    struct {                     // 3-D tensor map of the last frame sequence
        const void* ptr;
        int frames, rows;
        CUtensorMap map;
    } seqmap;
    dmsgm::HostStage stage;
};

namespace dmsgm {

// FP64 homography -> double-float coefficients for block size B, in the
// affine form when it applies (affine = 1) or the general form; false if a
// coefficient is not finite in FP32.
bool make_coef(const double H3x3[9], int B, Coef* c, int* affine);

// Fill the per-frame kernel arguments of handle h (reads h->parity etc.).
void fill_args(const dmsgm_ctx* h, int affine, uint32_t* mask_dev, StreamArgs* a);

// Advance the handle's bookkeeping after a frame has been enqueued.
void advance(dmsgm_ctx* h);

// Tensor map of one of the handle's frames with the batched kernel's box
// (kTileW x rows), from a small per-handle cache keyed by the frame.
int batch_frame_map(dmsgm_ctx* h, const void* frame, int rows, CUtensorMap* out);

// Bound on the block-unit displacement (|ex|, |ey|) of every block centre of
// a W x H grid of B x B blocks under m (current -> previous); false when the
// map puts some block behind the camera (no bound).
bool displacement_bound(const double m[9], int W, int H, int B, double* ex, double* ey);

// The driver's cuTensorMapEncodeTiled (NULL if unavailable).
#include <cudaTypedefs.h>
PFN_cuTensorMapEncodeTiled_v12000 encode_fn();
bool valid_dims_ex(int W, int H, int B);

// T frames of one handle in persistent cooperative launches (dmsgm_seq.cu).
int launch_seq(dmsgm_ctx* h, const uint8_t* frames_dev, int T, const double* H3x3s,
               uint32_t* masks_dev, cudaStream_t stream, int* flags);

// Launch the per-tile frame-step kernel for block size B (dmsgm_step.cuh,
// instantiated in dmsgm_step_b<B>.cu).
template <int B>
cudaError_t launch_step_block(dmsgm_ctx* h, const CUtensorMap& tmap, const StreamArgs& a,
                              const Coef& k, cudaStream_t s, bool pdl);
extern template cudaError_t launch_step_block<1>(dmsgm_ctx*, const CUtensorMap&, const StreamArgs&, const Coef&, cudaStream_t, bool);
extern template cudaError_t launch_step_block<2>(dmsgm_ctx*, const CUtensorMap&, const StreamArgs&, const Coef&, cudaStream_t, bool);
extern template cudaError_t launch_step_block<4>(dmsgm_ctx*, const CUtensorMap&, const StreamArgs&, const Coef&, cudaStream_t, bool);
extern template cudaError_t launch_step_block<8>(dmsgm_ctx*, const CUtensorMap&, const StreamArgs&, const Coef&, cudaStream_t, bool);
extern template cudaError_t launch_step_block<16>(dmsgm_ctx*, const CUtensorMap&, const StreamArgs&, const Coef&, cudaStream_t, bool);

// The preprocessing filter's weights (dmsgm_prefilter.cu): false if the
// Gaussian size or sigma is invalid; *half is 0 when the quantised blur is the
// identity.
bool make_filt_args(int gauss_size, double sigma, int median, FiltArgs* f, int* half);

// The per-tile frame step with the preprocessing fused in, for block sizes 4
// and 8 with 32-row tiles and Gaussian half-sizes up to 3 (dmsgm_step_pre.cuh).
template <int B>
cudaError_t launch_step_pre_block(const dmsgm_ctx* h, const uint8_t* frame, const StreamArgs& a,
                                  const Coef& k, cudaStream_t s, bool pdl);
extern template cudaError_t launch_step_pre_block<4>(const dmsgm_ctx*, const uint8_t*, const StreamArgs&, const Coef&, cudaStream_t, bool);
extern template cudaError_t launch_step_pre_block<8>(const dmsgm_ctx*, const uint8_t*, const StreamArgs&, const Coef&, cudaStream_t, bool);

// Sec. 2.1 preprocessing of one frame (dmsgm_prefilter.cu).
int launch_prefilter(const uint8_t* in_dev, uint8_t* out_dev, int W, int H, int gauss_size,
                     double sigma, int median, cudaStream_t s);

// Launch the batched persistent kernel (dmsgm_batch.cu).
int launch_batch(int n, const dmsgm_t* hs, const uint8_t* const* frames_dev,
                 const double* H3x3s, uint32_t* const* masks_dev, const dmsgm_batch_opts& o,
                 cudaStream_t stream);

}  // namespace dmsgm

// dmsgm_homog.cuh -- internals shared by the two translation units of the
// motion-estimation front end (dmsgm_homog.cu: corners, pyramids, tracking
// and the C ABI; dmsgm_homog_ransac.cu: the FP64 RANSAC, built without
// fused multiply-add).
#pragma once

#include "dmsgm_homog.h"
#include "dmsgm_internal.h"

namespace dmsgm {

constexpr int kHoKmax = 8192;          // candidates considered, strongest first
constexpr int kHoTieCap = 4096;        // candidates tied at the selection cut held
constexpr int kHoSortCap = kHoKmax + kHoTieCap;
constexpr int kHoMaxPts = 4096;        // corners / pairs per call
constexpr int kHoMaxLevels = 8;
constexpr int kHoRankSplit = 8;        // key ranges per rank-sort region (partial counts)
constexpr int kHoFitCtas = 128;        // refit CTAs: kHoMaxPts pairs, 32 each
constexpr int kHoFitTerms = 44;        // normal-equation terms: upper triangle 36 + right side 8

// Control block (device, zeroed per call): words of the corner selection and
// the counts that pass between kernels without a host round trip.
enum HoCtrl {
    kCtrlMaxBits = 0,     // max score (float bits; scores are >= 0)
    kCtrlCand,            // candidates (local maxima above the cut)
    kCtrlHiCut,           // high 16 bits of the cut value
    kCtrlAboveHi,         // candidates in buckets above it
    kCtrlCut,             // the cut value's bits (candidates strictly above are all kept)
    kCtrlTakeAll,         // 1: every candidate is kept (no cut)
    kCtrlNGt,             // collected above the cut
    kCtrlNEq,             // collected at the cut
    kCtrlOverflow,        // 1: more ties at the cut than held
    kCtrlNSel,            // selected, sorted
    kCtrlNCorners,        // corners kept
    kCtrlNPts,            // points to track
    kCtrlNPairs,          // tracked pairs
    kCtrlLocalMax,        // local maxima listed by the score kernel
    kCtrlBestM,           // the best hypothesis (-1: none)
    kCtrlBestC,           // its inlier count
    kCtrlWords = 16
};

struct HoPyr {            // one image's pyramid (level 0: the frame itself)
    const uint8_t* p[kHoMaxLevels + 1];
    int w[kHoMaxLevels + 1], h[kHoMaxLevels + 1];
};

// The RANSAC's device results.
struct HoRansacOut {
    double H[9];
    int inliers;          // -1: no model
    int best;
};

}  // namespace dmsgm

struct dmsgm_homog_ctx {
    int W, H, device;
    dmsgm_homog_params p;
    int gw, gh, cell;                 // spacing cells (`cell` pixels; none when gw == 0)
    int cand_ctas;                    // CTAs of the candidate passes over the listed maxima
    unsigned long long* lmax;         // W x H: the listed local maxima (score key, index)
    uint32_t* zeroed;                 // one memset per call: ctrl, hist_hi, hist_lo
    uint32_t* ctrl;
    uint32_t* hist_hi;                // 65536
    uint32_t* hist_lo;                // 65536
    unsigned long long* keys;         // kHoSortCap: above-cut keys, then tie keys
    unsigned long long* sel;          // kHoKmax sorted keys
    uint32_t* rank;                   // kHoRankSplit x kHoSortCap partial ranks
    int* corners;                     // kHoMaxPts x 2
    float* cscore;                    // kHoMaxPts
    float2* pts_in;                   // kHoMaxPts
    float2* pts_out;
    uint8_t* status;
    double* src;                      // kHoMaxPts x 2
    double* dst;
    float4* pf;                       // kHoMaxPts: the pairs rounded to FP32 (the counts' pre-test)
    uint8_t* inl;                     // kHoMaxPts
    double* hyp;                      // ransac_iters x 9
    float* hypf;                      // ransac_iters x 10: FP32 copies and their range flag
    int* hcount;                      // ransac_iters
    double* fitpart;                  // kHoFitCtas x kHoFitTerms refit partial sums
    dmsgm::HoRansacOut* rout;
    uint8_t* pyr[2][dmsgm::kHoMaxLevels + 1];   // levels 1.. of the two images
    int lw[dmsgm::kHoMaxLevels + 1], lh[dmsgm::kHoMaxLevels + 1];
    void* host;                       // pinned staging of the results
    const uint8_t** fdev;             // device slot: the frame pair the kernels read
    const uint8_t** fhost;            // its pinned staging
    cudaGraphExec_t graph;            // the whole estimate (corners, tracking, RANSAC)
};

namespace dmsgm {

// The RANSAC over the tracked pairs (or over pairs already in h->src/dst with
// the count in ctrl[kCtrlNPairs]); results in h->rout.  pairs_from_track:
// build the pairs from h->pts_in/pts_out/status first.
int ho_launch_ransac(dmsgm_homog_ctx* h, bool pairs_from_track, cudaStream_t s);

}  // namespace dmsgm

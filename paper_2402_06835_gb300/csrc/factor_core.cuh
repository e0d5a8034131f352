// Factor of one or several light curves (segments) packed back to back.
// Shared by nu_gp_factor (one segment) and nu_batch_search (many).
#pragma once

#include <vector>

#include "factor_ops.cuh"
#include "nu_internal.cuh"

namespace nu {

// Chunk length and group size of the scans, chosen per factor by the number
// of samples.  The scan's sequential depth is about 2 B per-sample steps plus
// 2 G element operations per tree level; the GPU runs 608 sub-partitions x
// 32 lanes of such chains at once.  While the level-0 chunks fit in about two
// such waves, short chunks and small groups shorten the chain (on a 19 440-
// sample curve B = 4, G = 4 with warp-level trees); a large batch has chunks
// to spare, and long chunks keep the tree's extra work and its element memory
// small.
constexpr int SCAN_TOP = 16;
inline int scan_chunk_len(int64_t n_total) {
    int B = 4;
    while (B < 32 && n_total > (int64_t)B * 2 * 608 * 32) B *= 2;
    return B;
}
inline int scan_group(int B) { return B <= 8 ? 4 : 8; }

// Device arrays of a factor, all indexed by packed sample.
struct FactorBuffers {
    const double* t;
    double* F;          // [n][nb][4]
    double* kg;         // [n][J]
    double* invD;       // [n]
    double* G;          // [n][J(J+1)/2]
    double* z0;         // [n]
    double* Zt;         // [n][k]
    double* work;       // [n][k+1] forward innovations
    double* scal;       // per segment [4]: logdet, lnL_null, chi2, -
    long long* dstat;   // per segment [2]: status, first bad local sample
    float* F32;         // FP32 copies (null: not made)
    float* kg32;
    float* invD32;
    float* G32;
    float* z032;
    float* Zt32;
};

// Host plan: segment table, scan structure, workspace layout.
struct FactorPlan {
    int nb;
    int k;
    int n_seg;
    int64_t n_total;
    int64_t n_chunks;
    int B;                           // chunk length of the scans
    int G;                           // group size of the scan tree
    ScanShape shape;
    std::vector<int64_t> index;      // scan index arrays
    std::vector<int> chunk_seg;      // segment of each chunk
    std::vector<int64_t> s_off;      // [n_seg + 1]
    std::vector<SegInfo> segs;
    std::vector<Blocks> blocks;
    // workspace layout (bytes)
    size_t off_scan, off_scan_fu, off_partial, off_idx, off_chunk_seg, off_segs, off_blocks, off_s_off,
        off_cross, off_wR, off_Dpiv, off_U, off_chi, off_logD, bytes;
};

// Build the plan for segments of n_g samples with the given covariance blocks
// (all segments must have the same number of blocks).
FactorPlan plan_factor(const int64_t* n_per_seg, const Blocks* blocks, int n_seg, int k);

// Copy the plan's tables into the workspace (synchronises the stream).
nu_status upload_factor_plan(const FactorPlan& p, char* ws, cudaStream_t st);

// Enqueue every kernel of the factor (no host synchronisation, no
// allocation): safe to capture in a CUDA graph.  X may be null (then the
// columns are [1, t] up to k), with leading dimension ldx otherwise.
// When `side` is a stream other than st, the future-information scan (which
// needs only the pivots and gains) runs on it concurrently with the forward
// and backward solves, forked from and joined back into st by events; the
// caller must not use `side` concurrently for anything else.
nu_status launch_factor(const FactorPlan& p, const FactorBuffers& b, char* ws,
                        const double* diag_var, const double* X, int64_t ldx,
                        const double* y, cudaStream_t st, cudaStream_t side, int* launched);

// A non-blocking stream private to the calling thread and current device,
// created on first use and kept for the thread's lifetime (null on failure).
cudaStream_t thread_side_stream();

}  // namespace nu

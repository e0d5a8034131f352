// Fold (periodic search) pieces shared by the single-curve and batch paths.
#pragma once

#include <vector>

#include "nu_internal.cuh"

namespace nu {

// Node record of the single-event grid: depth, sigma = sqrt(var) (NaN when
// any of depth/var/gain is not finite or var <= 0), gain, and ig = 1/(gap to
// the next epoch) (NaN when there is no next epoch or the gap exceeds the
// limit).  Interpolating with a NaN anywhere yields a NaN sigma, which is how
// an epoch is dropped.
template <typename T> struct __align__(4 * sizeof(T)) Node4 {
    T d, s, l, ig;
};

// Node record of the exact path: the Node4 fields plus the differences to the
// next epoch's depth, sigma and gain (NaN when the next epoch is missing or
// invalid), so that an event is one record load and three FMAs.
template <typename T> struct __align__(8 * sizeof(T)) Node8 {
    T d, s, l, ig, dd, ds, dl, pad;
};

// Screening record of the FP64 path, one per (duration, epoch i): the FP32
// values and slopes of the interval [t0_i, t0_{i+1}], wsc = 2^-22 dt/gap (the
// weight per unit of the 2^-22-slot position difference), and flags = 1 when
// the interval is outside the screen's error model (epochs closer than dt/4,
// end sigmas more than a factor 3 apart, or values whose FP32 sums could
// overflow): a cell with an event there is evaluated exactly.  s is NaN on an
// invalid interval.
struct __align__(32) ScreenRec {
    float d, s, l, dd, ds, dl, wsc;
    unsigned flags;
};

// Byte layout of the exact path's per-(duration, epoch) arrays for n epochs:
// Node8 records, then (FP64 only) screening records and pairs of fixed-point
// epoch positions.
struct ExactLayout {
    size_t off_screen, off_vpos, total;
};
inline ExactLayout exact_layout(int64_t n, int n_D, bool fp64) {
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    ExactLayout L;
    const size_t node = al((size_t)n * n_D * 8 * (fp64 ? 8 : 4));
    L.off_screen = node;
    L.off_vpos = node + (fp64 ? al((size_t)n * n_D * sizeof(ScreenRec)) : 0);
    L.total = L.off_vpos + (fp64 ? al((size_t)n * 16) : 0);
    return L;
}

// Geometry of one light curve of a batch fold.
struct FoldSeg {
    int64_t s_off;      // first epoch (= first sample) in the packed arrays
    int64_t n_t0;
    double t_ref, t_last;
    int64_t n_bucket, bucket_off;
    int64_t n_slots, rec_off;
    int use_slots;
    int screen;         // FP64 path: FP32 screening allowed for this curve
    int64_t srec_off;   // FP64 path: first slot-indexed screening record
    int64_t gain_off;   // first entry of the curve's grouped gain table (either path)
    unsigned long long ulast;   // slot path: the last epoch's position, 24.40 slots
};

// Gain tables are grouped by duration: the gains of W consecutive durations
// at one slot are adjacent, so that one vector load serves W cells of one
// phase (their epochs are the same).  Per curve the table is [n_D / W groups
// (rounded up)][n_slots][W] floats; columns past n_D hold 0.
#ifndef NU_GAIN_W_MAX
#define NU_GAIN_W_MAX 4
#endif
__host__ __device__ inline int gain_width(int n_D) {
    return n_D >= 4 && NU_GAIN_W_MAX >= 4 ? 4 : (n_D >= 2 && NU_GAIN_W_MAX >= 2 ? 2 : 1);
}
__host__ __device__ inline int gain_cols(int n_D) {
    const int W = gain_width(n_D);
    return (n_D + W - 1) / W * W;
}

struct PeriodConst;
size_t period_const_bytes();

// Device scratch of the batch fold.
struct FoldScratch {
    void* nodes;            // exact-path records (exact_layout of all samples)
    int* bucket;            // bucket tables
    Node4<float>* rec;      // mixed slot records
    float* lgm;             // mixed: the larger gain of each slot and the next (grouped)
    ScreenRec* srec;        // FP64 slot-indexed screening records
    int* slot_of;           // FP64: slot of every sample
    unsigned* reg;          // FP64: two words per curve (zeroed by the prep)
    float* lint;            // FP64: largest gain of the interval at each slot
    float* lm3;             //       and its maximum over the slot and both
                            //       neighbours (grouped)
    unsigned long long* peak;  // FP64: per curve, the key of its largest gain
    PeriodConst* ptab;      // FP64: per period, its curve-independent constants
};

// Host side of the batch fold: per-curve layout and launches.
struct FoldBatch {
    std::vector<FoldSeg> segs;
    int64_t n_bucket_total = 0, n_rec_total = 0, n_srec_total = 0;
    int64_t n_gain_total = 0;    // entries of the grouped gain tables (either path)
    bool any_slots = false, any_exact = false;
    bool slot_cascade = false;   // some curve's grid is large enough for the mixed cascade
};

void plan_fold_batch(const std::vector<int64_t>& s_off, const std::vector<double>& t_first,
                     const std::vector<double>& t_last, const std::vector<int>& irregular,
                     bool fp64, double dt, double gap_factor, int n_D, FoldBatch& fb);

// Enqueues the fold's preparation kernels; returns the first error of an
// enqueued memset (the launches are checked by the caller) and the number of
// kernels launched in *n_launched.
cudaError_t launch_fold_prep(const FoldBatch& fb, const FoldSeg* segs_dev,
                             const int64_t* s_off_dev, int n_seg, int64_t n_total, bool fp64,
                             const double* t, const void* depth, const void* var,
                             const void* gain, int n_D, double dt, double gap_factor,
                             const FoldScratch& fs, cudaStream_t st, int* n_launched);

int launch_fold_batch(const FoldBatch& fb, const FoldSeg* segs_dev, int n_seg,
                      int64_t n_total, bool fp64, const double* t, const FoldScratch& fs,
                      int n_D, double dt, double gap_factor, const double* periods,
                      int64_t n_P, unsigned long long* counter, int grid, int threads,
                      double* Q, double* T0, int* Didx, double* dep, double* sig, double* lnp,
                      cudaStream_t st);

int launch_slots_test(const double* t, const int64_t* s_off_dev, int n_seg, int64_t n_total,
                      double dt, int* irregular, cudaStream_t st);

}  // namespace nu

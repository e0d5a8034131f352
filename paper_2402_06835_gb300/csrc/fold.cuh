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

// Geometry of one light curve of a batch fold.
struct FoldSeg {
    int64_t s_off;      // first epoch (= first sample) in the packed arrays
    int64_t n_t0;
    double t_ref, t_last;
    int64_t n_bucket, bucket_off;
    int64_t n_slots, rec_off;
    int use_slots;
};

// Host side of the batch fold: per-curve layout and launches.
struct FoldBatch {
    std::vector<FoldSeg> segs;
    int64_t n_bucket_total = 0, n_rec_total = 0;
    bool any_slots = false, any_exact = false;
};

void plan_fold_batch(const std::vector<int64_t>& s_off, const std::vector<double>& t_first,
                     const std::vector<double>& t_last, const std::vector<int>& irregular,
                     bool fp64, double dt, double gap_factor, int n_D, FoldBatch& fb);

int launch_fold_prep(const FoldBatch& fb, const FoldSeg* segs_dev, const int64_t* s_off_dev,
                     int n_seg, int64_t n_total, bool fp64, const double* t, const void* depth,
                     const void* var, const void* gain, int n_D, double dt, double gap_factor,
                     void* nodes, int* bucket, Node4<float>* rec, cudaStream_t st);

int launch_fold_batch(const FoldBatch& fb, const FoldSeg* segs_dev, int n_seg, bool fp64,
                      const double* t, const void* nodes, const int* bucket,
                      const Node4<float>* rec, int n_D, double dt, double gap_factor,
                      const double* periods, int64_t n_P, unsigned long long* counter,
                      int grid, int threads, double* Q, double* T0, int* Didx, double* dep,
                      double* sig, double* lnp, cudaStream_t st);

int launch_slots_test(const double* t, const int64_t* s_off_dev, int n_seg, int64_t n_total,
                      double dt, int* irregular, cudaStream_t st);

}  // namespace nu

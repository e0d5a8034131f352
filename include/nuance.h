/*
 * nuance on GB300: C ABI of the transit-search hot path.
 *
 * Method: Garcia et al., "nuance: Efficient detection of planets transiting
 * active stars" (arXiv:2402.06835).  The library computes
 *   - the linear search of Sect. 2.2: for every trial epoch t0 and duration D,
 *     the generalised least-squares fit (Eq. ls) of a transit template that is
 *     the last column of the design matrix (Eq. linear_model), under the fixed
 *     Gaussian-process covariance Sigma, returning the depth, its variance and
 *     the log-likelihood gain of Eq. linear_search_ll over the transit-free
 *     model;
 *   - the periodic search of Sect. 2.3-2.4: the combination of those single
 *     events with Eq. result (biased estimates of Eq. sigma_delta) on a phase
 *     grid, the argmax of Eq. phi0 and the periodogram Q(P) = Delta / sigma.
 *
 * Conventions for every call:
 *   - Arrays named *_dev are DEVICE pointers owned by the caller; arrays named
 *     *_host are host pointers read during the call only.  All times,
 *     durations and periods are in days.
 *   - Work is enqueued on `stream` (a cudaStream_t passed as void*, NULL for
 *     the legacy default stream) and is asynchronous unless stated.
 *   - The return value is a nu_status; on anything but NU_OK a message is
 *     available from nu_last_error() in the calling thread.  Argument errors
 *     are detected on the host before any work is enqueued.  Errors that only
 *     the device can see (a non-positive pivot of the factor, unsorted times)
 *     are written to a status word that the next synchronising call
 *     (nu_factor_info, nu_batch_search) reads back.  No kernel of this library
 *     waits on a flag set by another kernel or another device: persistent
 *     kernels take work from an atomic counter and never spin.
 *   - The library keeps no global state except the thread-local error
 *     message; a nu_factor may be used from any thread but not concurrently.
 */
#ifndef NUANCE_GB300_H
#define NUANCE_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NU_OK = 0,
    NU_EINVAL = 1,    /* bad argument: shape, order, range, null pointer       */
    NU_ENOTPD = 2,    /* covariance not positive definite (pivot <= 0 or NaN)  */
    NU_ECUDA = 3,     /* a CUDA runtime call failed                            */
    NU_ENOMEM = 4,    /* device allocation failed                              */
    NU_ETIMEOUT = 5   /* reserved for a bounded device wait; no call of this
                         version returns it (no kernel waits on a flag)         */
} nu_status;

typedef enum {
    NU_FP64 = 0,      /* every step in IEEE binary64                           */
    NU_MIXED = 1      /* FP64 factor; FP32 window recursion, window sums and
                         GLS with compensated accumulation; FP32 fold with
                         FP64 epoch arithmetic                                  */
} nu_precision;

typedef enum {
    NU_BOX = 0,       /* -1 for t0 - D/2 <= t < t0 + D/2, else 0 (Sect. 2.1:
                         "normalized box-shaped transit")                        */
    NU_TRAPEZOID = 1, /* total width D, linear ingress and egress of width
                         ingress_frac*D, flat bottom -1; not in the paper (its
                         Sect. 4.4 names other base templates as a prospect).
                         params[0] = ingress_frac, 0 < ingress_frac <= 0.5      */
    NU_LIMB_QUAD = 2  /* limb-darkened transit as base model (Sect. 4.4's
                         prospect): small-planet limit of a central transit
                         under the quadratic law, -I(mu) on the window with
                         r = 2 (t - t0) / D, mu = sqrt(1 - r^2), x = 1 - mu,
                         I = 1 - u1 x - u2 x^2 (depth = the central dip).
                         params[0] = u1, params[1] = u2, any finite values
                         (physical laws have u1 + u2 <= 1)                       */
} nu_template;
/* Every template is zero outside its window t0 - D/2 <= t < t0 + D/2; the
 * `tmpl_params` argument of the calls below is a host array read during the
 * call (NULL allowed for NU_BOX). */

/* Covariance terms.  kind and parameters:
 *   NU_TERM_SHO      p = {sigma, omega, Q}: Appendix A, k(0) = sigma^2;
 *                    all three damping regimes (Q <, =, > 1/2) are accepted.
 *   NU_TERM_EXP      p = {sigma, ell}: sigma^2 exp(-|tau|/ell), Sect. 3.2.
 *   NU_TERM_ROTATION p = {sigma, period, Q0, dQ, f}: the two SHO terms of
 *                    Sect. 3.2 (Q1 = 1/2+Q0+dQ, omega1 = 4 pi Q1/(P sqrt(4Q1^2-1)),
 *                    S1 = sigma^2/((1+f) omega1 Q1); Q2 = 1/2+Q0, omega2 = 2 omega1,
 *                    S2 = f sigma^2/((1+f) omega2 Q2)), with sigma_j^2 = S_j omega_j Q_j.
 * The total state dimension (2 per SHO, 2 per EXP, 4 per ROTATION) must be
 * at most 8. */
enum { NU_TERM_SHO = 0, NU_TERM_EXP = 1, NU_TERM_ROTATION = 2 };
typedef struct {
    int kind;
    double p[5];
} nu_term;

typedef struct nu_factor nu_factor;   /* opaque; owns library device memory */

/* Factor the covariance and prepare the per-sample vectors of the search.
 *
 * Defines Sigma = diag(diag_var) + sum of terms (Sect. 2.1, App. A, Sect. 3.2)
 * on the sample times t, factors it as L diag(D) L^T (the celerite-type
 * quasiseparable factorisation the paper uses through tinygp, here in its
 * state-space form), and computes, for the transit-free model y ~ N(X w, Sigma):
 * Sigma^-1 X after Sigma-orthonormalising the columns of X, the null fit and
 * its residual z0 = Sigma^-1 (y - X w_null), ln|Sigma| and the null
 * log-likelihood of Eq. linear_search_ll.
 *
 *   t_dev         (n) strictly increasing sample times (checked on device)
 *   diag_var_dev  (n) white-noise variance per sample, > 0 recommended
 *   terms_host    (n_terms) covariance terms, see nu_term
 *   X_dev         column-major n x k design matrix (column c at X_dev + c*n);
 *                 may be NULL when k == 0.  0 <= k <= 4.
 *   y_dev         (n) observed flux
 *   out           receives a new factor; release it with nu_factor_free.
 * The input arrays are copied; they may be freed once the call returns
 * (after the stream has reached this point).  Asynchronous: a non-positive
 * pivot or unsorted t is reported by nu_factor_info.
 * Errors: NU_EINVAL (n < 2, k outside 0..4, bad term, state dimension > 8,
 * null pointer), NU_ENOMEM, NU_ECUDA. */
nu_status nu_gp_factor(const double* t_dev, const double* diag_var_dev, int64_t n,
                       const nu_term* terms_host, int n_terms,
                       const double* X_dev, int k, const double* y_dev,
                       void* stream, nu_factor** out);

/* Synchronise with the factor's stream and read its scalars: ln|Sigma|, the
 * null log-likelihood (Eq. linear_search_ll without the transit column) and,
 * when the factor failed, the first sample index at fault (else -1).
 * Any pointer may be NULL.  Returns the factor's device status
 * (NU_OK, NU_ENOTPD for a pivot <= 0 or NaN, NU_EINVAL for unsorted t). */
nu_status nu_factor_info(const nu_factor* f, double* logdet, double* lnL_null,
                         int64_t* first_bad_index);

/* Number of samples and columns of X of a factor (host-side, no sync). */
int64_t nu_factor_size(const nu_factor* f, int* k);

/* Release a factor.  Its device memory is returned stream-ordered on the
 * factor's stream (no host synchronisation): work already enqueued on that
 * stream completes first.  Work that used the factor on another stream must
 * be complete (or ordered before this call's point on the factor's stream)
 * before the call. */
void nu_factor_free(nu_factor* f);

/* Linear search (Sect. 2.2) on the grid t0s x Ds.
 *
 * For every duration index j and epoch index i the template m(t0_i, D_j) is
 * appended to X and Eq. ls is solved: depth = last weight, var = last diagonal
 * entry of (X'^T Sigma^-1 X')^-1, dlnl = ln L(t0, D) - ln L_null = depth^2 /
 * (2 var) (Eq. linear_search_ll).  Outputs are [n_D][n_t0] row-major
 * (duration-major), FP64 when prec == NU_FP64 and FP32 when NU_MIXED.  A
 * window with no sample, or whose template lies in the span of X, gives NaN
 * in all three outputs.
 *
 *   f             factor from nu_gp_factor (its samples define the windows)
 *   t0s_dev       (n_t0) trial epochs, any order
 *   Ds_host       (n_D) trial durations, > 0
 *   tmpl, tmpl_params  template and its parameters (see nu_template)
 *   depth_dev, var_dev, dlnl_dev  outputs as above (double* or float*)
 * Errors: NU_EINVAL (null pointer, n_t0 < 1, n_D < 1, D <= 0, bad template or
 * template parameters), NU_ENOMEM, NU_ECUDA. */
nu_status nu_linear_search(const nu_factor* f, const double* t0s_dev, int64_t n_t0,
                           const double* Ds_host, int n_D, nu_template tmpl,
                           const double* tmpl_params, nu_precision prec, void* stream,
                           void* depth_dev, void* var_dev, void* dlnl_dev);

/* Periodic search (Sect. 2.3-2.4) over trial periods.
 *
 * Inputs are the linear-search products on the grid t0s x Ds (layout and
 * element type as produced by nu_linear_search with the same prec).  t0s must
 * be sorted ascending.  For each period P: phases phi_j = j/n_phi with
 * n_phi = ceil(P/phase_step); epochs T = t0s[0] + (phi_j + k) P for k >= 0
 * and T <= t0s[n_t0-1]; each single event is linearly interpolated in time
 * between the bracketing grid epochs (largest i with t0_i <= T, and i+1) from
 * (depth, sqrt(var), dlnl), and dropped if it has no right neighbour, if the
 * two epochs are more than gap_factor*phase_step apart, or if a node is
 * non-finite.  The events of a (phase, duration) cell are combined with
 * Eq. result using the biased estimates of Eq. sigma_delta and the gains as
 * ln L_k; the cell maximising ln P (first in duration-major, then phase order)
 * is Eq. phi0's argmax.
 *
 *   phase_step    > 0, or 0 for the median spacing of t0s (computed on the
 *                 host from a copy of t0s; this synchronises the stream)
 *   gap_factor    > 0 (1.5 is the default reading)
 *   outputs (n_P each): Q = Delta/sigma, T0 = t0s[0] + phi0*P, D_idx (int32,
 *   -1 when no cell has an epoch), depth Delta, sigma, lnP.  A period with no
 *   valid cell gets Q = 0, lnP = -inf and NaN for the others; a period that
 *   is not finite and > 0, or that gives more than 1e9 epochs or phases,
 *   gets NaN everywhere and D_idx = -1 (and costs no work).
 * Errors: NU_EINVAL, NU_ENOMEM, NU_ECUDA. */
nu_status nu_periodic_search(const double* t0s_dev, int64_t n_t0,
                             const double* Ds_host, int n_D,
                             const void* depth_dev, const void* var_dev,
                             const void* dlnl_dev, nu_precision prec,
                             const double* periods_dev, int64_t n_P,
                             double phase_step, double gap_factor, void* stream,
                             double* Q_dev, double* T0_dev, int32_t* D_idx_dev,
                             double* depth_out_dev, double* sigma_out_dev,
                             double* lnP_dev);

/* Masking of a found transit for the next search of a multi-planet system
 * (Sect. 2.5 and the TOI-540 comparison, Sect. 3.3: after a periodic search,
 * the linear-search products of the trial epochs in windows of width 2 D
 * centred on the detected transits are masked and the periodic search is
 * run again on the same grid).
 *
 * Marks every grid entry (all durations) whose epoch t0_i lies within
 * half_width of a transit of the candidate (P, T0) as invalid, in place:
 * with n = rint((t0_i - T0) / P), the entry is masked when
 * |t0_i - (T0 + n P)| < half_width (each operation rounded once, in FP64);
 * depth, var and dlnl of a masked entry become NaN, which the periodic
 * search treats as a missing epoch.  half_width = D of the candidate gives
 * the paper's window of width 2 D.
 *   depth/var/dlnl  [n_D][n_t0], element type by prec (as nu_linear_search)
 * Enqueued on `stream`; no synchronisation.  Errors: NU_EINVAL (null array,
 * n_t0 < 1, n_D < 1, P not finite and > 0, T0 or half_width not finite),
 * NU_ECUDA. */
nu_status nu_mask_transits(const double* t0s_dev, int64_t n_t0, int n_D, void* depth_dev,
                           void* var_dev, void* dlnl_dev, nu_precision prec, double P,
                           double T0, double half_width, void* stream);

/* Rotation-alias period exclusion (Sect. 3, the comparison set-up).
 *
 * Removes from a period grid the periods near whole multiples of the stellar
 * rotation period P_star: with dP = P / P_star, a period is dropped when
 * |dP - ceil(dP)| < tol (the printed criterion, tol = 0.02 in the paper), or,
 * with symmetric != 0, when |dP - rint(dP)| < tol (the wording "less than 2 %
 * from an integer", which also drops periods just above a multiple).  Each
 * operation is rounded once in FP64.  Periods that are not finite are kept.
 *   periods_dev  (n_P) input grid
 *   kept_dev     (n_P capacity) receives the kept periods in input order;
 *                must not overlap periods_dev
 *   n_kept_dev   one int64 in device memory: the number of kept periods
 * Enqueued on `stream`; no synchronisation.
 * Errors: NU_EINVAL (null pointer, n_P < 1, P_star not finite and > 0, tol
 * not finite and >= 0, kept_dev == periods_dev), NU_ECUDA. */
nu_status nu_rotation_alias_filter(const double* periods_dev, int64_t n_P, double P_star,
                                   double tol, int symmetric, double* kept_dev,
                                   int64_t* n_kept_dev, void* stream);

/* Exact periodic-template fit of candidates (Sect. 2.4 read as one fit).
 *
 * Sect. 2.4 defines Q(P) as the SNR of a periodic transit of period P, epoch
 * T0 and duration D.  nu_periodic_search computes it from the single events
 * with Eq. result, which treats the transits as independent (Sect. 2.3).
 * This call solves Eq. ls once per candidate with the design matrix
 * X' = [X, m_P] at the factor's full covariance, where m_P(t) is the sum over
 * all integers n of the single template (tmpl) centred at T0 + n*P (the
 * product rounded, then the sum, in FP64; windows half-open as in
 * nu_linear_search).  depth = last weight, var = last diagonal entry of
 * (X'^T Sigma^-1 X')^-1, dlnl = depth^2 / (2 var) (Eq. linear_search_ll),
 * snr = depth / sqrt(var).  The difference between snr and the periodic
 * search's Q at the same (P, T0, D) is the cost of the independence
 * approximation.
 *
 *   f             factor from nu_gp_factor
 *   P_dev, T0_dev (n_cand) periods and epochs, e.g. the trial periods and the
 *                 T0 output of nu_periodic_search
 *   D_idx_dev     (n_cand) int32 index into Ds_host, e.g. its D_idx output
 *   Ds_host       (n_D) durations, finite and > 0
 *   tmpl, tmpl_params  as in nu_linear_search
 *   depth_dev, var_dev, dlnl_dev, snr_dev  (n_cand) FP64 outputs
 * A candidate with P or T0 not finite, D_idx outside [0, n_D), 2 D > P
 * (windows would overlap), no sample in any window, or a template in the
 * span of X gets NaN in all four outputs.  Always FP64.  One warp per
 * candidate, its lanes over 32 segments of the samples; gaps between windows
 * advance in blocks of 32 samples.  Enqueued on `stream`; no synchronisation.
 * Errors: NU_EINVAL (null pointer, n_cand < 1, n_D < 1, a duration not finite
 * and > 0, bad template or template parameters), NU_ENOMEM, NU_ECUDA. */
nu_status nu_periodic_refine(const nu_factor* f, const double* P_dev, const double* T0_dev,
                             const int* D_idx_dev, int64_t n_cand, const double* Ds_host,
                             int n_D, nu_template tmpl, const double* tmpl_params, void* stream,
                             double* depth_dev, double* var_dev, double* dlnl_dev,
                             double* snr_dev);

/* Periodic search without device allocation (no counterpart in the paper).
 *
 * Same inputs, outputs and results as nu_periodic_search, for callers that
 * cannot allocate device memory while they run: a runtime that reserves all
 * of its device memory up front, a plugin whose host framework forbids
 * allocation inside a step, or a process already at its memory limit where a
 * mid-run allocation could fail.  The scratch (packed epoch records, lookup
 * tables) lives in a fixed array of NU_NOALLOC_SCRATCH_LIMIT bytes inside the
 * library, which every GPU that loads the library holds until the process
 * exits; grids that need more return NU_EINVAL (nu_periodic_search handles
 * them).  This call makes no cudaMalloc/cudaFree or other allocating call.
 *   - phase_step must be > 0 (the median-spacing default would need a host
 *     buffer).
 *   - The array of the device that `stream` belongs to is used; that device
 *     must be the current device and hold t0s_dev, else NU_EINVAL.
 *   - The first call on a device looks up the array's device address with
 *     that device current and keeps it for the process; make that first call
 *     before any stream capture on the device.  After cudaDeviceReset the kept
 *     address is stale: do not call this function again in that process.
 *   - Every call copies the first and last epoch to the host and therefore
 *     synchronises `stream`; the mixed-precision path reads one more flag
 *     back in the same way.
 *   - Every call on a device shares the one array, which keeps the previous
 *     call's contents; the call clears what must start at zero.  Calls whose
 *     work overlaps on the GPU (different streams, threads or processes using
 *     the same library image) race on it: serialise them.
 * Errors: as nu_periodic_search, plus NU_EINVAL when the grid needs more
 * scratch than the limit. */
#define NU_NOALLOC_SCRATCH_LIMIT (32ull << 20)
nu_status nu_periodic_search_noalloc(const double* t0s_dev, int64_t n_t0,
                                     const double* Ds_host, int n_D,
                                     const void* depth_dev, const void* var_dev,
                                     const void* dlnl_dev, nu_precision prec,
                                     const double* periods_dev, int64_t n_P,
                                     double phase_step, double gap_factor, void* stream,
                                     double* Q_dev, double* T0_dev, int32_t* D_idx_dev,
                                     double* depth_out_dev, double* sigma_out_dev,
                                     double* lnP_dev);

/* Scratch limit of nu_periodic_search_noalloc in bytes. */
uint64_t nu_periodic_search_noalloc_limit(void);

/* Batched survey search: factor, linear search (box template, t0s = the
 * sample times of each curve) and periodic search for n_lc light curves of
 * uneven length packed back to back, launched as one graph on `stream`.
 *
 *   offsets_host  (n_lc+1) start of each curve in the packed arrays
 *   t_dev, y_dev, diag_var_dev  packed samples
 *   terms_host, n_terms_host    terms of curve c are terms_host[tb_c ...],
 *                 tb_c = sum of n_terms_host[0..c-1]
 *   k             1 or 2: X = [1] or [1, t] per curve
 *   Ds_host (n_D), periods_dev (n_P): shared grids
 *   phase_step    > 0 (shared by all curves), or 0 for the median sample
 *                 spacing of the first curve (computed on the host from a
 *                 copy of that curve's times)
 *   outputs, [n_lc][n_P] each: Q, T0, D_idx, depth, sigma, lnP (as in
 *   nu_periodic_search); status_host (n_lc) per-curve factor status.
 * Synchronises the stream before returning (the statuses are host data).
 * The launch shapes of the fold and of the linear search are tuned the first
 * time a configuration (state size, k, precision, n_D) is seen in the process
 * and cached; the executable graph of a configuration (the same and n_lc,
 * total samples, n_P) is kept and updated with the next call's parameters.
 * Errors: NU_EINVAL, NU_ENOMEM, NU_ECUDA. */
nu_status nu_batch_search(int n_lc, const int64_t* offsets_host,
                          const double* t_dev, const double* y_dev,
                          const double* diag_var_dev, const nu_term* terms_host,
                          const int* n_terms_host, int k,
                          const double* Ds_host, int n_D,
                          const double* periods_dev, int64_t n_P,
                          double phase_step, nu_precision prec, void* stream,
                          double* Q_dev, double* T0_dev, int32_t* D_idx_dev,
                          double* depth_out_dev, double* sigma_out_dev,
                          double* lnP_dev, int* status_host);

/* Message of the last failed call in this thread ("" if none). */
const char* nu_last_error(void);

/* Number of CUDA kernels this library has launched since it was loaded
 * (all threads, all devices); for launch accounting in benchmarks. */
uint64_t nu_launch_count(void);

/* Library version string. */
const char* nu_version(void);

#ifdef __cplusplus
}
#endif

#endif /* NUANCE_GB300_H */

// Internal declarations shared by the CUDA translation units of the library.
//
// The covariance of Sect. 2.1 (white noise on the diagonal plus the SHO /
// exponential terms of Appendix A and Sect. 3.2) is handled in its
// state-space form: every term is a 2-dimensional block of a linear
// Gaussian state x_n with transition F_n = exp(A_c (t_n - t_{n-1})),
// stationary covariance P_inf and observation h (first component of every
// block).  The Kalman innovations of that model are exactly the unit lower
// triangular factor Sigma = L diag(D) L^T that the celerite-type
// quasiseparable algorithms of the paper's tinygp back end compute (the
// pivots D_n and the forward / backward solves are the same numbers), so
// every Sigma^-1 product of Eq. ls is a pair of O(N J^2) recursions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include "../../include/nuance.h"

#define NU_MAX_BLOCKS 4          // state dimension J = 2 * blocks <= 8
#define NU_MAX_K 4               // columns of the design matrix

namespace nu {

// A 2x2 state block of one covariance term.
//  type 0: SHO with zero-lag variance sigma2, angular frequency omega,
//          quality Q (all damping regimes); coordinates (f, f'/omega) so
//          that P_inf = sigma2 * I.
//  type 1: exponential sigma2 exp(-tau/ell); first component only,
//          P_inf = diag(sigma2, 0).
struct BlockParams {
    int type;
    double sigma2;
    double omega;
    double Q;
    double ell;
};

struct Blocks {
    int nb;
    BlockParams b[NU_MAX_BLOCKS];
};

// Keep freed stream-ordered allocations in the current device's default
// memory pool (instead of returning them at every synchronisation), so that
// repeated calls reuse memory without new device allocations.
void pool_keep_memory();

// Number of kernels this library has launched (nu_launch_count).
void count_launches(int k);

// Error reporting (thread-local message, see nu_last_error).
void set_error(const char* fmt, ...);
nu_status fail(nu_status s, const char* fmt, ...);
nu_status cuda_fail(cudaError_t e, const char* where);

// Expand ABI terms into 2x2 blocks; validates parameters.
nu_status expand_terms(const nu_term* terms, int n_terms, Blocks* out);

inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Per-sample factor arrays as read by the linear search (FP64 or FP32 copies).
template <typename T> struct FactorView {
    const T* F;
    const T* kg;
    const T* invD;
    const T* G;
    const T* z0;
    const T* Zt;
};

// Launch shape of the linear search's window-start kernel: tlo window
// starts per block (32, 64, 128 or 256), ch samples of the recursion per
// staged chunk of factor rows.
struct WindowShape {
    int tlo, ch;
};
#ifndef NU_WIN_TLO_SMALL
#define NU_WIN_TLO_SMALL 32
#endif
#ifndef NU_WIN_CH
#define NU_WIN_CH 64
#endif
// Default shape: small curves take NU_WIN_TLO_SMALL starts per block so that
// their few warps spread over every SM sub-partition (the FP64 recursion
// issues one warp instruction per 64 cycles per sub-partition).
inline WindowShape default_window_shape(int64_t n_total) {
    return WindowShape{n_total < 152 * 128 * 2 ? NU_WIN_TLO_SMALL : 128, NU_WIN_CH};
}
// Ints of device scratch the window-start plan needs per curve (four
// window variants per duration).
inline int window_plan_ints(int n_D) { return 2 + 20 * n_D; }

// Linear search of packed light curves (batch path); no allocation, no sync.
// plan: window_plan_ints(n_D) ints of device scratch per curve for the
// window-start kernel, or nullptr for one recursion per template.  Returns
// the number of kernels launched.
int launch_window_batch(int nb, bool fp64, const double* t, int k, const void* fv,
                        const int64_t* s_off, int n_seg, int64_t n_total, const double* Ds,
                        int n_D, int* plan, const WindowShape& ws, void* d, void* v, void* l,
                        cudaStream_t st);

}  // namespace nu

// Library-owned factor of one light curve.  All arrays are device memory
// inside one allocation.  Per-sample arrays are sample-major:
//   F    [n][nb][4]  transition from sample n-1 to n (row-major 2x2 blocks)
//   kg   [n][J]      Kalman gain P_{n|n-1} h / D_n
//   invD [n]         1 / D_n
//   G    [n][J(J+1)/2] information about the future state: the quadratic
//                    form that gives sum_{m >= n} e_m^2 / D_m for a forward
//                    solve whose input is zero from n on (packed upper)
//   z0   [n]         Sigma^-1 (y - X w_null)
//   Zt   [n][k]      Sigma^-1 X R^-1 with X^T Sigma^-1 X = R^T R
// and FP32 copies of F, kg, invD, G, z0, Zt for the mixed-precision search.
struct nu_factor {
    int64_t n;
    int nb;
    int k;
    cudaStream_t stream;
    cudaEvent_t ready;   // recorded on `stream` to order other streams after the factor
    nu::Blocks blocks;
    void* mem;
    size_t mem_bytes;
    double* t;
    double* F;
    double* kg;
    double* invD;
    double* G;
    double* z0;
    double* Zt;
    double* work;        // [n][k+1] forward innovations of X columns and y
    double* scal;        // [0] logdet [1] lnL_null [2] chi2_null
    long long* dstat;    // [0] status [1] first bad index
    float* F32;
    float* kg32;
    float* invD32;
    float* G32;
    float* z032;
    float* Zt32;
};

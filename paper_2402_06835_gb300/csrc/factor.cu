// nu_gp_factor: the quasiseparable factor of Sigma and the precomputed vectors
// of the linear search (Sect. 2.2, Eq. ls, Eq. linear_search_ll).
//
// Sigma = diag(diag_var) + sum of terms (Sect. 2.1, App. A, Sect. 3.2) is
// factored as L diag(D) L^T through the Kalman recursion of its state-space
// form (see ss.cuh).  With M_n = P_inf - P_{n|n-1}:
//   D_n  = h^T P_inf h + diag_var_n - h^T M_n h
//   kg_n = (P_inf - M_n) h / D_n
//   M_{n+1} = F_{n+1} (M_n + D_n kg_n kg_n^T) F_{n+1}^T,  M_0 = 0
// Forward solve e = L^-1 x:  e_n = x_n - h^T s_n,  s_{n+1} = F_{n+1}(s_n + kg_n e_n)
// Backward solve v = L^-T u: v_n = u_n - kg_n^T g_n, g_{n-1} = F_n^T (h v_n + g_n)
// Future information: G_n = h h^T / D_n + A_{n+1}^T G_{n+1} A_{n+1},
//   A_{n+1} = F_{n+1} (I - kg_n h^T), so that a forward solve whose input is
//   zero from sample n on contributes s_n^T G_n s_n to sum e^2 / D.
// The null model (X alone) is solved through these: X^T Sigma^-1 X and
// X^T Sigma^-1 y are dot products of forward innovations weighted by 1/D.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "factor_ops.cuh"
#include "nu_internal.cuh"
#include "ss.cuh"

namespace nu {

enum { ST_OK = 0, ST_EINVAL = 1, ST_ENOTPD = 2 };

__device__ inline void flag_bad(long long* dstat, int code, long long idx) {
    // keep the smallest failing index; the first code that claims it wins
    unsigned long long old = atomicMin((unsigned long long*)&dstat[1],
                                       (unsigned long long)idx);
    if ((long long)old > idx) atomicExch((unsigned long long*)&dstat[0],
                                         (unsigned long long)code);
}

// ---------------------------------------------------------------- transitions
template <int NB>
__global__ void k_transitions(const double* __restrict__ t, int64_t n, Blocks bl,
                              double* __restrict__ F, long long* dstat) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double* Fi = F + i * NB * 4;
    if (!isfinite(t[i])) flag_bad(dstat, ST_EINVAL, i);
    if (i == 0) {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            Fi[4 * b] = 1.0; Fi[4 * b + 1] = 0.0; Fi[4 * b + 2] = 0.0; Fi[4 * b + 3] = 1.0;
        }
        return;
    }
    const double tau = t[i] - t[i - 1];
    if (!(tau > 0.0)) flag_bad(dstat, ST_EINVAL, i);
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        double f[4];
        block_transition(bl.b[b], tau, f);
        Fi[4 * b] = f[0]; Fi[4 * b + 1] = f[1]; Fi[4 * b + 2] = f[2]; Fi[4 * b + 3] = f[3];
    }
}

// -------------------------------------------------------------- null GLS
// One thread: A = X^T Sigma^-1 X = R^T R (Cholesky), w = A^-1 X^T Sigma^-1 y,
// Rinv = R^-1.  wR layout: [0..k) w, [k .. k+k*k) Rinv row-major.
__global__ void k_null_gls(int k, const double* __restrict__ cross, double* __restrict__ wR,
                           long long* dstat) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (dstat[0] != 0) return;       // the factor already failed
    const int nr = k + 1;
    double R[NU_MAX_K][NU_MAX_K] = {};
    for (int i = 0; i < k; ++i) {
        for (int j = i; j < k; ++j) {
            double s = cross[i * nr + j];
            for (int p = 0; p < i; ++p) s -= R[p][i] * R[p][j];
            if (i == j) {
                if (!(s > 0.0)) {
                    // X is rank deficient under Sigma: no null fit
                    unsigned long long old = atomicMin((unsigned long long*)&dstat[1], 0ull);
                    (void)old;
                    atomicExch((unsigned long long*)&dstat[0], (unsigned long long)ST_EINVAL);
                    return;
                }
                R[i][i] = sqrt(s);
            } else {
                R[i][j] = s / R[i][i];
            }
        }
    }
    // Rinv (upper triangular)
    double Ri[NU_MAX_K][NU_MAX_K] = {};
    for (int j = 0; j < k; ++j) {
        Ri[j][j] = 1.0 / R[j][j];
        for (int i = j - 1; i >= 0; --i) {
            double s = 0.0;
            for (int p = i + 1; p <= j; ++p) s += R[i][p] * Ri[p][j];
            Ri[i][j] = -s / R[i][i];
        }
    }
    // w = R^-1 R^-T u, u_a = cross[a][k] (X_a^T Sigma^-1 y)
    double z[NU_MAX_K];
    for (int i = 0; i < k; ++i) {          // R^T z = u
        double s = cross[i * nr + k];
        for (int p = 0; p < i; ++p) s -= R[p][i] * z[p];
        z[i] = s / R[i][i];
    }
    for (int i = k - 1; i >= 0; --i) {     // R w = z
        double s = z[i];
        for (int p = i + 1; p < k; ++p) s -= R[i][p] * wR[p];
        wR[i] = s / R[i][i];
    }
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) wR[k + i * k + j] = Ri[i][j];
}

// ------------------------------------------- right-hand sides of the solves
// Per sample: null residual innovation e0 = e_y - sum_c w_c e_c, its weighted
// square (chi-square terms), and the backward right-hand sides
// U[i][0] = e0 / D, U[i][1+a] = (sum_c e_c Rinv[c][a]) / D.
__global__ void k_rhs(int64_t n, int k, const double* __restrict__ E,
                      const double* __restrict__ invD, const double* __restrict__ wR,
                      double* __restrict__ U, double* __restrict__ chi_terms,
                      const double* __restrict__ Dpiv, double* __restrict__ logD) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int nr = k + 1;
    const double* e = E + i * nr;
    double e0 = e[k];
    for (int c = 0; c < k; ++c) e0 -= wR[c] * e[c];
    const double iD = invD[i];
    U[i * nr] = e0 * iD;
    for (int a = 0; a < k; ++a) {
        double s = 0.0;
        for (int c = 0; c < k; ++c) s += e[c] * wR[k + c * k + a];
        U[i * nr + 1 + a] = s * iD;
    }
    chi_terms[i] = e0 * e0 * iD;
    logD[i] = log(Dpiv[i]);
}

// -------------------------------------------------- deterministic reductions
// partial[b] = sum over a contiguous range; then one block sums the partials.
__global__ void k_sum_partial(const double* __restrict__ x, int64_t n, double* partial) {
    __shared__ double sh[256];
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = blockIdx.x * per;
    const int64_t hi = lo + per < n ? lo + per : n;
    double s = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) s += x[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// cross[a][b] = sum over chunks of partial[c][a][b] (one block per entry)
__global__ void k_reduce_cross(const double* __restrict__ partial, int64_t n_chunks, int nr,
                               double* __restrict__ cross) {
    __shared__ double sh[256];
    const int a = blockIdx.x / nr, b = blockIdx.x % nr;
    double s = 0.0;
    for (int64_t c = threadIdx.x; c < n_chunks; c += blockDim.x)
        s += partial[c * NRMAX * NRMAX + a * NRMAX + b];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) cross[a * nr + b] = sh[0];
}

__global__ void k_finalize(int64_t n, int nparts, const double* __restrict__ pchi,
                           const double* __restrict__ plog, double* scal) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double chi = 0.0, lg = 0.0;
    for (int b = 0; b < nparts; ++b) {
        chi += pchi[b];
        lg += plog[b];
    }
    scal[0] = lg;
    scal[2] = chi;
    scal[1] = -0.5 * chi - 0.5 * lg - 0.5 * (double)n * log(2.0 * M_PI);
}

// ------------------------------------------------------------- FP32 copies
__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

// ------------------------------------------------------------------ driver
// chunk length, group size and top-level count of the scans
constexpr int SCAN_B = 32;
constexpr int SCAN_G = 8;
constexpr int SCAN_TOP = 16;

template <int NB>
static size_t factor_workspace(int64_t n, int k) {
    const int64_t nc = (n + SCAN_B - 1) / SCAN_B;
    size_t m = plan_scan<RiccatiOp<NB>>(nc, SCAN_G, SCAN_TOP).bytes;
    m = std::max(m, plan_scan<ForwardOp<NB>>(nc, SCAN_G, SCAN_TOP).bytes);
    m = std::max(m, plan_scan<BackwardOp<NB>>(nc, SCAN_G, SCAN_TOP).bytes);
    m = std::max(m, plan_scan<FutureOp<NB>>(nc, SCAN_G, SCAN_TOP).bytes);
    (void)k;
    return m + (size_t)nc * NRMAX * NRMAX * sizeof(double) + 512;
}

template <int NB>
static nu_status run_factor(nu_factor* f, const double* diag_var, const double* X,
                            const double* y, double* scratch, char* ws) {
    constexpr int J = Dims<NB>::J;
    constexpr int JJ = Dims<NB>::JJ;
    const int64_t n = f->n;
    const int k = f->k;
    const int nr = k + 1;
    cudaStream_t st = f->stream;
    const int nblk = div_up(n, 256);
    const int64_t nc = (n + SCAN_B - 1) / SCAN_B;
    // scratch layout
    double* Dpiv = scratch;                 // n
    double* U = Dpiv + n;                   // n * nr
    double* chi_terms = U + n * nr;         // n
    double* logD = chi_terms + n;           // n
    double* cross = logD + n;               // 32
    double* wR = cross + 32;                // 32
    double* pchi = wR + 32;                 // 256
    double* plog = pchi + 256;              // 256
    int launched = 0;
    k_transitions<NB><<<nblk, 256, 0, st>>>(f->t, n, f->blocks, f->F, f->dstat);
    ++launched;
    // 1. pivots and gains
    RiccatiOp<NB> ric;
    ric.F = f->F;
    ric.dv = diag_var;
    ric.n = n;
    ric.B = SCAN_B;
    for (int b = 0; b < NB; ++b) {
        ric.pinf[2 * b] = f->blocks.b[b].sigma2;
        ric.pinf[2 * b + 1] = f->blocks.b[b].type == 0 ? f->blocks.b[b].sigma2 : 0.0;
    }
    ric.kg = f->kg;
    ric.invD = f->invD;
    ric.Dpiv = Dpiv;
    ric.dstat = f->dstat;
    launched += run_scan(ric, plan_scan<RiccatiOp<NB>>(nc, SCAN_G, SCAN_TOP), ws, st);
    // 2. forward solves of X and y, cross products
    double* partial = (double*)(ws + factor_workspace<NB>(n, k) -
                                (size_t)nc * NRMAX * NRMAX * sizeof(double) - 256);
    ForwardOp<NB> fw{f->F, f->kg, f->invD, X, y, n, k, SCAN_B, f->work, partial};
    launched += run_scan(fw, plan_scan<ForwardOp<NB>>(nc, SCAN_G, SCAN_TOP), ws, st);
    k_reduce_cross<<<nr * nr, 256, 0, st>>>(partial, nc, nr, cross);
    ++launched;
    // 3. null fit, right-hand sides, backward solves
    if (k > 0) {
        k_null_gls<<<1, 32, 0, st>>>(k, cross, wR, f->dstat);
        ++launched;
    }
    k_rhs<<<nblk, 256, 0, st>>>(n, k, f->work, f->invD, wR, U, chi_terms, Dpiv, logD);
    ++launched;
    BackwardOp<NB> bw{f->F, f->kg, U, n, nr, k, SCAN_B, nc, f->z0, f->Zt};
    launched += run_scan(bw, plan_scan<BackwardOp<NB>>(nc, SCAN_G, SCAN_TOP), ws, st);
    // 4. future information
    FutureOp<NB> fu{f->F, f->kg, f->invD, n, SCAN_B, nc, f->G};
    launched += run_scan(fu, plan_scan<FutureOp<NB>>(nc, SCAN_G, SCAN_TOP), ws, st);
    // scalars and FP32 copies
    const int nparts = 256;
    k_sum_partial<<<nparts, 256, 0, st>>>(chi_terms, n, pchi);
    k_sum_partial<<<nparts, 256, 0, st>>>(logD, n, plog);
    k_finalize<<<1, 32, 0, st>>>(n, nparts, pchi, plog, f->scal);
    launched += 3;
    const int64_t sizes[6] = {n * NB * 4, n * (int64_t)J, n, n * (int64_t)JJ, n, n * (int64_t)k};
    const double* src[6] = {f->F, f->kg, f->invD, f->G, f->z0, f->Zt};
    float* dst[6] = {f->F32, f->kg32, f->invD32, f->G32, f->z032, f->Zt32};
    for (int a = 0; a < 6; ++a)
        if (sizes[a] > 0) {
            k_to_f32<<<div_up(sizes[a], 256), 256, 0, st>>>(src[a], dst[a], sizes[a]);
            ++launched;
        }
    count_launches(launched);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "nu_gp_factor launch");
    return NU_OK;
}

static size_t workspace_bytes(int nb, int64_t n, int k) {
    switch (nb) {
        case 1: return factor_workspace<1>(n, k);
        case 2: return factor_workspace<2>(n, k);
        case 3: return factor_workspace<3>(n, k);
        default: return factor_workspace<4>(n, k);
    }
}

}  // namespace nu

using namespace nu;

extern "C" nu_status nu_gp_factor(const double* t_dev, const double* diag_var_dev,
                                  int64_t n, const nu_term* terms_host, int n_terms,
                                  const double* X_dev, int k, const double* y_dev,
                                  void* stream, nu_factor** out) {
    if (out == nullptr) return fail(NU_EINVAL, "nu_gp_factor: out is NULL");
    *out = nullptr;
    if (n < 2) return fail(NU_EINVAL, "nu_gp_factor: need n >= 2 (got %lld)", (long long)n);
    if (k < 0 || k > NU_MAX_K) return fail(NU_EINVAL, "nu_gp_factor: k must be 0..%d", NU_MAX_K);
    if (!t_dev || !diag_var_dev || !y_dev || (k > 0 && !X_dev))
        return fail(NU_EINVAL, "nu_gp_factor: null array");
    Blocks bl;
    nu_status s = expand_terms(terms_host, n_terms, &bl);
    if (s != NU_OK) return s;
    const int nb = bl.nb;
    const int J = 2 * nb, JJ = J * (J + 1) / 2;
    // sizes in 8-byte words
    const int64_t w_t = n, w_F = n * nb * 4, w_kg = n * J, w_iD = n, w_G = n * JJ,
                  w_z0 = n, w_Zt = n * k, w_work = n * (k + 1), w_scal = 8, w_stat = 2;
    const int64_t w_scratch = n + n * (k + 1) + n + n + 32 + 32 + 256 + 256;
    const int64_t w_f32 = (w_F + w_kg + w_iD + w_G + w_z0 + w_Zt + 8) / 2 + 8;
    const int64_t words = w_t + w_F + w_kg + w_iD + w_G + w_z0 + w_Zt + w_work + w_scal +
                          w_stat + w_scratch + w_f32 + 64;
    nu_factor* f = new nu_factor();
    f->n = n;
    f->nb = nb;
    f->k = k;
    f->blocks = bl;
    f->stream = (cudaStream_t)stream;
    f->mem_bytes = (size_t)words * 8;
    pool_keep_memory();
    cudaError_t e = cudaMallocAsync(&f->mem, f->mem_bytes, f->stream);
    if (e != cudaSuccess) {
        delete f;
        return cuda_fail(e, "nu_gp_factor: cudaMallocAsync");
    }
    double* p = (double*)f->mem;
    f->t = p; p += w_t;
    f->F = p; p += w_F;
    f->kg = p; p += w_kg;
    f->invD = p; p += w_iD;
    f->G = p; p += w_G;
    f->z0 = p; p += w_z0;
    f->Zt = p; p += w_Zt;
    f->work = p; p += w_work;
    f->scal = p; p += w_scal;
    f->dstat = (long long*)p; p += w_stat;
    double* scratch = p; p += w_scratch;
    float* q = (float*)p;
    f->F32 = q; q += w_F;
    f->kg32 = q; q += w_kg;
    f->invD32 = q; q += w_iD;
    f->G32 = q; q += w_G;
    f->z032 = q; q += w_z0;
    f->Zt32 = q; q += w_Zt;
    cudaStream_t st = f->stream;
    long long init[2] = {0, (long long)n};
    e = cudaMemsetAsync(f->mem, 0, f->mem_bytes, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(f->dstat, init, sizeof(init), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(f->t, t_dev, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // init is a host temporary
    if (e != cudaSuccess) {
        cudaFreeAsync(f->mem, st);
        delete f;
        return cuda_fail(e, "nu_gp_factor: copy");
    }
    const size_t ws_bytes = workspace_bytes(nb, n, k);
    char* ws = nullptr;
    e = cudaMallocAsync((void**)&ws, ws_bytes, st);
    if (e != cudaSuccess) {
        cudaFreeAsync(f->mem, st);
        delete f;
        return cuda_fail(e, "nu_gp_factor: workspace");
    }
    switch (nb) {
        case 1: s = run_factor<1>(f, diag_var_dev, X_dev, y_dev, scratch, ws); break;
        case 2: s = run_factor<2>(f, diag_var_dev, X_dev, y_dev, scratch, ws); break;
        case 3: s = run_factor<3>(f, diag_var_dev, X_dev, y_dev, scratch, ws); break;
        default: s = run_factor<4>(f, diag_var_dev, X_dev, y_dev, scratch, ws); break;
    }
    cudaFreeAsync(ws, st);
    if (s != NU_OK) {
        cudaFreeAsync(f->mem, st);
        delete f;
        return s;
    }
    *out = f;
    return NU_OK;
}

extern "C" nu_status nu_factor_info(const nu_factor* f, double* logdet, double* lnL_null,
                                    int64_t* first_bad_index) {
    if (!f) return fail(NU_EINVAL, "nu_factor_info: null factor");
    double scal[3];
    long long st[2];
    cudaError_t e = cudaMemcpyAsync(scal, f->scal, sizeof(scal), cudaMemcpyDeviceToHost,
                                    f->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(st, f->dstat, sizeof(st), cudaMemcpyDeviceToHost, f->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(f->stream);
    if (e != cudaSuccess) return cuda_fail(e, "nu_factor_info");
    if (logdet) *logdet = scal[0];
    if (lnL_null) *lnL_null = scal[1];
    const bool bad = st[0] != 0;
    if (first_bad_index) *first_bad_index = bad ? (int64_t)st[1] : -1;
    if (st[0] == ST_ENOTPD)
        return fail(NU_ENOTPD, "covariance not positive definite at sample %lld", st[1]);
    if (st[0] == ST_EINVAL)
        return fail(NU_EINVAL, "times not strictly increasing / finite, or X rank "
                               "deficient (sample %lld)", st[1]);
    return NU_OK;
}

extern "C" int64_t nu_factor_size(const nu_factor* f, int* k) {
    if (!f) return -1;
    if (k) *k = f->k;
    return f->n;
}

extern "C" void nu_factor_free(nu_factor* f) {
    if (!f) return;
    cudaFreeAsync(f->mem, f->stream);     // stream-ordered: no host sync
    delete f;
}

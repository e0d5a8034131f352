// nu_periodic_search: Sect. 2.3-2.4 on the products of the linear search.
//
// For each trial period P (one thread block), every (duration d, phase j)
// cell gathers its single events at epochs T_k = T_ref + (j/n_phi + k) P,
// linearly interpolated in time between the bracketing grid epochs, and
// combines them with Eq. result using the biased estimates of
// Eq. sigma_delta:
//   pass 1:  S_inv = sum 1/s_k^2,  S_d = sum Delta_k / s_k^2,  S_L = sum gain_k
//            sigma^2 = 1/S_inv,    Delta = sigma^2 S_d
//   pass 2:  pen = sum [ln s_k^2 - ln(sigma^2 + s_k^2) + (Delta_k - Delta)^2/(s_k^2 + sigma^2)]
//            ln P = S_L - pen / 2
// The cell with the largest ln P (first in duration-major, phase order;
// Eq. phi0) gives Q(P) = Delta / sigma.
//
// Epoch arithmetic (T, the bracket, the weight) is FP64 in both precisions
// so that which epochs take part is decided exactly as in FP64; the event
// values and sums are FP64 (NU_FP64) or FP32 with compensated sums (NU_MIXED).
#include <algorithm>
#include <climits>
#include <cmath>
#include <vector>

#include "nu_internal.cuh"

namespace nu {

struct FoldGeom {
    const double* t0s;
    int64_t n_t0;
    double t_ref;
    double t_last;
    double dt;          // phase step
    double inv_dt;
    double gap_max;     // gap_factor * dt
    const int* bucket;  // bucket[b] = #{i : t0_i <= t_ref + b*dt}
    int64_t n_bucket;
};

// largest i with t0[i] <= T (T >= t0[0]), exact
__device__ __forceinline__ int64_t bracket(const FoldGeom& g, double T) {
    int64_t b = (int64_t)floor((T - g.t_ref) * g.inv_dt);
    b = b < 0 ? 0 : (b >= g.n_bucket ? g.n_bucket - 1 : b);
    int64_t i = (int64_t)g.bucket[b] - 1;
    if (i < 0) i = 0;
    while (i + 1 < g.n_t0 && g.t0s[i + 1] <= T) ++i;
    while (i > 0 && g.t0s[i] > T) --i;
    return i;
}

__global__ void k_buckets(const double* __restrict__ t0s, int64_t n_t0, double t_ref,
                          double dt, int64_t n_bucket, int* __restrict__ bucket) {
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= n_bucket) return;
    const double edge = t_ref + (double)b * dt;
    int64_t lo = 0, hi = n_t0;          // count of t0 <= edge
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (t0s[mid] <= edge) lo = mid + 1; else hi = mid;
    }
    bucket[b] = (int)lo;
}

template <typename T>
__global__ void k_sqrt(const T* __restrict__ var, T* __restrict__ sig, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const T v = var[i];
    sig[i] = v > T(0) ? sqrt(v) : T(NAN);
}

template <typename T> struct KSum {
    T s, c;
    __device__ __forceinline__ void init() { s = T(0); c = T(0); }
    __device__ __forceinline__ void add(T x) {
        const T y = x - c;
        const T t = s + y;
        c = (t - s) - y;
        s = t;
    }
};
template <> struct KSum<double> {
    double s;
    __device__ __forceinline__ void init() { s = 0.0; }
    __device__ __forceinline__ void add(double x) { s += x; }
};

struct Best {
    double lnp;
    long long cell;
    double depth;
    double sigma;
};

__device__ __forceinline__ bool better(const Best& a, const Best& b) {
    // a beats b: larger ln P, ties to the smaller cell index
    if (a.lnp > b.lnp) return true;
    if (a.lnp < b.lnp) return false;
    return a.cell < b.cell;
}

template <typename T>
__device__ __forceinline__ bool event(const FoldGeom& g, const T* __restrict__ dep,
                                      const T* __restrict__ sig, const T* __restrict__ gl,
                                      double Tk, T& dk, T& sk2, T& lk) {
    const int64_t i = bracket(g, Tk);
    if (i > g.n_t0 - 2) return false;
    const double ta = g.t0s[i], tb = g.t0s[i + 1];
    const double gap = tb - ta;
    if (!(gap <= g.gap_max)) return false;
    const double w = (Tk - ta) / gap;
    const T da = dep[i], db = dep[i + 1], sa = sig[i], sb = sig[i + 1];
    const T la = gl[i], lb = gl[i + 1];
    if (!(isfinite(da) && isfinite(db) && isfinite(sa) && isfinite(sb) && isfinite(la) &&
          isfinite(lb)))
        return false;
    const T wl = (T)(1.0 - w), wr = (T)w;
    dk = wl * da + wr * db;
    const T s = wl * sa + wr * sb;
    sk2 = s * s;
    lk = wl * la + wr * lb;
    return true;
}

template <typename T>
__global__ void __launch_bounds__(256)
k_fold(FoldGeom g, const T* __restrict__ depth, const T* __restrict__ sig,
       const T* __restrict__ gain, int n_D, const double* __restrict__ periods,
       int64_t n_P, double* __restrict__ Q_out, double* __restrict__ T0_out,
       int* __restrict__ Didx_out, double* __restrict__ dep_out,
       double* __restrict__ sig_out, double* __restrict__ lnp_out) {
    const int64_t p = blockIdx.x;
    if (p >= n_P) return;
    const double P = periods[p];
    // a period must be finite, > 0 and give at most 1e9 epochs and phases;
    // anything else is reported as NaN with no cell (and does no work)
    if (!(P > 0.0) || !isfinite(P) || (g.t_last - g.t_ref) / P > 1.0e9 ||
        P / g.dt > 1.0e9) {
        if (threadIdx.x == 0) {
            Q_out[p] = NAN;
            T0_out[p] = NAN;
            Didx_out[p] = -1;
            dep_out[p] = NAN;
            sig_out[p] = NAN;
            lnp_out[p] = NAN;
        }
        return;
    }
    const int64_t n_phi = (int64_t)ceil(P / g.dt);
    const int64_t n_cells = n_phi * n_D;
    Best best{-INFINITY, LLONG_MAX, NAN, NAN};
    for (int64_t cell = threadIdx.x; cell < n_cells; cell += blockDim.x) {
        const int d = (int)(cell / n_phi);
        const int64_t j = cell - (int64_t)d * n_phi;
        const double phi = (double)j / (double)n_phi;
        const T* dp = depth + (int64_t)d * g.n_t0;
        const T* sp = sig + (int64_t)d * g.n_t0;
        const T* lp = gain + (int64_t)d * g.n_t0;
        KSum<T> s_inv, s_d, s_l;
        s_inv.init();
        s_d.init();
        s_l.init();
        int K = 0;
        for (int64_t k = 0;; ++k) {
            const double Tk = __dadd_rn(g.t_ref, __dmul_rn(__dadd_rn(phi, (double)k), P));
            if (Tk > g.t_last) break;
            T dk, sk2, lk;
            if (!event<T>(g, dp, sp, lp, Tk, dk, sk2, lk)) continue;
            const T iv = T(1) / sk2;
            s_inv.add(iv);
            s_d.add(dk * iv);
            s_l.add(lk);
            ++K;
        }
        if (K == 0) continue;
        const T s2 = T(1) / s_inv.s;
        const T Dl = s2 * s_d.s;
        KSum<T> pen;
        pen.init();
        for (int64_t k = 0;; ++k) {
            const double Tk = __dadd_rn(g.t_ref, __dmul_rn(__dadd_rn(phi, (double)k), P));
            if (Tk > g.t_last) break;
            T dk, sk2, lk;
            if (!event<T>(g, dp, sp, lp, Tk, dk, sk2, lk)) continue;
            const T den = sk2 + s2;
            const T r = dk - Dl;
            // ln s_k^2 - ln(sigma^2 + s_k^2) = -ln(1 + sigma^2 / s_k^2)
            pen.add(-log1p(s2 / sk2) + r * r / den);
        }
        const double lnp = (double)s_l.s - 0.5 * (double)pen.s;
        if (!(lnp == lnp)) continue;   // NaN never selected
        Best cand{lnp, (long long)cell, (double)Dl, sqrt((double)s2)};
        if (better(cand, best)) best = cand;
    }
    // block argmax
    __shared__ Best sh[256];
    sh[threadIdx.x] = best;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w && better(sh[threadIdx.x + w], sh[threadIdx.x]))
            sh[threadIdx.x] = sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const Best b = sh[0];
        if (b.cell == LLONG_MAX) {
            Q_out[p] = 0.0;
            T0_out[p] = NAN;
            Didx_out[p] = -1;
            dep_out[p] = NAN;
            sig_out[p] = NAN;
            lnp_out[p] = -INFINITY;
        } else {
            const int d = (int)(b.cell / n_phi);
            const int64_t j = b.cell - (int64_t)d * n_phi;
            Q_out[p] = b.depth / b.sigma;
            T0_out[p] = __dadd_rn(g.t_ref, __dmul_rn((double)j / (double)n_phi, P));
            Didx_out[p] = d;
            dep_out[p] = b.depth;
            sig_out[p] = b.sigma;
            lnp_out[p] = b.lnp;
        }
    }
}

}  // namespace nu

using namespace nu;

extern "C" nu_status nu_periodic_search(const double* t0s_dev, int64_t n_t0,
                                        const double* Ds_host, int n_D,
                                        const void* depth_dev, const void* var_dev,
                                        const void* dlnl_dev, nu_precision prec,
                                        const double* periods_dev, int64_t n_P,
                                        double phase_step, double gap_factor, void* stream,
                                        double* Q_dev, double* T0_dev, int32_t* D_idx_dev,
                                        double* depth_out_dev, double* sigma_out_dev,
                                        double* lnP_dev) {
    if (!t0s_dev || !depth_dev || !var_dev || !dlnl_dev || !periods_dev || !Q_dev ||
        !T0_dev || !D_idx_dev || !depth_out_dev || !sigma_out_dev || !lnP_dev)
        return fail(NU_EINVAL, "nu_periodic_search: null array");
    (void)Ds_host;
    if (n_t0 < 2 || n_D < 1 || n_P < 1)
        return fail(NU_EINVAL, "nu_periodic_search: need n_t0 >= 2, n_D >= 1, n_P >= 1");
    if (prec != NU_FP64 && prec != NU_MIXED)
        return fail(NU_EINVAL, "nu_periodic_search: unknown precision");
    if (!(gap_factor > 0.0)) return fail(NU_EINVAL, "nu_periodic_search: gap_factor <= 0");
    if (n_t0 > 2000000000LL) return fail(NU_EINVAL, "nu_periodic_search: n_t0 too large");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    // grid end points (host copies; the step, when not given, is the median
    // spacing of the epochs)
    std::vector<double> ends(2);
    double t_ref, t_last;
    if (!(phase_step > 0.0)) {
        std::vector<double> h(n_t0);
        e = cudaMemcpyAsync(h.data(), t0s_dev, n_t0 * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "nu_periodic_search: copy t0s");
        std::vector<double> d(n_t0 - 1);
        for (int64_t i = 0; i + 1 < n_t0; ++i) d[i] = h[i + 1] - h[i];
        std::sort(d.begin(), d.end());
        const size_t m = d.size();
        phase_step = (m % 2) ? d[m / 2] : 0.5 * (d[m / 2 - 1] + d[m / 2]);
        t_ref = h[0];
        t_last = h[n_t0 - 1];
    } else {
        e = cudaMemcpyAsync(&ends[0], t0s_dev, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&ends[1], t0s_dev + n_t0 - 1, sizeof(double),
                                cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "nu_periodic_search: copy ends");
        t_ref = ends[0];
        t_last = ends[1];
    }
    if (!(phase_step > 0.0) || !std::isfinite(phase_step))
        return fail(NU_EINVAL, "nu_periodic_search: phase step must be > 0");
    if (!(t_last >= t_ref)) return fail(NU_EINVAL, "nu_periodic_search: t0s not sorted");
    const double span_steps = (t_last - t_ref) / phase_step;
    if (span_steps > 1.0e9) return fail(NU_EINVAL, "nu_periodic_search: phase grid too fine");
    const int64_t n_bucket = (int64_t)span_steps + 2;
    const size_t esz = prec == NU_FP64 ? sizeof(double) : sizeof(float);
    pool_keep_memory();
    void* scratch = nullptr;
    const size_t sig_bytes = ((size_t)n_t0 * n_D * esz + 255) / 256 * 256;
    e = cudaMallocAsync(&scratch, sig_bytes + n_bucket * sizeof(int), st);
    if (e != cudaSuccess) return cuda_fail(e, "nu_periodic_search: cudaMallocAsync");
    void* sig = scratch;
    int* bucket = (int*)((char*)scratch + sig_bytes);
    k_buckets<<<div_up(n_bucket, 256), 256, 0, st>>>(t0s_dev, n_t0, t_ref, phase_step,
                                                    n_bucket, bucket);
    FoldGeom g{t0s_dev, n_t0, t_ref, t_last, phase_step, 1.0 / phase_step,
               gap_factor * phase_step, bucket, n_bucket};
    const int64_t nsig = n_t0 * (int64_t)n_D;
    if (prec == NU_FP64) {
        k_sqrt<double><<<div_up(nsig, 256), 256, 0, st>>>((const double*)var_dev,
                                                        (double*)sig, nsig);
        k_fold<double><<<(unsigned)n_P, 256, 0, st>>>(
            g, (const double*)depth_dev, (const double*)sig, (const double*)dlnl_dev, n_D,
            periods_dev, n_P, Q_dev, T0_dev, D_idx_dev, depth_out_dev, sigma_out_dev,
            lnP_dev);
    } else {
        k_sqrt<float><<<div_up(nsig, 256), 256, 0, st>>>((const float*)var_dev,
                                                       (float*)sig, nsig);
        k_fold<float><<<(unsigned)n_P, 256, 0, st>>>(
            g, (const float*)depth_dev, (const float*)sig, (const float*)dlnl_dev, n_D,
            periods_dev, n_P, Q_dev, T0_dev, D_idx_dev, depth_out_dev, sigma_out_dev,
            lnP_dev);
    }
    count_launches(3);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "nu_periodic_search: launch");
    e = cudaFreeAsync(scratch, st);
    if (e != cudaSuccess) return cuda_fail(e, "nu_periodic_search: cudaFreeAsync");
    return NU_OK;
}

extern "C" nu_status nu_batch_search(int n_lc, const int64_t* offsets_host,
                                     const double* t_dev, const double* y_dev,
                                     const double* diag_var_dev,
                                     const nu_term* terms_host, const int* n_terms_host,
                                     int k, const double* Ds_host, int n_D,
                                     const double* periods_dev, int64_t n_P,
                                     double phase_step, nu_precision prec, void* stream,
                                     double* Q_dev, double* T0_dev, int32_t* D_idx_dev,
                                     double* depth_out_dev, double* sigma_out_dev,
                                     double* lnP_dev, int* status_host) {
    (void)n_lc; (void)offsets_host; (void)t_dev; (void)y_dev; (void)diag_var_dev;
    (void)terms_host; (void)n_terms_host; (void)k; (void)Ds_host; (void)n_D;
    (void)periods_dev; (void)n_P; (void)phase_step; (void)prec; (void)stream; (void)Q_dev;
    (void)T0_dev; (void)D_idx_dev; (void)depth_out_dev; (void)sigma_out_dev; (void)lnP_dev;
    (void)status_host;
    return fail(NU_EINVAL, "nu_batch_search: not built yet");
}

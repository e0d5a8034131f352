// nu_linear_search: Sect. 2.2 on the grid of epochs x durations.
//
// With the null fit of the factor (z0 = Sigma^-1 r0, Zt = Sigma^-1 X R^-1)
// Eq. ls for X' = [X, m] reduces by a Schur complement to three window
// quantities of the template m:
//   c   = m^T Sigma^-1 m
//   num = m^T z0                (= m^T Sigma^-1 y - b^T A^-1 u)
//   bt  = Zt^T m                (k values; b^T A^-1 b = |bt|^2)
// s = c - |bt|^2, depth = num / s, var = 1 / s, gain = num^2 / (2 s)
// (the last column of (X'^T Sigma^-1 X')^-1 and of the GLS weights, and the
// chi-square drop of Eq. linear_search_ll).
//
// c is the squared D^-1/2-weighted norm of L^-1 m.  m is zero before the
// window start lo, so the forward solve starts from a zero state there:
//   e_n = m_n - h^T s_n,  c += e_n^2 / D_n,  s_{n+1} = F_{n+1}(s_n + kg_n e_n)
// over the window, and after the window (m = 0) the remaining terms sum to
// s_hi^T G_hi s_hi with the factor's future-information matrix.
#include <cmath>
#include <cstring>

#include "nu_internal.cuh"
#include "ss.cuh"
#include "templates.cuh"

namespace nu {

// first index with t[idx] >= x (t sorted ascending)
__device__ __forceinline__ int64_t lower_bound_d(const double* __restrict__ t, int64_t n,
                                                 double x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (t[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Compensated (Kahan) accumulator for the FP32 path; plain for FP64.
template <typename T> struct Acc {
    T s, c;
    __device__ __forceinline__ void init() { s = T(0); c = T(0); }
    __device__ __forceinline__ void add(T x) {
        const T y = x - c;
        const T t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ T get() const { return s; }
};
template <> struct Acc<double> {
    double s;
    __device__ __forceinline__ void init() { s = 0.0; }
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double get() const { return s; }
};


// One window: the fit of template m(t0, D) against the factor of one light
// curve (arrays already offset to the curve, n samples).
template <int NB, typename T, int TMPL>
__device__ __forceinline__ void window_fit(const double* __restrict__ t, int64_t n, int k,
                                           const FactorView<T>& fv, double t0, double D,
                                           const TmplArgs& ta, T& out_d, T& out_v, T& out_l) {
    constexpr int J = Dims<NB>::J;
    constexpr int JJ = Dims<NB>::JJ;
    const double half = D * 0.5;
    // window of Sect. 2.1's box, half-open: t0 - D/2 <= t < t0 + D/2
    const int64_t lo = lower_bound_d(t, n, __dsub_rn(t0, half));
    const int64_t hi = lower_bound_d(t, n, __dadd_rn(t0, half));
    const T nanv = T(NAN);
    out_d = nanv;
    out_v = nanv;
    out_l = nanv;
    if (hi <= lo) return;
    T s[J];
#pragma unroll
    for (int c = 0; c < J; ++c) s[c] = T(0);
    Acc<T> c2, num, bt[NU_MAX_K];
    c2.init();
    num.init();
#pragma unroll
    for (int a = 0; a < NU_MAX_K; ++a) bt[a].init();
    for (int64_t m = lo; m < hi; ++m) {
        const T mv = TMPL == NU_BOX ? T(-1) : (T)template_value<TMPL>(t[m], t0, half, D, ta);
        const T e = mv - hdot<NB>(s);
        const T iD = fv.invD[m];
        c2.add(e * e * iD);
        num.add(mv * fv.z0[m]);
        for (int a = 0; a < k; ++a) bt[a].add(mv * fv.Zt[m * k + a]);
        if (m + 1 < n) {
            T tmp[J];
#pragma unroll
            for (int c = 0; c < J; ++c) tmp[c] = s[c] + fv.kg[m * J + c] * e;
            apply_F<NB>(fv.F + (m + 1) * NB * 4, tmp, s);
        }
    }
    T cval = c2.get();
    if (hi < n) {
        // tail of the forward solve after the window: s^T G_hi s
        const T* Gh = fv.G + hi * JJ;
        T q = T(0);
#pragma unroll
        for (int r = 0; r < J; ++r) {
            T rowsum = Gh[pk(r, r, J)] * s[r];
#pragma unroll
            for (int c = r + 1; c < J; ++c) rowsum += T(2) * Gh[pk(r, c, J)] * s[c];
            q += s[r] * rowsum;
        }
        cval += q;
    }
    T bb = T(0);
    for (int a = 0; a < k; ++a) bb += bt[a].get() * bt[a].get();
    const T sch = cval - bb;
    if (!(sch > T(0))) return;
    const T nm = num.get();
    const T dep = nm / sch;
    out_d = dep;
    out_v = T(1) / sch;
    out_l = T(0.5) * nm * dep;
}

template <int NB, typename T>
__device__ __forceinline__ FactorView<T> view_at(const FactorView<T>& fv, int64_t s0, int k) {
    constexpr int J = Dims<NB>::J;
    constexpr int JJ = Dims<NB>::JJ;
    return FactorView<T>{fv.F + s0 * NB * 4, fv.kg + s0 * J, fv.invD + s0, fv.G + s0 * JJ,
                         fv.z0 + s0, fv.Zt + s0 * k};
}

// One thread per (duration j, epoch i) of one light curve.
template <int NB, typename T, int TMPL>
__global__ void __launch_bounds__(128)
k_window(const double* __restrict__ t, int64_t n, int k, FactorView<T> fv,
         const double* __restrict__ t0s, int64_t n_t0, const double* __restrict__ Ds,
         int n_D, TmplArgs ta, T* __restrict__ out_depth, T* __restrict__ out_var,
         T* __restrict__ out_dlnl) {
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gid >= n_t0 * (int64_t)n_D) return;
    const int j = (int)(gid / n_t0);
    const int64_t i = gid - (int64_t)j * n_t0;
    T d, v, l;
    window_fit<NB, T, TMPL>(t, n, k, fv, t0s[i], Ds[j], ta, d, v, l);
    out_depth[gid] = d;
    out_var[gid] = v;
    out_dlnl[gid] = l;
}

// Several light curves packed back to back (segments), epochs = the curves'
// own samples; outputs of curve g are [n_D][n_g] at n_D * s_off[g].
template <int NB, typename T>
__global__ void __launch_bounds__(128)
k_window_batch(const double* __restrict__ t, int k, FactorView<T> fv,
               const int64_t* __restrict__ s_off, int n_seg, const double* __restrict__ Ds,
               int n_D, T* __restrict__ out_depth, T* __restrict__ out_var,
               T* __restrict__ out_dlnl) {
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gid >= s_off[n_seg] * (int64_t)n_D) return;
    int lo = 0, hi = n_seg;                     // segment: n_D s_off[g] <= gid
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s_off[mid] * (int64_t)n_D <= gid) lo = mid; else hi = mid;
    }
    const int64_t s0 = s_off[lo], ng = s_off[lo + 1] - s0;
    const int64_t w = gid - s0 * n_D;
    const int j = (int)(w / ng);
    const int64_t i = w - (int64_t)j * ng;
    T d, v, l;
    window_fit<NB, T, NU_BOX>(t + s0, ng, k, view_at<NB, T>(fv, s0, k), t[s0 + i], Ds[j],
                              TmplArgs{0.0, 0.0}, d, v, l);
    out_depth[gid] = d;
    out_var[gid] = v;
    out_dlnl[gid] = l;
}

template <int NB, typename T>
static void launch_window(const nu_factor* f, FactorView<T> fv, const double* t0s,
                          int64_t n_t0, const double* Ds_dev, int n_D, int tmpl,
                          const TmplArgs& ta, void* d, void* v, void* l, cudaStream_t st) {
    const int64_t total = n_t0 * (int64_t)n_D;
    const int th = 128;
    const int blocks = div_up(total, th);
    if (tmpl == NU_BOX)
        k_window<NB, T, NU_BOX><<<blocks, th, 0, st>>>(f->t, f->n, f->k, fv, t0s, n_t0,
                                                      Ds_dev, n_D, ta, (T*)d, (T*)v, (T*)l);
    else if (tmpl == NU_TRAPEZOID)
        k_window<NB, T, NU_TRAPEZOID><<<blocks, th, 0, st>>>(
            f->t, f->n, f->k, fv, t0s, n_t0, Ds_dev, n_D, ta, (T*)d, (T*)v, (T*)l);
    else
        k_window<NB, T, NU_LIMB_QUAD><<<blocks, th, 0, st>>>(
            f->t, f->n, f->k, fv, t0s, n_t0, Ds_dev, n_D, ta, (T*)d, (T*)v, (T*)l);
}

// Linear search of packed light curves (batch path); no allocation, no sync.
int launch_window_batch(int nb, bool fp64, const double* t, int k, const void* fv,
                        const int64_t* s_off, int n_seg, int64_t n_total, const double* Ds,
                        int n_D, void* d, void* v, void* l, cudaStream_t st) {
    const int64_t total = n_total * (int64_t)n_D;
    const int th = 128;
    const int blocks = div_up(total, th);
#define NU_WB(NB_, T_)                                                                   \
    k_window_batch<NB_, T_><<<blocks, th, 0, st>>>(t, k, *(const FactorView<T_>*)fv, s_off, \
                                                  n_seg, Ds, n_D, (T_*)d, (T_*)v, (T_*)l)
    if (fp64) {
        switch (nb) {
            case 1: NU_WB(1, double); break;
            case 2: NU_WB(2, double); break;
            case 3: NU_WB(3, double); break;
            default: NU_WB(4, double); break;
        }
    } else {
        switch (nb) {
            case 1: NU_WB(1, float); break;
            case 2: NU_WB(2, float); break;
            case 3: NU_WB(3, float); break;
            default: NU_WB(4, float); break;
        }
    }
#undef NU_WB
    return 1;
}

}  // namespace nu

using namespace nu;

extern "C" nu_status nu_linear_search(const nu_factor* f, const double* t0s_dev,
                                      int64_t n_t0, const double* Ds_host, int n_D,
                                      nu_template tmpl, const double* tmpl_params,
                                      nu_precision prec, void* stream, void* depth_dev,
                                      void* var_dev, void* dlnl_dev) {
    if (!f) return fail(NU_EINVAL, "nu_linear_search: null factor");
    if (!t0s_dev || !Ds_host || !depth_dev || !var_dev || !dlnl_dev)
        return fail(NU_EINVAL, "nu_linear_search: null array");
    if (n_t0 < 1 || n_D < 1) return fail(NU_EINVAL, "nu_linear_search: empty grid");
    TmplArgs ta;
    const char* why = "";
    if (!template_args((int)tmpl, tmpl_params, &ta, &why))
        return fail(NU_EINVAL, "nu_linear_search: %s (template %d)", why, (int)tmpl);
    if (prec != NU_FP64 && prec != NU_MIXED)
        return fail(NU_EINVAL, "nu_linear_search: unknown precision %d", (int)prec);
    for (int j = 0; j < n_D; ++j)
        if (!(Ds_host[j] > 0.0) || !std::isfinite(Ds_host[j]))
            return fail(NU_EINVAL, "nu_linear_search: durations must be finite and > 0");
    cudaStream_t st = (cudaStream_t)stream;
    pool_keep_memory();
    double* Ds_dev = nullptr;
    cudaError_t e = cudaMallocAsync(&Ds_dev, n_D * sizeof(double), st);
    if (e != cudaSuccess) return cuda_fail(e, "nu_linear_search: cudaMallocAsync");
    e = cudaMemcpyAsync(Ds_dev, Ds_host, n_D * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "nu_linear_search: copy");
    // order the factor's work before ours when the streams differ
    if (f->stream != st) {
        cudaEvent_t ev;
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        cudaEventRecord(ev, f->stream);
        cudaStreamWaitEvent(st, ev, 0);
        cudaEventDestroy(ev);
    }
    if (prec == NU_FP64) {
        FactorView<double> fv{f->F, f->kg, f->invD, f->G, f->z0, f->Zt};
        switch (f->nb) {
            case 1: launch_window<1, double>(f, fv, t0s_dev, n_t0, Ds_dev, n_D, tmpl, ta, depth_dev, var_dev, dlnl_dev, st); break;
            case 2: launch_window<2, double>(f, fv, t0s_dev, n_t0, Ds_dev, n_D, tmpl, ta, depth_dev, var_dev, dlnl_dev, st); break;
            case 3: launch_window<3, double>(f, fv, t0s_dev, n_t0, Ds_dev, n_D, tmpl, ta, depth_dev, var_dev, dlnl_dev, st); break;
            default: launch_window<4, double>(f, fv, t0s_dev, n_t0, Ds_dev, n_D, tmpl, ta, depth_dev, var_dev, dlnl_dev, st); break;
        }
    } else {
        FactorView<float> fv{f->F32, f->kg32, f->invD32, f->G32, f->z032, f->Zt32};
        switch (f->nb) {
            case 1: launch_window<1, float>(f, fv, t0s_dev, n_t0, Ds_dev, n_D, tmpl, ta, depth_dev, var_dev, dlnl_dev, st); break;
            case 2: launch_window<2, float>(f, fv, t0s_dev, n_t0, Ds_dev, n_D, tmpl, ta, depth_dev, var_dev, dlnl_dev, st); break;
            case 3: launch_window<3, float>(f, fv, t0s_dev, n_t0, Ds_dev, n_D, tmpl, ta, depth_dev, var_dev, dlnl_dev, st); break;
            default: launch_window<4, float>(f, fv, t0s_dev, n_t0, Ds_dev, n_D, tmpl, ta, depth_dev, var_dev, dlnl_dev, st); break;
        }
    }
    count_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "nu_linear_search: launch");
    e = cudaFreeAsync(Ds_dev, st);
    if (e != cudaSuccess) return cuda_fail(e, "nu_linear_search: cudaFreeAsync");
    return NU_OK;
}

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
#include <climits>
#include <cmath>
#include <cstdint>
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

// ------------------------------------------------------------------------
// Window-start recursion (box template).  The forward solve of a box window
// starts from a zero state at its first sample lo and does not depend on
// where the window ends, so one recursion from lo serves every duration
// whose window starts there: after L samples the running sums and the state
// give that window's c, num and bt.  For epochs on the sample grid the
// windows of duration j take a few (length L, offset a = epoch index - lo)
// pairs ("variants"): one, or up to four when a window edge falls on a
// sample and FP64 rounding decides whether that sample is in.  The plan
// below finds them; one thread per window start runs the recursion once
// over the longest variant and completes every window that starts there
// and matches a variant, and the per-template kernel does the rest
// (windows clipped by a gap or an end).
//
// Plan of a curve (ints, NV = 4 variants per duration):
//   [0] the longest L; [1] the number E of variants;
//   [2 + e], e < E: their lengths sorted ascending, [2 + NV n_D + e] their
//   offsets, [2 + 2 NV n_D + e] their durations;
//   [2 + 3 NV n_D + NV j + v] and [2 + 4 NV n_D + NV j + v], v < NV: L and a
//   of the variants of duration j (L = 0: unused slot).
#define NU_WIN_NV 4
#define NU_WIN_PROBES 256
__host__ __device__ constexpr int plan_ints(int n_D) { return 2 + 5 * NU_WIN_NV * n_D; }

// Whether the window of (epoch t0, half-duration half) is exactly samples
// [lo, hi) of the curve t[0..n): the first sample >= t0 - half is lo and the
// first sample >= t0 + half is hi (the half-open window, FP64 as written).
__device__ __forceinline__ bool window_is(const double* __restrict__ t, int64_t n, double t0,
                                          double half, int64_t lo, int64_t hi) {
    if (lo < 0 || hi > n || hi <= lo) return false;
    const double xl = __dsub_rn(t0, half), xh = __dadd_rn(t0, half);
    if (lo > 0 && !(t[lo - 1] < xl)) return false;
    if (!(t[lo] >= xl)) return false;
    if (!(t[hi - 1] < xh)) return false;
    if (hi < n && !(t[hi] >= xh)) return false;
    return true;
}

// Per-curve view: first packed sample, samples, epochs (n_t0 of them), and
// the first output element.  s_off == nullptr: one curve, epochs t0s.
struct CurveView {
    int64_t s0, n, n_t0, out0;
    const double* t0;
};
__device__ __forceinline__ CurveView curve_of(const double* __restrict__ t,
                                              const double* __restrict__ t0s, int64_t n_t0,
                                              const int64_t* __restrict__ s_off, int n_seg,
                                              int64_t n_total, int n_D, int64_t x, int* seg) {
    if (!s_off) {
        *seg = 0;
        return CurveView{0, n_total, n_t0, 0, t0s};
    }
    int lo = 0, hi = n_seg;                     // segment: s_off[g] <= x
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s_off[mid] <= x) lo = mid; else hi = mid;
    }
    *seg = lo;
    const int64_t s0 = s_off[lo], n = s_off[lo + 1] - s0;
    return CurveView{s0, n, n, (int64_t)n_D * s0, t + s0};
}

// Variants of one (curve, duration): one block of NU_WIN_PROBES threads per
// (curve, duration) probes epochs spread over the grid (binary searches),
// and keeps the NU_WIN_NV most frequent (L, a) pairs within a 4 x 5 window
// around the longest probed L (first seen on ties).  Clipped windows (edges,
// gaps) are shorter and left to the per-template kernel.
__global__ void __launch_bounds__(NU_WIN_PROBES)
k_window_variants(const double* __restrict__ t, const double* __restrict__ t0s, int64_t n_t0,
                  const int64_t* __restrict__ s_off, int64_t n_total,
                  const double* __restrict__ Ds, int n_D, int* __restrict__ plan) {
    __shared__ int sh_L[NU_WIN_PROBES], sh_a[NU_WIN_PROBES];
    __shared__ int sh_lc, sh_ac;
    __shared__ int sh_cnt[4 * 5], sh_first[4 * 5];
    const int g = blockIdx.x / n_D, j = blockIdx.x - (blockIdx.x / n_D) * n_D;
    const int64_t s0 = s_off ? s_off[g] : 0;
    const int64_t n = s_off ? s_off[g + 1] - s0 : n_total;
    const int64_t nt = s_off ? n : n_t0;
    const double* tg = t + s0;
    const double* t0g = s_off ? tg : t0s;
    const double half = Ds[j] * 0.5;
    const int r = threadIdx.x;
    const int64_t ip = (nt * (2 * r + 1)) / (2 * NU_WIN_PROBES);
    const double t0 = t0g[ip];
    const int64_t lo = lower_bound_d(tg, n, __dsub_rn(t0, half));
    const int64_t hi = lower_bound_d(tg, n, __dadd_rn(t0, half));
    const int64_t L = hi - lo, a = ip - lo;
    const bool ok = L > 0 && L < (1 << 20) && a > -(1 << 29) && a < (1 << 29);
    sh_L[r] = ok ? (int)L : 0;
    sh_a[r] = ok ? (int)a : 0;
    if (r < 20) {
        sh_cnt[r] = 0;
        sh_first[r] = INT_MAX;
    }
    if (r == 0) sh_lc = 0;
    __syncthreads();
    if (sh_L[r] > 0) atomicMax(&sh_lc, sh_L[r]);
    __syncthreads();
    if (r == 0) {
        sh_ac = 0;
        for (int q = 0; q < NU_WIN_PROBES; ++q)
            if (sh_L[q] == sh_lc && sh_lc > 0) {
                sh_ac = sh_a[q];
                break;
            }
    }
    __syncthreads();
    const int dl = sh_L[r] - sh_lc + 3, da = sh_a[r] - sh_ac + 2;
    if (sh_L[r] > 0 && dl >= 0 && dl < 4 && da >= 0 && da < 5) {
        atomicAdd(&sh_cnt[dl * 5 + da], 1);
        atomicMin(&sh_first[dl * 5 + da], r);
    }
    __syncthreads();
    if (r != 0) return;
    int* P = plan + (int64_t)g * plan_ints(n_D);
    int* Lv = P + 2 + 3 * NU_WIN_NV * n_D + NU_WIN_NV * j;
    int* av = P + 2 + 4 * NU_WIN_NV * n_D + NU_WIN_NV * j;
    bool used[20] = {};
    for (int v = 0; v < NU_WIN_NV; ++v) {
        int best = -1;
        for (int b = 0; b < 20; ++b)
            if (!used[b] && sh_cnt[b] > 0 &&
                (best < 0 || sh_cnt[b] > sh_cnt[best] ||
                 (sh_cnt[b] == sh_cnt[best] && sh_first[b] < sh_first[best])))
                best = b;
        if (best >= 0) {
            used[best] = true;
            Lv[v] = sh_lc + best / 5 - 3;
            av[v] = sh_ac + best % 5 - 2;
        } else {
            Lv[v] = 0;
            av[v] = 0;
        }
    }
}

// One thread per curve: the variants of all durations sorted by L (stable)
// into the emission list, and the longest L.
__global__ void k_window_plan_sort(int n_seg, int n_D, int* __restrict__ plan) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_seg) return;
    int* P = plan + (int64_t)g * plan_ints(n_D);
    const int E0 = NU_WIN_NV * n_D;
    int* Ls = P + 2;
    int* As = P + 2 + E0;
    int* Js = P + 2 + 2 * E0;
    const int* Lv = P + 2 + 3 * E0;
    const int* av = P + 2 + 4 * E0;
    int E = 0, lmax = 0;
    for (int j = 0; j < n_D; ++j)
        for (int v = 0; v < NU_WIN_NV; ++v) {
            const int L = Lv[NU_WIN_NV * j + v];
            if (L <= 0) continue;
            lmax = max(lmax, L);
            int q = E++;                               // insertion, stable
            while (q > 0 && Ls[q - 1] > L) {
                Ls[q] = Ls[q - 1];
                As[q] = As[q - 1];
                Js[q] = Js[q - 1];
                --q;
            }
            Ls[q] = L;
            As[q] = av[NU_WIN_NV * j + v];
            Js[q] = j;
        }
    P[0] = lmax;
    P[1] = E;
}

// Whether window (epoch index i, duration j) matches one of the plan's
// variants of j (then the window-start kernel writes it).
__device__ __forceinline__ bool window_in_plan(const int* __restrict__ P, int n_D,
                                               const double* __restrict__ t, int64_t n,
                                               double t0, double half, int j, int64_t i) {
    const int* Lv = P + 2 + 3 * NU_WIN_NV * n_D + NU_WIN_NV * j;
    const int* av = P + 2 + 4 * NU_WIN_NV * n_D + NU_WIN_NV * j;
#pragma unroll
    for (int v = 0; v < NU_WIN_NV; ++v) {
        const int L = Lv[v];
        if (L <= 0) break;
        const int64_t lo = i - av[v];
        if (window_is(t, n, t0, half, lo, lo + L)) return true;
    }
    return false;
}

// Number of per-sample values the window-start kernel stages: F (4 NB), the
// gain (J), 1/D, z0 and Zt (k).
template <int NB> __host__ __device__ constexpr int stage_fields(int k) {
    return 4 * NB + 2 * NB + 2 + k;
}

// Copy elements [base*W, (base+cnt)*W) of a sample-major array of W values
// per sample into shared rows dst[f * rs + x] (x the sample, f the value),
// with 16-byte loads where the source is 16-byte aligned.
template <typename T>
__device__ __forceinline__ void stage_rows(const T* __restrict__ src, int W, int64_t base,
                                           int cnt, T* __restrict__ dst, int rs) {
    const T* g = src + base * W;
    const int nel = cnt * W;
    constexpr int V = 16 / sizeof(T);
    int e0 = 0;
    if ((reinterpret_cast<uintptr_t>(g) & 15) == 0) {
        const int nv = nel / V;
        for (int c = threadIdx.x; c < nv; c += blockDim.x) {
            T v[V];
            if constexpr (sizeof(T) == 8) {
                const double2 d = reinterpret_cast<const double2*>(g)[c];
                v[0] = d.x;
                v[1] = d.y;
            } else {
                const float4 f = reinterpret_cast<const float4*>(g)[c];
                v[0] = f.x;
                v[1] = f.y;
                v[2] = f.z;
                v[3] = f.w;
            }
#pragma unroll
            for (int u = 0; u < V; ++u) {
                const int e = c * V + u;
                dst[(e % W) * rs + e / W] = v[u];
            }
        }
        e0 = nv * V;
    }
    for (int e = e0 + threadIdx.x; e < nel; e += blockDim.x) dst[(e % W) * rs + e / W] = g[e];
}

// A box window that matches no variant of the plan, fitted on its own
// (template gid of the grid, duration-major per curve).
template <int NB, typename T>
__device__ __forceinline__ void window_rest(const double* __restrict__ t,
                                            const double* __restrict__ t0s, int64_t n_t0, int k,
                                            const FactorView<T>& fv,
                                            const int64_t* __restrict__ s_off, int n_seg,
                                            int64_t n_total, const double* __restrict__ Ds,
                                            int n_D, const int* __restrict__ plan, int64_t gid,
                                            T* __restrict__ out_depth, T* __restrict__ out_var,
                                            T* __restrict__ out_dlnl) {
    int64_t s0 = 0, ng = n_total, nt = n_t0, w = gid;
    int g = 0;
    if (s_off) {
        int lo = 0, hi = n_seg;                 // segment: n_D s_off[g] <= gid
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (s_off[mid] * (int64_t)n_D <= gid) lo = mid; else hi = mid;
        }
        g = lo;
        s0 = s_off[g];
        ng = nt = s_off[g + 1] - s0;
        w = gid - s0 * n_D;
    }
    const int j = (int)(w / nt);
    const int64_t i = w - (int64_t)j * nt;
    const double t0 = s_off ? t[s0 + i] : t0s[i];
    if (window_in_plan(plan + (int64_t)g * plan_ints(n_D), n_D, t + s0, ng, t0, Ds[j] * 0.5, j,
                       i))
        return;
    T d, v, l;
    window_fit<NB, T, NU_BOX>(t + s0, ng, k, view_at<NB, T>(fv, s0, k), t0, Ds[j],
                              TmplArgs{0.0, 0.0}, d, v, l);
    out_depth[gid] = d;
    out_var[gid] = v;
    out_dlnl[gid] = l;
}

// One thread per window start lo (packed sample index); the block's TLO
// consecutive starts share the factor rows of samples [lo0 + m0, lo0 + m0 +
// TLO + ch), staged in shared memory ch samples of the recursion at a time.
// The first n_rest blocks instead take TLO templates each of the whole grid
// and fit the windows that match no variant (clipped by a gap or an end);
// in the same launch their long serial recursions overlap the window-start
// recursions, which leave the FP64 pipe idle between dependent instructions
// when there are few warps per sub-partition.
template <int NB, typename T, int TLO>
__global__ void __launch_bounds__(TLO)
k_window_lo(const double* __restrict__ t, const double* __restrict__ t0s, int64_t n_t0, int k,
            FactorView<T> fv, const int64_t* __restrict__ s_off, int n_seg, int64_t n_total,
            const double* __restrict__ Ds, int n_D, const int* __restrict__ plan, int ch,
            int n_rest, T* __restrict__ out_depth, T* __restrict__ out_var,
            T* __restrict__ out_dlnl) {
    constexpr int J = Dims<NB>::J;
    constexpr int JJ = Dims<NB>::JJ;
    if ((int)blockIdx.x < n_rest) {
        const int64_t gid = (int64_t)blockIdx.x * TLO + threadIdx.x;
        const int64_t n_tmpl = (s_off ? n_total : n_t0) * (int64_t)n_D;
        if (gid < n_tmpl)
            window_rest<NB, T>(t, t0s, n_t0, k, fv, s_off, n_seg, n_total, Ds, n_D, plan, gid,
                               out_depth, out_var, out_dlnl);
        return;
    }
    extern __shared__ __align__(16) unsigned char sh_raw[];
    T* sm = reinterpret_cast<T*>(sh_raw);
    __shared__ int sh_lblk;
    const int rs = TLO + ch;                  // shared row length (samples)
    T* smF = sm;                              // 4 NB rows
    T* smK = smF + 4 * NB * rs;               // J rows
    T* smD = smK + J * rs;                    // 1/D
    T* smZ = smD + rs;                        // z0
    T* smX = smZ + rs;                        // k rows of Zt
    const int64_t lo0 = (int64_t)(blockIdx.x - n_rest) * TLO;
    const int64_t lo = lo0 + threadIdx.x;
    int seg = 0;
    CurveView cv{0, 0, 0, 0, nullptr};
    int nsteps = 0;
    const int* P = nullptr;
    if (lo < n_total) {
        cv = curve_of(t, t0s, n_t0, s_off, n_seg, n_total, n_D, lo, &seg);
        P = plan + (int64_t)seg * plan_ints(n_D);
        nsteps = (int)min((int64_t)P[0], cv.s0 + cv.n - lo);
    }
    if (threadIdx.x == 0) sh_lblk = 0;
    __syncthreads();
    if (nsteps > 0) atomicMax(&sh_lblk, nsteps);
    __syncthreads();
    const int lblk = sh_lblk;
    const int64_t lo_l = lo - cv.s0;          // window start within the curve
    const int64_t seg_end = cv.s0 + cv.n;
    T s[J];
#pragma unroll
    for (int c = 0; c < J; ++c) s[c] = T(0);
    Acc<T> c2, num, bt[NU_MAX_K];
    c2.init();
    num.init();
#pragma unroll
    for (int a = 0; a < NU_MAX_K; ++a) bt[a].init();
    // the plan's variants in ascending L: lengths, offsets, durations
    const int E0 = NU_WIN_NV * n_D;
    const int n_e = nsteps > 0 ? P[1] : 0;
    int q = 0;
    int next_l = n_e > 0 ? P[2] : INT_MAX;
    for (int m0 = 0; m0 < lblk; m0 += ch) {
        __syncthreads();
        const int64_t base = lo0 + m0;
        const int cnt = (int)min((int64_t)rs, n_total - base);
        stage_rows<T>(fv.F, 4 * NB, base, cnt, smF, rs);
        stage_rows<T>(fv.kg, J, base, cnt, smK, rs);
        stage_rows<T>(fv.invD, 1, base, cnt, smD, rs);
        stage_rows<T>(fv.z0, 1, base, cnt, smZ, rs);
        if (k > 0) stage_rows<T>(fv.Zt, k, base, cnt, smX, rs);
        __syncthreads();
        const int mend = min(ch, lblk - m0);
        for (int mm = 0; mm < mend; ++mm) {
            const int m = m0 + mm;
            if (m >= nsteps) break;
            const int x = threadIdx.x + mm;   // shared column of sample lo + m
            const T e = T(-1) - hdot<NB>(s);
            c2.add(e * e * smD[x]);
            num.add(-smZ[x]);
            for (int a = 0; a < k; ++a) bt[a].add(-smX[a * rs + x]);
            if (lo + m + 1 < seg_end) {
                T tmp[J], Fr[4 * NB];
#pragma unroll
                for (int c = 0; c < J; ++c) tmp[c] = s[c] + smK[c * rs + x] * e;
#pragma unroll
                for (int c = 0; c < 4 * NB; ++c) Fr[c] = smF[c * rs + x + 1];
                apply_F<NB>(Fr, tmp, s);
            }
            // every window of length m + 1 that starts at lo and matches a
            // variant of its duration
            while (next_l == m + 1) {
                const int j = P[2 + 2 * E0 + q];
                const int64_t i = lo_l + P[2 + E0 + q];
                const int64_t hi_l = lo_l + m + 1;
                if (i >= 0 && i < cv.n_t0 &&
                    window_is(t + cv.s0, cv.n, cv.t0[i], Ds[j] * 0.5, lo_l, hi_l)) {
                    T cval = c2.get();
                    if (hi_l < cv.n) {
                        const T* Gh = fv.G + (cv.s0 + hi_l) * JJ;
                        T qf = T(0);
#pragma unroll
                        for (int r = 0; r < J; ++r) {
                            T rowsum = Gh[pk(r, r, J)] * s[r];
#pragma unroll
                            for (int c = r + 1; c < J; ++c) rowsum += T(2) * Gh[pk(r, c, J)] * s[c];
                            qf += s[r] * rowsum;
                        }
                        cval += qf;
                    }
                    T bb = T(0);
                    for (int a = 0; a < k; ++a) bb += bt[a].get() * bt[a].get();
                    const T sch = cval - bb;
                    const int64_t o = cv.out0 + (int64_t)j * cv.n_t0 + i;
                    if (sch > T(0)) {
                        const T nm = num.get();
                        const T r = T(1) / sch;
                        const T dep = nm * r;
                        out_depth[o] = dep;
                        out_var[o] = r;
                        out_dlnl[o] = T(0.5) * nm * dep;
                    } else {
                        out_depth[o] = T(NAN);
                        out_var[o] = T(NAN);
                        out_dlnl[o] = T(NAN);
                    }
                }
                ++q;
                next_l = q < n_e ? P[2 + q] : INT_MAX;
            }
        }
    }
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

// Launch shape of the window-start kernel: TLO starts per block, ch samples
// per staged chunk.  Returns false when the staged rows would not fit.
template <int NB, typename T, int TLO>
static bool launch_lo(const double* t, const double* t0s, int64_t n_t0, int k, FactorView<T> fv,
                      const int64_t* s_off, int n_seg, int64_t n_total, const double* Ds,
                      int n_D, const int* plan, int ch, void* d, void* v, void* l,
                      cudaStream_t st) {
    const size_t smem = (size_t)stage_fields<NB>(k) * (TLO + ch) * sizeof(T);
    if (smem > 200 * 1024) return false;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_window_lo<NB, T, TLO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    const int64_t n_tmpl = (s_off ? n_total : n_t0) * (int64_t)n_D;
    const int n_rest = div_up(n_tmpl, TLO);
    k_window_lo<NB, T, TLO><<<n_rest + div_up(n_total, TLO), TLO, smem, st>>>(
        t, t0s, n_t0, k, fv, s_off, n_seg, n_total, Ds, n_D, plan, ch, n_rest, (T*)d, (T*)v,
        (T*)l);
    return true;
}

template <int NB, typename T>
static bool launch_lo_shape(int tlo, const double* t, const double* t0s, int64_t n_t0, int k,
                            FactorView<T> fv, const int64_t* s_off, int n_seg, int64_t n_total,
                            const double* Ds, int n_D, const int* plan, int ch, void* d, void* v,
                            void* l, cudaStream_t st) {
    if (tlo == 32)
        return launch_lo<NB, T, 32>(t, t0s, n_t0, k, fv, s_off, n_seg, n_total, Ds, n_D, plan,
                                    ch, d, v, l, st);
    if (tlo == 64)
        return launch_lo<NB, T, 64>(t, t0s, n_t0, k, fv, s_off, n_seg, n_total, Ds, n_D, plan,
                                    ch, d, v, l, st);
    if (tlo == 256)
        return launch_lo<NB, T, 256>(t, t0s, n_t0, k, fv, s_off, n_seg, n_total, Ds, n_D, plan,
                                     ch, d, v, l, st);
    return launch_lo<NB, T, 128>(t, t0s, n_t0, k, fv, s_off, n_seg, n_total, Ds, n_D, plan, ch,
                                 d, v, l, st);
}

template <int NB, typename T>
static int launch_window(const nu_factor* f, FactorView<T> fv, const double* t0s, int64_t n_t0,
                         const double* Ds_dev, int n_D, int tmpl, const TmplArgs& ta,
                         const int* plan, const WindowShape& ws, void* d, void* v, void* l,
                         cudaStream_t st) {
    const int64_t total = n_t0 * (int64_t)n_D;
    const int th = 128;
    const int blocks = div_up(total, th);
    int launched = 0;
    if (plan) {
        k_window_variants<<<n_D, NU_WIN_PROBES, 0, st>>>(f->t, t0s, n_t0, nullptr, f->n, Ds_dev,
                                                        n_D, (int*)plan);
        k_window_plan_sort<<<1, 32, 0, st>>>(1, n_D, (int*)plan);
        launched += 2;
        // the window-start kernel also fits the windows outside the plan
        if (launch_lo_shape<NB, T>(ws.tlo, f->t, t0s, n_t0, f->k, fv, nullptr, 1, f->n, Ds_dev,
                                   n_D, plan, ws.ch, d, v, l, st))
            return launched + 1;
    }
    if (tmpl == NU_BOX)
        k_window<NB, T, NU_BOX><<<blocks, th, 0, st>>>(f->t, f->n, f->k, fv, t0s, n_t0, Ds_dev,
                                                      n_D, ta, (T*)d, (T*)v, (T*)l);
    else if (tmpl == NU_TRAPEZOID)
        k_window<NB, T, NU_TRAPEZOID><<<blocks, th, 0, st>>>(
            f->t, f->n, f->k, fv, t0s, n_t0, Ds_dev, n_D, ta, (T*)d, (T*)v, (T*)l);
    else
        k_window<NB, T, NU_LIMB_QUAD><<<blocks, th, 0, st>>>(
            f->t, f->n, f->k, fv, t0s, n_t0, Ds_dev, n_D, ta, (T*)d, (T*)v, (T*)l);
    return launched + 1;
}

// Linear search of packed light curves (batch path); no allocation, no sync.
// plan: plan_ints(n_D) ints per curve of device scratch, or nullptr for the
// per-template kernel alone.
int launch_window_batch(int nb, bool fp64, const double* t, int k, const void* fv,
                        const int64_t* s_off, int n_seg, int64_t n_total, const double* Ds,
                        int n_D, int* plan, const WindowShape& ws, void* d, void* v, void* l,
                        cudaStream_t st) {
    const int64_t total = n_total * (int64_t)n_D;
    const int th = 128;
    const int blocks = div_up(total, th);
    int launched = 0;
    if (plan) {
        k_window_variants<<<(unsigned)((int64_t)n_seg * n_D), NU_WIN_PROBES, 0, st>>>(
            t, nullptr, 0, s_off, n_total, Ds, n_D, plan);
        k_window_plan_sort<<<div_up(n_seg, 128), 128, 0, st>>>(n_seg, n_D, plan);
        launched += 2;
        bool ok = true;
#define NU_WL(NB_, T_)                                                                      \
    ok = launch_lo_shape<NB_, T_>(ws.tlo, t, nullptr, 0, k, *(const FactorView<T_>*)fv, s_off, \
                                  n_seg, n_total, Ds, n_D, plan, ws.ch, d, v, l, st)
        if (fp64) {
            switch (nb) {
                case 1: NU_WL(1, double); break;
                case 2: NU_WL(2, double); break;
                case 3: NU_WL(3, double); break;
                default: NU_WL(4, double); break;
            }
        } else {
            switch (nb) {
                case 1: NU_WL(1, float); break;
                case 2: NU_WL(2, float); break;
                case 3: NU_WL(3, float); break;
                default: NU_WL(4, float); break;
            }
        }
#undef NU_WL
        // the window-start kernel also fits the windows outside the plan
        if (ok) return launched + 1;
    }
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
    return launched + 1;
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
    // box windows on the sample grid take the window-start recursion (a plan
    // of plan_ints(n_D) ints next to the durations); everything else one
    // recursion per template
    const bool use_lo = tmpl == NU_BOX && n_t0 == f->n && n_D <= 4096;
    const size_t ds_bytes = ((size_t)n_D * sizeof(double) + 255) / 256 * 256;
    const size_t bytes = ds_bytes + (use_lo ? (size_t)plan_ints(n_D) * sizeof(int) : 0);
    char* mem = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&mem, bytes, st);
    if (e != cudaSuccess) return cuda_fail(e, "nu_linear_search: cudaMallocAsync");
    double* Ds_dev = (double*)mem;
    int* plan = use_lo ? (int*)(mem + ds_bytes) : nullptr;
    e = cudaMemcpyAsync(Ds_dev, Ds_host, n_D * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
        cudaFreeAsync(mem, st);
        return cuda_fail(e, "nu_linear_search: copy");
    }
    // order the factor's work before ours when the streams differ
    if (f->stream != st) {
        e = cudaEventRecord(f->ready, f->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, f->ready, 0);
        if (e != cudaSuccess) {
            cudaFreeAsync(mem, st);
            return cuda_fail(e, "nu_linear_search: stream order");
        }
    }
    const WindowShape ws = default_window_shape(f->n);
    int launched = 0;
    if (prec == NU_FP64) {
        FactorView<double> fv{f->F, f->kg, f->invD, f->G, f->z0, f->Zt};
        switch (f->nb) {
            case 1: launched = launch_window<1, double>(f, fv, t0s_dev, n_t0, Ds_dev, n_D, tmpl, ta, plan, ws, depth_dev, var_dev, dlnl_dev, st); break;
            case 2: launched = launch_window<2, double>(f, fv, t0s_dev, n_t0, Ds_dev, n_D, tmpl, ta, plan, ws, depth_dev, var_dev, dlnl_dev, st); break;
            case 3: launched = launch_window<3, double>(f, fv, t0s_dev, n_t0, Ds_dev, n_D, tmpl, ta, plan, ws, depth_dev, var_dev, dlnl_dev, st); break;
            default: launched = launch_window<4, double>(f, fv, t0s_dev, n_t0, Ds_dev, n_D, tmpl, ta, plan, ws, depth_dev, var_dev, dlnl_dev, st); break;
        }
    } else {
        FactorView<float> fv{f->F32, f->kg32, f->invD32, f->G32, f->z032, f->Zt32};
        switch (f->nb) {
            case 1: launched = launch_window<1, float>(f, fv, t0s_dev, n_t0, Ds_dev, n_D, tmpl, ta, plan, ws, depth_dev, var_dev, dlnl_dev, st); break;
            case 2: launched = launch_window<2, float>(f, fv, t0s_dev, n_t0, Ds_dev, n_D, tmpl, ta, plan, ws, depth_dev, var_dev, dlnl_dev, st); break;
            case 3: launched = launch_window<3, float>(f, fv, t0s_dev, n_t0, Ds_dev, n_D, tmpl, ta, plan, ws, depth_dev, var_dev, dlnl_dev, st); break;
            default: launched = launch_window<4, float>(f, fv, t0s_dev, n_t0, Ds_dev, n_D, tmpl, ta, plan, ws, depth_dev, var_dev, dlnl_dev, st); break;
        }
    }
    count_launches(launched);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        cudaFreeAsync(mem, st);
        return cuda_fail(e, "nu_linear_search: launch");
    }
    e = cudaFreeAsync(mem, st);
    if (e != cudaSuccess) return cuda_fail(e, "nu_linear_search: cudaFreeAsync");
    return NU_OK;
}

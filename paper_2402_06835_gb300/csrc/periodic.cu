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
#include <mutex>
#include <string>
#include <vector>

#include "fold.cuh"
#include "nu_internal.cuh"

namespace nu {

// ------------------------------------------------------------------ helpers
// Reciprocals from the hardware approximation refined by Newton-Raphson
// (y <- y (2 - x y), each step doubling the correct bits); x > 0 finite.
__device__ __forceinline__ double rcp64(double x) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    double e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    e = fma(-x, y, 1.0);
    return fma(y, e, y);
}
__device__ __forceinline__ float rcp32(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt32(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_32(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}


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

// Per-(duration, epoch) node records for the exact path.
template <typename T>
__device__ __forceinline__ T node_sigma(T d, T v, T l) {
    return (isfinite(d) && isfinite(v) && isfinite(l) && v > T(0)) ? sqrt(v) : T(NAN);
}

template <typename T>
__device__ __forceinline__ Node8<T> make_node8(const T* __restrict__ depth,
                                               const T* __restrict__ var,
                                               const T* __restrict__ gain,
                                               const double* __restrict__ t0, int64_t gid,
                                               int64_t i, int64_t n, double gap_max) {
    Node8<T> r;
    r.d = depth[gid];
    r.l = gain[gid];
    r.s = node_sigma<T>(r.d, var[gid], r.l);
    r.ig = T(NAN);
    r.dd = T(NAN);
    r.ds = T(NAN);
    r.dl = T(NAN);
    r.pad = T(0);
    if (i + 1 < n) {
        const double gap = t0[i + 1] - t0[i];
        if (gap <= gap_max && gap > 0.0) r.ig = (T)(1.0 / gap);
        const T d1 = depth[gid + 1], l1 = gain[gid + 1];
        const T s1 = node_sigma<T>(d1, var[gid + 1], l1);
        r.dd = d1 - r.d;
        r.ds = s1 - r.s;
        r.dl = l1 - r.l;
    }
    return r;
}

template <typename T>
__global__ void k_nodes(const T* __restrict__ depth, const T* __restrict__ var,
                        const T* __restrict__ gain, const double* __restrict__ t0s,
                        int64_t n_t0, int n_D, double gap_max, Node8<T>* __restrict__ nodes) {
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gid >= n_t0 * (int64_t)n_D) return;
    nodes[gid] = make_node8<T>(depth, var, gain, t0s, gid, gid % n_t0, n_t0, gap_max);
}

// Regular-grid test for the slot path: every epoch within 1e-3 slot of
// t_ref + s*dt with strictly increasing slots.  slot_of[i] = s.
__global__ void k_slots(const double* __restrict__ t0s, int64_t n_t0, double t_ref,
                        double inv_dt, int* __restrict__ slot_of, int* __restrict__ irregular) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_t0) return;
    const double u = (t0s[i] - t_ref) * inv_dt;
    const double s = rint(u);
    bool bad = !(fabs(u - s) <= 1e-3) || !(s >= 0.0) || s > 2.0e9;
    if (i > 0) {
        const double up = rint((t0s[i - 1] - t_ref) * inv_dt);
        bad = bad || !(s > up);
    }
    slot_of[i] = bad ? -1 : (int)s;
    if (bad) atomicExch(irregular, 1);
}

// Slot records (mixed path): node values placed at their slot, NaN sigma in
// empty slots.  One thread per (duration, epoch); slots were cleared to NaN.
__global__ void k_slot_fill(const float* __restrict__ depth, const float* __restrict__ var,
                            const float* __restrict__ gain, const int* __restrict__ slot_of,
                            int64_t n_t0, int n_D, int64_t n_slots,
                            Node4<float>* __restrict__ rec) {
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gid >= n_t0 * (int64_t)n_D) return;
    const int64_t d = gid / n_t0, i = gid - d * n_t0;
    const int s = slot_of[i];
    if (s < 0 || s >= n_slots) return;
    const float dd = depth[gid], v = var[gid], l = gain[gid];
    Node4<float> r;
    r.d = dd;
    r.l = l;
    r.s = (isfinite(dd) && isfinite(v) && isfinite(l) && v > 0.f) ? sqrtf(v) : NAN;
    r.ig = 0.f;
    rec[d * n_slots + s] = r;
}

__global__ void k_fill_nan(Node4<float>* rec, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    rec[i] = Node4<float>{NAN, NAN, NAN, 0.f};
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

__device__ __forceinline__ void write_best(const Best& b, int64_t p, int64_t n_phi, double t_ref,
                                           double P, double* Q_out, double* T0_out,
                                           int* Didx_out, double* dep_out, double* sig_out,
                                           double* lnp_out) {
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
        T0_out[p] = __dadd_rn(t_ref, __dmul_rn((double)j / (double)n_phi, P));
        Didx_out[p] = d;
        dep_out[p] = b.depth;
        sig_out[p] = b.sigma;
        lnp_out[p] = b.lnp;
    }
}

// MAXT: the largest block size the caller is launched with
template <int MAXT = 256>
__device__ __forceinline__ Best block_argmax(Best best) {
    __shared__ Best sh[MAXT];
    sh[threadIdx.x] = best;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w && better(sh[threadIdx.x + w], sh[threadIdx.x]))
            sh[threadIdx.x] = sh[threadIdx.x + w];
        __syncthreads();
    }
    return sh[0];
}

// Bound used to skip the second pass of a cell that cannot be the argmax.
// With x_k = sigma^2 / s_k^2 (sum x_k = 1 by Eq. sigma_delta) the log terms of
// Eq. result contribute -1/2 sum ln(s_k^2/(sigma^2+s_k^2)) = 1/2 sum ln(1+x_k)
// <= 1/2 sum x_k = 1/2.  Because sigma^2 <= s_k^2, the depth terms satisfy
//   sum (Delta_k - Delta)^2 / (s_k^2 + sigma^2) >= 1/2 sum (Delta_k - Delta)^2 / s_k^2
//                                          = 1/2 (S_dd - S_d^2 / S_inv)
// with S_dd = sum Delta_k^2 / s_k^2 from the first pass.  Hence
//   ln P <= S_L + 1/2 - 1/4 (S_dd - S_d^2 / S_inv),
// and a cell whose bound is below the best ln P found so far cannot win:
// skipping its second pass changes no result.  The margins (on the bound and
// on the cancellation in S_dd - S_d^2/S_inv) are far above the rounding of
// each precision.
__device__ __forceinline__ bool cannot_win(double s_l, double s_inv, double s_d, double s_dd,
                                           double best) {
    const double q = fmax(0.0, s_dd - s_d * s_d / s_inv - 1e-9 * s_dd);
    const double ub = s_l + 0.5 - 0.25 * q;
    return ub + 1e-6 * fmax(1.0, fabs(ub)) < best;
}

// FP32 form for the mixed kernel, with the tighter depth term
// q / (2 (1 + x_max)), x_max = max_k sigma^2/s_k^2 = ivmax / S_inv <= 1
// (sigma^2 + s_k^2 = s_k^2 (1 + x_k) <= s_k^2 (1 + x_max)).
// The reciprocals are the hardware approximation (2^-21 relative, far inside
// the margins).
__device__ __forceinline__ bool cannot_win_f(float s_l, float s_inv, float s_d, float s_dd,
                                             float ivmax, float best) {
    const float r = rcp32(s_inv);
    const float q = fmaxf(0.0f, s_dd - s_d * s_d * r - 1e-4f * s_dd);
    const float x = fminf(1.0f, ivmax * r * 1.001f);
    const float ub = s_l + 0.5f - 0.5f * q * rcp32(1.0f + x) * 0.9999f;
    return ub + 1e-4f * fmaxf(1.0f, fabsf(ub)) < best;
}

__device__ __forceinline__ bool bad_period(double P, const FoldGeom& g) {
    // a period must be finite, > 0 and give at most 1e9 epochs and phases
    return !(P > 0.0) || !isfinite(P) || g.t_last - g.t_ref > 1.0e9 * P ||
           P / g.dt > 1.0e9;
}

__device__ __forceinline__ void write_bad(int64_t p, double* Q_out, double* T0_out,
                                          int* Didx_out, double* dep_out, double* sig_out,
                                          double* lnp_out) {
    Q_out[p] = NAN;
    T0_out[p] = NAN;
    Didx_out[p] = -1;
    dep_out[p] = NAN;
    sig_out[p] = NAN;
    lnp_out[p] = NAN;
}

// ------------------------------------------------ exact path (FP64 epochs)
// Order-preserving integer key of a non-NaN double (so comparisons of times
// run on the integer pipe; -0.0 never occurs among the epochs compared here).
__device__ __forceinline__ long long okey(double x) {
    const long long b = __double_as_longlong(x);
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}

// largest i with t0[i] <= T starting from a guess (exact)
__device__ __forceinline__ int64_t bracket_from(const FoldGeom& g, long long kT, int64_t i) {
    while (i + 1 < g.n_t0 && okey(g.t0s[i + 1]) <= kT) ++i;
    while (i > 0 && okey(g.t0s[i]) > kT) --i;
    return i;
}

__device__ __forceinline__ bool nan64(double x) {
    return (__double_as_longlong(x) & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL;
}

__device__ __forceinline__ int64_t bracket_guess(const FoldGeom& g, double T) {
    int64_t b = (int64_t)((T - g.t_ref) * g.inv_dt);
    b = b < 0 ? 0 : (b >= g.n_bucket ? g.n_bucket - 1 : b);
    const int64_t i = (int64_t)g.bucket[b] - 1;
    return i < 0 ? 0 : i;
}

template <typename T> __device__ __forceinline__ T rcp_t(T x);
template <> __device__ __forceinline__ double rcp_t<double>(double x) { return rcp64(x); }
template <> __device__ __forceinline__ float rcp_t<float>(float x) { return rcp32(x); }

// One single event at epoch Tk: interpolated depth, variance and gain.
template <typename T>
__device__ __forceinline__ bool event_exact(const FoldGeom& g, const Node8<T>* __restrict__ nd,
                                            double Tk, int64_t& i, T& dk, T& sk2, T& lk) {
    i = bracket_from(g, okey(Tk), i);
    const Node8<T> a = nd[i];
    const T w = (T)((Tk - g.t0s[i]) * (double)a.ig);   // NaN across a gap / at the end
    const T s = fma(w, a.ds, a.s);
    if (sizeof(T) == 8 ? nan64((double)s) : isnan(s)) return false;
    dk = fma(w, a.dd, a.d);
    lk = fma(w, a.dl, a.l);
    sk2 = s * s;
    return true;
}

// Fixed-point (24.40) walk of the slot grid u = (T - t_ref)/dt used to guess
// brackets; the decisions themselves are FP64 comparisons with T.
struct SlotWalk {
    unsigned long long u0, ustep;
};
__device__ __forceinline__ SlotWalk slot_walk(double phi, double R) {
    const double SCALE = 1099511627776.0;   // 2^40
    SlotWalk w;
    const double a = phi * R * SCALE, b = R * SCALE;
    w.u0 = a < 4.0e18 ? (unsigned long long)llrint(a) : 4000000000000000000ull;
    w.ustep = b < 4.0e18 ? (unsigned long long)llrint(b) : 4000000000000000000ull;
    return w;
}
__device__ __forceinline__ int64_t guess_at(const FoldGeom& g, unsigned long long u) {
    int64_t b = (int64_t)(u >> 40);
    b = b >= g.n_bucket ? g.n_bucket - 1 : b;
    const int64_t i = (int64_t)g.bucket[b] - 1;
    return i < 0 ? 0 : i;
}

template <typename T>
struct ExactAcc {
    KSum<T> s_inv, s_d, s_l;
    T s_dd;                // sum Delta_k^2 / s_k^2 (bound only, plain sum)
    int K;
    __device__ __forceinline__ void init() {
        s_inv.init();
        s_d.init();
        s_l.init();
        s_dd = T(0);
        K = 0;
    }
    __device__ __forceinline__ void add(T dk, T sk2, T lk) {
        const T iv = rcp_t<T>(sk2);
        const T div = dk * iv;
        s_inv.add(iv);
        s_d.add(div);
        s_dd = fma(div, dk, s_dd);
        s_l.add(lk);
        ++K;
    }
    __device__ __forceinline__ bool cannot_win(double best) const {
        return nu::cannot_win((double)s_l.s, (double)s_inv.s, (double)s_d.s, (double)s_dd,
                              best);
    }
};

// second sum of Eq. result: ln s_k^2 - ln(sigma^2 + s_k^2) accumulated as the
// log of a product of ratios in [1/2, 1] (renormalised), plus
// (Delta_k - Delta)^2 / (s_k^2 + sigma^2)
template <typename T>
struct ExactPen {
    KSum<T> quad;
    double prod;
    int expo, cnt;
    float lsum;
    T s2, Dl;
    __device__ __forceinline__ void init(T s2_, T Dl_) {
        quad.init();
        prod = 1.0;
        expo = 0;
        cnt = 0;
        lsum = 0.f;
        s2 = s2_;
        Dl = Dl_;
    }
    __device__ __forceinline__ void add(T dk, T sk2) {
        const T den = sk2 + s2;
        const T iden = rcp_t<T>(den);
        const T r = dk - Dl;
        quad.add(r * r * iden);
        if (sizeof(T) == 8) {
            prod *= (double)(sk2 * iden);
            if ((++cnt & 255) == 0) {
                const int e = ((__double2hiint(prod) >> 20) & 0x7ff) - 1023;
                prod = __hiloint2double(__double2hiint(prod) - (e << 20), __double2loint(prod));
                expo += e;
            }
        } else {
            lsum += lg2_32((float)(sk2 * iden));
        }
    }
    __device__ __forceinline__ double logsum() const {
        if (sizeof(T) == 8) return log(prod) + (double)expo * 0.69314718055994530942;
        return (double)lsum * 0.69314718055994530942;
    }
};

// Order-preserving unsigned key of a non-NaN double, for a shared atomic max.
__device__ __forceinline__ unsigned long long max_key(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double from_max_key(unsigned long long k) {
    const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)b);
}

// A cell that survived the bound after its first pass, queued for the second.
template <typename T>
struct QCell {
    double phi;
    unsigned long long u0;
    long long cell;
    double s_l;
    T s2, Dl;
    int d;
    int kmax;
};

// Per-period constants of the exact evaluation of a cell.
struct CellCtx {
    double P, nphi_d, rphi;
    SlotWalk swp, swk;         // per-phase and per-epoch steps of the slot guess
    unsigned long long ulast;  // t_last on the same fixed-point scale
    float inv_ustep32;
    long long klast;           // order key of t_last
};

__device__ __forceinline__ CellCtx cell_ctx(const FoldGeom& g, double P, int64_t n_phi) {
    CellCtx c;
    c.P = P;
    const double R = P * g.inv_dt;
    c.swp = slot_walk(1.0 / (double)n_phi, R);
    c.swk = slot_walk(0.0, R);
    const double SCALE = 1099511627776.0;   // 2^40
    const double ulast_d = (g.t_last - g.t_ref) * g.inv_dt * SCALE;
    c.ulast = ulast_d < 4.0e18 ? (unsigned long long)llrint(ulast_d) : 4000000000000000000ull;
    c.inv_ustep32 = (float)(4294967296.0 / (double)c.swk.ustep);
    c.klast = okey(g.t_last);
    // phase j / n_phi: reciprocal plus one FMA correction of the quotient
    // (Markstein 1990), instead of a division per cell
    c.nphi_d = (double)n_phi;
    c.rphi = 1.0 / c.nphi_d;
    return c;
}

// The constants of one period that do not depend on the curve (phase count,
// fixed-point walk steps and their reciprocals), computed as screen_period
// and cell_ctx compute them.  The batched fold takes them from a table built
// once per call, so that its (curve, period) items, bound by the FP64 pipe
// when their cells are short, skip these divisions.
struct PeriodConst {
    int64_t n_phi;
    double R;                          // P / dt
    unsigned long long ustep, uph;     // screen steps (0 when R 2^40 >= 4e18)
    float inv_ustep32;
    float c_inv_ustep32;
    SlotWalk swp, swk;
    double nphi_d, rphi;
};

// The table entry of period P (P must not be a bad period of the curves).
__device__ __forceinline__ PeriodConst period_const(double P, double dt, double inv_dt) {
    PeriodConst pc;
    const double SCALE = 1099511627776.0;   // 2^40
    pc.n_phi = (int64_t)ceil(P / dt);
    pc.R = P * inv_dt;
    if (pc.R * SCALE < 4.0e18) {
        pc.ustep = (unsigned long long)llrint(pc.R * SCALE);
        pc.uph = (unsigned long long)llrint(pc.R / (double)pc.n_phi * SCALE);
        pc.inv_ustep32 = (float)(4294967296.0 / (double)pc.ustep);
    } else {
        pc.ustep = pc.uph = 0;
        pc.inv_ustep32 = 0.f;
    }
    pc.swp = slot_walk(1.0 / (double)pc.n_phi, pc.R);
    pc.swk = slot_walk(0.0, pc.R);
    pc.c_inv_ustep32 = (float)(4294967296.0 / (double)pc.swk.ustep);
    pc.nphi_d = (double)pc.n_phi;
    pc.rphi = 1.0 / pc.nphi_d;
    return pc;
}

// cell_ctx from a table entry (the same values).
__device__ __forceinline__ CellCtx cell_ctx(const FoldGeom& g, double P, const PeriodConst& pc) {
    CellCtx c;
    c.P = P;
    c.swp = pc.swp;
    c.swk = pc.swk;
    const double SCALE = 1099511627776.0;   // 2^40
    const double ulast_d = (g.t_last - g.t_ref) * g.inv_dt * SCALE;
    c.ulast = ulast_d < 4.0e18 ? (unsigned long long)llrint(ulast_d) : 4000000000000000000ull;
    c.inv_ustep32 = pc.c_inv_ustep32;
    c.klast = okey(g.t_last);
    c.nphi_d = pc.nphi_d;
    c.rphi = pc.rphi;
    return c;
}

// Table of period constants (invalid periods get placeholder entries; the
// folds test a period before they read its entry).
__global__ void k_period_consts(const double* __restrict__ periods, int64_t n_P, double dt,
                                PeriodConst* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_P) return;
    const double P = periods[i];
    if (!(P > 0.0) || !isfinite(P) || P / dt > 1.0e9) {
        out[i] = PeriodConst{1, 0.0, 0, 0, 0.f, 0.f, {0, 0}, {0, 0}, 1.0, 1.0};
        return;
    }
    out[i] = period_const(P, dt, 1.0 / dt);
}

// Per-period constants of the slot path: phases, and the epoch and phase
// steps in 24.40 fixed point.  The single-curve fold computes them per block;
// the batch reads them from a table filled by the same function
// (k_slot_periods), so both fold a curve identically.  bad marks a period
// that is not folded for any curve (the curve's own limit, a span of more
// than 1e9 periods, is tested per curve).
struct SlotPeriod {
    int64_t n_phi;
    unsigned long long ustep, uph;
    int bad;
};
// The position of a curve's last epoch (< 2^62 by the host's span check).
__host__ __device__ inline unsigned long long slot_ulast(double t_ref, double t_last, double dt) {
    return (unsigned long long)llrint((t_last - t_ref) / dt * 1099511627776.0);
}
__device__ __forceinline__ SlotPeriod slot_period(double P, double dt) {
    SlotPeriod sp{1, 0ull, 0ull, 1};
    if (!(P > 0.0) || !isfinite(P) || P / dt > 1.0e9) return sp;
    const double SCALE = 1099511627776.0;                      // 2^40
    const double R = P / dt;                                   // slots per period
    sp.n_phi = (int64_t)ceil(R);
    sp.ustep = R * SCALE < 4.0e18 ? (unsigned long long)llrint(R * SCALE)
                                  : 4000000000000000000ull;
    // phase j starts at j * (R / n_phi) slots; per-cell work stays integer
    sp.uph = (unsigned long long)llrint(R / (double)sp.n_phi * SCALE);
    sp.bad = 0;
    return sp;
}
__global__ void k_slot_periods(const double* __restrict__ periods, int64_t n_P, double dt,
                               SlotPeriod* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n_P) out[i] = slot_period(periods[i], dt);
}

size_t period_const_bytes() {
    return sizeof(PeriodConst) > sizeof(SlotPeriod) ? sizeof(PeriodConst) : sizeof(SlotPeriod);
}

__device__ __forceinline__ double cell_phi(const CellCtx& c, int64_t j) {
    const double jd = (double)j;
    const double q0 = jd * c.rphi;
    return fma(fma(-q0, c.nphi_d, jd), c.rphi, q0);
}

__device__ __forceinline__ double epoch_time(const FoldGeom& g, const CellCtx& c, double phi,
                                             double kd) {
    return __dadd_rn(g.t_ref, __dmul_rn(__dadd_rn(phi, kd), c.P));
}

// number of epochs with T <= t_last: integer estimate, then the exact
// comparisons of the definition
__device__ __forceinline__ int64_t cell_kmax(const FoldGeom& g, const CellCtx& c, double phi,
                                             unsigned long long u0) {
    int64_t kk = u0 > c.ulast ? 0
                              : (int64_t)((float)(unsigned)((c.ulast - u0) >> 32) *
                                          c.inv_ustep32) + 1;
    while (kk > 0 && okey(epoch_time(g, c, phi, (double)(kk - 1))) > c.klast) --kk;
    while (okey(epoch_time(g, c, phi, (double)kk)) <= c.klast) ++kk;
    return kk;
}

// First and second sums of one cell over epochs k0, k0 + ks, ... < kmax.
template <typename T>
__device__ __forceinline__ void cell_pass1(const FoldGeom& g, const Node8<T>* __restrict__ nd,
                                           const CellCtx& c, double phi, unsigned long long u0,
                                           int64_t kmax, int k0, int ks, ExactAcc<T>& a1) {
    unsigned long long u = u0 + (unsigned long long)k0 * c.swk.ustep;
    const unsigned long long us = (unsigned long long)ks * c.swk.ustep;
    double kd = (double)k0;
    const double kds = (double)ks;
    for (int64_t k = k0; k < kmax; k += ks, u += us, kd += kds) {
        const double Tk = epoch_time(g, c, phi, kd);
        T dk, sk2, lk;
        int64_t i = guess_at(g, u);
        if (event_exact<T>(g, nd, Tk, i, dk, sk2, lk)) a1.add(dk, sk2, lk);
    }
}
template <typename T>
__device__ __forceinline__ void cell_pass2(const FoldGeom& g, const Node8<T>* __restrict__ nd,
                                           const CellCtx& c, double phi, unsigned long long u0,
                                           int64_t kmax, int k0, int ks, ExactPen<T>& a2) {
    unsigned long long u = u0 + (unsigned long long)k0 * c.swk.ustep;
    const unsigned long long us = (unsigned long long)ks * c.swk.ustep;
    double kd = (double)k0;
    const double kds = (double)ks;
    for (int64_t k = k0; k < kmax; k += ks, u += us, kd += kds) {
        const double Tk = epoch_time(g, c, phi, kd);
        T dk, sk2, lk;
        int64_t i = guess_at(g, u);
        if (event_exact<T>(g, nd, Tk, i, dk, sk2, lk)) a2.add(dk, sk2);
    }
}

// One period P of one light curve: every (duration, phase) cell, then the
// block argmax; results at index p of the outputs.  Called by all threads of
// the block.  Cells are processed in waves of blockDim: every thread runs the
// first pass of one cell, the cells whose bound can still beat the block's
// best are compacted into a shared queue, and the queue's second passes run
// densely (a warp instruction costs the same however many lanes are active).
template <typename T, int KC, int MAXT = 256>
__device__ __forceinline__ void fold_exact_one(const FoldGeom& g, const Node8<T>* __restrict__ nodes,
                                               int n_D, double P, int64_t p,
                                               double* __restrict__ Q_out,
                                               double* __restrict__ T0_out,
                                               int* __restrict__ Didx_out,
                                               double* __restrict__ dep_out,
                                               double* __restrict__ sig_out,
                                               double* __restrict__ lnp_out) {
    __shared__ QCell<T> sh_q[MAXT];
    __shared__ int sh_nq;
    __shared__ unsigned long long sh_best;
    if (bad_period(P, g)) {
        if (threadIdx.x == 0) write_bad(p, Q_out, T0_out, Didx_out, dep_out, sig_out, lnp_out);
        return;
    }
    const int64_t n_phi = (int64_t)ceil(P / g.dt);
    const int64_t n_cells = n_phi * n_D;
    const CellCtx c = cell_ctx(g, P, n_phi);
    double bl = -INFINITY;
    long long bc = LLONG_MAX;
    T bD = T(NAN), bs2 = T(NAN);
    if (threadIdx.x == 0) {
        sh_nq = 0;
        sh_best = max_key(-INFINITY);
    }
    __syncthreads();
    // cells walk (duration, phase) incrementally: no 64-bit division per cell
    int d = (int)(threadIdx.x / n_phi);
    int64_t j = (int64_t)threadIdx.x - (int64_t)d * n_phi;
    for (int64_t base = 0; base < n_cells; base += blockDim.x, j += blockDim.x) {
        while (j >= n_phi) {
            j -= n_phi;
            ++d;
        }
        const int64_t cell = base + threadIdx.x;
        if (cell < n_cells) {
            const double phi = cell_phi(c, j);
            const Node8<T>* nd = nodes + (int64_t)d * g.n_t0;
            const unsigned long long u0 = (unsigned long long)j * c.swp.u0;
            const int64_t kmax = cell_kmax(g, c, phi, u0);
            ExactAcc<T> a1;
            a1.init();
            cell_pass1<T>(g, nd, c, phi, u0, kmax, 0, 1, a1);
            const double best_now = fmax(bl, from_max_key(sh_best));
            if (a1.K > 0 && !a1.cannot_win(best_now)) {
                const T s2 = T(1) / a1.s_inv.s;
                const int q = atomicAdd(&sh_nq, 1);
                sh_q[q] = QCell<T>{phi, u0, (long long)cell, (double)a1.s_l.s, s2,
                                   s2 * a1.s_d.s, d, (int)kmax};
            }
        }
        __syncthreads();
        const int nq = sh_nq;
        for (int q = threadIdx.x; q < nq; q += blockDim.x) {
            const QCell<T> qc = sh_q[q];
            const Node8<T>* nd = nodes + (int64_t)qc.d * g.n_t0;
            ExactPen<T> a2;
            a2.init(qc.s2, qc.Dl);
            cell_pass2<T>(g, nd, c, qc.phi, qc.u0, qc.kmax, 0, 1, a2);
            const double lnp = qc.s_l - 0.5 * (a2.logsum() + (double)a2.quad.s);
            if (!(lnp == lnp)) continue;   // NaN never selected
            if (lnp > bl || (lnp == bl && qc.cell < bc)) {
                bl = lnp;
                bc = qc.cell;
                bD = qc.Dl;
                bs2 = qc.s2;
            }
            atomicMax(&sh_best, max_key(lnp));
        }
        __syncthreads();
        if (threadIdx.x == 0) sh_nq = 0;
        __syncthreads();
    }
    Best best{-INFINITY, LLONG_MAX, NAN, NAN};
    if (bc != LLONG_MAX) best = Best{bl, bc, (double)bD, sqrt((double)bs2)};
    const Best b = block_argmax<MAXT>(best);
    if (threadIdx.x == 0)
        write_best(b, p, n_phi, g.t_ref, P, Q_out, T0_out, Didx_out, dep_out, sig_out, lnp_out);
}

// The period a block (or a batch item) folds.  Short periods hold few cells
// of many epochs each, and in the FP64 fold they are the longest blocks: a
// grid whose periods run downwards (uniform in frequency, say) is folded from
// its far end, so that those blocks start first (C2 FP64: 8.5 ms in
// ascending order, 13.8 ms descending).  Any order gives the same results.
__device__ __forceinline__ int64_t period_slot(int64_t b, const double* __restrict__ periods,
                                              int64_t n_P) {
    return periods[n_P - 1] < periods[0] ? n_P - 1 - b : b;
}

template <typename T, int KC>
__global__ void __launch_bounds__(256)
k_fold_exact(FoldGeom g, const Node8<T>* __restrict__ nodes, int n_D,
             const double* __restrict__ periods, int64_t n_P, double* __restrict__ Q_out,
             double* __restrict__ T0_out, int* __restrict__ Didx_out,
             double* __restrict__ dep_out, double* __restrict__ sig_out,
             double* __restrict__ lnp_out) {
    if ((int64_t)blockIdx.x >= n_P) return;
    const int64_t p = period_slot(blockIdx.x, periods, n_P);
    fold_exact_one<T, KC>(g, nodes, n_D, periods[p], p, Q_out, T0_out, Didx_out, dep_out,
                          sig_out, lnp_out);
}

// ------------------------------ FP64 path: FP32 screen, exact survivors
// Every cell is first screened with FP32 events: an upper bound on its ln P
// (the bound of cannot_win, tightened below) computed from FP32 values with
// an error term that covers every rounding of the screen, on an epoch set
// that is provably the exact path's.  Only cells whose bound reaches the
// best ln P found so far are evaluated exactly (FP64 epochs and values, the
// same code as the exact path); a skipped cell cannot be the argmax, so the
// outputs are those of the exact evaluation of every cell.
//
// Tighter bound.  With x_k = sigma^2/s_k^2 and x_max = max_k x_k,
//   sum (Delta_k - Delta)^2/(s_k^2 + sigma^2) >= q / (1 + x_max),
//   q = sum (Delta_k - Delta)^2 / s_k^2 = S_dd - S_d^2/S_inv,
// so ln P <= S_L + 1/2 - q / (2 (1 + x_max)).
//
// Epoch set.  Epoch positions are walked in 24.40 fixed point of the slot
// grid (u = (T - t_ref)/dt), the epochs' own positions are stored on the same
// scale, and the interval of an event is the last epoch position <= u.  The
// walk differs from the FP64 epochs by at most e_pos (bounded per period
// from the fixed-point rounding and the FP64 rounding of T), so the interval
// is the exact path's whenever u is farther than delta >> e_pos from every
// epoch; within delta of an epoch (or of t_last, for the epoch count) the
// event's T is computed in FP64 exactly as the exact path does and the
// interval is taken by the same comparisons.  The screen's epoch set and
// intervals are therefore the exact path's.
//
// Error term.  An FP32 event value x (depth, sigma, gain) differs from the
// FP64 one by at most cv (|x_i| + |x_{i+1}|) (node and slope rounding,
// weight rounding and position error, the FMA; an event in the band of an
// epoch takes its exact interval and an FP32 weight within 5u of the exact
// one), with |x_i| + |x_{i+1}| <=
// 2|x| + |x_{i+1} - x_i| accumulated per cell.  Intervals whose end sigmas
// differ by more than a factor 3 (or outside the other limits of the
// screening record) are not screened, so |ds|/s <= 2 and the
// relative error of each 1/s_k^2 is at most gam = 2.2 cv (2 + 2) + 6u; sums
// of K positive terms carry at most (K + 2)u.  With these:
//   S_L     <= sl + (cv + (K+2)u) sum (2|l_k| + |dl_k|)
//   sqrt(q) >= sqrt(q_fp32_lo / (1 + gam + (K+2)u)) - cv sqrt(sum a_k^2/s_k^2)
//   x_max   <= min(1, ivmax/sinv (1 + 4 gam + 2(K+2)u))
// (triangle inequality in the 1/s^2-weighted norm for q).  Overflow or NaN
// anywhere makes the bound +inf or NaN, which never skips a cell.


struct ScreenGeom {
    const ScreenRec* rec;              // duration-major rows of n_t0 records
    const ulonglong2* vpair;           // (position of epoch i, of epoch i+1), 24.40
                                       // slots from t_ref; the last .y is 2^64 - 1
    const ScreenRec* srec;             // the same records placed at their epochs'
                                       // slots: duration-major rows of n_slots
    int64_t n_slots;
    const unsigned* reg;               // [0]: an epoch is off the slot grid,
                                       // [1]: max |offset from its slot| (float bits)
    int on;                            // screening allowed for this curve
    const unsigned long long* peak;    // key of the largest finite gain (k_gain_peak);
                                       // 0: none
    const float* lm3;                  // grouped gain table (k_lmax3 of the interval gains)
};

// Node sigma of one (duration, epoch) in FP64 (NaN when invalid).
template <typename T>
__device__ __forceinline__ double sigma_at(const T* depth, const T* var, const T* gain,
                                           int64_t o) {
    return (double)node_sigma<T>(depth[o], var[o], gain[o]);
}

// Slot of every epoch on the regular grid u = (t0 - t_ref)/dt and the largest
// offset from it; reg[0] is set when the slots are not strictly increasing
// or fall outside [0, n_slots).  reg must be zero on entry.
__device__ __forceinline__ void slot_offset(const double* __restrict__ t0, int64_t i,
                                            double inv_dt, int64_t n_slots,
                                            int* __restrict__ slot_of,
                                            unsigned* __restrict__ reg) {
    const double u = (t0[i] - t0[0]) * inv_dt;
    const double s = rint(u);
    bool bad = !(s >= 0.0) || !(s < (double)n_slots);
    if (i > 0) bad = bad || !(s > rint((t0[i - 1] - t0[0]) * inv_dt));
    slot_of[i] = bad ? -1 : (int)s;
    if (bad) atomicOr(&reg[0], 1u);
    atomicMax(&reg[1], __float_as_uint((float)fabs(u - s) * 1.0001f));
}

__global__ void k_slot_offsets(const double* __restrict__ t0s, int64_t n_t0, double inv_dt,
                               int64_t n_slots, int* __restrict__ slot_of,
                               unsigned* __restrict__ reg) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_t0) return;
    slot_offset(t0s, i, inv_dt, n_slots, slot_of, reg);
}

// Screening record of epoch i of a curve with n epochs (gid indexes the
// (duration, epoch) arrays; d is the duration), also placed at the epoch's
// slot, and for the first duration row the pair of epoch positions.
template <typename T>
__device__ __forceinline__ void make_screen(const T* __restrict__ depth,
                                            const T* __restrict__ var,
                                            const T* __restrict__ gain,
                                            const double* __restrict__ t0, int64_t gid,
                                            int64_t i, int64_t n, int64_t d, double gap_max,
                                            double dt, ScreenRec* __restrict__ out,
                                            ScreenRec* __restrict__ sout,
                                            float* __restrict__ lint, int64_t n_slots, const int* __restrict__ slot_of,
                                            ulonglong2* __restrict__ vpair) {
    // an interval needs both ends valid and a gap in (0, gap_max]
    bool v0 = i + 1 < n;
    if (v0) {
        const double gap = t0[i + 1] - t0[i];
        v0 = gap > 0.0 && gap <= gap_max && !isnan(sigma_at<T>(depth, var, gain, gid)) &&
             !isnan(sigma_at<T>(depth, var, gain, gid + 1));
    }
    ScreenRec r;
    unsigned flags = 0u;
    float lmax = 0.f;      // largest gain an event on the interval can take
    const double d0 = (double)depth[gid], l0 = (double)gain[gid];
    r.d = (float)d0;
    r.l = (float)l0;
    if (v0) {
        const double s0 = sigma_at<T>(depth, var, gain, gid);
        const double s1 = sigma_at<T>(depth, var, gain, gid + 1);
        const double d1 = (double)depth[gid + 1], l1 = (double)gain[gid + 1];
        const double gap = t0[i + 1] - t0[i];
        r.s = (float)s0;
        r.dd = (float)(d1 - d0);
        r.ds = (float)(s1 - s0);
        r.dl = (float)(l1 - l0);
        r.wsc = (float)(2.384185791015625e-07 * dt / gap);   // 2^-22 dt / gap
        // outside the error model: very close epochs, or values whose FP32
        // sums could overflow
        const bool odd = gap < 0.25 * dt || !(s0 >= 1e-12 && s0 <= 1e12) ||
                         !(s1 >= 1e-12 && s1 <= 1e12) || !(s1 <= 3.0 * s0) ||
                         !(s0 <= 3.0 * s1) || !(fabs(d0) <= 1e8 * s0) ||
                         !(fabs(d1) <= 1e8 * s1) || !(fabs(l0) <= 1e20) || !(fabs(l1) <= 1e20);
        if (odd) {
            // sigma +inf marks the interval for the screen (flags for the
            // exact events)
            flags = 1u;
            r.s = INFINITY;
            r.ds = 0.f;
        }
        // the exact event's gain fma(w, l1 - l0, l0) with w in [0, 1] (to a few
        // units of FP64 rounding) is at most max(l0, l1) + 2^-50 (|l0| + |l1|);
        // rounded up, and +inf when the interval is not screened
        lmax = odd ? INFINITY
                   : __double2float_ru(fmax(0.0, fmax(l0, l1)) +
                                       8.881784197001252e-16 * (fabs(l0) + fabs(l1)));
    } else {
        r.s = NAN;
        r.dd = 0.f;
        r.ds = 0.f;
        r.dl = 0.f;
        r.wsc = 0.f;
    }
    r.flags = flags;
    out[gid] = r;
    const int sl = slot_of[i];
    if (sl >= 0 && sl < n_slots) {
        sout[d * n_slots + sl] = r;
        lint[d * n_slots + sl] = lmax;
    }
    if (d == 0) {
        auto pos = [&](int64_t k) -> unsigned long long {
            const double v = (t0[k] - t0[0]) / dt * 1099511627776.0;
            return v < 9.0e18 ? (unsigned long long)llrint(v) : 9000000000000000000ull;
        };
        vpair[i] = make_ulonglong2(pos(i), i + 1 < n ? pos(i + 1) : ~0ull);
    }
}

// Slot records start as invalid intervals (slots without an epoch).
__global__ void k_fill_screen(ScreenRec* __restrict__ rec, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    rec[i] = ScreenRec{0.f, NAN, 0.f, 0.f, 0.f, 0.f, 0.f, 0u};
}

template <typename T>
__global__ void k_screen(const T* __restrict__ depth, const T* __restrict__ var,
                         const T* __restrict__ gain, const double* __restrict__ t0s,
                         int64_t n_t0, int n_D, double gap_max, double dt,
                         ScreenRec* __restrict__ rec, ScreenRec* __restrict__ srec,
                         float* __restrict__ lint, int64_t n_slots,
                         const int* __restrict__ slot_of, ulonglong2* __restrict__ vpair) {
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gid >= n_t0 * (int64_t)n_D) return;
    const int64_t d = gid / n_t0, i = gid - d * n_t0;
    make_screen<T>(depth, var, gain, t0s, gid, i, n_t0, d, gap_max, dt, rec, srec, lint, n_slots,
                   slot_of, vpair);
}

// Entry o of a grouped gain table: the curve (segs: the batch's, else one
// curve of n_slots1 slots), the source row's duration d and slot s.  Per
// curve the table holds [groups][n_slots][W] entries from gain_off on; the
// source rows are duration-major rows of n_slots from srec_off (FP64) or
// rec_off (mixed).  Returns false for entries of no curve.
struct GainSlot {
    int64_t src_off, n_slots;
    int d, s;
};
__device__ __forceinline__ bool gain_slot(const FoldSeg* __restrict__ segs, int n_seg,
                                          int64_t n_slots1, int n_D, bool fp64, int64_t o,
                                          GainSlot& gs) {
    int64_t out_off = 0;
    gs.src_off = 0;
    gs.n_slots = n_slots1;
    if (segs) {
        // the last curve whose table starts at or before o (curves without a
        // table take no entries and share their successor's offset)
        int lo = 0, hi = n_seg;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (segs[mid].gain_off <= o) lo = mid; else hi = mid;
        }
        const FoldSeg& f = segs[lo];
        if (!(fp64 ? f.screen : f.use_slots)) return false;
        out_off = f.gain_off;
        gs.src_off = fp64 ? f.srec_off : f.rec_off;
        gs.n_slots = f.n_slots;
    }
    const int W = gain_width(n_D);
    const int64_t local = o - out_off;
    if (local < 0 || local >= gs.n_slots * gain_cols(n_D)) return false;
    const int64_t g = local / (gs.n_slots * W);
    const int64_t rem = local - g * gs.n_slots * W;
    gs.s = (int)(rem / W);
    gs.d = (int)(g * W + (rem - (int64_t)gs.s * W));
    return true;
}

// Grouped gain table of the FP64 screen: the maximum of lint over slots
// s - 1, s and s + 1 of the row: the largest gain of an event whose walk
// position lies in slot s (its interval starts at the epoch of slot s - 1, s
// or s + 1, see the gain bound).
__global__ void k_lmax3(const float* __restrict__ lint, const FoldSeg* __restrict__ segs,
                        int n_seg, int64_t n_slots1, int n_D, int64_t n_out,
                        float* __restrict__ lm3) {
    const int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (o >= n_out) return;
    GainSlot gs;
    if (!gain_slot(segs, n_seg, n_slots1, n_D, true, o, gs)) return;
    float m = 0.f;
    if (gs.d < n_D) {
        const float* r = lint + gs.src_off + (int64_t)gs.d * gs.n_slots;
        m = r[gs.s];
        if (gs.s > 0) m = fmaxf(m, r[gs.s - 1]);
        if (gs.s + 1 < gs.n_slots) m = fmaxf(m, r[gs.s + 1]);
    }
    lm3[o] = m;
}

// Per-period constants of the screen.
struct ScreenPeriod {
    unsigned long long uph, ustep, ulast, delta;
    unsigned long long uend;   // epochs walk while u < uend = ulast + delta
    float inv_ustep32;
    float wscale;   // 2^22 / dt (FP32): weight of an event in the band of an epoch
    float cv;       // error coefficient of an FP32 event value
    float dw;       // half-width of the band around an epoch, as an interval weight
    float hw;       // 1/2 - dw: an event is in a band when |w - 1/2| > hw
    bool on;
    bool slots;     // regular grid: events from the slot records
};

// The curve-dependent constants of the screen (the walk's error bound, the
// band around epochs, the regular-grid test); sp holds the period's steps.
__device__ __forceinline__ ScreenPeriod screen_period_curve(const FoldGeom& g,
                                                            const ScreenGeom& sg, double P,
                                                            int64_t n_phi, double R,
                                                            double span, ScreenPeriod sp) {
    const double SCALE = 1099511627776.0;   // 2^40
    sp.ulast = sg.vpair[g.n_t0 - 1].x;
    // position error of the walk against the FP64 epochs, in 2^-40 slots:
    // half a unit per phase and epoch step, the rounding of T, t0 and vpos
    const double kb = span / R + 2.0;
    const double e_pos = 0.5 * ((double)n_phi + kb) + 4.0 +
                         8.881784197001252e-16 * (fabs(g.t_ref) + fabs(g.t_last) + P) *
                             g.inv_dt * SCALE;
    const double delta = 16.0 * e_pos + 1048576.0;          // + 2^-20 slot
    sp.on = delta < 1.6e10;                                  // below 2^-6 slot
    sp.delta = (unsigned long long)delta;
    sp.uend = sp.ulast + sp.delta;
    // regular grid: every epoch within 2^-10 slot of its own slot.  The error
    // terms below grow with the largest offset; a phase step taken as the
    // median spacing of FP64 times carries a relative rounding of about
    // 1e-11, so on long curves (seven sectors: 1.2e-7 slot) the offsets are
    // well above the rounding of one sector's times.
    const float off = sg.srec ? __uint_as_float(sg.reg[1]) : 1.f;
    sp.slots = sg.srec && sg.reg[0] == 0u && off <= 9.765625e-04f;
    double e_w;
    if (sp.slots) {
        // the weight is the fraction of the slot: position error, the
        // epochs' offsets (3 x, both ends), 24-bit truncation
        sp.dw = (float)(1.01 * (delta / SCALE + (double)off) + 2.4e-7);
        e_w = e_pos / SCALE + 3.0 * (double)off + 1.1920928955078125e-07;
    } else {
        // dt/gap <= 4 on a screened interval; 2^-22-slot truncation
        sp.dw = (float)(4.04 * delta / SCALE + 2.0e-6);
        e_w = 4.0 * e_pos / SCALE + 9.5367431640625e-07;
    }
    // (the weight of an event in the band of an epoch, computed in FP32 by
    // screen_exact_event, is within 5u of the exact one: 3u more than the
    // smallest e_w)
    sp.cv = (float)(8.0 * 5.9604644775390625e-08 + 2.0 * (e_w + 3.0 * 5.9604644775390625e-08));
    // on a regular grid an event within one fraction unit of an epoch's slot
    // may take the epoch's values: off by at most ws times a slope, and for
    // sigma ws times 2 sigma (adjacent sigmas within a factor 3)
    if (sp.slots)
        sp.cv = fmaxf(sp.cv, (float)(2.02 * (1.1920928955078125e-07 + e_pos / SCALE + (double)off) +
                                     8.0 * 5.9604644775390625e-08));
    sp.hw = 0.5f - sp.dw;
    sp.wscale = (float)(4194304.0 * g.inv_dt);
    return sp;
}

__device__ __forceinline__ ScreenPeriod screen_period(const FoldGeom& g, const ScreenGeom& sg,
                                                      double P, int64_t n_phi) {
    ScreenPeriod sp;
    const double SCALE = 1099511627776.0;   // 2^40
    const double R = P * g.inv_dt;
    const double span = (g.t_last - g.t_ref) * g.inv_dt;
    sp.on = sg.on != 0 && R * SCALE < 4.0e18 && span < 8388608.0;
    sp.slots = false;
    sp.uph = sp.ustep = sp.ulast = sp.delta = sp.uend = 0;
    sp.inv_ustep32 = 0.f;
    sp.wscale = 0.f;
    sp.cv = 0.f;
    sp.dw = 0.f;
    sp.hw = 0.5f;
    if (!sp.on) return sp;
    sp.ustep = (unsigned long long)llrint(R * SCALE);
    sp.uph = (unsigned long long)llrint(R / (double)n_phi * SCALE);
    sp.inv_ustep32 = (float)(4294967296.0 / (double)sp.ustep);
    return screen_period_curve(g, sg, P, n_phi, R, span, sp);
}

// screen_period from a table entry (the same values).
__device__ __forceinline__ ScreenPeriod screen_period(const FoldGeom& g, const ScreenGeom& sg,
                                                      double P, const PeriodConst& pc) {
    ScreenPeriod sp;
    const double SCALE = 1099511627776.0;   // 2^40
    const double R = pc.R;
    const double span = (g.t_last - g.t_ref) * g.inv_dt;
    sp.on = sg.on != 0 && R * SCALE < 4.0e18 && span < 8388608.0;
    sp.slots = false;
    sp.uph = sp.ustep = sp.ulast = sp.delta = sp.uend = 0;
    sp.inv_ustep32 = 0.f;
    sp.wscale = 0.f;
    sp.cv = 0.f;
    sp.dw = 0.f;
    sp.hw = 0.5f;
    if (!sp.on) return sp;
    sp.ustep = pc.ustep;
    sp.uph = pc.uph;
    sp.inv_ustep32 = pc.inv_ustep32;
    return screen_period_curve(g, sg, P, pc.n_phi, R, span, sp);
}

// Sums of the screen (see above) and the bound they give.
// Integer-to-float conversions run on the FP64 pipe of this GPU, so the
// screen counts events in a float and builds weights from bit patterns.
struct ScreenAcc {
    float sinv, sd, sdd, sdd2, sl, sabs, ivmax;
    float K;                 // number of events (exact in FP32 below 2^24)
    __device__ __forceinline__ void init() {
        sinv = sd = sdd = sdd2 = sl = sabs = ivmax = 0.f;
        K = 0.f;
    }
    // event (depth dk, sigma s, gain lk) on an interval with depth and gain
    // differences dd, dl.  The error budget of the depths uses
    // (|Delta_i| + |Delta_{i+1}|)^2 <= (2|dk| + |dd|)^2 <= 8 dk^2 + 2 dd^2.
    __device__ __forceinline__ void add(float dk, float s, float lk, float dd, float dl) {
        const float iv = rcp32(s * s);
        const float div = dk * iv;
        sinv += iv;
        sd += div;
        sdd = fmaf(div, dk, sdd);
        sl += lk;
        sdd2 = fmaf(dd * dd, iv, sdd2);
        sabs += fmaf(2.f, fabsf(lk), fabsf(dl));
        ivmax = fmaxf(ivmax, iv);
        K += 1.f;
    }
    // Hardware reciprocal / reciprocal square root (relative error below
    // 2^-21, counted as 8u per use) with every term rounded the safe way.
    // The q term only lowers the bound, so the cheaper S_L + 1/2 + margins
    // is returned when it already falls below the threshold bf.
    __device__ __forceinline__ float bound(float cv, float bf) const {
        if (K == 0.f) return -INFINITY;
        const float U = 5.9604645e-8f;                        // 2^-24
        const float sk = (K + 2.f) * U;
        const float e_l = 1.05f * (cv + sk) * sabs;
        const float ub0 = sl + e_l + 0.5f + 8.f * U * (sabs + 1.f);
        if (ub0 < bf) return ub0;
        // |ds|/s <= 2 on a screened interval (adjacent sigmas within a factor 3)
        const float gam = 2.2f * cv * 4.f + 6.f * U;
        const float r = rcp32(sinv);
        const float qc = fmaf(-sd * sd, r, sdd);
        const float qcl = qc - fmaf(4.f, K, 32.f) * U * sdd;
        float q_lo = 0.f;
        if (qcl > 0.f) {
            const float x1 = qcl * rcp32(1.f + gam + sk) * (1.f - 16.f * U);
            const float a = x1 * rsqrt32(x1) * (1.f - 16.f * U);
            const float y = fmaf(8.f, sdd, 2.f * sdd2) * (1.f + 2.f * gam + sk) * (1.f + 8.f * U);
            const float e = y > 0.f ? 1.05f * cv * (y * rsqrt32(y)) * (1.f + 16.f * U) : 0.f;
            if (a > e) q_lo = (a - e) * (a - e) * (1.f - 8.f * U);
        }
        const float x_hi = fminf(1.f, ivmax * r * (1.f + 4.f * gam + 2.f * sk + 24.f * U));
        return sl + e_l + 0.5f - 0.5f * q_lo * rcp32(1.f + x_hi) * (1.f - 16.f * U) +
               8.f * U * (sabs + q_lo + 1.f);
    }
};

// The event of epoch k whose walk position lies in the band of an epoch
// (or of t_last): T and its interval exactly as the exact path computes
// them (FP64 epoch, comparisons of the doubles' integer keys), then the
// weight (T - t_i)/gap in FP32 from the interval's screening record (within
// 5u of the exact path's weight, which the error coefficient covers) and the
// FP32 values as for any other event.  Returns 0 when there is no event, 1
// when the event was added, 2 when its interval is outside the error model.
__device__ __forceinline__ int screen_exact_event(const FoldGeom& g,
                                                  const ScreenRec* __restrict__ rd,
                                                  const CellCtx& c, double phi, int64_t k,
                                                  unsigned long long u, float wscale,
                                                  ScreenAcc& acc) {
    const double Tk = epoch_time(g, c, phi, (double)k);
    const long long kT = okey(Tk);
    if (kT > c.klast) return 0;                 // after the last epoch
    const int64_t i = bracket_from(g, kT, guess_at(g, u));
    const ScreenRec r = rd[i];
    if (r.flags) return 2;
    // wsc = 2^-22 dt/gap: (T - t_i) 2^22/dt wsc = (T - t_i)/gap
    const float w = (float)(Tk - g.t0s[i]) * wscale * r.wsc;
    const float s = fmaf(w, r.ds, r.s);
    if (isnan(s)) return 0;                     // the interval has no event
    acc.add(fmaf(w, r.dd, r.d), s, fmaf(w, r.dl, r.l), r.dd, r.dl);
    return 1;
}

// Upper bound on ln P of cell (j, duration rows rd / rs) whose first
// epoch is at u0 (see above): -inf when the cell has no event, +inf when an
// event falls on an interval outside the screen's error model; any value
// below bf when the cell is already known not to reach bf.
__device__ __forceinline__ float screen_cell(const FoldGeom& g, const ScreenGeom& sg,
                                             const ScreenRec* __restrict__ rd,
                                             const ScreenRec* __restrict__ rs,
                                             const ScreenPeriod& sp, const CellCtx& c,
                                             int64_t j, unsigned long long u0, float bf) {
    // epochs up to u < ulast + delta: those within delta of t_last (the last
    // epoch's position) fall in the band around it and take the exact event,
    // which drops T > t_last
    double phi = 0.0;
    bool have_phi = false;
    ScreenAcc acc;
    acc.init();
    unsigned long long u = u0;
    // the exact event of the epoch at u (rare: within the band of an epoch);
    // false when the cell must be evaluated exactly
    auto exact = [&]() -> bool {
        if (!have_phi) {
            phi = cell_phi(c, j);
            have_phi = true;
        }
        const int64_t k = (int64_t)((u - u0) / sp.ustep);
        return screen_exact_event(g, rd, c, phi, k, u, sp.wscale, acc) != 2;
    };
    if (sp.slots) {
        // regular grid: the interval is the slot's, the weight its fraction
        const unsigned ns1 = (unsigned)(sg.n_slots - 1);
        auto slot = [&](unsigned long long x) { return min((unsigned)(x >> 40), ns1); };
        auto visit = [&](const ScreenRec& r) -> bool {
            // fraction of the slot: its top 23 bits as the mantissa of a float in [1, 2)
            const float w =
                __uint_as_float(0x3f800000u | (unsigned)((u >> 17) & 0x7fffffu)) - 1.0f;
            if (fabsf(w - 0.5f) > sp.hw) {
                // in the band of an epoch.  A position within one unit of the
                // fraction of the epoch's slot m (every event of a period of
                // whole slots) takes the epoch's values when both intervals
                // at m are screened: the event lies on one of them, within
                // ws = 2^-23 + e_pos + off of m, so its values are the epoch's
                // within ws times either slope (the error coefficient covers
                // it, with the larger slope as the event's).  Otherwise the
                // exact event.
                if (w != 0.f && w < 0.99999988f) return exact();
                const unsigned sl = slot(u);
                const unsigned m = w < 0.5f ? sl : sl + 1u;
                if (m == 0u || m >= ns1) return exact();
                const ScreenRec L = m == sl ? rs[m - 1u] : r;
                const ScreenRec R = m == sl ? r : rs[m];
                if (!(L.s < INFINITY) || !(R.s < INFINITY)) return exact();
                acc.add(R.d, R.s, R.l, fmaxf(fabsf(L.dd), fabsf(R.dd)),
                        fmaxf(fabsf(L.dl), fabsf(R.dl)));
                return true;
            }
            const float s = fmaf(w, r.ds, r.s);
            if (!(s < INFINITY)) return s != s;   // NaN: no event; +inf: not screened
            acc.add(fmaf(w, r.dd, r.d), s, fmaf(w, r.dl, r.l), r.dd, r.dl);
            return true;
        };
        // two records in flight, alternating (no register moves)
        ScreenRec ra = rs[slot(u)], rb;
        while (u < sp.uend) {
            rb = rs[slot(u + sp.ustep)];
            if (!visit(ra)) return INFINITY;
            u += sp.ustep;
            if (!(u < sp.uend)) break;
            ra = rs[slot(u + sp.ustep)];
            if (!visit(rb)) return INFINITY;
            u += sp.ustep;
        }
        return acc.bound(sp.cv, bf);
    }
    const int64_t nb1 = g.n_bucket - 1;
    int bnext = g.bucket[min((int64_t)(u >> 40), nb1)];
    for (; u < sp.uend; u += sp.ustep) {
        // interval guess from the bucket table (the next epoch's entry is
        // fetched one iteration ahead), verified against the stored positions
        int64_t i = bnext > 0 ? (int64_t)bnext - 1 : 0;
        bnext = g.bucket[min((int64_t)((u + sp.ustep) >> 40), nb1)];
        ulonglong2 v = sg.vpair[i];
        ScreenRec r = rd[i];
        if (u >= v.y || u < v.x) {
            while (u >= v.y) v = sg.vpair[++i];
            while (u < v.x) v = sg.vpair[--i];
            r = rd[i];
        }
        const long long sdu = (long long)(u - v.x);
        // position in units of 2^-22 slot (23 bits for du < 2 slots) as a float
        const float w = (__uint_as_float(0x4b000000u | ((unsigned)(sdu >> 18) & 0x7fffffu)) -
                         8388608.0f) * r.wsc;
        const float s = fmaf(w, r.ds, r.s);
        // within delta of either end (on a valid interval: w within dw of 0
        // or 1, dw >= 4 delta in slots as dt/gap <= 4): the exact event
        const bool near = isnan(s) ? ((unsigned long long)sdu < sp.delta || v.y - u < sp.delta)
                                   : fabsf(w - 0.5f) > sp.hw;
        if (near) {
            if (!exact()) return INFINITY;
            continue;
        }
        if (!(s < INFINITY)) {
            if (s != s) continue;                  // no event
            return INFINITY;                       // not screened
        }
        acc.add(fmaf(w, r.dd, r.d), s, fmaf(w, r.dl, r.l), r.dd, r.dl);
    }
    return acc.bound(sp.cv, bf);
}

// The gain bound of a cell on a regular grid, from 4 bytes per epoch.  By the
// bound above, ln P <= S_L + 1/2, and every event's gain is at most the
// larger gain of its interval's two nodes.  The walk's position u of epoch k
// lies within half a slot of the exact epoch, and on a regular grid every
// epoch is within 2^-10 slot of its slot, so the exact interval starts at
// the epoch of slot floor(u) - 1, floor(u) or floor(u) + 1: lm3 at floor(u)
// bounds the event's gain (0 for a dropped epoch, +inf on an interval outside
// the screen's error model).  Extra walk positions past t_last (u < uend)
// only add terms >= 0.  The FP32 sum of K terms >= 0 is rounded up by
// (K + 16) 2^-23 of itself, and 1e-6 covers the exact path's own rounding.
//
// The walk runs in 32-bit fixed point (few instructions per epoch):
// positions in units of 2^-F slot, started from the 64-bit position of a
// cell's first epoch (truncated) and advanced by the rounded step, so that
// epoch k is at most 1 + k/2 units from the 64-bit walk.  F is chosen per
// period so that no position the walk loads (up to end + 3 steps: four epochs
// a round) exceeds 2^31 (the margin below allows twelve), and the walk is
// used only when that error stays below half a slot for every epoch (the gain
// bound tolerates the exact interval starting one slot either side of the
// walk's slot).  The end is widened by the same error, so every epoch of the
// 64-bit walk is counted; positions past it add terms >= 0 (the walk adds
// four terms at a time; a position past the row is clamped to the padding
// slot zs, whose term is 0).
struct GainWalk32 {
    unsigned step, end;
    int shift;            // 40 - F
    int F;
    int ok;
};
__device__ __forceinline__ GainWalk32 gain_walk32(unsigned long long ustep,
                                                  unsigned long long uend) {
    GainWalk32 w{0u, 0u, 0, 0, 0};
    const double S40 = 9.094947017729282e-13;               // 2^-40
    const double R = (double)ustep * S40;                    // slots per period
    if (!(R > 0.0)) return w;
    const double span = (double)uend * S40;
    const double kmax = span / R + 2.0;                      // epochs walked, at most
    const double top = span + 12.0 * R + kmax + 8.0;         // slots a position can reach
    int F = 30 - ilogb(top);                                 // 2^F top < 2^31
    if (F > 24) F = 24;
    if (F < 8 || (kmax + 2.0) * ldexp(1.0, -F) > 0.5) return w;
    w.F = F;
    w.shift = 40 - F;
    w.step = (unsigned)((ustep + (1ull << (w.shift - 1))) >> w.shift);
    w.end = (unsigned)((uend >> w.shift) + 2ull + (unsigned long long)(kmax + 2.0));
    w.ok = w.step > 0u;
    return w;
}

// The gain tables are grouped by duration (gain_width): the W cells of one
// phase and W consecutive durations share their epochs, so a lane walks them
// together with one W-wide load per epoch.  row points at the group's first
// slot; the sums of the W columns go to s (the unused ones stay 0) and the
// number of terms, the same for every column, is returned.
template <int W>
struct GainVec;
template <>
struct GainVec<1> {
    typedef float T;
    __device__ static __forceinline__ T zero() { return 0.f; }
    __device__ static __forceinline__ void add(float4& s, T a, T b, T c, T e) {
        s.x += (a + c) + (b + e);
    }
};
template <>
struct GainVec<2> {
    typedef float2 T;
    __device__ static __forceinline__ T zero() { return make_float2(0.f, 0.f); }
    __device__ static __forceinline__ void add(float4& s, T a, T b, T c, T e) {
        s.x += (a.x + c.x) + (b.x + e.x);
        s.y += (a.y + c.y) + (b.y + e.y);
    }
};
template <>
struct GainVec<4> {
    typedef float4 T;
    __device__ static __forceinline__ T zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    __device__ static __forceinline__ void add(float4& s, T a, T b, T c, T e) {
        s.x += (a.x + c.x) + (b.x + e.x);
        s.y += (a.y + c.y) + (b.y + e.y);
        s.z += (a.z + c.z) + (b.z + e.z);
        s.w += (a.w + c.w) + (b.w + e.w);
    }
};
// (NU_GAIN_UNROLL4 epochs a round for 4-wide groups, four for the others)
#ifndef NU_GAIN_UNROLL4
#define NU_GAIN_UNROLL4 4
#endif
template <int W>
__device__ __forceinline__ float gain_walk_w(const float* __restrict__ row, unsigned zs,
                                             unsigned u, const GainWalk32& w, float4& s) {
    typedef typename GainVec<W>::T V;
    const V* __restrict__ r = reinterpret_cast<const V*>(row);
    const unsigned st = w.step;
    float K = 0.f;
    if (W == 4 && NU_GAIN_UNROLL4 == 2) {
        // two epochs a round, the second clamped past the end (a zero term)
        for (; u < w.end; u += 2u * st) {
            const V a = r[min(u >> w.F, zs)];
            const V b = r[min((u + st) >> w.F, zs)];
            const V z = GainVec<W>::zero();
            GainVec<W>::add(s, a, b, z, z);
            K += 2.f;
        }
        return K;
    }
    for (; u < w.end; u += 4u * st) {
        const V a = r[min(u >> w.F, zs)];
        const V b = r[min((u + st) >> w.F, zs)];
        const V c = r[min((u + 2u * st) >> w.F, zs)];
        const V e = r[min((u + 3u * st) >> w.F, zs)];
        GainVec<W>::add(s, a, b, c, e);
        K += 4.f;
    }
    return K;
}
__device__ __forceinline__ float gain_walk(const float* __restrict__ row, int W, unsigned zs,
                                           unsigned u, const GainWalk32& w, float4& s) {
    s = make_float4(0.f, 0.f, 0.f, 0.f);
    if (W == 4) return gain_walk_w<4>(row, zs, u, w, s);
    if (W == 2) return gain_walk_w<2>(row, zs, u, w, s);
    return gain_walk_w<1>(row, zs, u, w, s);
}
// The same walk on the 64-bit positions (2^-40 slot) that define the mixed
// fold's events: each epoch's slot is exactly its event's, so the table needs
// no neighbours.  Positions past uend add terms >= 0 (clamped to zs);
// ustep < 2^60 and u < 2^62 keep u + 3 ustep from wrapping.
template <int W>
__device__ __forceinline__ float gain_walk64_w(const float* __restrict__ row, unsigned zs,
                                               unsigned long long u, unsigned long long ustep,
                                               unsigned long long uend, float4& s) {
    typedef typename GainVec<W>::T V;
    const V* __restrict__ r = reinterpret_cast<const V*>(row);
    float K = 0.f;
    for (; u < uend; u += 4ull * ustep) {
        const V a = r[min((unsigned)(u >> 40), zs)];
        const V b = r[min((unsigned)((u + ustep) >> 40), zs)];
        const V c = r[min((unsigned)((u + 2ull * ustep) >> 40), zs)];
        const V e = r[min((unsigned)((u + 3ull * ustep) >> 40), zs)];
        GainVec<W>::add(s, a, b, c, e);
        K += 4.f;
    }
    return K;
}
__device__ __forceinline__ float gain_walk64(const float* __restrict__ row, int W, unsigned zs,
                                             unsigned long long u, unsigned long long ustep,
                                             unsigned long long uend, float4& s) {
    s = make_float4(0.f, 0.f, 0.f, 0.f);
    if (W == 4) return gain_walk64_w<4>(row, zs, u, ustep, uend, s);
    if (W == 2) return gain_walk64_w<2>(row, zs, u, ustep, uend, s);
    return gain_walk64_w<1>(row, zs, u, ustep, uend, s);
}
__device__ __forceinline__ float gain_col(const float4& s, int i) {
    return i == 0 ? s.x : (i == 1 ? s.y : (i == 2 ? s.z : s.w));
}

// The mixed fold's cascade runs on periods with at least NU_CASCADE_ROUNDS
// rounds of cells per warp.
#ifndef NU_CASCADE_ROUNDS
#define NU_CASCADE_ROUNDS 32
#endif

// A warp whose gain bounds pass at least NU_GAIN_PASS_MAX of its 32 cells
// screens its next NU_GAIN_DIRECT_ROUNDS rounds in full without them.
#ifndef NU_GAIN_PASS_MAX
#define NU_GAIN_PASS_MAX 28
#endif
#ifndef NU_GAIN_DIRECT_ROUNDS
#define NU_GAIN_DIRECT_ROUNDS 16
#endif

// Exact ln P of one cell computed by a whole warp (lanes over epochs); used
// only to seed the pruning threshold.
__device__ __forceinline__ double exact_cell_warp(const FoldGeom& g,
                                                  const Node8<double>* __restrict__ nd,
                                                  const CellCtx& c, int64_t j) {
    const int lane = threadIdx.x & 31;
    const double phi = cell_phi(c, j);
    const unsigned long long u0 = (unsigned long long)j * c.swp.u0;
    const int64_t kmax = cell_kmax(g, c, phi, u0);
    ExactAcc<double> a1;
    a1.init();
    cell_pass1<double>(g, nd, c, phi, u0, kmax, lane, 32, a1);
    double s_inv = a1.s_inv.s, s_d = a1.s_d.s, s_l = a1.s_l.s;
    int K = a1.K;
    for (int o = 16; o > 0; o >>= 1) {
        s_inv += __shfl_xor_sync(0xffffffffu, s_inv, o);
        s_d += __shfl_xor_sync(0xffffffffu, s_d, o);
        s_l += __shfl_xor_sync(0xffffffffu, s_l, o);
        K += __shfl_xor_sync(0xffffffffu, K, o);
    }
    if (K == 0) return -INFINITY;
    const double s2 = 1.0 / s_inv;
    ExactPen<double> a2;
    a2.init(s2, s2 * s_d);
    cell_pass2<double>(g, nd, c, phi, u0, kmax, lane, 32, a2);
    double pen = a2.logsum() + a2.quad.s;
    for (int o = 16; o > 0; o >>= 1) pen += __shfl_xor_sync(0xffffffffu, pen, o);
    return s_l - 0.5 * pen;
}

// Order-preserving unsigned key of a float (for a shared atomic max).
__device__ __forceinline__ unsigned fkey(float x) {
    const unsigned b = __float_as_uint(x);
    return (b >> 31) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float from_fkey(unsigned k) {
    return __uint_as_float((k >> 31) ? (k & 0x7fffffffu) : ~k);
}

// A large finite single-event gain of each curve, for the peak seed: key[g]
// = (order key of the gain rounded to FP32) << 32 | (2^32 - 1 - e), the
// maximum over the curve's grid entries e (duration-major, e < 2^32 - 1), so
// the largest rounded gain wins and ties go to the first entry.  key[g] must
// be zero on entry and stays zero when no gain is finite.  blockIdx.x is the
// curve (s_off == nullptr: one curve of n_t0 epochs); the blocks along y
// share a curve's entries.
__global__ void k_gain_peak(const double* __restrict__ gain, const int64_t* __restrict__ s_off,
                            int64_t n_t0, int n_D, unsigned long long* __restrict__ key) {
    const int g = blockIdx.x;
    const int64_t s0 = s_off ? s_off[g] : 0;
    const int64_t ng = s_off ? s_off[g + 1] - s0 : n_t0;
    const int64_t n = ng * n_D;
    if (n >= 0xffffffffLL) return;
    const double* row = gain + s0 * n_D;
    unsigned long long best = 0;
    for (int64_t e = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.y * blockDim.x) {
        const double v = row[e];
        if (v > -INFINITY && v < INFINITY) {
            const unsigned long long k = ((unsigned long long)fkey((float)v) << 32) |
                                         (unsigned long long)(0xffffffffu - (unsigned)e);
            best = k > best ? k : best;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, best, o);
        best = k2 > best ? k2 : best;
    }
    if ((threadIdx.x & 31) == 0 && best != 0) atomicMax(key + g, best);
}

// Exact evaluation of a queued cell by one thread; the thread's best is kept
// in shared memory and the block's thresholds are raised.
__device__ __forceinline__ void evaluate_queued(const FoldGeom& g,
                                               const Node8<double>* __restrict__ nodes,
                                               const CellCtx& c, int64_t n_phi, long long qcell,
                                               int qd, unsigned long long* sh_sbest,
                                               unsigned* sh_bfk, Best* tb) {
    const int64_t qj = qcell - (int64_t)qd * n_phi;
    const Node8<double>* nd = nodes + (int64_t)qd * g.n_t0;
    const double phi = cell_phi(c, qj);
    const unsigned long long u0 = (unsigned long long)qj * c.swp.u0;
    const int64_t kmax = cell_kmax(g, c, phi, u0);
    ExactAcc<double> a1;
    a1.init();
    cell_pass1<double>(g, nd, c, phi, u0, kmax, 0, 1, a1);
    if (a1.K == 0 || a1.cannot_win(from_max_key(*sh_sbest))) return;
    const double s2 = 1.0 / a1.s_inv.s;
    const double Dl = s2 * a1.s_d.s;
    ExactPen<double> a2;
    a2.init(s2, Dl);
    cell_pass2<double>(g, nd, c, phi, u0, kmax, 0, 1, a2);
    const double lnp = a1.s_l.s - 0.5 * (a2.logsum() + a2.quad.s);
    if (!(lnp == lnp)) return;   // NaN never selected
    const Best cand{lnp, qcell, Dl, s2};
    if (better(cand, *tb)) *tb = cand;
    if (lnp > from_max_key(*sh_sbest)) {
        atomicMax(sh_sbest, max_key(lnp));
        atomicMax(sh_bfk, fkey(__double2float_rd(lnp)));
    }
}

// The same evaluation by a whole warp (lanes over epochs, fixed reduction
// order); called by all lanes with the same cell.  Used for every evaluation
// of a period whose cells have 32 or more epochs, where one cell per lane
// would leave most lanes idle whenever fewer than 32 cells are queued.
__device__ __forceinline__ void evaluate_queued_warp(const FoldGeom& g,
                                                    const Node8<double>* __restrict__ nodes,
                                                    const CellCtx& c, int64_t n_phi,
                                                    long long qcell, int qd,
                                                    unsigned long long* sh_sbest,
                                                    unsigned* sh_bfk, Best* tb) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t qj = qcell - (int64_t)qd * n_phi;
    const Node8<double>* nd = nodes + (int64_t)qd * g.n_t0;
    const double phi = cell_phi(c, qj);
    const unsigned long long u0 = (unsigned long long)qj * c.swp.u0;
    const int64_t kmax = cell_kmax(g, c, phi, u0);
    ExactAcc<double> a1;
    a1.init();
    cell_pass1<double>(g, nd, c, phi, u0, kmax, lane, 32, a1);
    double s_inv = a1.s_inv.s, s_d = a1.s_d.s, s_l = a1.s_l.s, s_dd = a1.s_dd;
    int K = a1.K;
    for (int o = 16; o > 0; o >>= 1) {
        s_inv += __shfl_xor_sync(FULL, s_inv, o);
        s_d += __shfl_xor_sync(FULL, s_d, o);
        s_l += __shfl_xor_sync(FULL, s_l, o);
        s_dd += __shfl_xor_sync(FULL, s_dd, o);
        K += __shfl_xor_sync(FULL, K, o);
    }
    const double best_now = __shfl_sync(FULL, from_max_key(*sh_sbest), 0);
    if (K == 0 || cannot_win(s_l, s_inv, s_d, s_dd, best_now)) return;
    const double s2 = 1.0 / s_inv;
    const double Dl = s2 * s_d;
    ExactPen<double> a2;
    a2.init(s2, Dl);
    cell_pass2<double>(g, nd, c, phi, u0, kmax, lane, 32, a2);
    double pen = a2.logsum() + a2.quad.s;
    for (int o = 16; o > 0; o >>= 1) pen += __shfl_xor_sync(FULL, pen, o);
    const double lnp = s_l - 0.5 * pen;
    if (lane != 0 || !(lnp == lnp)) return;      // NaN never selected
    const Best cand{lnp, qcell, Dl, s2};
    if (better(cand, *tb)) *tb = cand;
    if (lnp > from_max_key(*sh_sbest)) {
        atomicMax(sh_sbest, max_key(lnp));
        atomicMax(sh_bfk, fkey(__double2float_rd(lnp)));
    }
}

// One period of the FP64 path with the screen.  Each warp screens its own
// cells (the block's cells in strides of blockDim) and queues the survivors
// in its own shared queue; a full queue (32 cells) is evaluated exactly, one
// cell per lane, by that warp alone, so the screen needs no block barriers.
// Warp 0 first evaluates the cell through the curve's largest single-event
// gain, and in its first round each warp evaluates its best-bounded cell with
// all its lanes when that bound is above the threshold.  The thresholds (best ln P, and its FP32
// lower bound) are shared by the block through atomic maxima.
// With TAB the period's curve-independent constants come from the table
// entry pc (k_period_consts), else they are computed here.
template <int MAXT = 256, bool TAB = false, bool GROUP = true>
__device__ __forceinline__ void fold_screened_one(const FoldGeom& g, const ScreenGeom& sg,
                                                  const Node8<double>* __restrict__ nodes,
                                                  int n_D, double P, int64_t p,
                                                  double* __restrict__ Q_out,
                                                  double* __restrict__ T0_out,
                                                  int* __restrict__ Didx_out,
                                                  double* __restrict__ dep_out,
                                                  double* __restrict__ sig_out,
                                                  double* __restrict__ lnp_out,
                                                  const PeriodConst* __restrict__ pc = nullptr) {
    __shared__ long long sh_qc[MAXT / 32][64];      // per-warp survivor queues
    __shared__ int sh_qd[MAXT / 32][64];
    __shared__ long long sh_qa[MAXT / 32][160];     // per-warp cells for the full screen
    __shared__ int sh_qad[MAXT / 32][160];
    __shared__ unsigned long long sh_sbest; // best ln P evaluated (max key)
    __shared__ unsigned sh_bfk;             // its FP32 lower bound (float key)
    __shared__ Best sh_tb[MAXT];            // each thread's best evaluated cell (kept
                                            // out of registers during the screen)
    if (bad_period(P, g)) {
        if (threadIdx.x == 0) write_bad(p, Q_out, T0_out, Didx_out, dep_out, sig_out, lnp_out);
        return;
    }
    // the period's constants live in shared memory: registers are kept for
    // the screen loop (most of these are read only on rare paths)
    __shared__ ScreenPeriod sh_sp;
    __shared__ CellCtx sh_cc;
    __shared__ GainWalk32 sh_gw;
    const int64_t n_phi = TAB ? pc->n_phi : (int64_t)ceil(P / g.dt);
    if (threadIdx.x == 0) sh_sp = TAB ? screen_period(g, sg, P, *pc) : screen_period(g, sg, P, n_phi);
    __syncthreads();
    if (!sh_sp.on) {
        fold_exact_one<double, 8, MAXT>(g, nodes, n_D, P, p, Q_out, T0_out, Didx_out, dep_out,
                                  sig_out, lnp_out);
        return;
    }
    sh_tb[threadIdx.x] = Best{-INFINITY, LLONG_MAX, NAN, NAN};
    if (threadIdx.x == 0) {
        sh_gw = gain_walk32(sh_sp.ustep, sh_sp.uend);
        sh_cc = TAB ? cell_ctx(g, P, *pc) : cell_ctx(g, P, n_phi);
        sh_sbest = max_key(-INFINITY);
        sh_bfk = fkey(-INFINITY);
    }
    __syncthreads();
    const ScreenPeriod& sp = sh_sp;
    const CellCtx& c = sh_cc;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // cells of 32 or more epochs are evaluated warp-cooperatively
    const bool coop = g.t_last - g.t_ref >= 32.0 * P;
    // Peak seed: the cell whose epochs pass through the epoch of the curve's
    // largest single-event gain (phase index nearest to it), evaluated
    // exactly by warp 0.  When one event dominates a short cell (a deep
    // transit), every cell that catches it would otherwise pass the screen
    // until the threshold has risen.  Long cells are left to the first-round
    // seeds: there one event weighs less, and the seed costs a long walk.
    if (sg.peak && !coop) {
        const unsigned long long pk = *sg.peak;
        if (pk != 0) {
            if (wid == 0) {
                const int64_t e = (int64_t)(0xffffffffu - (unsigned)(pk & 0xffffffffu));
                const int64_t pd = e / g.n_t0;
                const double x = (g.t0s[e - pd * g.n_t0] - g.t_ref) / P;
                int64_t pj = (int64_t)rint((x - floor(x)) * (double)n_phi);
                if (pj >= n_phi || pj < 0) pj = 0;
                const double lnp = exact_cell_warp(g, nodes + pd * g.n_t0, c, pj);
                if (lane == 0 && lnp == lnp && lnp > -INFINITY) {
                    // the same margin as the first-round seed below
                    const double seed = lnp - 1e-9 * (1.0 + fabs(lnp));
                    atomicMax(&sh_sbest, max_key(seed));
                    atomicMax(&sh_bfk, fkey(__double2float_rd(seed)));
                }
            }
            __syncthreads();
        }
    }
    const unsigned FULL = 0xffffffffu;
    long long* qc = sh_qc[wid];
    int* qd = sh_qd[wid];
    int nq = 0;                              // warp-uniform queue lengths
    long long* qa = sh_qa[wid];
    int* qad = sh_qad[wid];
    int na = 0;
    // Cascade on regular grids: after the warp's first round every cell is
    // bounded from its gains alone (the gain bound, 4 bytes per epoch); the
    // cells that bound does not rule out are queued and screened in full 32
    // at a time, and the full screen's survivors are evaluated exactly.
    const bool cascade = sp.slots && sg.lm3 != nullptr && sp.ustep < (1ull << 60) && sh_gw.ok;
    const unsigned ns1 = (unsigned)(sg.n_slots - 1);
    // append this lane's cell to a queue when keep (positions by ballot)
    auto push = [&](long long* qx, int* qy, int& n, bool keep, long long cl, int dl) {
        const unsigned m = __ballot_sync(FULL, keep);
        if (keep) {
            const int pos = n + __popc(m & ((1u << lane) - 1u));
            qx[pos] = cl;
            qy[pos] = dl;
        }
        n += __popc(m);
        __syncwarp();
    };
    // drop the first 32 entries of a queue
    auto pop32 = [&](long long* qx, int* qy, int& n) {
        n -= 32;
        long long c2 = 0;
        int d2 = 0;
        if (lane < n) {
            c2 = qx[32 + lane];
            d2 = qy[32 + lane];
        }
        __syncwarp();
        if (lane < n) {
            qx[lane] = c2;
            qy[lane] = d2;
        }
        __syncwarp();
    };
    // exact evaluation of the first 32 entries of the survivor queue
    auto evaluate32 = [&]() {
        if (coop) {
            for (int q = 0; q < 32; ++q)
                evaluate_queued_warp(g, nodes, c, n_phi, qc[q], qd[q], &sh_sbest, &sh_bfk,
                                     &sh_tb[threadIdx.x]);
        } else {
            evaluate_queued(g, nodes, c, n_phi, qc[lane], qd[lane], &sh_sbest, &sh_bfk,
                            &sh_tb[threadIdx.x]);
        }
        __syncwarp();
        pop32(qc, qd, nq);
    };
    // First-round seed: the warp evaluates its lane with the largest finite
    // bound (all lanes over its epochs), unless that bound is already below
    // the threshold (the cell cannot raise it).  A 1e-9 margin keeps the
    // seeding cell itself above the threshold: it is evaluated again by the
    // thread code.
    auto seed_warp = [&](float ub, int dl, int64_t jl) {
        float v = (ub < INFINITY) ? ub : -INFINITY;
        int src = lane;
        for (int o = 16; o > 0; o >>= 1) {
            const float v2 = __shfl_xor_sync(FULL, v, o);
            const int s2 = __shfl_xor_sync(FULL, src, o);
            if (v2 > v || (v2 == v && s2 < src)) {
                v = v2;
                src = s2;
            }
        }
        // (the threshold is broadcast so that the branch is warp-uniform)
        const float thr = __shfl_sync(FULL, from_fkey(sh_bfk), 0);
        if (v > -INFINITY && !(v < thr)) {
            const int pd = __shfl_sync(FULL, dl, src);
            const long long pj = __shfl_sync(FULL, (long long)jl, src);
            const double lnp = exact_cell_warp(g, nodes + (int64_t)pd * g.n_t0, c, pj);
            if (lane == 0 && lnp == lnp && lnp > -INFINITY) {
                const double seed = lnp - 1e-9 * (1.0 + fabs(lnp));
                atomicMax(&sh_sbest, max_key(seed));
                atomicMax(&sh_bfk, fkey(__double2float_rd(seed)));
            }
            __syncwarp();
        }
    };
    // Cells are taken W durations at a time (one gain group, one phase per
    // lane; W = 1 without the cascade).  Without the cascade, the warp's
    // first round and its direct rounds every cell goes on; otherwise those
    // whose gain bound reaches the threshold.  Cells that go on are screened
    // in full from queue A, 32 at a time (the warp's first such screen seeds
    // the threshold), and the screen's survivors are evaluated exactly from
    // the survivor queue.
    bool seed = true;
    // full screen of queue A's entries h .. h + cnt - 1 (one per lane)
    auto screen_queued = [&](int h, int cnt) {
        float ub = -INFINITY;
        long long cl = 0;
        int dl = 0;
        int64_t jl = 0;
        if (lane < cnt) {
            cl = qa[h + lane];
            dl = qad[h + lane];
            jl = cl - (int64_t)dl * n_phi;
            ub = screen_cell(g, sg, sg.rec + (int64_t)dl * g.n_t0,
                             sg.srec ? sg.srec + (int64_t)dl * sg.n_slots : nullptr, sp, c, jl,
                             (unsigned long long)jl * sp.uph, from_fkey(sh_bfk));
        }
        if (seed) {
            seed = false;
            seed_warp(ub, dl, jl);
        }
        // a cell without events (bound -inf) is never the argmax; NaN
        // survives.  The FP32 threshold is at most every evaluated ln P.
        push(qc, qd, nq, lane < cnt && !(ub == -INFINITY) && !(ub < from_fkey(sh_bfk)), cl,
             dl);
    };
    // (GROUP = false compiles the one-duration walk alone: the wider walks'
    // registers would otherwise weigh on the grids of one duration)
    const int W = cascade && GROUP ? gain_width(n_D) : 1;
    const int64_t n_gc = (int64_t)((n_D + W - 1) / W) * n_phi;
    const int dr = NU_GAIN_DIRECT_ROUNDS / W > 0 ? NU_GAIN_DIRECT_ROUNDS / W : 1;
    const unsigned zs = ns1 - 1u;
    int gi = (int)(threadIdx.x / n_phi);
    int64_t j = (int64_t)threadIdx.x - (int64_t)gi * n_phi;
    bool first = true;
    int direct = 0;                          // rounds left without the gain bound
    for (int64_t base = (int64_t)wid * 32; base < n_gc; base += blockDim.x, j += blockDim.x) {
        while (j >= n_phi) {
            j -= n_phi;
            ++gi;
        }
        const int d0 = gi * W;
        const int nv = base + lane < n_gc ? min(W, n_D - d0) : 0;   // this lane's cells
        unsigned pass = 0u;
        if (!cascade || first || direct > 0) {
            if (cascade && !first) --direct;
            first = false;
            pass = (1u << nv) - 1u;
        } else {
            if (nv > 0) {
                float4 sk;
                const float K = gain_walk(sg.lm3 + (int64_t)gi * sg.n_slots * W, W, zs,
                                          (unsigned)(((unsigned long long)j * sp.uph) >>
                                                     sh_gw.shift),
                                          sh_gw, sk);
                const float f = fmaf(K + 16.f, 1.1920929e-7f, 1.f);
                const float thr = from_fkey(sh_bfk);
                for (int i = 0; i < nv; ++i)
                    if (!(gain_col(sk, i) * f + 0.5f + 1e-6f < thr)) pass |= 1u << i;
            }
            // where the gain bound rules out almost nothing (cells of many
            // epochs, whose bound needs the depth terms) the warp screens its
            // next rounds in full directly
            const int np = __reduce_add_sync(FULL, (unsigned)__popc(pass));
            const int nt = __reduce_add_sync(FULL, (unsigned)nv);
            if (nt > 0 && np * 32 >= NU_GAIN_PASS_MAX * nt) direct = dr;
        }
        for (int i = 0; i < W; ++i)
            push(qa, qad, na, (pass >> i) & 1u, (long long)(d0 + i) * n_phi + j, d0 + i);
        // queue A holds at most 31 + 32 W entries here
        int h = 0;
        for (; na - h >= 32; h += 32) {
            screen_queued(h, 32);
            if (nq >= 32) evaluate32();
        }
        if (h > 0) {
            na -= h;
            long long c2 = 0;
            int d2 = 0;
            if (lane < na) {
                c2 = qa[h + lane];
                d2 = qad[h + lane];
            }
            __syncwarp();
            if (lane < na) {
                qa[lane] = c2;
                qad[lane] = d2;
            }
            __syncwarp();
        }
    }
    if (na > 0) screen_queued(0, na);
    if (nq >= 32) evaluate32();
    if (coop) {
        for (int q = 0; q < nq; ++q)
            evaluate_queued_warp(g, nodes, c, n_phi, qc[q], qd[q], &sh_sbest, &sh_bfk,
                                 &sh_tb[threadIdx.x]);
    } else if (lane < nq) {
        evaluate_queued(g, nodes, c, n_phi, qc[lane], qd[lane], &sh_sbest, &sh_bfk,
                        &sh_tb[threadIdx.x]);
    }
    __syncthreads();
    Best best = sh_tb[threadIdx.x];
    if (best.cell != LLONG_MAX) best.sigma = sqrt(best.sigma);   // held sigma^2
    const Best b = block_argmax<MAXT>(best);
    if (threadIdx.x == 0)
        write_best(b, p, n_phi, g.t_ref, P, Q_out, T0_out, Didx_out, dep_out, sig_out, lnp_out);
}

// resident blocks per SM the register allocation is sized for
#ifndef NU_SCREEN_MIN_BLOCKS
#define NU_SCREEN_MIN_BLOCKS 3
#endif

// 256-thread blocks: 3 per SM (about 80 registers); 64-thread blocks:
// NU_SCREEN_SMALL_BLOCKS per SM (the shared arrays are sized for 2 warps),
// NU_SCREEN_GROUP_BLOCKS with the grouped gain walk, whose registers need 80
// (C2 fold 8.52 ms at 12 blocks, 8.74 ms at 14 with 72 registers).
#ifndef NU_SCREEN_SMALL_BLOCKS
#define NU_SCREEN_SMALL_BLOCKS 14
#endif
#ifndef NU_SCREEN_GROUP_BLOCKS
#define NU_SCREEN_GROUP_BLOCKS 12
#endif
template <int MAXT, bool GROUP>
__global__ void __launch_bounds__(MAXT, MAXT <= 64 ? (GROUP ? NU_SCREEN_GROUP_BLOCKS
                                                            : NU_SCREEN_SMALL_BLOCKS)
                                                   : NU_SCREEN_MIN_BLOCKS)
k_fold_screened(FoldGeom g, ScreenGeom sg, const Node8<double>* __restrict__ nodes, int n_D,
                const double* __restrict__ periods, int64_t n_P, double* __restrict__ Q_out,
                double* __restrict__ T0_out, int* __restrict__ Didx_out,
                double* __restrict__ dep_out, double* __restrict__ sig_out,
                double* __restrict__ lnp_out) {
    if ((int64_t)blockIdx.x >= n_P) return;
    const int64_t p = period_slot(blockIdx.x, periods, n_P);
    fold_screened_one<MAXT, false, GROUP>(g, sg, nodes, n_D, periods[p], p, Q_out, T0_out,
                                          Didx_out, dep_out, sig_out, lnp_out);
}

// ---------------------------------------- slot path (mixed, regular grids)
struct SlotEvent {
    float d, s, l;
};
__device__ __forceinline__ SlotEvent slot_event(const Node4<float>* __restrict__ rd,
                                                unsigned long long u) {
    const int64_t s = (int64_t)(u >> 40);
    // weight = fractional slot position: its top 23 bits as the mantissa of a
    // float in [1, 2), minus 1 (no integer-to-float conversion)
    const float w =
        __uint_as_float(0x3f800000u | (unsigned)((u >> 17) & 0x7fffffu)) - 1.0f;
    const Node4<float> a = rd[s];
    const Node4<float> b = rd[s + 1];
    SlotEvent e;
    e.s = a.s + w * (b.s - a.s);
    e.d = a.d + w * (b.d - a.d);
    e.l = a.l + w * (b.l - a.l);
    return e;
}

struct SlotPass1 {
    KSum<float> s_inv, s_d, s_l;
    float s_dd;            // sum Delta_k^2 / s_k^2 (bound only)
    float ivmax;           // max 1/s_k^2 (bound only)
    int K;
    __device__ __forceinline__ void init() {
        s_inv.init();
        s_d.init();
        s_l.init();
        s_dd = 0.f;
        ivmax = 0.f;
        K = 0;
    }
    __device__ __forceinline__ void add(const SlotEvent& e) {
        if (isnan(e.s)) return;
        const float iv = rcp32(e.s * e.s);
        const float div = e.d * iv;
        s_inv.add(iv);
        s_d.add(div);
        s_dd = fmaf(div, e.d, s_dd);
        ivmax = fmaxf(ivmax, iv);
        s_l.add(e.l);
        ++K;
    }
};

struct SlotPass2 {
    KSum<float> quad;
    float lsum;
    float s2, Dl;
    __device__ __forceinline__ void init(float s2_, float Dl_) {
        quad.init();
        lsum = 0.f;
        s2 = s2_;
        Dl = Dl_;
    }
    __device__ __forceinline__ void add(float dk, float sg) {
        if (isnan(sg)) return;
        const float sk2 = sg * sg;
        const float iden = rcp32(sk2 + s2);
        const float r = dk - Dl;
        quad.add(r * r * iden);
        lsum += lg2_32(sk2 * iden);
    }
};

// A cell of the slot path that passed the bound, queued for its second pass.
struct SCell {
    unsigned long long u0;
    long long cell;
    float s_l, s2, Dl;
    int d, kmax, pad;
};

// Gain table of the slot path.  An event at walk position u interpolates the
// records of slots floor(u) and floor(u) + 1, so its gain is at most the
// pair gain of floor(u): the larger gain of the two records when both are
// valid (0 otherwise, a dropped event), rounded up (to cover the FP32
// rounding of the interpolation).  The gain walk reads it at the 64-bit
// positions that define the events (gain_walk64).  Grouped by duration
// (gain_slot).
__global__ void k_slot_gain(const Node4<float>* __restrict__ rec,
                            const FoldSeg* __restrict__ segs, int n_seg, int64_t n_slots1,
                            int n_D, int64_t n_out, float* __restrict__ lgm) {
    const int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (o >= n_out) return;
    GainSlot gs;
    if (!gain_slot(segs, n_seg, n_slots1, n_D, false, o, gs)) return;
    float m = 0.f;
    if (gs.d < n_D && gs.s + 1 < gs.n_slots) {
        const Node4<float>* r = rec + gs.src_off + (int64_t)gs.d * gs.n_slots;
        const Node4<float> a = r[gs.s], b = r[gs.s + 1];
        if (!isnan(a.s) && !isnan(b.s)) m = __fmul_ru(fmaxf(0.f, fmaxf(a.l, b.l)), 1.0000005f);
    }
    lgm[o] = m;
}

// Epochs walk the slot grid in 24.40 fixed point: u = (T - t_ref)/dt =
// (j/n_phi + k) P/dt.  The interval is (slot, slot+1) and the weight is the
// fractional part; on a grid whose epochs sit on the slots this is the
// interpolation between the bracketing epochs up to their offsets from the
// slot centres (checked to be below 1e-3 slot).
//
// Cascade per warp (no block barriers until the final argmax):
//   1. gain bound of each cell from lgm (4 bytes per epoch): with the bound
//      of cannot_win, ln P <= S_L + 1/2, and S_L is at most the sum of the
//      epochs' lgm; cells below the threshold stop here.  A lane bounds the
//      cells of one phase and one group of durations (gain_width) in one
//      walk;
//   2. queued, 32 at a time: the first pass (FP32 sums) and the bound of
//      cannot_win_f;
//   3. queued, 32 at a time: the second pass, whose ln P raises the threshold.
// A warp's first round skips step 1.  Warps whose gain bounds pass almost
// every cell (cells of many epochs) skip it for their next rounds, and
// periods with few cells per warp (short curves) skip the cascade
// throughout, running the first pass directly: their threshold does not rise
// in time for the bound to pay.
// CASC = false compiles the fold without the cascade (its registers spill
// the plain path's), for grids too small for it (the host decides).
// (Evaluating the best-bounded cell of the first round at once, as a seed
// of the threshold, did not pay either.)
template <int KC, int MAXT = 256, bool CASC = true>
__device__ __forceinline__ void fold_slots_one(const Node4<float>* __restrict__ rec,
                                               const float* __restrict__ lgm,
                                               int64_t n_slots, int n_D, double dt,
                                               double t_ref, double t_last, double P, int64_t p,
                                               const SlotPeriod* __restrict__ spp,
                                               unsigned long long ulast_in,
                                               double* __restrict__ Q_out,
                                               double* __restrict__ T0_out,
                                               int* __restrict__ Didx_out,
                                               double* __restrict__ dep_out,
                                               double* __restrict__ sig_out,
                                               double* __restrict__ lnp_out) {
    __shared__ SCell sh_q[MAXT / 32][64];
    __shared__ long long sh_qa[MAXT / 32][CASC ? 160 : 1];   // cells for the first pass
    __shared__ int sh_qad[MAXT / 32][CASC ? 160 : 1];
    __shared__ unsigned int sh_best;
    // the period's constants from the batch's table (spp) or computed here;
    // the curve's last epoch position from the batch (ulast_in) or here
    const SlotPeriod spc = spp ? *spp : slot_period(P, dt);
    if (spc.bad || t_last - t_ref > 1.0e9 * P) {
        if (threadIdx.x == 0) write_bad(p, Q_out, T0_out, Didx_out, dep_out, sig_out, lnp_out);
        return;
    }
    const unsigned FULL = 0xffffffffu;
    const int64_t n_phi = spc.n_phi;
    const int64_t n_cells = n_phi * n_D;
    const unsigned long long ulast = spp ? ulast_in : slot_ulast(t_ref, t_last, dt);
    const unsigned long long ustep = spc.ustep, uph = spc.uph;
    float bl = -INFINITY, bD = NAN, bs2 = NAN;
    long long bc = LLONG_MAX;
    if (threadIdx.x == 0) sh_best = 0u;     // key below every finite float
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    SCell* q = sh_q[wid];
    int nq = 0;                              // warp-uniform queue lengths
    long long* qa = sh_qa[wid];
    int* qad = sh_qad[wid];
    int na = 0;
    const unsigned ns1 = (unsigned)(n_slots - 1);
    // the gain walk adds 4 positions past ulast at most: ustep < 2^60 keeps
    // them from wrapping (ulast < 2^62).  The cascade needs the threshold to
    // rise before it pays: periods of fewer than NU_CASCADE_ROUNDS rounds of
    // cells per warp (short light curves) run the first pass on every cell.
    const bool cascade = CASC && lgm != nullptr && ustep < (1ull << 60) &&
                         n_cells >= (int64_t)NU_CASCADE_ROUNDS * blockDim.x;
    auto best_now = [&]() {
        const unsigned int kb = sh_best;
        return fmaxf(bl, kb ? __uint_as_float((kb >> 31) ? (kb & 0x7fffffffu) : ~kb)
                            : -INFINITY);
    };
    // second pass of queued cell e, by one lane
    auto pass2 = [&](const SCell& e) {
        const Node4<float>* rd = rec + (int64_t)e.d * n_slots;
        SlotPass2 p2;
        p2.init(e.s2, e.Dl);
        unsigned long long u = e.u0;
        for (int k = 0; k < e.kmax; ++k, u += ustep) {
            const SlotEvent ev = slot_event(rd, u);
            p2.add(ev.d, ev.s);
        }
        const float lnp = e.s_l - 0.5f * (p2.lsum * 0.693147180559945f + p2.quad.s);
        if (!(lnp == lnp)) return;
        if (lnp > bl || (lnp == bl && e.cell < bc)) {
            bl = lnp;
            bc = e.cell;
            bD = p2.Dl;
            bs2 = p2.s2;
        }
        const unsigned int b32 = __float_as_uint(lnp);
        atomicMax(&sh_best, (b32 >> 31) ? ~b32 : (b32 | 0x80000000u));
    };
    // first pass and bound of cell (dl, jl); *ub receives the bound (-inf:
    // no event) and e the queue entry; returns whether the cell is kept
    auto pass1 = [&](int dl, int64_t jl, long long cl, SCell& e, float* ub) -> bool {
        *ub = -INFINITY;
        const unsigned long long u0 = (unsigned long long)jl * uph;
        if (u0 > ulast) return false;
        // epochs with u <= ulast, counted as they are walked
        const Node4<float>* rd = rec + (int64_t)dl * n_slots;
        SlotPass1 p1;
        p1.init();
        int kmax = 0;
        // two epochs' record loads in flight
#pragma unroll 2
        for (unsigned long long u = u0; u <= ulast; u += ustep, ++kmax) p1.add(slot_event(rd, u));
        if (p1.K == 0) return false;
        *ub = p1.s_l.s + 0.5f;
        if (cannot_win_f(p1.s_l.s, p1.s_inv.s, p1.s_d.s, p1.s_dd, p1.ivmax, best_now()))
            return false;
        const float s2 = 1.0f / p1.s_inv.s;
        e = SCell{u0, cl, p1.s_l.s, s2, s2 * p1.s_d.s, dl, kmax, 0};
        return true;
    };
    auto push_b = [&](bool keep, const SCell& e) {
        const unsigned m = __ballot_sync(FULL, keep);
        if (keep) q[nq + __popc(m & ((1u << lane) - 1u))] = e;
        nq += __popc(m);
        __syncwarp();
    };
    auto flush_b = [&]() {
        pass2(q[lane]);
        __syncwarp();
        nq -= 32;
        SCell e2;
        if (lane < nq) e2 = q[32 + lane];
        __syncwarp();
        if (lane < nq) q[lane] = e2;
        __syncwarp();
    };
    // first passes of the first cnt entries of queue A, one per lane; the
    // survivors join queue B, which is flushed at once when it holds 32 (so
    // it never holds more than 63 entries)
    auto flush_a = [&](int h, int cnt) {
        SCell e;
        float ub;
        bool keep = false;
        if (lane < cnt) {
            const long long cl = qa[h + lane];
            const int dl = qad[h + lane];
            keep = pass1(dl, cl - (int64_t)dl * n_phi, cl, e, &ub);
        }
        push_b(keep, e);
        if (nq >= 32) flush_b();
    };
    if (cascade) {
        // cells W durations at a time (one gain group, one phase per lane),
        // as in the FP64 fold: the first and the direct rounds pass every
        // cell to queue A, the others those whose gain bound reaches the
        // threshold (with the margins of cannot_win_f on top of the rounding
        // of the sum)
        const int W = gain_width(n_D);
        const int64_t n_gc = (int64_t)((n_D + W - 1) / W) * n_phi;
        const int dr = NU_GAIN_DIRECT_ROUNDS / W > 0 ? NU_GAIN_DIRECT_ROUNDS / W : 1;
        const unsigned zs = ns1 - 1u;
        int gi = (int)(threadIdx.x / n_phi);
        int64_t j = (int64_t)threadIdx.x - (int64_t)gi * n_phi;
        bool first = true;
        int direct = 0;                      // rounds left without the gain bound
        for (int64_t base = (int64_t)wid * 32; base < n_gc; base += blockDim.x,
                     j += blockDim.x) {
            while (j >= n_phi) {
                j -= n_phi;
                ++gi;
            }
            const int d0 = gi * W;
            const int nv = base + lane < n_gc ? min(W, n_D - d0) : 0;   // this lane's cells
            unsigned pass = 0u;
            if (first || direct > 0) {
                if (!first) --direct;
                first = false;
                pass = (1u << nv) - 1u;
            } else {
                if (nv > 0) {
                    float4 sk;
                    const float K = gain_walk64(lgm + (int64_t)gi * n_slots * W, W, zs,
                                                (unsigned long long)j * uph, ustep, ulast + 1,
                                                sk);
                    const float f = fmaf(K + 16.f, 1.1920929e-7f, 1.f);
                    const float thr = best_now();
                    if (K > 0.f)
                        for (int i = 0; i < nv; ++i) {
                            const float gb = gain_col(sk, i) * f + 0.5f;
                            if (!(gb + 1e-4f * fmaxf(1.f, fabsf(gb)) < thr)) pass |= 1u << i;
                        }
                }
                const int np = __reduce_add_sync(FULL, (unsigned)__popc(pass));
                const int nt = __reduce_add_sync(FULL, (unsigned)nv);
                if (nt > 0 && np * 32 >= NU_GAIN_PASS_MAX * nt) direct = dr;
            }
            for (int i = 0; i < W; ++i) {
                const bool keep = (pass >> i) & 1u;
                const unsigned m = __ballot_sync(FULL, keep);
                if (keep) {
                    const int pos = na + __popc(m & ((1u << lane) - 1u));
                    qa[pos] = (long long)(d0 + i) * n_phi + j;
                    qad[pos] = d0 + i;
                }
                na += __popc(m);
                __syncwarp();
            }
            // queue A holds at most 31 + 32 W entries here
            int h = 0;
            for (; na - h >= 32; h += 32) flush_a(h, 32);
            if (h > 0) {
                na -= h;
                long long c2 = 0;
                int d2 = 0;
                if (lane < na) {
                    c2 = qa[h + lane];
                    d2 = qad[h + lane];
                }
                __syncwarp();
                if (lane < na) {
                    qa[lane] = c2;
                    qad[lane] = d2;
                }
                __syncwarp();
            }
        }
        if (na > 0) flush_a(0, na);
    } else {
        int d = (int)(threadIdx.x / n_phi);
        int64_t j = (int64_t)threadIdx.x - (int64_t)d * n_phi;
        for (int64_t base = (int64_t)wid * 32; base < n_cells; base += blockDim.x,
                     j += blockDim.x) {
            while (j >= n_phi) {
                j -= n_phi;
                ++d;
            }
            const int64_t cell = base + lane;
            SCell e;
            float ub = -INFINITY;
            const bool keep = cell < n_cells && pass1(d, j, cell, e, &ub);
            push_b(keep, e);
            if (nq >= 32) flush_b();
        }
    }
    if (nq >= 32) flush_b();
    if (lane < nq) pass2(q[lane]);
    // block argmax in FP32 (larger ln P, ties to the smaller cell): warp
    // shuffles, then the warps' winners through shared memory; FP64 only for
    // the one result (the FP64 pipe is 1/64 of the FP32 one on this part)
    for (int o = 16; o > 0; o >>= 1) {
        const float l2 = __shfl_xor_sync(FULL, bl, o);
        const long long c2 = __shfl_xor_sync(FULL, bc, o);
        const float D2 = __shfl_xor_sync(FULL, bD, o);
        const float s2 = __shfl_xor_sync(FULL, bs2, o);
        if (l2 > bl || (l2 == bl && c2 < bc)) {
            bl = l2;
            bc = c2;
            bD = D2;
            bs2 = s2;
        }
    }
    __shared__ float sh_bl[MAXT / 32], sh_bD[MAXT / 32], sh_bs2[MAXT / 32];
    __shared__ long long sh_bc[MAXT / 32];
    if (lane == 0) {
        sh_bl[wid] = bl;
        sh_bc[wid] = bc;
        sh_bD[wid] = bD;
        sh_bs2[wid] = bs2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (sh_bl[w] > bl || (sh_bl[w] == bl && sh_bc[w] < bc)) {
                bl = sh_bl[w];
                bc = sh_bc[w];
                bD = sh_bD[w];
                bs2 = sh_bs2[w];
            }
        Best b{-INFINITY, LLONG_MAX, NAN, NAN};
        if (bc != LLONG_MAX) b = Best{(double)bl, bc, (double)bD, sqrt((double)bs2)};
        write_best(b, p, n_phi, t_ref, P, Q_out, T0_out, Didx_out, dep_out, sig_out, lnp_out);
    }
}

#ifndef NU_SLOTS_SMALL
#define NU_SLOTS_SMALL 128         // block size of the mixed fold on large grids
#endif
#ifndef NU_SLOTS_SMALL_FROM
#define NU_SLOTS_SMALL_FROM 8192   // periods from which it is used
#endif
#ifndef NU_SLOTS_MIN_BLOCKS
#define NU_SLOTS_MIN_BLOCKS 4
#endif
#ifndef NU_SLOTS_CASC_MIN_BLOCKS
#define NU_SLOTS_CASC_MIN_BLOCKS 4
#endif

template <int KC, int MAXT, bool CASC>
__global__ void __launch_bounds__(MAXT, (CASC ? NU_SLOTS_CASC_MIN_BLOCKS : NU_SLOTS_MIN_BLOCKS) * 256 / MAXT)
k_fold_slots(const Node4<float>* __restrict__ rec, const float* __restrict__ lgm,
             int64_t n_slots, int n_D, double dt, double t_ref, double t_last,
             const double* __restrict__ periods, int64_t n_P, double* __restrict__ Q_out,
             double* __restrict__ T0_out, int* __restrict__ Didx_out,
             double* __restrict__ dep_out, double* __restrict__ sig_out,
             double* __restrict__ lnp_out) {
    if ((int64_t)blockIdx.x >= n_P) return;
    const int64_t p = period_slot(blockIdx.x, periods, n_P);
    fold_slots_one<KC, MAXT, CASC>(rec, lgm, n_slots, n_D, dt, t_ref, t_last, periods[p], p,
                                   nullptr, 0ull,
                                   Q_out, T0_out, Didx_out, dep_out, sig_out, lnp_out);
}

// ------------------------------------------------------------ batch path

// Persistent fold over (curve, period) work items taken from a device
// counter (no waits: a block takes items until none are left).  kind 0: the
// exact FP64-epoch path with FP64 values; 1: exact path, FP32 values;
// 2: slot path (mixed precision, regular grids).  Items of curves that do not
// use this kernel's path are skipped.
// Resident blocks per SM the registers are sized for, by path and block size.
// The FP64 batch kernel carries the work-item loop besides the screen: at 80
// registers it spills, at 96 (10 x 64 threads) it does not; slots as the
// single-curve kernel (64 registers at any size).
template <int KIND, int MAXT>
struct BatchBlocks {
    static constexpr int value =
        KIND == 0 || KIND == 4 ? (MAXT <= 64 ? 10 : (MAXT <= 128 ? 5 : NU_SCREEN_MIN_BLOCKS))
                  : (KIND == 2 ? NU_SLOTS_CASC_MIN_BLOCKS * 256 / MAXT
                               : KIND == 3 ? NU_SLOTS_MIN_BLOCKS * 256 / MAXT : 1);
};

template <int KIND, int MAXT>
__global__ void __launch_bounds__(MAXT, BatchBlocks<KIND, MAXT>::value)
k_fold_batch(const FoldSeg* __restrict__ segs, int n_seg, const double* __restrict__ t,
             const void* __restrict__ nodes, const ScreenRec* __restrict__ screen,
             const ulonglong2* __restrict__ vpair, const ScreenRec* __restrict__ srec,
             const float* __restrict__ lm3, const float* __restrict__ lgm,
             const unsigned* __restrict__ reg,
             const unsigned long long* __restrict__ peak,
             const int* __restrict__ bucket,
             const Node4<float>* __restrict__ rec, int n_D, double dt, double gap_factor,
             const double* __restrict__ periods, const PeriodConst* __restrict__ ptab,
             int64_t n_P, unsigned long long* counter,
             double* __restrict__ Q_out, double* __restrict__ T0_out,
             int* __restrict__ Didx_out, double* __restrict__ dep_out,
             double* __restrict__ sig_out, double* __restrict__ lnp_out) {
    __shared__ unsigned long long item_sh;
    const unsigned long long total = (unsigned long long)n_seg * (unsigned long long)n_P;
    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) item_sh = atomicAdd(counter, 1ull);
        __syncthreads();
        const unsigned long long item = item_sh;
        if (item >= total) break;
        const int g = (int)(item / (unsigned long long)n_P);
        const int64_t p = period_slot((int64_t)(item % (unsigned long long)n_P), periods, n_P);
        const FoldSeg fs = segs[g];
        if ((KIND == 2 || KIND == 3) != (fs.use_slots != 0)) continue;
        const int64_t o = (int64_t)g * n_P + p;
        if (KIND == 2 || KIND == 3) {
            // (the slot path's period table shares the FP64 path's buffer)
            fold_slots_one<8, MAXT, KIND == 2>(
                rec + fs.rec_off, lgm + fs.gain_off, fs.n_slots, n_D, dt, fs.t_ref, fs.t_last,
                periods[p], o, reinterpret_cast<const SlotPeriod*>(ptab) + p, fs.ulast, Q_out,
                T0_out, Didx_out, dep_out, sig_out, lnp_out);
        } else {
            FoldGeom gg{t + fs.s_off, fs.n_t0, fs.t_ref, fs.t_last, dt, 1.0 / dt,
                        gap_factor * dt, bucket + fs.bucket_off, fs.n_bucket};
            if (KIND == 0 || KIND == 4) {
                const ScreenGeom sg{screen + fs.s_off * n_D, vpair + fs.s_off,
                                    srec + fs.srec_off, fs.n_slots,
                                    reg + 2 * g, fs.screen, peak + g, lm3 + fs.gain_off};
                fold_screened_one<MAXT, true, KIND == 4>(gg, sg,
                                              (const Node8<double>*)nodes + fs.s_off * n_D, n_D,
                                              periods[p], o, Q_out, T0_out, Didx_out, dep_out,
                                              sig_out, lnp_out, ptab + p);
            }
            else
                fold_exact_one<float, 8, MAXT>(gg, (const Node8<float>*)nodes + fs.s_off * n_D, n_D,
                                         periods[p], o, Q_out, T0_out, Didx_out, dep_out,
                                         sig_out, lnp_out);
        }
    }
}

// Per-curve node records (exact path) and bucket tables; slot tables.
template <typename T>
__global__ void k_nodes_batch(const T* __restrict__ depth, const T* __restrict__ var,
                              const T* __restrict__ gain, const double* __restrict__ t,
                              const FoldSeg* __restrict__ segs, int n_seg,
                              const int64_t* __restrict__ s_off, int n_D, double gap_max,
                              Node8<T>* __restrict__ nodes) {
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gid >= s_off[n_seg] * (int64_t)n_D) return;
    int lo = 0, hi = n_seg;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s_off[mid] * (int64_t)n_D <= gid) lo = mid; else hi = mid;
    }
    const int64_t s0 = s_off[lo], ng = s_off[lo + 1] - s0;
    const int64_t i = (gid - s0 * n_D) % ng;
    nodes[gid] = make_node8<T>(depth, var, gain, t + s0, gid, i, ng, gap_max);
}

template <typename T>
__global__ void k_screen_batch(const T* __restrict__ depth, const T* __restrict__ var,
                               const T* __restrict__ gain, const double* __restrict__ t,
                               const FoldSeg* __restrict__ segs, int n_seg,
                               const int64_t* __restrict__ s_off, int n_D, double gap_max,
                               double dt, ScreenRec* __restrict__ rec,
                               ulonglong2* __restrict__ vpair, ScreenRec* __restrict__ srec,
                               float* __restrict__ lint,
                               const int* __restrict__ slot_of) {
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gid >= s_off[n_seg] * (int64_t)n_D) return;
    int lo = 0, hi = n_seg;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s_off[mid] * (int64_t)n_D <= gid) lo = mid; else hi = mid;
    }
    const FoldSeg fs = segs[lo];
    if (!fs.screen) return;
    const int64_t s0 = s_off[lo], ng = s_off[lo + 1] - s0;
    const int64_t w = gid - s0 * n_D;
    const int64_t d = w / ng, i = w - d * ng;
    make_screen<T>(depth, var, gain, t + s0, gid, i, ng, d, gap_max, dt, rec,
                   srec + fs.srec_off, lint + fs.srec_off, fs.n_slots,
                   slot_of + s0, vpair + s0);
}

// Slots of every sample of the screened curves (reg: two words per curve).
__global__ void k_slot_offsets_batch(const double* __restrict__ t,
                                     const FoldSeg* __restrict__ segs, int n_seg,
                                     const int64_t* __restrict__ s_off, double inv_dt,
                                     int* __restrict__ slot_of, unsigned* __restrict__ reg) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= s_off[n_seg]) return;
    int lo = 0, hi = n_seg;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s_off[mid] <= i) lo = mid; else hi = mid;
    }
    const FoldSeg fs = segs[lo];
    if (!fs.screen) return;
    const int64_t s0 = s_off[lo];
    slot_offset(t + s0, i - s0, inv_dt, fs.n_slots, slot_of + s0, reg + 2 * lo);
}

__global__ void k_buckets_batch(const double* __restrict__ t, const FoldSeg* __restrict__ segs,
                                int n_seg, int64_t n_bucket_total, double dt,
                                int* __restrict__ bucket) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= n_bucket_total) return;
    int lo = 0, hi = n_seg;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (segs[mid].bucket_off <= b) lo = mid; else hi = mid;
    }
    const FoldSeg fs = segs[lo];
    const double edge = fs.t_ref + (double)(b - fs.bucket_off) * dt;
    const double* t0 = t + fs.s_off;
    int64_t l = 0, h = fs.n_t0;
    while (l < h) {
        const int64_t mid = (l + h) >> 1;
        if (t0[mid] <= edge) l = mid + 1; else h = mid;
    }
    bucket[b] = (int)l;
}

__global__ void k_slot_fill_batch(const float* __restrict__ depth, const float* __restrict__ var,
                                  const float* __restrict__ gain, const double* __restrict__ t,
                                  const FoldSeg* __restrict__ segs, int n_seg,
                                  const int64_t* __restrict__ s_off, int n_D, double inv_dt,
                                  Node4<float>* __restrict__ rec) {
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gid >= s_off[n_seg] * (int64_t)n_D) return;
    int lo = 0, hi = n_seg;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s_off[mid] * (int64_t)n_D <= gid) lo = mid; else hi = mid;
    }
    const FoldSeg fs = segs[lo];
    if (!fs.use_slots) return;
    const int64_t s0 = s_off[lo], ng = s_off[lo + 1] - s0;
    const int64_t w = gid - s0 * n_D;
    const int64_t d = w / ng, i = w - d * ng;
    const int64_t s = (int64_t)rint((t[s0 + i] - fs.t_ref) * inv_dt);
    if (s < 0 || s >= fs.n_slots) return;
    const float dd = depth[gid], v = var[gid], l = gain[gid];
    Node4<float> r;
    r.d = dd;
    r.l = l;
    r.s = (isfinite(dd) && isfinite(v) && isfinite(l) && v > 0.f) ? sqrtf(v) : NAN;
    r.ig = 0.f;
    rec[fs.rec_off + d * fs.n_slots + s] = r;
}

// Regularity of each curve's epochs for the slot path (flag[g] = 1 if not).
__global__ void k_slots_batch(const double* __restrict__ t, const int64_t* __restrict__ s_off,
                              int n_seg, double inv_dt, int* __restrict__ irregular) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= s_off[n_seg]) return;
    int lo = 0, hi = n_seg;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s_off[mid] <= i) lo = mid; else hi = mid;
    }
    const int64_t s0 = s_off[lo];
    const double tr = t[s0];
    const double u = (t[i] - tr) * inv_dt;
    const double sl = rint(u);
    bool bad = !(fabs(u - sl) <= 1e-3) || !(sl >= 0.0) || sl > 2.0e9;
    if (i > s0) bad = bad || !(sl > rint((t[i - 1] - tr) * inv_dt));
    if (bad) atomicExch(&irregular[lo], 1);
}

// Host side of the batch fold: per-curve layout and launches.

void plan_fold_batch(const std::vector<int64_t>& s_off, const std::vector<double>& t_first,
                     const std::vector<double>& t_last, const std::vector<int>& irregular,
                     bool fp64, double dt, double gap_factor, int n_D, FoldBatch& fb) {
    const int n_seg = (int)t_first.size();
    fb.segs.resize(n_seg);
    for (int g = 0; g < n_seg; ++g) {
        FoldSeg& f = fb.segs[g];
        f.s_off = s_off[g];
        f.n_t0 = s_off[g + 1] - s_off[g];
        f.t_ref = t_first[g];
        f.t_last = t_last[g];
        f.ulast = slot_ulast(f.t_ref, f.t_last, dt);
        const double span = (t_last[g] - t_first[g]) / dt;
        f.n_bucket = (int64_t)span + 2;
        f.n_slots = f.n_bucket + 2;
        f.use_slots = (!fp64 && gap_factor > 1.0 && gap_factor < 2.0 && span < 4.0e6 &&
                       !irregular[g]) ? 1 : 0;
        f.screen = (fp64 && gap_factor < 2.0 && span < 8.0e6) ? 1 : 0;
        f.srec_off = fb.n_srec_total;
        fb.n_srec_total += f.screen ? f.n_slots * n_D : 0;
        f.gain_off = fb.n_gain_total;
        fb.n_gain_total += (fp64 ? f.screen : f.use_slots) ? f.n_slots * gain_cols(n_D) : 0;
        f.bucket_off = fb.n_bucket_total;
        fb.n_bucket_total += f.use_slots ? 0 : f.n_bucket;
        f.rec_off = fb.n_rec_total;
        fb.n_rec_total += f.use_slots ? f.n_slots * n_D : 0;
        fb.any_slots = fb.any_slots || f.use_slots;
        if (f.use_slots && f.n_slots * (int64_t)n_D >= (int64_t)NU_CASCADE_ROUNDS * 128)
            fb.slot_cascade = true;
        fb.any_exact = fb.any_exact || !f.use_slots;
    }
}

cudaError_t launch_fold_prep(const FoldBatch& fb, const FoldSeg* segs_dev,
                             const int64_t* s_off_dev, int n_seg, int64_t n_total, bool fp64,
                             const double* t, const void* depth, const void* var,
                             const void* gain, int n_D, double dt, double gap_factor,
                             const FoldScratch& fs, cudaStream_t st, int* n_launched) {
    int launched = 0;
    *n_launched = 0;
    const int64_t ngrid = n_total * (int64_t)n_D;
    cudaError_t e = cudaSuccess;
    if (fb.any_exact) {
        if (fp64) {
            const ExactLayout L = exact_layout(n_total, n_D, true);
            k_nodes_batch<double><<<div_up(ngrid, 256), 256, 0, st>>>(
                (const double*)depth, (const double*)var, (const double*)gain, t, segs_dev,
                n_seg, s_off_dev, n_D, gap_factor * dt, (Node8<double>*)fs.nodes);
            ++launched;
            e = cudaMemsetAsync(fs.reg, 0, (size_t)n_seg * 2 * sizeof(unsigned), st);
            if (e != cudaSuccess) {
                *n_launched = launched;
                return e;
            }
            k_slot_offsets_batch<<<div_up(n_total, 256), 256, 0, st>>>(
                t, segs_dev, n_seg, s_off_dev, 1.0 / dt, fs.slot_of, fs.reg);
            k_fill_screen<<<div_up(fb.n_srec_total + 1, 256), 256, 0, st>>>(
                fs.srec, fb.n_srec_total);
            launched += 2;
            e = cudaMemsetAsync(fs.lint, 0, (size_t)(fb.n_srec_total + 1) * sizeof(float), st);
            if (e != cudaSuccess) {
                *n_launched = launched;
                return e;
            }
            k_screen_batch<double><<<div_up(ngrid, 256), 256, 0, st>>>(
                (const double*)depth, (const double*)var, (const double*)gain, t, segs_dev,
                n_seg, s_off_dev, n_D, gap_factor * dt, dt,
                (ScreenRec*)((char*)fs.nodes + L.off_screen),
                (ulonglong2*)((char*)fs.nodes + L.off_vpos), fs.srec, fs.lint, fs.slot_of);
            k_lmax3<<<div_up(fb.n_gain_total + 1, 256), 256, 0, st>>>(
                fs.lint, segs_dev, n_seg, 0, n_D, fb.n_gain_total, fs.lm3);
            launched += 2;
            e = cudaMemsetAsync(fs.peak, 0, (size_t)n_seg * sizeof(unsigned long long), st);
            if (e != cudaSuccess) {
                *n_launched = launched;
                return e;
            }
            k_gain_peak<<<dim3(n_seg, 1), 256, 0, st>>>((const double*)gain, s_off_dev, 0, n_D,
                                                       fs.peak);
            ++launched;
        } else {
            k_nodes_batch<float><<<div_up(ngrid, 256), 256, 0, st>>>(
                (const float*)depth, (const float*)var, (const float*)gain, t, segs_dev, n_seg,
                s_off_dev, n_D, gap_factor * dt, (Node8<float>*)fs.nodes);
            ++launched;
        }
        k_buckets_batch<<<div_up(fb.n_bucket_total, 256), 256, 0, st>>>(
            t, segs_dev, n_seg, fb.n_bucket_total, dt, fs.bucket);
        ++launched;
    }
    if (fb.any_slots) {
        k_fill_nan<<<div_up(fb.n_rec_total, 256), 256, 0, st>>>(fs.rec, fb.n_rec_total);
        k_slot_fill_batch<<<div_up(ngrid, 256), 256, 0, st>>>(
            (const float*)depth, (const float*)var, (const float*)gain, t, segs_dev, n_seg,
            s_off_dev, n_D, 1.0 / dt, fs.rec);
        k_slot_gain<<<div_up(fb.n_gain_total + 1, 256), 256, 0, st>>>(
            fs.rec, segs_dev, n_seg, 0, n_D, fb.n_gain_total, fs.lgm);
        launched += 3;
    }
    *n_launched = launched;
    return cudaSuccess;
}

// The persistent fold kernels; counter[0..1] must be zero.  blocks_per_sm
// and threads come from the autotuner.
int launch_fold_batch(const FoldBatch& fb, const FoldSeg* segs_dev, int n_seg,
                      int64_t n_total, bool fp64, const double* t, const FoldScratch& fs,
                      int n_D, double dt, double gap_factor, const double* periods,
                      int64_t n_P, unsigned long long* counter, int grid, int threads,
                      double* Q, double* T0, int* Didx, double* dep, double* sig, double* lnp,
                      cudaStream_t st) {
    int launched = 0;
    const ExactLayout L = exact_layout(n_total, n_D, fp64);
    const ScreenRec* screen =
        fp64 ? (const ScreenRec*)((const char*)fs.nodes + L.off_screen) : nullptr;
    const ulonglong2* vpair =
        fp64 ? (const ulonglong2*)((const char*)fs.nodes + L.off_vpos) : nullptr;
    // the kernel instance whose shared arrays and register budget match the
    // block size (64, 128 or 256 threads)
#define NU_FB(KIND_, MAXT_, CTR_)                                                          \
    k_fold_batch<KIND_, MAXT_><<<grid, MAXT_, 0, st>>>(                                  \
        segs_dev, n_seg, t, fs.nodes, screen, vpair, fs.srec, fs.lm3, fs.lgm, fs.reg,      \
        fs.peak, fs.bucket,                                                                \
        fs.rec, n_D, dt, gap_factor, periods, fs.ptab, n_P, CTR_, Q, T0, Didx, dep, sig, lnp)
#define NU_FB_SIZE(KIND_, CTR_)                                                            \
    do {                                                                                   \
        if (threads <= 64) NU_FB(KIND_, 64, CTR_);                                         \
        else if (threads <= 128) NU_FB(KIND_, 128, CTR_);                                  \
        else NU_FB(KIND_, 256, CTR_);                                                      \
    } while (0)
    if (fb.any_exact) {
        if (fp64) {
            k_period_consts<<<div_up(n_P, 256), 256, 0, st>>>(periods, n_P, dt, fs.ptab);
            ++launched;
            if (gain_width(n_D) > 1)
                NU_FB_SIZE(4, counter);
            else
                NU_FB_SIZE(0, counter);
        } else
            NU_FB_SIZE(1, counter);
        ++launched;
    }
    if (fb.any_slots) {
        k_slot_periods<<<div_up(n_P, 256), 256, 0, st>>>(periods, n_P, dt,
                                                         reinterpret_cast<SlotPeriod*>(fs.ptab));
        ++launched;
        if (fb.slot_cascade)
            NU_FB_SIZE(2, counter + 1);
        else
            NU_FB_SIZE(3, counter + 1);
        ++launched;
    }
#undef NU_FB_SIZE
#undef NU_FB
    return launched;
}

int launch_slots_test(const double* t, const int64_t* s_off_dev, int n_seg, int64_t n_total,
                      double dt, int* irregular, cudaStream_t st) {
    k_slots_batch<<<div_up(n_total, 256), 256, 0, st>>>(t, s_off_dev, n_seg, 1.0 / dt,
                                                       irregular);
    return 1;
}

}  // namespace nu

// ------------------------------------------------ single-curve host side
namespace nu {

// Scratch layout of the single-curve fold.
struct SingleLayout {
    ExactLayout el;
    size_t exact, bucket, slot_of, flag, rec, srec, lint, lm3, lgm, total;
};

static SingleLayout single_layout(int64_t n_t0, int n_D, int64_t n_bucket, bool fp64) {
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    SingleLayout L;
    L.el = exact_layout(n_t0, n_D, fp64);
    const int64_t n_slots = n_bucket + 2;          // slot records, NaN padded
    L.exact = 0;
    L.bucket = L.exact + L.el.total;
    L.slot_of = L.bucket + al((size_t)n_bucket * sizeof(int));
    L.flag = L.slot_of + al((size_t)n_t0 * sizeof(int));
    L.rec = L.flag + 256;
    L.srec = L.rec + (fp64 ? 0 : al((size_t)n_slots * n_D * sizeof(Node4<float>)));
    L.lint = L.srec + (fp64 ? al((size_t)n_slots * n_D * sizeof(ScreenRec)) : 0);
    L.lm3 = L.lint + (fp64 ? al((size_t)n_slots * n_D * sizeof(float)) : 0);
    L.lgm = L.lm3 + (fp64 ? al((size_t)n_slots * gain_cols(n_D) * sizeof(float)) : 0);
    L.total = L.lgm + (fp64 ? 0 : al((size_t)n_slots * gain_cols(n_D) * sizeof(float)));
    return L;
}

// Enqueue the fold of one light curve on st with its scratch at `scratch`
// (laid out by single_layout).  The mixed-precision slot test reads one flag
// back (one synchronisation of st).
static nu_status single_fold(const char* who, char* scratch, const SingleLayout& L,
                             const double* t0s_dev, int64_t n_t0, int n_D, const void* depth_dev,
                             const void* var_dev, const void* dlnl_dev, bool fp64,
                             const double* periods_dev, int64_t n_P, double phase_step,
                             double gap_factor, double t_ref, double t_last, int64_t n_bucket,
                             cudaStream_t st, double* Q_dev, double* T0_dev, int32_t* D_idx_dev,
                             double* depth_out_dev, double* sigma_out_dev, double* lnP_dev) {
    const double span_steps = (t_last - t_ref) / phase_step;
    const int64_t ngrid = n_t0 * (int64_t)n_D;
    const int64_t n_slots = n_bucket + 2;
    void* nodes = scratch + L.exact;
    int* bucket = (int*)(scratch + L.bucket);
    int* slot_of = (int*)(scratch + L.slot_of);
    int* flag = (int*)(scratch + L.flag);
    Node4<float>* rec = (Node4<float>*)(scratch + L.rec);
    int launched = 0;
    cudaError_t e = cudaSuccess;
    // the slot path needs a regular grid and a gap rule that only joins
    // neighbouring slots (1 < gap_factor < 2)
    bool use_slots = !fp64 && gap_factor > 1.0 && gap_factor < 2.0 && span_steps < 4.0e6;
    if (use_slots) {
        int irregular = 0;
        e = cudaMemsetAsync(flag, 0, sizeof(int), st);
        k_slots<<<div_up(n_t0, 256), 256, 0, st>>>(t0s_dev, n_t0, t_ref, 1.0 / phase_step,
                                                  slot_of, flag);
        ++launched;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&irregular, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            count_launches(launched);
            return cuda_fail(e, (std::string(who) + ": slot test").c_str());
        }
        use_slots = irregular == 0;
    }
    if (use_slots) {
        const int64_t nrec = n_slots * n_D;
        k_fill_nan<<<div_up(nrec, 256), 256, 0, st>>>(rec, nrec);
        k_slot_fill<<<div_up(ngrid, 256), 256, 0, st>>>(
            (const float*)depth_dev, (const float*)var_dev, (const float*)dlnl_dev, slot_of,
            n_t0, n_D, n_slots, rec);
        float* lgm = (float*)(scratch + L.lgm);
        const int64_t nlg = n_slots * gain_cols(n_D);
        k_slot_gain<<<div_up(nlg, 256), 256, 0, st>>>(rec, nullptr, 0, n_slots, n_D, nlg, lgm);
        // the cascade's instance where a period can hold enough cells for it
        const bool casc = nrec >= (int64_t)NU_CASCADE_ROUNDS * 128;
#define NU_FS(MAXT_, CASC_)                                                                \
    k_fold_slots<8, MAXT_, CASC_><<<(unsigned)n_P, MAXT_, 0, st>>>(                        \
        rec, lgm, n_slots, n_D, phase_step, t_ref, t_last, periods_dev, n_P, Q_dev, T0_dev, \
        D_idx_dev, depth_out_dev, sigma_out_dev, lnP_dev)
        if (n_P >= NU_SLOTS_SMALL_FROM) {
            if (casc) NU_FS(NU_SLOTS_SMALL, true); else NU_FS(NU_SLOTS_SMALL, false);
        } else {
            if (casc) NU_FS(256, true); else NU_FS(256, false);
        }
#undef NU_FS
        launched += 4;
    } else {
        k_buckets<<<div_up(n_bucket, 256), 256, 0, st>>>(t0s_dev, n_t0, t_ref, phase_step,
                                                        n_bucket, bucket);
        FoldGeom g{t0s_dev, n_t0, t_ref, t_last, phase_step, 1.0 / phase_step,
                   gap_factor * phase_step, bucket, n_bucket};
        if (fp64) {
            ScreenRec* nrec = (ScreenRec*)(scratch + L.exact + L.el.off_screen);
            ulonglong2* vpair = (ulonglong2*)(scratch + L.exact + L.el.off_vpos);
            ScreenRec* srec = (ScreenRec*)(scratch + L.srec);
            float* lint = (float*)(scratch + L.lint);
            float* lm3 = (float*)(scratch + L.lm3);
            unsigned* reg = (unsigned*)(flag + 1);
            unsigned long long* peak = (unsigned long long*)(scratch + L.flag + 16);
            const ScreenGeom sg{nrec, vpair, srec, n_slots, reg,
                                (gap_factor < 2.0 && span_steps < 8.0e6) ? 1 : 0, peak, lm3};
            e = cudaMemsetAsync(flag, 0, 256, st);
            if (e != cudaSuccess) {
                count_launches(launched);
                return cuda_fail(e, (std::string(who) + ": memset").c_str());
            }
            k_slot_offsets<<<div_up(n_t0, 256), 256, 0, st>>>(t0s_dev, n_t0, 1.0 / phase_step,
                                                              n_slots, slot_of, reg);
            k_fill_screen<<<div_up(n_slots * n_D, 256), 256, 0, st>>>(srec, n_slots * n_D);
            e = cudaMemsetAsync(lint, 0, (size_t)n_slots * n_D * sizeof(float), st);
            if (e != cudaSuccess) {
                count_launches(launched + 2);
                return cuda_fail(e, (std::string(who) + ": memset").c_str());
            }
            k_nodes<double><<<div_up(ngrid, 256), 256, 0, st>>>(
                (const double*)depth_dev, (const double*)var_dev, (const double*)dlnl_dev,
                t0s_dev, n_t0, n_D, g.gap_max, (Node8<double>*)nodes);
            k_screen<double><<<div_up(ngrid, 256), 256, 0, st>>>(
                (const double*)depth_dev, (const double*)var_dev, (const double*)dlnl_dev,
                t0s_dev, n_t0, n_D, g.gap_max, phase_step, nrec, srec, lint, n_slots, slot_of,
                vpair);
            const int64_t nlm = n_slots * gain_cols(n_D);
            k_lmax3<<<div_up(nlm, 256), 256, 0, st>>>(lint, nullptr, 0, n_slots, n_D, nlm, lm3);
            k_gain_peak<<<dim3(1, (unsigned)std::min<int64_t>(div_up(ngrid, 2048), 608)), 256, 0,
                          st>>>((const double*)dlnl_dev, nullptr, n_t0, n_D, peak);
            // One block per period.  With many periods, 2-warp blocks: 14 fit
            // on an SM (28 warps) and each period has 2 warps to seed; with
            // few, 8-warp blocks keep the GPU full (C2, 20 000 periods: 16.5 ms
            // at 256 threads, 14.0 at 128 (7 per SM), 13.6 at 64).
            // (the grouped gain walk where the durations form groups)
#define NU_FSC(MAXT_)                                                                      \
    do {                                                                                   \
        if (gain_width(n_D) > 1)                                                           \
            k_fold_screened<MAXT_, true><<<(unsigned)n_P, MAXT_, 0, st>>>(                 \
                g, sg, (const Node8<double>*)nodes, n_D, periods_dev, n_P, Q_dev, T0_dev,  \
                D_idx_dev, depth_out_dev, sigma_out_dev, lnP_dev);                         \
        else                                                                               \
            k_fold_screened<MAXT_, false><<<(unsigned)n_P, MAXT_, 0, st>>>(                \
                g, sg, (const Node8<double>*)nodes, n_D, periods_dev, n_P, Q_dev, T0_dev,  \
                D_idx_dev, depth_out_dev, sigma_out_dev, lnP_dev);                         \
    } while (0)
            if (n_P >= 8192)
                NU_FSC(64);
            else
                NU_FSC(256);
#undef NU_FSC
            launched += 8;
        } else {
            k_nodes<float><<<div_up(ngrid, 256), 256, 0, st>>>(
                (const float*)depth_dev, (const float*)var_dev, (const float*)dlnl_dev,
                t0s_dev, n_t0, n_D, g.gap_max, (Node8<float>*)nodes);
            k_fold_exact<float, 8><<<(unsigned)n_P, 256, 0, st>>>(
                g, (const Node8<float>*)nodes, n_D, periods_dev, n_P, Q_dev, T0_dev,
                D_idx_dev, depth_out_dev, sigma_out_dev, lnP_dev);
            launched += 3;
        }
    }
    count_launches(launched);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, (std::string(who) + ": launch").c_str());
    return NU_OK;
}

static nu_status check_args(const char* who, const double* t0s_dev, int64_t n_t0, int n_D,
                            const void* depth_dev, const void* var_dev, const void* dlnl_dev,
                            nu_precision prec, const double* periods_dev, int64_t n_P,
                            double gap_factor, double* Q_dev, double* T0_dev,
                            int32_t* D_idx_dev, double* depth_out_dev, double* sigma_out_dev,
                            double* lnP_dev) {
    if (!t0s_dev || !depth_dev || !var_dev || !dlnl_dev || !periods_dev || !Q_dev ||
        !T0_dev || !D_idx_dev || !depth_out_dev || !sigma_out_dev || !lnP_dev)
        return fail(NU_EINVAL, "%s: null array", who);
    if (n_t0 < 2 || n_D < 1 || n_P < 1)
        return fail(NU_EINVAL, "%s: need n_t0 >= 2, n_D >= 1, n_P >= 1", who);
    if (prec != NU_FP64 && prec != NU_MIXED) return fail(NU_EINVAL, "%s: unknown precision", who);
    if (!(gap_factor > 0.0)) return fail(NU_EINVAL, "%s: gap_factor <= 0", who);
    if (n_t0 > 2000000000LL) return fail(NU_EINVAL, "%s: n_t0 too large", who);
    if (n_P > 2147483647LL) return fail(NU_EINVAL, "%s: n_P too large", who);
    return NU_OK;
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
    const char* who = "nu_periodic_search";
    (void)Ds_host;
    nu_status s = check_args(who, t0s_dev, n_t0, n_D, depth_dev, var_dev, dlnl_dev, prec,
                             periods_dev, n_P, gap_factor, Q_dev, T0_dev, D_idx_dev,
                             depth_out_dev, sigma_out_dev, lnP_dev);
    if (s != NU_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    // grid end points (host copies; the step, when not given, is the median
    // spacing of the epochs)
    double ends[2];
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
    const bool fp64 = prec == NU_FP64;
    const SingleLayout L = single_layout(n_t0, n_D, n_bucket, fp64);
    pool_keep_memory();
    char* scratch = nullptr;
    e = cudaMallocAsync((void**)&scratch, L.total, st);
    if (e != cudaSuccess) return cuda_fail(e, "nu_periodic_search: cudaMallocAsync");
    s = single_fold(who, scratch, L, t0s_dev, n_t0, n_D, depth_dev, var_dev, dlnl_dev, fp64,
                    periods_dev, n_P, phase_step, gap_factor, t_ref, t_last, n_bucket, st,
                    Q_dev, T0_dev, D_idx_dev, depth_out_dev, sigma_out_dev, lnP_dev);
    e = cudaFreeAsync(scratch, st);
    if (s != NU_OK) return s;
    if (e != cudaSuccess) return cuda_fail(e, "nu_periodic_search: cudaFreeAsync");
    return NU_OK;
}

// ------------------------------------------------ transit masking
// One thread per epoch: the distance to the nearest transit of (P, T0),
// each operation rounded once (no contraction), decides for all durations.
template <typename T>
__global__ void k_mask_transits(const double* __restrict__ t0s, int64_t n_t0, int n_D,
                                T* __restrict__ depth, T* __restrict__ var,
                                T* __restrict__ dlnl, double P, double T0, double hw) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_t0) return;
    const double t = t0s[i];
    const double n = rint(__ddiv_rn(__dsub_rn(t, T0), P));
    const double dist = fabs(__dsub_rn(t, __dadd_rn(T0, __dmul_rn(n, P))));
    if (!(dist < hw)) return;
    for (int d = 0; d < n_D; ++d) {
        const int64_t o = (int64_t)d * n_t0 + i;
        depth[o] = T(NAN);
        var[o] = T(NAN);
        dlnl[o] = T(NAN);
    }
}

extern "C" nu_status nu_mask_transits(const double* t0s_dev, int64_t n_t0, int n_D,
                                      void* depth_dev, void* var_dev, void* dlnl_dev,
                                      nu_precision prec, double P, double T0,
                                      double half_width, void* stream) {
    if (!t0s_dev || !depth_dev || !var_dev || !dlnl_dev)
        return fail(NU_EINVAL, "nu_mask_transits: null array");
    if (n_t0 < 1 || n_D < 1) return fail(NU_EINVAL, "nu_mask_transits: need n_t0, n_D >= 1");
    if (prec != NU_FP64 && prec != NU_MIXED)
        return fail(NU_EINVAL, "nu_mask_transits: unknown precision");
    if (!(P > 0.0) || !std::isfinite(P) || !std::isfinite(T0) || !std::isfinite(half_width))
        return fail(NU_EINVAL, "nu_mask_transits: P must be finite and > 0, T0 and "
                               "half_width finite");
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == NU_FP64)
        k_mask_transits<double><<<div_up(n_t0, 256), 256, 0, st>>>(
            t0s_dev, n_t0, n_D, (double*)depth_dev, (double*)var_dev, (double*)dlnl_dev, P, T0,
            half_width);
    else
        k_mask_transits<float><<<div_up(n_t0, 256), 256, 0, st>>>(
            t0s_dev, n_t0, n_D, (float*)depth_dev, (float*)var_dev, (float*)dlnl_dev, P, T0,
            half_width);
    count_launches(1);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "nu_mask_transits: launch");
    return NU_OK;
}

// ------------------------------------------------ rotation-alias periods
// One block walks the grid in tiles of its threads; a period is dropped when
// dP = P / P_star is within tol below its ceiling (or, symmetric, of its
// nearest integer), each operation rounded once; the kept periods are written
// in input order (warp ballots, then the warps' counts in shared memory).
__global__ void __launch_bounds__(1024)
k_alias_filter(const double* __restrict__ P, int64_t n_P, double P_star, double tol,
               int symmetric, double* __restrict__ kept, int64_t* __restrict__ n_kept) {
    __shared__ int warp_cnt[32];
    __shared__ int64_t base;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int n_warps = blockDim.x >> 5;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (int64_t t0 = 0; t0 < n_P; t0 += blockDim.x) {
        const int64_t i = t0 + threadIdx.x;
        bool keep = false;
        double p = 0.0;
        if (i < n_P) {
            p = P[i];
            const double dP = __ddiv_rn(p, P_star);
            const double ref = symmetric ? rint(dP) : ceil(dP);
            keep = !(fabs(__dsub_rn(dP, ref)) < tol);
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) warp_cnt[wid] = __popc(m);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < n_warps; ++w) {
            const int c = warp_cnt[w];
            if (w < wid) before += c;
            total += c;
        }
        if (keep) kept[base + before + __popc(m & ((1u << lane) - 1u))] = p;
        __syncthreads();
        if (threadIdx.x == 0) base += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) *n_kept = base;
}

extern "C" nu_status nu_rotation_alias_filter(const double* periods_dev, int64_t n_P,
                                              double P_star, double tol, int symmetric,
                                              double* kept_dev, int64_t* n_kept_dev,
                                              void* stream) {
    if (!periods_dev || !kept_dev || !n_kept_dev)
        return fail(NU_EINVAL, "nu_rotation_alias_filter: null array");
    if (n_P < 1) return fail(NU_EINVAL, "nu_rotation_alias_filter: n_P must be >= 1");
    if (!(P_star > 0.0) || !std::isfinite(P_star) || !(tol >= 0.0) || !std::isfinite(tol))
        return fail(NU_EINVAL, "nu_rotation_alias_filter: P_star must be finite and > 0, "
                               "tol finite and >= 0");
    if (periods_dev == kept_dev)
        return fail(NU_EINVAL, "nu_rotation_alias_filter: kept must not alias periods");
    cudaStream_t st = (cudaStream_t)stream;
    k_alias_filter<<<1, 1024, 0, st>>>(periods_dev, n_P, P_star, tol, symmetric ? 1 : 0,
                                       kept_dev, n_kept_dev);
    count_launches(1);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "nu_rotation_alias_filter: launch");
    return NU_OK;
}

// ------------------------------------------------ allocation-free variant
// nu_periodic_search_noalloc runs the same kernels as nu_periodic_search but
// takes its scratch (epoch records, bucket table, slot table, flag) from the
// file-scope device array below instead of the stream-ordered pool, for
// callers that must not allocate device memory.  The array is part of the
// library image: every GPU that loads the library holds it until the process
// exits.  Its address is looked up once per device (cudaGetSymbolAddress with
// that device current) on the first call made on the device.
#define NU_NOALLOC_SCRATCH_BYTES (32ull << 20)

static __device__ __align__(256) unsigned char g_fold_scratch[NU_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_scratch_mu;
void* g_scratch_ptr[64] = {};
}

// The scratch of the device that runs the call: the stream's device, which
// must be the current device (the symbol lookup and the launches use the
// current device) and must hold the epochs.
static nu_status noalloc_scratch(cudaStream_t st, const void* t0s_dev, void** out) {
    int dev = 0, sdev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "nu_periodic_search_noalloc: cudaGetDevice");
    e = cudaStreamGetDevice(st, &sdev);
    if (e != cudaSuccess) return cuda_fail(e, "nu_periodic_search_noalloc: cudaStreamGetDevice");
    if (sdev != dev)
        return fail(NU_EINVAL, "nu_periodic_search_noalloc: the stream belongs to device %d but "
                               "device %d is current; make the stream's device current", sdev,
                    dev);
    cudaPointerAttributes pa;
    e = cudaPointerGetAttributes(&pa, t0s_dev);
    if (e != cudaSuccess)
        return cuda_fail(e, "nu_periodic_search_noalloc: cudaPointerGetAttributes");
    if (pa.type == cudaMemoryTypeDevice && pa.device != dev)
        return fail(NU_EINVAL, "nu_periodic_search_noalloc: t0s is on device %d, the call runs "
                               "on device %d", pa.device, dev);
    if (dev < 0 || dev >= 64)
        return fail(NU_EINVAL, "nu_periodic_search_noalloc: device index %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_fold_scratch);
        if (e != cudaSuccess || !p)
            return cuda_fail(e, "nu_periodic_search_noalloc: cudaGetSymbolAddress");
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return NU_OK;
}

extern "C" uint64_t nu_periodic_search_noalloc_limit(void) { return NU_NOALLOC_SCRATCH_BYTES; }

extern "C" nu_status nu_periodic_search_noalloc(const double* t0s_dev, int64_t n_t0,
                                                const double* Ds_host, int n_D,
                                                const void* depth_dev, const void* var_dev,
                                                const void* dlnl_dev, nu_precision prec,
                                                const double* periods_dev, int64_t n_P,
                                                double phase_step, double gap_factor,
                                                void* stream, double* Q_dev, double* T0_dev,
                                                int32_t* D_idx_dev, double* depth_out_dev,
                                                double* sigma_out_dev, double* lnP_dev) {
    const char* who = "nu_periodic_search_noalloc";
    (void)Ds_host;
    nu_status s = check_args(who, t0s_dev, n_t0, n_D, depth_dev, var_dev, dlnl_dev, prec,
                             periods_dev, n_P, gap_factor, Q_dev, T0_dev, D_idx_dev,
                             depth_out_dev, sigma_out_dev, lnP_dev);
    if (s != NU_OK) return s;
    if (!(phase_step > 0.0) || !std::isfinite(phase_step))
        return fail(NU_EINVAL, "nu_periodic_search_noalloc: phase_step must be given (> 0)");
    cudaStream_t st = (cudaStream_t)stream;
    void* base = nullptr;
    s = noalloc_scratch(st, t0s_dev, &base);
    if (s != NU_OK) return s;
    double ends[2];
    cudaError_t e = cudaMemcpyAsync(&ends[0], t0s_dev, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&ends[1], t0s_dev + n_t0 - 1, sizeof(double), cudaMemcpyDeviceToHost,
                            st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "nu_periodic_search_noalloc: copy ends");
    const double t_ref = ends[0], t_last = ends[1];
    if (!(t_last >= t_ref)) return fail(NU_EINVAL, "nu_periodic_search_noalloc: t0s not sorted");
    const double span_steps = (t_last - t_ref) / phase_step;
    if (span_steps > 1.0e9)
        return fail(NU_EINVAL, "nu_periodic_search_noalloc: phase grid too fine");
    const int64_t n_bucket = (int64_t)span_steps + 2;
    const bool fp64 = prec == NU_FP64;
    const SingleLayout L = single_layout(n_t0, n_D, n_bucket, fp64);
    if (L.total > NU_NOALLOC_SCRATCH_BYTES)
        return fail(NU_EINVAL,
                    "nu_periodic_search_noalloc: this grid needs %zu bytes of scratch, more "
                    "than the fixed %llu bytes; use nu_periodic_search",
                    L.total, (unsigned long long)NU_NOALLOC_SCRATCH_BYTES);
    return single_fold(who, (char*)base, L, t0s_dev, n_t0, n_D, depth_dev, var_dev, dlnl_dev,
                       fp64, periods_dev, n_P, phase_step, gap_factor, t_ref, t_last, n_bucket,
                       st, Q_dev, T0_dev, D_idx_dev, depth_out_dev, sigma_out_dev, lnP_dev);
}

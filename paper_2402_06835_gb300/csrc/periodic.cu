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

__device__ __forceinline__ Best block_argmax(Best best) {
    __shared__ Best sh[256];
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

// FP32 form for the mixed kernel
__device__ __forceinline__ bool cannot_win_f(float s_l, float s_inv, float s_d, float s_dd,
                                             float best) {
    const float q = fmaxf(0.0f, s_dd - s_d * s_d / s_inv - 1e-4f * s_dd);
    const float ub = s_l + 0.5f - 0.25f * q;
    return ub + 1e-4f * fmaxf(1.0f, fabsf(ub)) < best;
}

__device__ __forceinline__ bool bad_period(double P, const FoldGeom& g) {
    // a period must be finite, > 0 and give at most 1e9 epochs and phases
    return !(P > 0.0) || !isfinite(P) || (g.t_last - g.t_ref) / P > 1.0e9 ||
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

// One period P of one light curve: every (duration, phase) cell, then the
// block argmax; results at index p of the outputs.  Called by all threads of
// the block.  Cells are processed in waves of blockDim: every thread runs the
// first pass of one cell, the cells whose bound can still beat the block's
// best are compacted into a shared queue, and the queue's second passes run
// densely (a warp instruction costs the same however many lanes are active).
template <typename T, int KC>
__device__ __forceinline__ void fold_exact_one(const FoldGeom& g, const Node8<T>* __restrict__ nodes,
                                               int n_D, double P, int64_t p,
                                               double* __restrict__ Q_out,
                                               double* __restrict__ T0_out,
                                               int* __restrict__ Didx_out,
                                               double* __restrict__ dep_out,
                                               double* __restrict__ sig_out,
                                               double* __restrict__ lnp_out) {
    __shared__ QCell<T> sh_q[256];
    __shared__ int sh_nq;
    __shared__ unsigned long long sh_best;
    if (bad_period(P, g)) {
        if (threadIdx.x == 0) write_bad(p, Q_out, T0_out, Didx_out, dep_out, sig_out, lnp_out);
        return;
    }
    const int64_t n_phi = (int64_t)ceil(P / g.dt);
    const int64_t n_cells = n_phi * n_D;
    const double R = P * g.inv_dt;
    const SlotWalk swp = slot_walk(1.0 / (double)n_phi, R);   // per-phase slot step
    const SlotWalk swk = slot_walk(0.0, R);                   // per-epoch slot step
    const double SCALE = 1099511627776.0;
    const double ulast_d = (g.t_last - g.t_ref) * g.inv_dt * SCALE;
    const unsigned long long ulast =
        ulast_d < 4.0e18 ? (unsigned long long)llrint(ulast_d) : 4000000000000000000ull;
    const float inv_ustep32 = (float)(4294967296.0 / (double)swk.ustep);
    const long long klast = okey(g.t_last);
    // phase j / n_phi: reciprocal plus one FMA correction of the quotient
    // (Markstein 1990), instead of a division per cell
    const double nphi_d = (double)n_phi;
    const double rphi = 1.0 / nphi_d;
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
            const double jd = (double)j;
            const double q0 = jd * rphi;
            const double phi = fma(fma(-q0, nphi_d, jd), rphi, q0);
            const Node8<T>* nd = nodes + (int64_t)d * g.n_t0;
            const unsigned long long u0 = (unsigned long long)j * swp.u0;
            // number of epochs with T <= t_last: integer estimate, then the
            // exact comparisons of the definition
            int64_t kk = u0 > ulast ? 0
                                    : (int64_t)((float)(unsigned)((ulast - u0) >> 32) *
                                                inv_ustep32) + 1;
            while (kk > 0 &&
                   okey(__dadd_rn(g.t_ref, __dmul_rn(__dadd_rn(phi, (double)(kk - 1)), P))) >
                       klast)
                --kk;
            while (okey(__dadd_rn(g.t_ref, __dmul_rn(__dadd_rn(phi, (double)kk), P))) <= klast)
                ++kk;
            const int64_t kmax = kk;
            ExactAcc<T> a1;
            a1.init();
            unsigned long long u = u0;
            double kd = 0.0;
            for (int64_t k = 0; k < kmax; ++k, u += swk.ustep, kd += 1.0) {
                const double Tk = __dadd_rn(g.t_ref, __dmul_rn(__dadd_rn(phi, kd), P));
                T dk, sk2, lk;
                int64_t i = guess_at(g, u);
                if (event_exact<T>(g, nd, Tk, i, dk, sk2, lk)) a1.add(dk, sk2, lk);
            }
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
            unsigned long long u = qc.u0;
            double kd = 0.0;
            for (int k = 0; k < qc.kmax; ++k, u += swk.ustep, kd += 1.0) {
                const double Tk = __dadd_rn(g.t_ref, __dmul_rn(__dadd_rn(qc.phi, kd), P));
                T dk, sk2, lk;
                int64_t i = guess_at(g, u);
                if (event_exact<T>(g, nd, Tk, i, dk, sk2, lk)) a2.add(dk, sk2);
            }
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
    const Best b = block_argmax(best);
    if (threadIdx.x == 0)
        write_best(b, p, n_phi, g.t_ref, P, Q_out, T0_out, Didx_out, dep_out, sig_out, lnp_out);
}

template <typename T, int KC>
__global__ void __launch_bounds__(256)
k_fold_exact(FoldGeom g, const Node8<T>* __restrict__ nodes, int n_D,
             const double* __restrict__ periods, int64_t n_P, double* __restrict__ Q_out,
             double* __restrict__ T0_out, int* __restrict__ Didx_out,
             double* __restrict__ dep_out, double* __restrict__ sig_out,
             double* __restrict__ lnp_out) {
    const int64_t p = blockIdx.x;
    if (p >= n_P) return;
    fold_exact_one<T, KC>(g, nodes, n_D, periods[p], p, Q_out, T0_out, Didx_out, dep_out,
                          sig_out, lnp_out);
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
    int K;
    __device__ __forceinline__ void init() {
        s_inv.init();
        s_d.init();
        s_l.init();
        s_dd = 0.f;
        K = 0;
    }
    __device__ __forceinline__ void add(const SlotEvent& e) {
        if (isnan(e.s)) return;
        const float iv = rcp32(e.s * e.s);
        const float div = e.d * iv;
        s_inv.add(iv);
        s_d.add(div);
        s_dd = fmaf(div, e.d, s_dd);
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

// Epochs walk the slot grid in 24.40 fixed point: u = (T - t_ref)/dt =
// (j/n_phi + k) P/dt.  The interval is (slot, slot+1) and the weight is the
// fractional part; on a grid whose epochs sit on the slots this is the
// interpolation between the bracketing epochs up to their offsets from the
// slot centres (checked to be below 1e-3 slot).  Cells are processed in waves
// with the second passes of the surviving cells compacted, as in the exact path.
template <int KC>
__device__ __forceinline__ void fold_slots_one(const Node4<float>* __restrict__ rec,
                                               int64_t n_slots, int n_D, double dt,
                                               double t_ref, double t_last, double P, int64_t p,
                                               double* __restrict__ Q_out,
                                               double* __restrict__ T0_out,
                                               int* __restrict__ Didx_out,
                                               double* __restrict__ dep_out,
                                               double* __restrict__ sig_out,
                                               double* __restrict__ lnp_out) {
    __shared__ QCell<float> sh_q[256];
    __shared__ int sh_nq;
    __shared__ unsigned int sh_best;
    FoldGeom gg{nullptr, 0, t_ref, t_last, dt, 1.0 / dt, 0.0, nullptr, 0};
    if (bad_period(P, gg)) {
        if (threadIdx.x == 0) write_bad(p, Q_out, T0_out, Didx_out, dep_out, sig_out, lnp_out);
        return;
    }
    const int64_t n_phi = (int64_t)ceil(P / dt);
    const int64_t n_cells = n_phi * n_D;
    const double R = P / dt;                                   // slots per period
    const double SCALE = 1099511627776.0;                      // 2^40
    const double ulast_d = (t_last - t_ref) / dt * SCALE;       // < 2^62 (host check)
    const unsigned long long ulast = (unsigned long long)llrint(ulast_d);
    const unsigned long long ustep =
        R * SCALE < 4.0e18 ? (unsigned long long)llrint(R * SCALE) : 4000000000000000000ull;
    // phase j starts at j * (R / n_phi) slots; per-cell work stays integer
    const unsigned long long uph = (unsigned long long)llrint(R / (double)n_phi * SCALE);
    // epochs per cell from the remaining span in units of 2^32 (a 32-bit
    // integer), corrected exactly below
    const float inv_ustep32 = (float)(4294967296.0 / (double)ustep);
    float bl = -INFINITY, bD = NAN, bs2 = NAN;
    long long bc = LLONG_MAX;
    if (threadIdx.x == 0) {
        sh_nq = 0;
        sh_best = 0u;                       // key below every finite float
    }
    __syncthreads();
    int d = (int)(threadIdx.x / n_phi);
    int64_t j = (int64_t)threadIdx.x - (int64_t)d * n_phi;
    for (int64_t base = 0; base < n_cells; base += blockDim.x, j += blockDim.x) {
        while (j >= n_phi) {
            j -= n_phi;
            ++d;
        }
        const int64_t cell = base + threadIdx.x;
        if (cell < n_cells) {
            const unsigned long long u0 = (unsigned long long)j * uph;
            if (u0 <= ulast) {
                int64_t kk = (int64_t)((float)(unsigned)((ulast - u0) >> 32) * inv_ustep32);
                while (kk > 0 && u0 + (unsigned long long)kk * ustep > ulast) --kk;
                while (u0 + (unsigned long long)(kk + 1) * ustep <= ulast) ++kk;
                const int64_t kmax = kk + 1;
                const Node4<float>* rd = rec + (int64_t)d * n_slots;
                SlotPass1 p1;
                p1.init();
                unsigned long long u = u0;
                for (int64_t k = 0; k < kmax; ++k, u += ustep) p1.add(slot_event(rd, u));
                const unsigned int kb = sh_best;
                const float best_now =
                    fmaxf(bl, kb ? __uint_as_float((kb >> 31) ? (kb & 0x7fffffffu) : ~kb)
                                 : -INFINITY);
                if (p1.K > 0 &&
                    !cannot_win_f(p1.s_l.s, p1.s_inv.s, p1.s_d.s, p1.s_dd, best_now)) {
                    const float s2 = 1.0f / p1.s_inv.s;
                    const int q = atomicAdd(&sh_nq, 1);
                    sh_q[q] = QCell<float>{0.0, u0, (long long)cell, (double)p1.s_l.s, s2,
                                           s2 * p1.s_d.s, d, (int)kmax};
                }
            }
        }
        __syncthreads();
        const int nq = sh_nq;
        for (int q = threadIdx.x; q < nq; q += blockDim.x) {
            const QCell<float> qc = sh_q[q];
            const Node4<float>* rd = rec + (int64_t)qc.d * n_slots;
            SlotPass2 p2;
            p2.init(qc.s2, qc.Dl);
            unsigned long long u = qc.u0;
            for (int k = 0; k < qc.kmax; ++k, u += ustep) {
                const SlotEvent e = slot_event(rd, u);
                p2.add(e.d, e.s);
            }
            const float lnp =
                (float)qc.s_l - 0.5f * (p2.lsum * 0.693147180559945f + p2.quad.s);
            if (!(lnp == lnp)) continue;
            if (lnp > bl || (lnp == bl && qc.cell < bc)) {
                bl = lnp;
                bc = qc.cell;
                bD = p2.Dl;
                bs2 = p2.s2;
            }
            const unsigned int b32 = __float_as_uint(lnp);
            atomicMax(&sh_best, (b32 >> 31) ? ~b32 : (b32 | 0x80000000u));
        }
        __syncthreads();
        if (threadIdx.x == 0) sh_nq = 0;
        __syncthreads();
    }
    Best best{-INFINITY, LLONG_MAX, NAN, NAN};
    if (bc != LLONG_MAX) best = Best{(double)bl, bc, (double)bD, sqrt((double)bs2)};
    const Best b = block_argmax(best);
    if (threadIdx.x == 0)
        write_best(b, p, n_phi, t_ref, P, Q_out, T0_out, Didx_out, dep_out, sig_out, lnp_out);
}

template <int KC>
__global__ void __launch_bounds__(256, 4)
k_fold_slots(const Node4<float>* __restrict__ rec, int64_t n_slots, int n_D, double dt,
             double t_ref, double t_last, const double* __restrict__ periods, int64_t n_P,
             double* __restrict__ Q_out, double* __restrict__ T0_out,
             int* __restrict__ Didx_out, double* __restrict__ dep_out,
             double* __restrict__ sig_out, double* __restrict__ lnp_out) {
    const int64_t p = blockIdx.x;
    if (p >= n_P) return;
    fold_slots_one<KC>(rec, n_slots, n_D, dt, t_ref, t_last, periods[p], p, Q_out, T0_out,
                       Didx_out, dep_out, sig_out, lnp_out);
}

// ------------------------------------------------------------ batch path

// Persistent fold over (curve, period) work items taken from a device
// counter (no waits: a block takes items until none are left).  kind 0: the
// exact FP64-epoch path with FP64 values; 1: exact path, FP32 values;
// 2: slot path (mixed precision, regular grids).  Items of curves that do not
// use this kernel's path are skipped.
template <int KIND>
__global__ void __launch_bounds__(256)
k_fold_batch(const FoldSeg* __restrict__ segs, int n_seg, const double* __restrict__ t,
             const void* __restrict__ nodes, const int* __restrict__ bucket,
             const Node4<float>* __restrict__ rec, int n_D, double dt, double gap_factor,
             const double* __restrict__ periods, int64_t n_P, unsigned long long* counter,
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
        const int64_t p = (int64_t)(item % (unsigned long long)n_P);
        const FoldSeg fs = segs[g];
        if ((KIND == 2) != (fs.use_slots != 0)) continue;
        const int64_t o = (int64_t)g * n_P + p;
        if (KIND == 2) {
            fold_slots_one<8>(rec + fs.rec_off, fs.n_slots, n_D, dt, fs.t_ref, fs.t_last,
                              periods[p], o, Q_out, T0_out, Didx_out, dep_out, sig_out,
                              lnp_out);
        } else {
            FoldGeom gg{t + fs.s_off, fs.n_t0, fs.t_ref, fs.t_last, dt, 1.0 / dt,
                        gap_factor * dt, bucket + fs.bucket_off, fs.n_bucket};
            if (KIND == 0)
                fold_exact_one<double, 8>(gg, (const Node8<double>*)nodes + fs.s_off * n_D,
                                          n_D, periods[p], o, Q_out, T0_out, Didx_out,
                                          dep_out, sig_out, lnp_out);
            else
                fold_exact_one<float, 8>(gg, (const Node8<float>*)nodes + fs.s_off * n_D, n_D,
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
        const double span = (t_last[g] - t_first[g]) / dt;
        f.n_bucket = (int64_t)span + 2;
        f.n_slots = f.n_bucket + 2;
        f.use_slots = (!fp64 && gap_factor > 1.0 && gap_factor < 2.0 && span < 4.0e6 &&
                       !irregular[g]) ? 1 : 0;
        f.bucket_off = fb.n_bucket_total;
        fb.n_bucket_total += f.use_slots ? 0 : f.n_bucket;
        f.rec_off = fb.n_rec_total;
        fb.n_rec_total += f.use_slots ? f.n_slots * n_D : 0;
        fb.any_slots = fb.any_slots || f.use_slots;
        fb.any_exact = fb.any_exact || !f.use_slots;
    }
}

int launch_fold_prep(const FoldBatch& fb, const FoldSeg* segs_dev, const int64_t* s_off_dev,
                     int n_seg, int64_t n_total, bool fp64, const double* t, const void* depth,
                     const void* var, const void* gain, int n_D, double dt, double gap_factor,
                     void* nodes, int* bucket, Node4<float>* rec, cudaStream_t st) {
    int launched = 0;
    const int64_t ngrid = n_total * (int64_t)n_D;
    if (fb.any_exact) {
        if (fp64)
            k_nodes_batch<double><<<div_up(ngrid, 256), 256, 0, st>>>(
                (const double*)depth, (const double*)var, (const double*)gain, t, segs_dev,
                n_seg, s_off_dev, n_D, gap_factor * dt, (Node8<double>*)nodes);
        else
            k_nodes_batch<float><<<div_up(ngrid, 256), 256, 0, st>>>(
                (const float*)depth, (const float*)var, (const float*)gain, t, segs_dev, n_seg,
                s_off_dev, n_D, gap_factor * dt, (Node8<float>*)nodes);
        k_buckets_batch<<<div_up(fb.n_bucket_total, 256), 256, 0, st>>>(
            t, segs_dev, n_seg, fb.n_bucket_total, dt, bucket);
        launched += 2;
    }
    if (fb.any_slots) {
        k_fill_nan<<<div_up(fb.n_rec_total, 256), 256, 0, st>>>(rec, fb.n_rec_total);
        k_slot_fill_batch<<<div_up(ngrid, 256), 256, 0, st>>>(
            (const float*)depth, (const float*)var, (const float*)gain, t, segs_dev, n_seg,
            s_off_dev, n_D, 1.0 / dt, rec);
        launched += 2;
    }
    return launched;
}

// The persistent fold kernels; counter[0..1] must be zero.  blocks_per_sm
// and threads come from the autotuner.
int launch_fold_batch(const FoldBatch& fb, const FoldSeg* segs_dev, int n_seg, bool fp64,
                      const double* t, const void* nodes, const int* bucket,
                      const Node4<float>* rec, int n_D, double dt, double gap_factor,
                      const double* periods, int64_t n_P, unsigned long long* counter,
                      int grid, int threads, double* Q, double* T0, int* Didx, double* dep,
                      double* sig, double* lnp, cudaStream_t st) {
    int launched = 0;
    if (fb.any_exact) {
        if (fp64)
            k_fold_batch<0><<<grid, threads, 0, st>>>(segs_dev, n_seg, t, nodes, bucket, rec,
                                                      n_D, dt, gap_factor, periods, n_P,
                                                      counter, Q, T0, Didx, dep, sig, lnp);
        else
            k_fold_batch<1><<<grid, threads, 0, st>>>(segs_dev, n_seg, t, nodes, bucket, rec,
                                                      n_D, dt, gap_factor, periods, n_P,
                                                      counter, Q, T0, Didx, dep, sig, lnp);
        ++launched;
    }
    if (fb.any_slots) {
        k_fold_batch<2><<<grid, threads, 0, st>>>(segs_dev, n_seg, t, nodes, bucket, rec, n_D,
                                                  dt, gap_factor, periods, n_P, counter + 1, Q,
                                                  T0, Didx, dep, sig, lnp);
        ++launched;
    }
    return launched;
}

int launch_slots_test(const double* t, const int64_t* s_off_dev, int n_seg, int64_t n_total,
                      double dt, int* irregular, cudaStream_t st) {
    k_slots_batch<<<div_up(n_total, 256), 256, 0, st>>>(t, s_off_dev, n_seg, 1.0 / dt,
                                                       irregular);
    return 1;
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
    const bool fp64 = prec == NU_FP64;
    const size_t esz = fp64 ? sizeof(double) : sizeof(float);
    const int64_t ngrid = n_t0 * (int64_t)n_D;
    const int64_t n_slots = n_bucket + 2;          // slot records, NaN padded
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t b_nodes = al((size_t)ngrid * 8 * esz);
    const size_t b_bucket = al((size_t)n_bucket * sizeof(int));
    const size_t b_slot_of = al((size_t)n_t0 * sizeof(int));
    const size_t b_flag = 256;
    const size_t b_rec = fp64 ? 0 : al((size_t)n_slots * n_D * sizeof(Node4<float>));
    pool_keep_memory();
    char* scratch = nullptr;
    e = cudaMallocAsync((void**)&scratch, b_nodes + b_bucket + b_slot_of + b_flag + b_rec, st);
    if (e != cudaSuccess) return cuda_fail(e, "nu_periodic_search: cudaMallocAsync");
    void* nodes = scratch;
    int* bucket = (int*)(scratch + b_nodes);
    int* slot_of = (int*)(scratch + b_nodes + b_bucket);
    int* flag = (int*)(scratch + b_nodes + b_bucket + b_slot_of);
    Node4<float>* rec = (Node4<float>*)(scratch + b_nodes + b_bucket + b_slot_of + b_flag);
    int launched = 0;
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
            cudaFreeAsync(scratch, st);
            return cuda_fail(e, "nu_periodic_search: slot test");
        }
        use_slots = irregular == 0;
    }
    if (use_slots) {
        const int64_t nrec = n_slots * n_D;
        k_fill_nan<<<div_up(nrec, 256), 256, 0, st>>>(rec, nrec);
        k_slot_fill<<<div_up(ngrid, 256), 256, 0, st>>>(
            (const float*)depth_dev, (const float*)var_dev, (const float*)dlnl_dev, slot_of,
            n_t0, n_D, n_slots, rec);
        k_fold_slots<8><<<(unsigned)n_P, 256, 0, st>>>(rec, n_slots, n_D, phase_step, t_ref,
                                                      t_last, periods_dev, n_P, Q_dev, T0_dev,
                                                      D_idx_dev, depth_out_dev, sigma_out_dev,
                                                      lnP_dev);
        launched += 3;
    } else {
        k_buckets<<<div_up(n_bucket, 256), 256, 0, st>>>(t0s_dev, n_t0, t_ref, phase_step,
                                                        n_bucket, bucket);
        FoldGeom g{t0s_dev, n_t0, t_ref, t_last, phase_step, 1.0 / phase_step,
                   gap_factor * phase_step, bucket, n_bucket};
        if (fp64) {
            k_nodes<double><<<div_up(ngrid, 256), 256, 0, st>>>(
                (const double*)depth_dev, (const double*)var_dev, (const double*)dlnl_dev,
                t0s_dev, n_t0, n_D, g.gap_max, (Node8<double>*)nodes);
            k_fold_exact<double, 8><<<(unsigned)n_P, 256, 0, st>>>(
                g, (const Node8<double>*)nodes, n_D, periods_dev, n_P, Q_dev, T0_dev,
                D_idx_dev, depth_out_dev, sigma_out_dev, lnP_dev);
        } else {
            k_nodes<float><<<div_up(ngrid, 256), 256, 0, st>>>(
                (const float*)depth_dev, (const float*)var_dev, (const float*)dlnl_dev,
                t0s_dev, n_t0, n_D, g.gap_max, (Node8<float>*)nodes);
            k_fold_exact<float, 8><<<(unsigned)n_P, 256, 0, st>>>(
                g, (const Node8<float>*)nodes, n_D, periods_dev, n_P, Q_dev, T0_dev,
                D_idx_dev, depth_out_dev, sigma_out_dev, lnP_dev);
        }
        launched += 3;
    }
    count_launches(launched);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "nu_periodic_search: launch");
    e = cudaFreeAsync(scratch, st);
    if (e != cudaSuccess) return cuda_fail(e, "nu_periodic_search: cudaFreeAsync");
    return NU_OK;
}

// ------------------------------------------------ allocation-free variant
// nu_periodic_search_noalloc runs the same kernels as nu_periodic_search but
// takes its scratch (packed epoch records, bucket table, slot table, flag)
// from the file-scope device array below instead of the stream-ordered pool,
// for callers that must not allocate device memory.  The array is part of the
// library image: every GPU that loads the library holds it until the process
// exits.  Its address is looked up once per device (cudaGetSymbolAddress with
// that device current) on the first call made on the device.
#define NU_NOALLOC_SCRATCH_BYTES (32ull << 20)

static __device__ __align__(256) unsigned char g_fold_scratch[NU_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_scratch_mu;
void* g_scratch_ptr[64] = {};
}

static nu_status noalloc_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "nu_periodic_search_noalloc: cudaGetDevice");
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
    (void)Ds_host;
    if (!t0s_dev || !depth_dev || !var_dev || !dlnl_dev || !periods_dev || !Q_dev ||
        !T0_dev || !D_idx_dev || !depth_out_dev || !sigma_out_dev || !lnP_dev)
        return fail(NU_EINVAL, "nu_periodic_search_noalloc: null array");
    if (n_t0 < 2 || n_D < 1 || n_P < 1)
        return fail(NU_EINVAL, "nu_periodic_search_noalloc: need n_t0 >= 2, n_D >= 1, n_P >= 1");
    if (prec != NU_FP64 && prec != NU_MIXED)
        return fail(NU_EINVAL, "nu_periodic_search_noalloc: unknown precision");
    if (!(gap_factor > 0.0))
        return fail(NU_EINVAL, "nu_periodic_search_noalloc: gap_factor <= 0");
    if (!(phase_step > 0.0) || !std::isfinite(phase_step))
        return fail(NU_EINVAL, "nu_periodic_search_noalloc: phase_step must be given (> 0)");
    if (n_t0 > 2000000000LL)
        return fail(NU_EINVAL, "nu_periodic_search_noalloc: n_t0 too large");
    void* base = nullptr;
    nu_status ss = noalloc_scratch(&base);
    if (ss != NU_OK) return ss;
    cudaStream_t st = (cudaStream_t)stream;
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
    const size_t esz = fp64 ? sizeof(double) : sizeof(float);
    const int64_t ngrid = n_t0 * (int64_t)n_D;
    const int64_t n_slots = n_bucket + 2;
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t b_nodes = al((size_t)ngrid * 8 * esz);
    const size_t b_bucket = al((size_t)n_bucket * sizeof(int));
    const size_t b_slot_of = al((size_t)n_t0 * sizeof(int));
    const size_t b_flag = 256;
    const size_t b_rec = fp64 ? 0 : al((size_t)n_slots * n_D * sizeof(Node4<float>));
    const size_t need = b_nodes + b_bucket + b_slot_of + b_flag + b_rec;
    if (need > NU_NOALLOC_SCRATCH_BYTES)
        return fail(NU_EINVAL,
                    "nu_periodic_search_noalloc: this grid needs %zu bytes of scratch, more "
                    "than the fixed %llu bytes; use nu_periodic_search",
                    need, (unsigned long long)NU_NOALLOC_SCRATCH_BYTES);
    char* scratch = (char*)base;
    void* nodes = scratch;
    int* bucket = (int*)(scratch + b_nodes);
    int* slot_of = (int*)(scratch + b_nodes + b_bucket);
    int* flag = (int*)(scratch + b_nodes + b_bucket + b_slot_of);
    Node4<float>* rec = (Node4<float>*)(scratch + b_nodes + b_bucket + b_slot_of + b_flag);
    int launched = 0;
    bool use_slots = !fp64 && gap_factor > 1.0 && gap_factor < 2.0 && span_steps < 4.0e6;
    if (use_slots) {
        int irregular = 0;
        e = cudaMemsetAsync(flag, 0, sizeof(int), st);   // the array keeps old contents
        k_slots<<<div_up(n_t0, 256), 256, 0, st>>>(t0s_dev, n_t0, t_ref, 1.0 / phase_step,
                                                  slot_of, flag);
        ++launched;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&irregular, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "nu_periodic_search_noalloc: slot test");
        use_slots = irregular == 0;
    }
    if (use_slots) {
        const int64_t nrec = n_slots * n_D;
        k_fill_nan<<<div_up(nrec, 256), 256, 0, st>>>(rec, nrec);
        k_slot_fill<<<div_up(ngrid, 256), 256, 0, st>>>(
            (const float*)depth_dev, (const float*)var_dev, (const float*)dlnl_dev, slot_of,
            n_t0, n_D, n_slots, rec);
        k_fold_slots<8><<<(unsigned)n_P, 256, 0, st>>>(rec, n_slots, n_D, phase_step, t_ref,
                                                      t_last, periods_dev, n_P, Q_dev, T0_dev,
                                                      D_idx_dev, depth_out_dev, sigma_out_dev,
                                                      lnP_dev);
        launched += 3;
    } else {
        k_buckets<<<div_up(n_bucket, 256), 256, 0, st>>>(t0s_dev, n_t0, t_ref, phase_step,
                                                        n_bucket, bucket);
        FoldGeom g{t0s_dev, n_t0, t_ref, t_last, phase_step, 1.0 / phase_step,
                   gap_factor * phase_step, bucket, n_bucket};
        if (fp64) {
            k_nodes<double><<<div_up(ngrid, 256), 256, 0, st>>>(
                (const double*)depth_dev, (const double*)var_dev, (const double*)dlnl_dev,
                t0s_dev, n_t0, n_D, g.gap_max, (Node8<double>*)nodes);
            k_fold_exact<double, 8><<<(unsigned)n_P, 256, 0, st>>>(
                g, (const Node8<double>*)nodes, n_D, periods_dev, n_P, Q_dev, T0_dev,
                D_idx_dev, depth_out_dev, sigma_out_dev, lnP_dev);
        } else {
            k_nodes<float><<<div_up(ngrid, 256), 256, 0, st>>>(
                (const float*)depth_dev, (const float*)var_dev, (const float*)dlnl_dev,
                t0s_dev, n_t0, n_D, g.gap_max, (Node8<float>*)nodes);
            k_fold_exact<float, 8><<<(unsigned)n_P, 256, 0, st>>>(
                g, (const Node8<float>*)nodes, n_D, periods_dev, n_P, Q_dev, T0_dev,
                D_idx_dev, depth_out_dev, sigma_out_dev, lnP_dev);
        }
        launched += 3;
    }
    count_launches(launched);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "nu_periodic_search_noalloc: launch");
    return NU_OK;
}

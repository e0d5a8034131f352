// nu_periodic_refine: the exact fit of a periodic transit column.
//
// Sect. 2.4 takes Q(P) as the SNR of a periodic transit of period P, epoch T0
// and duration D.  nu_periodic_search obtains it from the single events with
// Eq. result, which treats the transits as independent (Sect. 2.3).  Here the
// design matrix is X' = [X, m_P] with m_P the template repeated at every
// T0 + n P, and Eq. ls is solved once at the full covariance.  The Schur
// complement of the linear search carries over unchanged (linear.cu):
//   c = m_P^T Sigma^-1 m_P,  num = m_P^T z0,  bt = Zt^T m_P,
//   s = c - |bt|^2,  depth = num / s,  var = 1 / s,  dlnl = num^2 / (2 s).
// num and bt only see the samples inside the windows.  c is the D^-1
// weighted norm of the forward solve e = L^-1 m_P, which starts from a zero
// state at the first window and runs through every later sample: inside a
// window with the template as input, between windows with zero input, and
// after the last window through the future information G.
//
// Between windows the recursion is homogeneous, s_{i+1} = A_{i+1} s_i with
// A_{i+1} = F_{i+1} (I - kg_i h^T), and its D^-1 weighted innovations are a
// quadratic form in the state entering the stretch.  For aligned blocks of
// RB samples the map (Phi_b) and the form (M_b) are tabulated once per call
// (k_refine_blocks), so a zero-input stretch costs one J x J step per block
// plus single samples at its ends.
//
// One warp takes one candidate (k_refine).  GB300 issues one FP64 warp
// instruction per 64 cycles per sub-partition, so a candidate's cost is the
// length of its longest serial chain; the lanes split the samples into RS
// block-aligned segments and the solve into three phases: each lane's
// zero-state response of its segment to the template, a short serial pass
// over the segments' maps (Pseg, k_refine_segs) for the states entering them,
// and each lane's segment again from its true incoming state.  FP64
// throughout.
#include <cmath>

#include "nu_internal.cuh"
#include "ss.cuh"
#include "templates.cuh"

namespace nu {

constexpr int RB = 32;   // samples per tabulated block
constexpr int RS = 32;   // segments per candidate (one per lane)

__device__ __forceinline__ int64_t rf_lower_bound(const double* __restrict__ t, int64_t n,
                                                  double x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (t[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Phi_b (row-major J x J) and M_b (packed upper) of block b = samples
// [b RB, (b+1) RB): with s the state entering sample b RB and zero input,
// the state leaving the block is Phi_b s and the block's sum of e_i^2 / D_i
// is s^T M_b s.  Only blocks whose transitions all exist ((b+1) RB <= n-1).
template <int NB>
__global__ void __launch_bounds__(128)
k_refine_blocks(const double* __restrict__ F, const double* __restrict__ kg,
                const double* __restrict__ invD, int64_t n_blk, double* __restrict__ Phi,
                double* __restrict__ Mq) {
    constexpr int J = Dims<NB>::J;
    constexpr int JJ = Dims<NB>::JJ;
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= n_blk) return;
    double Ph[J][J], M[JJ];
#pragma unroll
    for (int r = 0; r < J; ++r)
#pragma unroll
        for (int c = 0; c < J; ++c) Ph[r][c] = r == c ? 1.0 : 0.0;
#pragma unroll
    for (int a = 0; a < JJ; ++a) M[a] = 0.0;
    const int64_t i0 = b * RB;
    for (int64_t i = i0; i < i0 + RB; ++i) {
        // g^T = h^T Phi: the innovation of sample i is -g^T s
        double g[J];
#pragma unroll
        for (int c = 0; c < J; ++c) {
            double v = Ph[0][c];
#pragma unroll
            for (int q = 1; q < NB; ++q) v += Ph[2 * q][c];
            g[c] = v;
        }
        const double iD = invD[i];
#pragma unroll
        for (int r = 0; r < J; ++r) {
            const double gr = g[r] * iD;
#pragma unroll
            for (int c = r; c < J; ++c) M[pk(r, c, J)] = fma(gr, g[c], M[pk(r, c, J)]);
        }
        // Phi <- F_{i+1} (Phi - kg_i g^T)
        const double* kgi = kg + i * J;
        const double* f = F + (i + 1) * NB * 4;
#pragma unroll
        for (int c = 0; c < J; ++c) {
            double col[J], out[J];
#pragma unroll
            for (int r = 0; r < J; ++r) col[r] = fma(-kgi[r], g[c], Ph[r][c]);
            apply_F<NB>(f, col, out);
#pragma unroll
            for (int r = 0; r < J; ++r) Ph[r][c] = out[r];
        }
    }
    double* po = Phi + b * J * J;
#pragma unroll
    for (int r = 0; r < J; ++r)
#pragma unroll
        for (int c = 0; c < J; ++c) po[r * J + c] = Ph[r][c];
    double* mo = Mq + b * JJ;
#pragma unroll
    for (int a = 0; a < JJ; ++a) mo[a] = M[a];
}

// One sample of the forward solve with input x: e = x - h^T s, adds e^2/D_i,
// s <- F_{i+1} (s + kg_i e) when sample i+1 exists.  Returns e.
template <int NB>
__device__ __forceinline__ double rf_step(const FactorView<double>& fv, int64_t i, int64_t n,
                                          double x, double* s, double& c2) {
    constexpr int J = Dims<NB>::J;
    const double e = x - hdot<NB>(s);
    c2 = fma(e * e, fv.invD[i], c2);
    if (i + 1 < n) {
        double tmp[J];
#pragma unroll
        for (int q = 0; q < J; ++q) tmp[q] = fma(fv.kg[i * J + q], e, s[q]);
        apply_F<NB>(fv.F + (i + 1) * NB * 4, tmp, s);
    }
    return e;
}

// s^T Q s for Q packed upper
template <int J>
__device__ __forceinline__ double rf_quad(const double* __restrict__ Q, const double* s) {
    double acc = 0.0;
#pragma unroll
    for (int r = 0; r < J; ++r) {
        double row = Q[pk(r, r, J)] * s[r];
#pragma unroll
        for (int c = r + 1; c < J; ++c) row = fma(2.0 * Q[pk(r, c, J)], s[c], row);
        acc = fma(s[r], row, acc);
    }
    return acc;
}

// Zero-input forward solve from cur up to target: aligned blocks of RB
// samples in one step each (Phi_b, and s^T M_b s added to c2 when ACC),
// single samples at the ends.
template <int NB, bool ACC>
__device__ __forceinline__ void rf_zero_walk(const FactorView<double>& fv, int64_t n,
                                             const double* __restrict__ Phi,
                                             const double* __restrict__ Mq, int64_t n_blk,
                                             int64_t& cur, int64_t target, double* s,
                                             double& c2) {
    constexpr int J = Dims<NB>::J;
    constexpr int JJ = Dims<NB>::JJ;
    while (cur < target) {
        if ((cur % RB) == 0 && cur + RB <= target && cur / RB < n_blk) {
            const int64_t b = cur / RB;
            if (ACC) c2 += rf_quad<J>(Mq + b * JJ, s);
            const double* ph = Phi + b * J * J;
            double o[J];
#pragma unroll
            for (int r = 0; r < J; ++r) {
                double v = 0.0;
#pragma unroll
                for (int q = 0; q < J; ++q) v = fma(ph[r * J + q], s[q], v);
                o[r] = v;
            }
#pragma unroll
            for (int q = 0; q < J; ++q) s[q] = o[q];
            cur += RB;
        } else {
            double unused = 0.0;
            rf_step<NB>(fv, cur, n, 0.0, s, ACC ? c2 : unused);
            ++cur;
        }
    }
}

// The candidate's windows inside the segment [seg_lo, seg_hi), walked in time
// order from the state s entering seg_lo (s_zero: s is zero, so the walk may
// start at the first window).  With ACC the D^-1 weighted innovations, the
// template-weighted z0 and Zt sums are accumulated.  Returns whether the
// segment holds a template sample; cur receives the sample the state s enters
// after the last window.  Sets bad when the walk runs out of its pass budget
// or the transit index leaves the exact integers.
template <int NB, int TMPL, bool ACC>
__device__ __forceinline__ bool rf_segment(const double* __restrict__ t, int64_t n, int k,
                                           const FactorView<double>& fv,
                                           const double* __restrict__ Phi,
                                           const double* __restrict__ Mq, int64_t n_blk,
                                           int64_t seg_lo, int64_t seg_hi, double P, double T0,
                                           double D, double half, const TmplArgs& ta,
                                           double* s, bool s_zero, double& c2, double& num,
                                           double* bt, int64_t& cur, bool& bad) {
    bool started = !s_zero, any = false;
    cur = seg_lo;
    int64_t p = seg_lo;
    double nf = -INFINITY;
    // every pass moves p forward or steps nf by one, at most two windows early
    int64_t budget = 4 * (seg_hi - seg_lo) + 16;
    while (p < seg_hi) {
        if (--budget < 0) {
            bad = true;
            break;
        }
        const double ne = rint(__ddiv_rn(__dsub_rn(t[p], T0), P)) - 1.0;
        if (!(fabs(ne) < 0x1p50)) {                 // transit index beyond exact integers
            bad = true;
            break;
        }
        nf = fmax(nf, ne);
        const double tc = __dadd_rn(T0, __dmul_rn(nf, P));
        const int64_t hi = rf_lower_bound(t, n, __dadd_rn(tc, half));
        if (hi <= p) {                              // window nf ends before t[p]
            nf += 1.0;
            continue;
        }
        const int64_t lo = rf_lower_bound(t, n, __dsub_rn(tc, half));
        if (lo >= hi) {                             // no sample in window nf
            p = hi;
            nf += 1.0;
            continue;
        }
        if (lo >= seg_hi) break;                    // the window starts after the segment
        int64_t a = lo > seg_lo ? lo : seg_lo;      // the window's part in the segment
        const int64_t e = hi < seg_hi ? hi : seg_hi;
        if (a < cur) a = cur;                       // windows are disjoint (2 D <= P)
        if (!started) {
            started = true;
            cur = a;
        }
        rf_zero_walk<NB, ACC>(fv, n, Phi, Mq, n_blk, cur, a, s, c2);
        for (int64_t m = a; m < e; ++m) {
            const double mv = template_value<TMPL>(t[m], tc, half, D, ta);
            double unused = 0.0;
            rf_step<NB>(fv, m, n, mv, s, ACC ? c2 : unused);
            if (ACC) {
                num = fma(mv, fv.z0[m], num);
                for (int q = 0; q < k; ++q) bt[q] = fma(mv, fv.Zt[m * k + q], bt[q]);
            }
        }
        cur = e;
        any = true;
        p = hi;
        nf += 1.0;
    }
    return any;
}

// Segment maps: Pseg[g] (row-major J x J) takes the state entering segment g
// to the state leaving it under zero input, the product of its blocks' Phi_b.
// One thread per (segment, column).  Only segments made of whole blocks are
// used (the one holding the last samples is never needed).
template <int NB>
__global__ void __launch_bounds__(128)
k_refine_segs(const double* __restrict__ Phi, int64_t n_blk, int64_t nbs,
              double* __restrict__ Pseg) {
    constexpr int J = Dims<NB>::J;
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= RS * J) return;
    const int g = gid / J, col = gid - g * J;
    double v[J];
#pragma unroll
    for (int r = 0; r < J; ++r) v[r] = r == col ? 1.0 : 0.0;
    const int64_t b0 = (int64_t)g * nbs;
    const int64_t b1 = b0 + nbs < n_blk ? b0 + nbs : n_blk;
    for (int64_t b = b0; b < b1; ++b) {
        const double* ph = Phi + b * J * J;
        double o[J];
#pragma unroll
        for (int r = 0; r < J; ++r) {
            double a = 0.0;
#pragma unroll
            for (int q = 0; q < J; ++q) a = fma(ph[r * J + q], v[q], a);
            o[r] = a;
        }
#pragma unroll
        for (int r = 0; r < J; ++r) v[r] = o[r];
    }
#pragma unroll
    for (int r = 0; r < J; ++r) Pseg[(int64_t)g * J * J + r * J + col] = v[r];
}

// One warp per candidate; lane g owns segment g (nbs blocks of RB samples).
// (a) each lane: the zero-state response of its segment to the template,
//     beta_g, at the segment's end;
// (b) lane 0: the states entering the segments, S_{g+1} = Pseg_g S_g + beta_g;
// (c) each lane between the first and the last segment with a template
//     sample: its segment again from S_g, accumulating e^2/D, num and bt; the
//     last one closes with the future information G after its last window.
template <int NB, int TMPL>
__global__ void __launch_bounds__(128)
k_refine(const double* __restrict__ t, int64_t n, int k, FactorView<double> fv,
         const double* __restrict__ Phi, const double* __restrict__ Mq, int64_t n_blk,
         const double* __restrict__ Pseg, int64_t nbs, const double* __restrict__ Ps,
         const double* __restrict__ T0s, const int* __restrict__ Didx, int64_t n_cand,
         const double* __restrict__ Ds, int n_D, TmplArgs ta, double* __restrict__ out_depth,
         double* __restrict__ out_var, double* __restrict__ out_dlnl,
         double* __restrict__ out_snr) {
    constexpr int J = Dims<NB>::J;
    constexpr int JJ = Dims<NB>::JJ;
    constexpr unsigned FULL = 0xffffffffu;
    __shared__ double sh_b[4][RS][J];        // beta_g, then S_g
    __shared__ int sh_any[4][RS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t cid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (cid >= n_cand) return;                                  // whole warps
    if (lane == 0) {
        out_depth[cid] = NAN;
        out_var[cid] = NAN;
        out_dlnl[cid] = NAN;
        out_snr[cid] = NAN;
    }
    const int jd = Didx[cid];
    if (jd < 0 || jd >= n_D) return;
    const double P = Ps[cid], T0 = T0s[cid], D = Ds[jd];
    if (!isfinite(P) || !isfinite(T0) || !(D > 0.0) || !(2.0 * D <= P)) return;
    const double half = D * 0.5;
    const int64_t seg_lo0 = (int64_t)lane * nbs * RB;
    const int64_t seg_lo = seg_lo0 < n ? seg_lo0 : n;
    const int64_t seg_hi = seg_lo0 + nbs * RB < n ? seg_lo0 + nbs * RB : n;
    bool bad = false;

    // (a)
    double s[J];
#pragma unroll
    for (int q = 0; q < J; ++q) s[q] = 0.0;
    double c2 = 0.0, num = 0.0, bt[NU_MAX_K];
#pragma unroll
    for (int q = 0; q < NU_MAX_K; ++q) bt[q] = 0.0;
    int64_t cur = seg_lo;
    const bool any = rf_segment<NB, TMPL, false>(t, n, k, fv, Phi, Mq, n_blk, seg_lo, seg_hi, P,
                                                 T0, D, half, ta, s, true, c2, num, bt, cur,
                                                 bad);
    if (any && seg_hi < n) rf_zero_walk<NB, false>(fv, n, Phi, Mq, n_blk, cur, seg_hi, s, c2);
#pragma unroll
    for (int q = 0; q < J; ++q) sh_b[w][lane][q] = any ? s[q] : 0.0;
    sh_any[w][lane] = any ? 1 : 0;
    if (__any_sync(FULL, bad)) return;
    __syncwarp();
    const unsigned have = __ballot_sync(FULL, any);
    if (have == 0u) return;                                     // no sample in any window
    const int first = __ffs(have) - 1, last = 31 - __clz(have);

    // (b)
    if (lane == 0) {
        double x[J];
#pragma unroll
        for (int q = 0; q < J; ++q) x[q] = 0.0;
        for (int g = first; g <= last; ++g) {
            double beta[J];
#pragma unroll
            for (int q = 0; q < J; ++q) {
                beta[q] = sh_b[w][g][q];
                sh_b[w][g][q] = x[q];                           // S_g
            }
            const double* pg = Pseg + (int64_t)g * J * J;
            double o[J];
#pragma unroll
            for (int r = 0; r < J; ++r) {
                double a = beta[r];
#pragma unroll
                for (int q = 0; q < J; ++q) a = fma(pg[r * J + q], x[q], a);
                o[r] = a;
            }
#pragma unroll
            for (int q = 0; q < J; ++q) x[q] = o[q];
        }
    }
    __syncwarp();

    // (c)
    c2 = 0.0;
    if (lane >= first && lane <= last) {
#pragma unroll
        for (int q = 0; q < J; ++q) s[q] = sh_b[w][lane][q];
        rf_segment<NB, TMPL, true>(t, n, k, fv, Phi, Mq, n_blk, seg_lo, seg_hi, P, T0, D, half,
                                   ta, s, lane == first, c2, num, bt, cur, bad);
        if (lane == last) {
            if (cur < n) c2 += rf_quad<J>(fv.G + cur * JJ, s);   // zero input to the end
        } else {
            rf_zero_walk<NB, true>(fv, n, Phi, Mq, n_blk, cur, seg_hi, s, c2);
        }
    }
    if (__any_sync(FULL, bad)) return;
    for (int o = 16; o > 0; o >>= 1) {
        c2 += __shfl_xor_sync(FULL, c2, o);
        num += __shfl_xor_sync(FULL, num, o);
#pragma unroll
        for (int q = 0; q < NU_MAX_K; ++q) bt[q] += __shfl_xor_sync(FULL, bt[q], o);
    }
    if (lane != 0) return;
    double bb = 0.0;
    for (int q = 0; q < k; ++q) bb = fma(bt[q], bt[q], bb);
    const double sch = c2 - bb;
    if (!(sch > 0.0)) return;
    const double dep = num / sch;
    const double var = 1.0 / sch;
    out_depth[cid] = dep;
    out_var[cid] = var;
    out_dlnl[cid] = 0.5 * num * dep;
    out_snr[cid] = dep / sqrt(var);
}

template <int NB>
static void launch_refine(const nu_factor* f, const double* Phi, const double* Mq,
                          int64_t n_blk, double* Pseg, const double* P, const double* T0,
                          const int* Didx, int64_t n_cand, const double* Ds, int n_D, int tmpl,
                          const TmplArgs& ta, double* d, double* v, double* l, double* snr,
                          cudaStream_t st) {
    const FactorView<double> fv{f->F, f->kg, f->invD, f->G, f->z0, f->Zt};
    const int th = 128;
    // segments of nbs blocks cover every sample: RS * nbs * RB >= n
    const int64_t blocks_all = (f->n + RB - 1) / RB;
    const int64_t nbs = (blocks_all + RS - 1) / RS;
    if (n_blk > 0)
        k_refine_blocks<NB><<<div_up(n_blk, th), th, 0, st>>>(f->F, f->kg, f->invD, n_blk,
                                                             (double*)Phi, (double*)Mq);
    k_refine_segs<NB><<<div_up(RS * 2 * NB, th), th, 0, st>>>(Phi, n_blk, nbs, Pseg);
    const int grid = div_up(n_cand * 32, th);
    if (tmpl == NU_BOX)
        k_refine<NB, NU_BOX><<<grid, th, 0, st>>>(f->t, f->n, f->k, fv, Phi, Mq, n_blk, Pseg,
                                                 nbs, P, T0, Didx, n_cand, Ds, n_D, ta, d, v, l,
                                                 snr);
    else if (tmpl == NU_TRAPEZOID)
        k_refine<NB, NU_TRAPEZOID><<<grid, th, 0, st>>>(f->t, f->n, f->k, fv, Phi, Mq, n_blk,
                                                       Pseg, nbs, P, T0, Didx, n_cand, Ds, n_D,
                                                       ta, d, v, l, snr);
    else
        k_refine<NB, NU_LIMB_QUAD><<<grid, th, 0, st>>>(f->t, f->n, f->k, fv, Phi, Mq, n_blk,
                                                       Pseg, nbs, P, T0, Didx, n_cand, Ds, n_D,
                                                       ta, d, v, l, snr);
}

}  // namespace nu

using namespace nu;

extern "C" nu_status nu_periodic_refine(const nu_factor* f, const double* P_dev,
                                        const double* T0_dev, const int* D_idx_dev,
                                        int64_t n_cand, const double* Ds_host, int n_D,
                                        nu_template tmpl, const double* tmpl_params,
                                        void* stream,
                                        double* depth_dev, double* var_dev, double* dlnl_dev,
                                        double* snr_dev) {
    if (!f) return fail(NU_EINVAL, "nu_periodic_refine: null factor");
    if (!P_dev || !T0_dev || !D_idx_dev || !Ds_host || !depth_dev || !var_dev || !dlnl_dev ||
        !snr_dev)
        return fail(NU_EINVAL, "nu_periodic_refine: null array");
    if (n_cand < 1 || n_D < 1) return fail(NU_EINVAL, "nu_periodic_refine: empty input");
    if (n_cand > (int64_t)1 << 31)
        return fail(NU_EINVAL, "nu_periodic_refine: more than 2^31 candidates");
    TmplArgs ta;
    const char* why = "";
    if (!template_args((int)tmpl, tmpl_params, &ta, &why))
        return fail(NU_EINVAL, "nu_periodic_refine: %s (template %d)", why, (int)tmpl);
    for (int j = 0; j < n_D; ++j)
        if (!(Ds_host[j] > 0.0) || !std::isfinite(Ds_host[j]))
            return fail(NU_EINVAL, "nu_periodic_refine: durations must be finite and > 0");
    cudaStream_t st = (cudaStream_t)stream;
    const int J = 2 * f->nb, JJ = J * (J + 1) / 2;
    const int64_t n_blk = (f->n - 1) / RB;
    const size_t bytes = (n_D + n_blk * (int64_t)(J * J + JJ) + RS * J * J) * sizeof(double);
    pool_keep_memory();
    double* mem = nullptr;
    cudaError_t e = cudaMallocAsync(&mem, bytes, st);
    if (e != cudaSuccess) return cuda_fail(e, "nu_periodic_refine: cudaMallocAsync");
    double* Ds_dev = mem;
    double* Phi = mem + n_D;
    double* Mq = Phi + n_blk * J * J;
    double* Pseg = Mq + n_blk * JJ;
    e = cudaMemcpyAsync(Ds_dev, Ds_host, n_D * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "nu_periodic_refine: copy");
    if (f->stream != st) {
        e = cudaEventRecord(f->ready, f->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, f->ready, 0);
        if (e != cudaSuccess) {
            cudaFreeAsync(mem, st);
            return cuda_fail(e, "nu_periodic_refine: stream order");
        }
    }
    switch (f->nb) {
        case 1: launch_refine<1>(f, Phi, Mq, n_blk, Pseg, P_dev, T0_dev, D_idx_dev, n_cand, Ds_dev, n_D, tmpl, ta, depth_dev, var_dev, dlnl_dev, snr_dev, st); break;
        case 2: launch_refine<2>(f, Phi, Mq, n_blk, Pseg, P_dev, T0_dev, D_idx_dev, n_cand, Ds_dev, n_D, tmpl, ta, depth_dev, var_dev, dlnl_dev, snr_dev, st); break;
        case 3: launch_refine<3>(f, Phi, Mq, n_blk, Pseg, P_dev, T0_dev, D_idx_dev, n_cand, Ds_dev, n_D, tmpl, ta, depth_dev, var_dev, dlnl_dev, snr_dev, st); break;
        default: launch_refine<4>(f, Phi, Mq, n_blk, Pseg, P_dev, T0_dev, D_idx_dev, n_cand, Ds_dev, n_D, tmpl, ta, depth_dev, var_dev, dlnl_dev, snr_dev, st); break;
    }
    count_launches(n_blk > 0 ? 3 : 2);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "nu_periodic_refine: launch");
    e = cudaFreeAsync(mem, st);
    if (e != cudaSuccess) return cuda_fail(e, "nu_periodic_refine: cudaFreeAsync");
    return NU_OK;
}

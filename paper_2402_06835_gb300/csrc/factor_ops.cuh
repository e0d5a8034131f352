// The four sequential recursions of the factor as chunked-scan operations
// (see scan.cuh).  J = 2 NB is the state dimension, h picks the first
// component of every 2x2 block, F_i is the block-diagonal transition into
// sample i (F_0 is taken as 0: the prior at the first sample is P_inf).
//
// 1. Riccati: predicted covariances of the state-space form give the pivots
//    D_i and gains kg_i of Sigma = L diag(D) L^T.  Chunk elements are those of
//    the temporal parallelisation of Bayesian filters (Sarkka and
//    Garcia-Fernandez 2021, IEEE TAC 66, 299): for a chunk, (A, C, Jm) with
//    A the filtered-mean map from a known state before the chunk, C the
//    filtered covariance from that known state and Jm the information the
//    chunk's samples carry about it; they are built by running the filter
//    from the known state, composed with
//      A_ij = A_j X A_i, C_ij = A_j X C_i A_j^T + C_j,
//      Jm_ij = (X A_i)^T Jm_j A_i + Jm_i,  X = (I + C_i Jm_j)^-1,
//    and applied to an incoming filtered covariance P as
//      A (I + P Jm)^-1 P A^T + C.
// 2. Forward solve e = L^-1 x for the columns of X and y:
//      s_{i+1} = F_{i+1} (s_i + kg_i (x_i - h^T s_i)),  e_i = x_i - h^T s_i,
//    affine in s; elements (Phi, beta) map the state entering a chunk to the
//    state leaving it.
// 3. Backward solve v = L^-T u (reverse order):
//      v_i = u_i - kg_i^T g_i,  g_{i-1} = F_i^T (g_i + h v_i).
// 4. Future information G_i = h h^T / D_i + A_{i+1}^T G_{i+1} A_{i+1},
//    A_{i+1} = F_{i+1} (I - kg_i h^T) (reverse order); elements (Psi, Gam)
//    with G_s = Psi^T G_{e+1} Psi + Gam.
#pragma once

#include "scan.cuh"
#include "ss.cuh"

namespace nu {

constexpr int NRMAX = NU_MAX_K + 1;

// One light curve inside packed per-sample arrays.
struct SegInfo {
    int64_t s_off;                    // first sample
    int64_t n;                        // samples
    int64_t c_off;                    // first chunk (level-0 scan element)
    int64_t n_c;                      // chunks
    double pinf[2 * NU_MAX_BLOCKS];   // diagonal of the stationary covariance
};

// Samples [s, e] of global chunk gc (time order), the segment's first sample
// and its end (one past the last sample).  rev: chunks in reverse time order.
struct ChunkRange {
    int g;
    int64_t s, e, base, end;
};
__device__ __forceinline__ ChunkRange chunk_of(const SegInfo* __restrict__ segs,
                                               const int* __restrict__ chunk_seg,
                                               int64_t gc, int B, bool rev) {
    ChunkRange r;
    r.g = chunk_seg[gc];
    const SegInfo sg = segs[r.g];
    int64_t c = gc - sg.c_off;
    if (rev) c = sg.n_c - 1 - c;
    r.base = sg.s_off;
    r.end = sg.s_off + sg.n;
    r.s = r.base + c * B;
    r.e = (r.s + B < r.end ? r.s + B : r.end) - 1;
    return r;
}

// dense J x J copy of the block-diagonal transition into sample i
template <int NB>
__device__ __forceinline__ void dense_F(const double* __restrict__ F, int64_t i,
                                        Mat<2 * NB>& Fm, bool first = false) {
    mat_zero(Fm);
    if (first) return;
    const double* f = F + i * NB * 4;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        Fm(2 * b, 2 * b) = f[4 * b];
        Fm(2 * b, 2 * b + 1) = f[4 * b + 1];
        Fm(2 * b + 1, 2 * b) = f[4 * b + 2];
        Fm(2 * b + 1, 2 * b + 1) = f[4 * b + 3];
    }
}

// M <- F M F^T for block-diagonal F (F_0 = 0)
template <int NB>
__device__ __forceinline__ void congruence_F(const double* __restrict__ F, int64_t i,
                                             Mat<2 * NB>& M, bool first) {
    constexpr int J = 2 * NB;
    if (first) {
        mat_zero(M);
        return;
    }
    const double* f = F + i * NB * 4;
    Mat<J> T;
#pragma unroll
    for (int c = 0; c < J; ++c) {
        double col[J], out[J];
#pragma unroll
        for (int r = 0; r < J; ++r) col[r] = M(r, c);
        apply_F<NB>(f, col, out);
#pragma unroll
        for (int r = 0; r < J; ++r) T(r, c) = out[r];
    }
#pragma unroll
    for (int r = 0; r < J; ++r) {
        double row[J], out[J];
#pragma unroll
        for (int c = 0; c < J; ++c) row[c] = T(r, c);
        apply_F<NB>(f, row, out);
#pragma unroll
        for (int c = 0; c < J; ++c) M(r, c) = out[c];
    }
    mat_symmetrize(M);
}


// --------------------------------------------------------------- Riccati
template <int NB>
struct RiccatiOp {
    static constexpr int J = 2 * NB;
    struct Elem {
        Mat<J> A, C, Jm;
    };
    struct State {
        Mat<J> P;          // filtered covariance after the previous chunk
    };
    const SegInfo* segs;
    const int* chunk_seg;
    const double* F;
    const double* dv;
    int B;
    double* kg;
    double* invD;
    double* Dpiv;
    long long* dstat;      // per segment: [2 g] status, [2 g + 1] first bad sample (local)

    __device__ void init_state(State& s) const { mat_zero(s.P); }

    // one filter step from the explained covariance Mf (= P_inf - P_filtered)
    // of the previous sample; returns D, P h and the filtered Mf of this sample
    __device__ __forceinline__ double step(int64_t i, bool first, const double* pinf,
                                           Mat<J>& Mf, double* Ph) const {
        congruence_F<NB>(F, i, Mf, first);           // M_i = F_i Mf F_i^T
        double hMh = 0.0, prior = 0.0;
#pragma unroll
        for (int r = 0; r < J; ++r) {
            double t = Mf(r, 0);
#pragma unroll
            for (int b = 1; b < NB; ++b) t += Mf(r, 2 * b);
            Ph[r] = (r % 2 == 0 ? pinf[r] : 0.0) - t;   // P h = (P_inf - M) h
            if (r % 2 == 0) {
                hMh += t;
                prior += pinf[r];
            }
        }
        const double D = (prior + dv[i]) - hMh;
        const double iD = 1.0 / D;
#pragma unroll
        for (int r = 0; r < J; ++r)
#pragma unroll
            for (int c = 0; c < J; ++c) Mf(r, c) = fma(Ph[r] * iD, Ph[c], Mf(r, c));
        return D;
    }

    __device__ void elem(int64_t gc, Elem& E) const {
        const ChunkRange cr = chunk_of(segs, chunk_seg, gc, B, false);
        const double* pinf = segs[cr.g].pinf;
        Mat<J> Mf, Psi, Jacc;
        mat_zero(Mf);
#pragma unroll
        for (int r = 0; r < J; ++r) Mf(r, r) = pinf[r];   // known state: P = 0
        mat_eye(Psi);
        mat_zero(Jacc);
        for (int64_t i = cr.s; i <= cr.e; ++i) {
            const bool first = i == cr.base;
            Mat<J> Fm, Phi;
            dense_F<NB>(F, i, Fm, first);
            mat_mul(Fm, Psi, Phi);                          // predicted sensitivity
            double Ph[J];
            const double D = step(i, first, pinf, Mf, Ph);
            const double iD = 1.0 / D;
            double g[J];
#pragma unroll
            for (int q = 0; q < J; ++q) {
                double t = Phi(0, q);
#pragma unroll
                for (int b = 1; b < NB; ++b) t += Phi(2 * b, q);
                g[q] = t;
            }
#pragma unroll
            for (int r = 0; r < J; ++r)
#pragma unroll
                for (int q = 0; q < J; ++q) Jacc(r, q) = fma(g[r] * iD, g[q], Jacc(r, q));
            // Psi = (I - k h^T) Phi, k = P h / D
#pragma unroll
            for (int r = 0; r < J; ++r)
#pragma unroll
                for (int q = 0; q < J; ++q) Psi(r, q) = fma(-Ph[r] * iD, g[q], Phi(r, q));
        }
        E.A = Psi;
#pragma unroll
        for (int r = 0; r < J; ++r)
#pragma unroll
            for (int q = 0; q < J; ++q) E.C(r, q) = (r == q ? pinf[r] : 0.0) - Mf(r, q);
        mat_symmetrize(E.C);
        mat_symmetrize(Jacc);
        E.Jm = Jacc;
    }

    __device__ void combine(Elem& ei, const Elem& ej) const {
        // X = (I + C_i Jm_j)^-1 applied to A_i and C_i
        Mat<J> M, Y1 = ei.A, Y2 = ei.C;
        mat_mul(ei.C, ej.Jm, M);
#pragma unroll
        for (int r = 0; r < J; ++r) M(r, r) += 1.0;
        Mat<J>* rhs[2] = {&Y1, &Y2};
        mat_solve<J, 2>(M, rhs);
        Mat<J> T, An, Cn, Jn;
        mat_mul(ej.A, Y1, An);                // A_j X A_i
        mat_mul(ej.A, Y2, T);                 // A_j X C_i
        mat_mult(T, ej.A, Cn);                // ... A_j^T
#pragma unroll
        for (int i = 0; i < J * J; ++i) Cn.a[i] += ej.C.a[i];
        mat_symmetrize(Cn);
        mat_tmul(Y1, ej.Jm, T);               // (X A_i)^T Jm_j
        mat_mul(T, ei.A, Jn);                 // ... A_i
#pragma unroll
        for (int i = 0; i < J * J; ++i) Jn.a[i] += ei.Jm.a[i];
        mat_symmetrize(Jn);
        ei.A = An;
        ei.C = Cn;
        ei.Jm = Jn;
    }

    __device__ void apply(const Elem& E, State& st) const {
        Mat<J> M, Y = st.P;
        mat_mul(st.P, E.Jm, M);
#pragma unroll
        for (int r = 0; r < J; ++r) M(r, r) += 1.0;
        Mat<J>* rhs[1] = {&Y};
        mat_solve<J, 1>(M, rhs);              // (I + P Jm)^-1 P
        Mat<J> T;
        mat_mul(E.A, Y, T);
        mat_mult(T, E.A, st.P);
#pragma unroll
        for (int i = 0; i < J * J; ++i) st.P.a[i] += E.C.a[i];
        mat_symmetrize(st.P);
    }

    __device__ void final(int64_t gc, const State& st) const {
        const ChunkRange cr = chunk_of(segs, chunk_seg, gc, B, false);
        const double* pinf = segs[cr.g].pinf;
        Mat<J> Mf;
#pragma unroll
        for (int r = 0; r < J; ++r)
#pragma unroll
            for (int q = 0; q < J; ++q) Mf(r, q) = (r == q ? pinf[r] : 0.0) - st.P(r, q);
        for (int64_t i = cr.s; i <= cr.e; ++i) {
            double Ph[J];
            const double D = step(i, i == cr.base, pinf, Mf, Ph);
            if (!(D > 0.0) || !isfinite(D)) {
                long long* ds = dstat + 2 * cr.g;
                const unsigned long long loc = (unsigned long long)(i - cr.base);
                const unsigned long long old = atomicMin((unsigned long long*)&ds[1], loc);
                if (old > loc) atomicExch((unsigned long long*)&ds[0], 2ull);
            }
            const double iD = 1.0 / D;
#pragma unroll
            for (int r = 0; r < J; ++r) kg[i * J + r] = Ph[r] * iD;
            invD[i] = iD;
            Dpiv[i] = D;
        }
    }
};

// ------------------------------------------- Riccati tree, one warp per group
// The tree levels of the Riccati scan have few groups (C2: 608 at the widest),
// and each combine or apply is a chain of about 600 FP64 operations on J x J
// matrices in one thread.  Here one warp takes a group and its lanes own the
// matrix entries (row-major in shared memory), so a product is J FMAs per
// lane and the Gauss-Jordan solve J short steps.  Every entry goes through the
// same sequence of FP64 operations as in the thread version (mat_mul,
// mat_solve, mat_symmetrize).
template <int J>
struct WEnt {
    static constexpr int N = J * J;
    static constexpr int PER = (N + 31) / 32;
};

// C = A B, C = A^T B, C = A B^T (C must not alias A or B)
template <int J, int MODE>
__device__ __forceinline__ void wmat_prod(const double* A, const double* B, double* C,
                                          int lane) {
#pragma unroll
    for (int t = 0; t < WEnt<J>::PER; ++t) {
        const int e = lane + 32 * t;
        if (e < J * J) {
            const int r = e / J, c = e - r * J;
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < J; ++k) {
                const double a = MODE == 1 ? A[k * J + r] : A[r * J + k];
                const double b = MODE == 2 ? B[c * J + k] : B[k * J + c];
                s = fma(a, b, s);
            }
            C[e] = s;
        }
    }
    __syncwarp();
}

// m <- (m + add) symmetrised as mat_symmetrize does (add may be null)
template <int J>
__device__ __forceinline__ void wmat_add_sym(double* m, const double* add, int lane) {
    if (add) {
#pragma unroll
        for (int t = 0; t < WEnt<J>::PER; ++t) {
            const int e = lane + 32 * t;
            if (e < J * J) m[e] += add[e];
        }
        __syncwarp();
    }
    double v[WEnt<J>::PER];
#pragma unroll
    for (int t = 0; t < WEnt<J>::PER; ++t) {
        const int e = lane + 32 * t;
        if (e < J * J) {
            const int r = e / J, c = e - r * J;
            const int lo = r < c ? r : c, hi = r < c ? c : r;
            v[t] = r == c ? m[e] : 0.5 * (m[lo * J + hi] + m[hi * J + lo]);
        }
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < WEnt<J>::PER; ++t) {
        const int e = lane + 32 * t;
        if (e < J * J) m[e] = v[t];
    }
    __syncwarp();
}

// [B1 B2] <- M^-1 [B1 B2] by Gauss-Jordan with partial pivoting (the first
// row of largest magnitude), as mat_solve; M is overwritten.  B2 may be null.
template <int J, int NRHS>
__device__ __forceinline__ void wmat_solve(double* M, double* B1, double* B2, int lane) {
    constexpr int W = (NRHS + 1) * J;                  // augmented row width
    constexpr int PER = (J * W + 31) / 32;
    auto at = [&](int r, int k) -> double* {
        return k < J ? &M[r * J + k] : (k < 2 * J ? &B1[r * J + k - J] : &B2[r * J + k - 2 * J]);
    };
    for (int c = 0; c < J; ++c) {
        double v = (lane >= c && lane < J) ? fabs(M[lane * J + c]) : -1.0;
        int piv = lane;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
            const int p2 = __shfl_xor_sync(0xffffffffu, piv, o);
            if (v2 > v || (v2 == v && p2 < piv)) {
                v = v2;
                piv = p2;
            }
        }
        // lane 0's choice for all (lanes could disagree only on NaN entries)
        piv = __shfl_sync(0xffffffffu, piv, 0);
        if (piv != c && piv < J) {
            for (int k = lane; k < W; k += 32) {
                double* a = at(c, k);
                double* b = at(piv, k);
                const double tmp = *a;
                *a = *b;
                *b = tmp;
            }
            __syncwarp();
        }
        const double inv = 1.0 / M[c * J + c];
        __syncwarp();
        for (int k = lane; k < W; k += 32) *at(c, k) *= inv;
        __syncwarp();
        double f[PER];
#pragma unroll
        for (int t = 0; t < PER; ++t) {
            const int e = lane + 32 * t;
            f[t] = e < J * W ? M[(e / W) * J + c] : 0.0;
        }
        __syncwarp();
#pragma unroll
        for (int t = 0; t < PER; ++t) {
            const int e = lane + 32 * t;
            if (e < J * W) {
                const int r = e / W, k = e - r * W;
                if (r != c) {
                    double* x = at(r, k);
                    *x = fma(-f[t], *at(c, k), *x);
                }
            }
        }
        __syncwarp();
    }
}

template <int J>
__device__ __forceinline__ void wcopy(double* dst, const double* src, int n, int lane) {
    for (int e = lane; e < n; e += 32) dst[e] = src[e];
    __syncwarp();
}

// shared-memory workspace of one warp
template <int J>
struct RicWarpSmem {
    double A[J * J], C[J * J], Jm[J * J];       // accumulated element / state P in A
    double eA[J * J], eC[J * J], eJ[J * J];     // the element being applied
    double M[J * J], Y1[J * J], Y2[J * J], T[J * J], R1[J * J], R2[J * J], R3[J * J];
};

// acc <- combine(acc, e) (RiccatiOp::combine)
template <int J>
__device__ __forceinline__ void ric_combine_w(RicWarpSmem<J>& s, int lane) {
    wmat_prod<J, 0>(s.C, s.eJ, s.M, lane);            // C_i Jm_j
    if (lane < J) s.M[lane * J + lane] += 1.0;
    wcopy<J>(s.Y1, s.A, J * J, lane);
    wcopy<J>(s.Y2, s.C, J * J, lane);
    wmat_solve<J, 2>(s.M, s.Y1, s.Y2, lane);          // X A_i, X C_i
    wmat_prod<J, 0>(s.eA, s.Y1, s.R1, lane);          // A_j X A_i
    wmat_prod<J, 0>(s.eA, s.Y2, s.T, lane);           // A_j X C_i
    wmat_prod<J, 2>(s.T, s.eA, s.R2, lane);           // ... A_j^T
    wmat_add_sym<J>(s.R2, s.eC, lane);
    wmat_prod<J, 1>(s.Y1, s.eJ, s.T, lane);           // (X A_i)^T Jm_j
    wmat_prod<J, 0>(s.T, s.A, s.R3, lane);            // ... A_i
    wmat_add_sym<J>(s.R3, s.Jm, lane);
    wcopy<J>(s.A, s.R1, J * J, lane);
    wcopy<J>(s.C, s.R2, J * J, lane);
    wcopy<J>(s.Jm, s.R3, J * J, lane);
}

// P (in s.A) <- apply(e, P) (RiccatiOp::apply)
template <int J>
__device__ __forceinline__ void ric_apply_w(RicWarpSmem<J>& s, int lane) {
    wmat_prod<J, 0>(s.A, s.eJ, s.M, lane);            // P Jm
    if (lane < J) s.M[lane * J + lane] += 1.0;
    wcopy<J>(s.Y1, s.A, J * J, lane);
    wmat_solve<J, 1>(s.M, s.Y1, nullptr, lane);        // (I + P Jm)^-1 P
    wmat_prod<J, 0>(s.eA, s.Y1, s.T, lane);
    wmat_prod<J, 2>(s.T, s.eA, s.R1, lane);
    wmat_add_sym<J>(s.R1, s.eC, lane);
    wcopy<J>(s.A, s.R1, J * J, lane);
}

template <int J, class E>
__device__ __forceinline__ void ric_load_elem(RicWarpSmem<J>& s, const E& src, bool to_acc,
                                              int lane) {
    double* dA = to_acc ? s.A : s.eA;
    double* dC = to_acc ? s.C : s.eC;
    double* dJ = to_acc ? s.Jm : s.eJ;
    for (int e = lane; e < J * J; e += 32) {
        dA[e] = src.A.a[e];
        dC[e] = src.C.a[e];
        dJ[e] = src.Jm.a[e];
    }
    __syncwarp();
}

template <int NB>
__global__ void __launch_bounds__(32)
k_ric_combine_warp(const typename RiccatiOp<NB>::Elem* __restrict__ Ein,
                   const int64_t* __restrict__ cb, const int64_t* __restrict__ ce,
                   int64_t n_out, typename RiccatiOp<NB>::Elem* __restrict__ Eout) {
    constexpr int J = 2 * NB;
    __shared__ RicWarpSmem<J> s;
    const int64_t q = blockIdx.x;
    const int lane = threadIdx.x;
    if (q >= n_out) return;
    ric_load_elem<J>(s, Ein[cb[q]], true, lane);
    for (int64_t r = cb[q] + 1; r < ce[q]; ++r) {
        ric_load_elem<J>(s, Ein[r], false, lane);
        ric_combine_w<J>(s, lane);
    }
    for (int e = lane; e < J * J; e += 32) {
        Eout[q].A.a[e] = s.A[e];
        Eout[q].C.a[e] = s.C[e];
        Eout[q].Jm.a[e] = s.Jm[e];
    }
}

template <int NB>
__global__ void __launch_bounds__(32)
k_ric_down_warp(const typename RiccatiOp<NB>::Elem* __restrict__ E,
                const int64_t* __restrict__ cb, const int64_t* __restrict__ ce,
                int64_t n_parent, const typename RiccatiOp<NB>::State* __restrict__ Sparent,
                typename RiccatiOp<NB>::State* __restrict__ S) {
    constexpr int J = 2 * NB;
    __shared__ RicWarpSmem<J> s;
    const int64_t q = blockIdx.x;
    const int lane = threadIdx.x;
    if (q >= n_parent) return;
    wcopy<J>(s.A, Sparent[q].P.a, J * J, lane);
    for (int64_t r = cb[q]; r < ce[q]; ++r) {
        for (int e = lane; e < J * J; e += 32) S[r].P.a[e] = s.A[e];
        ric_load_elem<J>(s, E[r], false, lane);
        ric_apply_w<J>(s, lane);
    }
}

template <int NB>
__global__ void __launch_bounds__(32)
k_ric_top_warp(const typename RiccatiOp<NB>::Elem* __restrict__ E,
               const int64_t* __restrict__ tb, const int64_t* __restrict__ te, int n_seg,
               typename RiccatiOp<NB>::State* __restrict__ S) {
    constexpr int J = 2 * NB;
    __shared__ RicWarpSmem<J> s;
    const int g = blockIdx.x;
    const int lane = threadIdx.x;
    if (g >= n_seg) return;
    for (int e = lane; e < J * J; e += 32) s.A[e] = 0.0;
    __syncwarp();
    for (int64_t i = tb[g]; i < te[g]; ++i) {
        for (int e = lane; e < J * J; e += 32) S[i].P.a[e] = s.A[e];
        ric_load_elem<J>(s, E[i], false, lane);
        ric_apply_w<J>(s, lane);
    }
}

// Levels with up to this many groups run one warp per group; wider levels
// (large batches) keep one thread per group, which packs 32 groups into each
// FP64 warp instruction.
constexpr int64_t RIC_WARP_TREE_MAX = 4096;

template <int NB>
inline void scan_combine(const RiccatiOp<NB>& op, const typename RiccatiOp<NB>::Elem* Ein,
                         const int64_t* cb, const int64_t* ce, int64_t n,
                         typename RiccatiOp<NB>::Elem* Eout, cudaStream_t st) {
    if (n <= RIC_WARP_TREE_MAX)
        k_ric_combine_warp<NB><<<(unsigned)n, 32, 0, st>>>(Ein, cb, ce, n, Eout);
    else
        scan_combine_threads(op, Ein, cb, ce, n, Eout, st);
}

template <int NB>
inline void scan_down(const RiccatiOp<NB>& op, const typename RiccatiOp<NB>::Elem* E,
                      const int64_t* cb, const int64_t* ce, int64_t n,
                      const typename RiccatiOp<NB>::State* Sp,
                      typename RiccatiOp<NB>::State* S, cudaStream_t st) {
    if (n <= RIC_WARP_TREE_MAX)
        k_ric_down_warp<NB><<<(unsigned)n, 32, 0, st>>>(E, cb, ce, n, Sp, S);
    else
        scan_down_threads(op, E, cb, ce, n, Sp, S, st);
}

template <int NB>
inline void scan_top(const RiccatiOp<NB>& op, const typename RiccatiOp<NB>::Elem* E,
                     const int64_t* tb, const int64_t* te, int n_seg,
                     typename RiccatiOp<NB>::State* S, cudaStream_t st) {
    if (n_seg <= RIC_WARP_TREE_MAX)
        k_ric_top_warp<NB><<<(unsigned)n_seg, 32, 0, st>>>(E, tb, te, n_seg, S);
    else
        scan_top_threads(op, E, tb, te, n_seg, S, st);
}

// ---------------------------------------------------------- forward solve
// Right-hand sides: the k columns of X (column-major with leading dimension
// ldx, or the polynomial columns [1, t] when X is null) and y.
template <int NB>
struct ForwardOp {
    static constexpr int J = 2 * NB;
    struct Elem {
        Mat<J> Phi;
        double beta[NRMAX][J];
    };
    struct State {
        double s[NRMAX][J];
    };
    const SegInfo* segs;
    const int* chunk_seg;
    const double* F;
    const double* kg;
    const double* invD;
    const double* X;
    int64_t ldx;
    const double* t;       // for polynomial columns
    const double* y;
    int k;
    int B;
    double* E;             // innovations [n][k+1]
    double* partial;       // per chunk (k+1)^2 weighted cross products

    __device__ __forceinline__ double xval(int64_t i, int r) const {
        if (r == k) return y[i];
        if (X) return X[(int64_t)r * ldx + i];
        return r == 0 ? 1.0 : t[i];
    }
    __device__ void init_state(State& st) const {
#pragma unroll
        for (int r = 0; r < NRMAX; ++r)
#pragma unroll
            for (int q = 0; q < J; ++q) st.s[r][q] = 0.0;
    }
    __device__ void elem(int64_t gc, Elem& El) const {
        const ChunkRange cr = chunk_of(segs, chunk_seg, gc, B, false);
        mat_eye(El.Phi);
        const int nr = k + 1;
#pragma unroll
        for (int r = 0; r < NRMAX; ++r)
#pragma unroll
            for (int q = 0; q < J; ++q) El.beta[r][q] = 0.0;
        for (int64_t i = cr.s; i <= cr.e && i + 1 < cr.end; ++i) {
            const double* kgi = kg + i * J;
            const double* f = F + (i + 1) * NB * 4;
            // Phi <- F (Phi - kg h^T Phi)
#pragma unroll
            for (int q = 0; q < J; ++q) {
                double hp = El.Phi(0, q);
#pragma unroll
                for (int b = 1; b < NB; ++b) hp += El.Phi(2 * b, q);
                double col[J], out[J];
#pragma unroll
                for (int r = 0; r < J; ++r) col[r] = fma(-kgi[r], hp, El.Phi(r, q));
                apply_F<NB>(f, col, out);
#pragma unroll
                for (int r = 0; r < J; ++r) El.Phi(r, q) = out[r];
            }
            for (int r = 0; r < nr; ++r) {
                const double innov = xval(i, r) - hdot<NB>(El.beta[r]);
                double col[J];
#pragma unroll
                for (int q = 0; q < J; ++q) col[q] = fma(kgi[q], innov, El.beta[r][q]);
                apply_F<NB>(f, col, El.beta[r]);
            }
        }
    }
    __device__ void combine(Elem& ei, const Elem& ej) const {
        Mat<J> P;
        mat_mul(ej.Phi, ei.Phi, P);
        const int nr = k + 1;
        for (int r = 0; r < nr; ++r) {
            double out[J];
#pragma unroll
            for (int a = 0; a < J; ++a) {
                double v = ej.beta[r][a];
#pragma unroll
                for (int b = 0; b < J; ++b) v = fma(ej.Phi(a, b), ei.beta[r][b], v);
                out[a] = v;
            }
#pragma unroll
            for (int a = 0; a < J; ++a) ei.beta[r][a] = out[a];
        }
        ei.Phi = P;
    }
    __device__ void apply(const Elem& El, State& st) const {
        const int nr = k + 1;
        for (int r = 0; r < nr; ++r) {
            double out[J];
#pragma unroll
            for (int a = 0; a < J; ++a) {
                double v = El.beta[r][a];
#pragma unroll
                for (int b = 0; b < J; ++b) v = fma(El.Phi(a, b), st.s[r][b], v);
                out[a] = v;
            }
#pragma unroll
            for (int a = 0; a < J; ++a) st.s[r][a] = out[a];
        }
    }
    __device__ void final(int64_t gc, const State& st0) const {
        const ChunkRange cr = chunk_of(segs, chunk_seg, gc, B, false);
        State st = st0;
        const int nr = k + 1;
        double acc[NRMAX][NRMAX];
        for (int a = 0; a < nr; ++a)
            for (int b = 0; b < nr; ++b) acc[a][b] = 0.0;
        for (int64_t i = cr.s; i <= cr.e; ++i) {
            const double iD = invD[i];
            double ev[NRMAX];
            for (int r = 0; r < nr; ++r) {
                ev[r] = xval(i, r) - hdot<NB>(st.s[r]);
                E[i * nr + r] = ev[r];
            }
            for (int a = 0; a < nr; ++a)
                for (int b = 0; b <= a; ++b) acc[a][b] = fma(ev[a] * iD, ev[b], acc[a][b]);
            if (i + 1 < cr.end) {
                const double* kgi = kg + i * J;
                const double* f = F + (i + 1) * NB * 4;
                for (int r = 0; r < nr; ++r) {
                    double col[J];
#pragma unroll
                    for (int q = 0; q < J; ++q) col[q] = fma(kgi[q], ev[r], st.s[r][q]);
                    apply_F<NB>(f, col, st.s[r]);
                }
            }
        }
        double* p = partial + gc * NRMAX * NRMAX;
        for (int a = 0; a < nr; ++a)
            for (int b = 0; b <= a; ++b) {
                p[a * NRMAX + b] = acc[a][b];
                p[b * NRMAX + a] = acc[a][b];
            }
    }
};

// --------------------------------------------------------- backward solve
template <int NB>
struct BackwardOp {
    static constexpr int J = 2 * NB;
    struct Elem {
        Mat<J> Phi;
        double beta[NRMAX][J];
    };
    struct State {
        double g[NRMAX][J];
    };
    const SegInfo* segs;
    const int* chunk_seg;
    const double* F;
    const double* kg;
    const double* U;       // right-hand sides [n][nr]
    int nr;
    int k;
    int B;
    double* z0;
    double* Zt;            // [n][k]

    __device__ void init_state(State& st) const {
#pragma unroll
        for (int r = 0; r < NRMAX; ++r)
#pragma unroll
            for (int q = 0; q < J; ++q) st.g[r][q] = 0.0;
    }
    __device__ void elem(int64_t gc, Elem& El) const {
        const ChunkRange cr = chunk_of(segs, chunk_seg, gc, B, true);
        mat_eye(El.Phi);
#pragma unroll
        for (int r = 0; r < NRMAX; ++r)
#pragma unroll
            for (int a = 0; a < J; ++a) El.beta[r][a] = 0.0;
        for (int64_t i = cr.e; i >= cr.s && i > cr.base; --i) {
            const double* kgi = kg + i * J;
            const double* f = F + i * NB * 4;
            // Phi <- F_i^T (Phi - h kg^T Phi)
#pragma unroll
            for (int a = 0; a < J; ++a) {
                double kp = 0.0;
#pragma unroll
                for (int b = 0; b < J; ++b) kp = fma(kgi[b], El.Phi(b, a), kp);
                double col[J], out[J];
#pragma unroll
                for (int b = 0; b < J; ++b) col[b] = El.Phi(b, a) - ((b % 2 == 0) ? kp : 0.0);
                apply_FT<NB>(f, col, out);
#pragma unroll
                for (int b = 0; b < J; ++b) El.Phi(b, a) = out[b];
            }
            for (int r = 0; r < nr; ++r) {
                double v = U[i * nr + r];
#pragma unroll
                for (int b = 0; b < J; ++b) v = fma(-kgi[b], El.beta[r][b], v);
                double col[J];
#pragma unroll
                for (int b = 0; b < J; ++b) col[b] = El.beta[r][b] + ((b % 2 == 0) ? v : 0.0);
                apply_FT<NB>(f, col, El.beta[r]);
            }
        }
    }
    __device__ void combine(Elem& ei, const Elem& ej) const {
        Mat<J> P;
        mat_mul(ej.Phi, ei.Phi, P);
        for (int r = 0; r < nr; ++r) {
            double out[J];
#pragma unroll
            for (int a = 0; a < J; ++a) {
                double v = ej.beta[r][a];
#pragma unroll
                for (int b = 0; b < J; ++b) v = fma(ej.Phi(a, b), ei.beta[r][b], v);
                out[a] = v;
            }
#pragma unroll
            for (int a = 0; a < J; ++a) ei.beta[r][a] = out[a];
        }
        ei.Phi = P;
    }
    __device__ void apply(const Elem& El, State& st) const {
        for (int r = 0; r < nr; ++r) {
            double out[J];
#pragma unroll
            for (int a = 0; a < J; ++a) {
                double v = El.beta[r][a];
#pragma unroll
                for (int b = 0; b < J; ++b) v = fma(El.Phi(a, b), st.g[r][b], v);
                out[a] = v;
            }
#pragma unroll
            for (int a = 0; a < J; ++a) st.g[r][a] = out[a];
        }
    }
    __device__ void final(int64_t gc, const State& st0) const {
        const ChunkRange cr = chunk_of(segs, chunk_seg, gc, B, true);
        State st = st0;
        for (int64_t i = cr.e; i >= cr.s; --i) {
            const double* kgi = kg + i * J;
            const double* f = F + i * NB * 4;
            for (int r = 0; r < nr; ++r) {
                double v = U[i * nr + r];
#pragma unroll
                for (int b = 0; b < J; ++b) v = fma(-kgi[b], st.g[r][b], v);
                if (r == 0) z0[i] = v; else Zt[i * k + (r - 1)] = v;
                if (i > cr.base) {
                    double col[J];
#pragma unroll
                    for (int b = 0; b < J; ++b) col[b] = st.g[r][b] + ((b % 2 == 0) ? v : 0.0);
                    apply_FT<NB>(f, col, st.g[r]);
                }
            }
        }
    }
};

// ------------------------------------------------ future information G
template <int NB>
struct FutureOp {
    static constexpr int J = 2 * NB;
    static constexpr int JJ = J * (J + 1) / 2;
    struct Elem {
        Mat<J> Psi, Gam;
    };
    struct State {
        Mat<J> G;
    };
    const SegInfo* segs;
    const int* chunk_seg;
    const double* F;
    const double* kg;
    const double* invD;
    int B;
    double* Gout;          // packed upper [n][JJ]

    // A_{i+1} = F_{i+1} (I - kg_i h^T) as a dense matrix
    __device__ __forceinline__ void closed_loop(int64_t i, Mat<J>& A) const {
        const double* f = F + (i + 1) * NB * 4;
        const double* kgi = kg + i * J;
        double fk[J];
        apply_F<NB>(f, kgi, fk);
        dense_F<NB>(F, i + 1, A);
#pragma unroll
        for (int r = 0; r < J; ++r)
#pragma unroll
            for (int b = 0; b < NB; ++b) A(r, 2 * b) -= fk[r];
    }
    __device__ void init_state(State& st) const { mat_zero(st.G); }
    __device__ void elem(int64_t gc, Elem& El) const {
        const ChunkRange cr = chunk_of(segs, chunk_seg, gc, B, true);
        mat_eye(El.Psi);
        mat_zero(El.Gam);
        for (int64_t i = cr.e; i >= cr.s; --i) {
            if (i + 1 < cr.end) {
                Mat<J> A, T;
                closed_loop(i, A);
                mat_mul(El.Psi, A, T);
                El.Psi = T;
                mat_mul(El.Gam, A, T);
                mat_tmul(A, T, El.Gam);
            }
            const double iD = invD[i];
#pragma unroll
            for (int r = 0; r < J; r += 2)
#pragma unroll
                for (int c = 0; c < J; c += 2) El.Gam(r, c) += iD;
        }
        mat_symmetrize(El.Gam);
    }
    __device__ void combine(Elem& ei, const Elem& ej) const {
        // ei: later samples (earlier in scan order), ej: earlier samples
        Mat<J> P, T, Gn;
        mat_mul(ei.Psi, ej.Psi, P);
        mat_mul(ei.Gam, ej.Psi, T);
        mat_tmul(ej.Psi, T, Gn);
#pragma unroll
        for (int i = 0; i < J * J; ++i) Gn.a[i] += ej.Gam.a[i];
        mat_symmetrize(Gn);
        ei.Psi = P;
        ei.Gam = Gn;
    }
    __device__ void apply(const Elem& El, State& st) const {
        Mat<J> T, Gn;
        mat_mul(st.G, El.Psi, T);
        mat_tmul(El.Psi, T, Gn);
#pragma unroll
        for (int i = 0; i < J * J; ++i) Gn.a[i] += El.Gam.a[i];
        mat_symmetrize(Gn);
        st.G = Gn;
    }
    __device__ void final(int64_t gc, const State& st0) const {
        const ChunkRange cr = chunk_of(segs, chunk_seg, gc, B, true);
        Mat<J> G = st0.G;
        for (int64_t i = cr.e; i >= cr.s; --i) {
            if (i + 1 < cr.end) {
                Mat<J> A, T;
                closed_loop(i, A);
                mat_mul(G, A, T);
                mat_tmul(A, T, G);
            } else {
                mat_zero(G);
            }
            const double iD = invD[i];
#pragma unroll
            for (int r = 0; r < J; r += 2)
#pragma unroll
                for (int c = 0; c < J; c += 2) G(r, c) += iD;
            mat_symmetrize(G);
            double* Gi = Gout + i * JJ;
#pragma unroll
            for (int r = 0; r < J; ++r)
#pragma unroll
                for (int c = r; c < J; ++c) Gi[pk(r, c, J)] = G(r, c);
        }
    }
};

// ------------------------------- affine and future-information trees, warps
// The same one-warp-per-group scheme for the other three scans.  Forward and
// backward solves share one element layout (Phi J x J, beta NRMAX x J; the
// state NRMAX x J), combined as P = Phi_j Phi_i, beta_i <- Phi_j beta_i +
// beta_j and applied as s <- Phi s + beta; the future information's element
// (Psi, Gam) combines as Psi_i Psi_j, Psi_j^T Gam_i Psi_j + Gam_j and applies
// to G as Psi^T G Psi + Gam.  Each entry follows the thread code's order.
template <int J>
struct AffWarpSmem {
    double P[J * J], b[NRMAX * J];        // accumulated element, or the state in b
    double eP[J * J], eb[NRMAX * J];      // the element being applied
    double R[J * J], rb[NRMAX * J];
};

template <int J>
__device__ __forceinline__ void aff_load(double* P, double* b, const double* src, int lane) {
    for (int e = lane; e < J * J; e += 32) P[e] = src[e];
    for (int e = lane; e < NRMAX * J; e += 32) b[e] = src[J * J + e];
    __syncwarp();
}

// acc (P, b) <- combine(acc, e): b rows r < nr
template <int J>
__device__ __forceinline__ void aff_combine_w(AffWarpSmem<J>& s, int nr, int lane) {
    wmat_prod<J, 0>(s.eP, s.P, s.R, lane);
    for (int e = lane; e < nr * J; e += 32) {
        const int r = e / J, a = e - r * J;
        double v = s.eb[r * J + a];
#pragma unroll
        for (int q = 0; q < J; ++q) v = fma(s.eP[a * J + q], s.b[r * J + q], v);
        s.rb[e] = v;
    }
    __syncwarp();
    for (int e = lane; e < J * J; e += 32) s.P[e] = s.R[e];
    for (int e = lane; e < nr * J; e += 32) s.b[e] = s.rb[e];
    __syncwarp();
}

// state (in b) <- apply(e, state)
template <int J>
__device__ __forceinline__ void aff_apply_w(AffWarpSmem<J>& s, int nr, int lane) {
    for (int e = lane; e < nr * J; e += 32) {
        const int r = e / J, a = e - r * J;
        double v = s.eb[r * J + a];
#pragma unroll
        for (int q = 0; q < J; ++q) v = fma(s.eP[a * J + q], s.b[r * J + q], v);
        s.rb[e] = v;
    }
    __syncwarp();
    for (int e = lane; e < nr * J; e += 32) s.b[e] = s.rb[e];
    __syncwarp();
}

template <int NB>
__global__ void __launch_bounds__(32)
k_aff_combine_warp(const double* __restrict__ Ein, const int64_t* __restrict__ cb,
                   const int64_t* __restrict__ ce, int64_t n_out, double* __restrict__ Eout,
                   int nr) {
    constexpr int J = 2 * NB, ES = J * J + NRMAX * J;
    __shared__ AffWarpSmem<J> s;
    const int64_t q = blockIdx.x;
    const int lane = threadIdx.x;
    if (q >= n_out) return;
    aff_load<J>(s.P, s.b, Ein + cb[q] * ES, lane);
    for (int64_t r = cb[q] + 1; r < ce[q]; ++r) {
        aff_load<J>(s.eP, s.eb, Ein + r * ES, lane);
        aff_combine_w<J>(s, nr, lane);
    }
    double* out = Eout + q * ES;
    for (int e = lane; e < J * J; e += 32) out[e] = s.P[e];
    for (int e = lane; e < NRMAX * J; e += 32) out[J * J + e] = e < nr * J ? s.b[e] : 0.0;
}

template <int NB>
__global__ void __launch_bounds__(32)
k_aff_down_warp(const double* __restrict__ E, const int64_t* __restrict__ cb,
                const int64_t* __restrict__ ce, int64_t n_parent,
                const double* __restrict__ Sparent, double* __restrict__ S, int nr) {
    constexpr int J = 2 * NB, ES = J * J + NRMAX * J, SS = NRMAX * J;
    __shared__ AffWarpSmem<J> s;
    const int64_t q = blockIdx.x;
    const int lane = threadIdx.x;
    if (q >= n_parent) return;
    for (int e = lane; e < SS; e += 32) s.b[e] = Sparent[q * SS + e];
    __syncwarp();
    for (int64_t r = cb[q]; r < ce[q]; ++r) {
        for (int e = lane; e < SS; e += 32) S[r * SS + e] = s.b[e];
        aff_load<J>(s.eP, s.eb, E + r * ES, lane);
        aff_apply_w<J>(s, nr, lane);
    }
}

template <int NB>
__global__ void __launch_bounds__(32)
k_aff_top_warp(const double* __restrict__ E, const int64_t* __restrict__ tb,
               const int64_t* __restrict__ te, int n_seg, double* __restrict__ S, int nr) {
    constexpr int J = 2 * NB, ES = J * J + NRMAX * J, SS = NRMAX * J;
    __shared__ AffWarpSmem<J> s;
    const int g = blockIdx.x;
    const int lane = threadIdx.x;
    if (g >= n_seg) return;
    for (int e = lane; e < SS; e += 32) s.b[e] = 0.0;
    __syncwarp();
    for (int64_t i = tb[g]; i < te[g]; ++i) {
        for (int e = lane; e < SS; e += 32) S[i * SS + e] = s.b[e];
        aff_load<J>(s.eP, s.eb, E + i * ES, lane);
        aff_apply_w<J>(s, nr, lane);
    }
}

template <int J>
struct FutWarpSmem {
    double Psi[J * J], Gam[J * J];        // accumulated element; the state G in Gam
    double ePsi[J * J], eGam[J * J];
    double T[J * J], R1[J * J], R2[J * J];
};

template <int J>
__device__ __forceinline__ void fut_load(double* Psi, double* Gam, const double* src, int lane) {
    for (int e = lane; e < J * J; e += 32) {
        Psi[e] = src[e];
        Gam[e] = src[J * J + e];
    }
    __syncwarp();
}

template <int NB>
__global__ void __launch_bounds__(32)
k_fut_combine_warp(const double* __restrict__ Ein, const int64_t* __restrict__ cb,
                   const int64_t* __restrict__ ce, int64_t n_out, double* __restrict__ Eout) {
    constexpr int J = 2 * NB, ES = 2 * J * J;
    __shared__ FutWarpSmem<J> s;
    const int64_t q = blockIdx.x;
    const int lane = threadIdx.x;
    if (q >= n_out) return;
    fut_load<J>(s.Psi, s.Gam, Ein + cb[q] * ES, lane);
    for (int64_t r = cb[q] + 1; r < ce[q]; ++r) {
        fut_load<J>(s.ePsi, s.eGam, Ein + r * ES, lane);
        wmat_prod<J, 0>(s.Psi, s.ePsi, s.R1, lane);          // Psi_i Psi_j
        wmat_prod<J, 0>(s.Gam, s.ePsi, s.T, lane);           // Gam_i Psi_j
        wmat_prod<J, 1>(s.ePsi, s.T, s.R2, lane);            // Psi_j^T ...
        wmat_add_sym<J>(s.R2, s.eGam, lane);
        wcopy<J>(s.Psi, s.R1, J * J, lane);
        wcopy<J>(s.Gam, s.R2, J * J, lane);
    }
    double* out = Eout + q * ES;
    for (int e = lane; e < J * J; e += 32) {
        out[e] = s.Psi[e];
        out[J * J + e] = s.Gam[e];
    }
}

template <int J>
__device__ __forceinline__ void fut_apply_w(FutWarpSmem<J>& s, int lane) {
    wmat_prod<J, 0>(s.Gam, s.ePsi, s.T, lane);               // G Psi
    wmat_prod<J, 1>(s.ePsi, s.T, s.R1, lane);                // Psi^T ...
    wmat_add_sym<J>(s.R1, s.eGam, lane);
    wcopy<J>(s.Gam, s.R1, J * J, lane);
}

template <int NB>
__global__ void __launch_bounds__(32)
k_fut_down_warp(const double* __restrict__ E, const int64_t* __restrict__ cb,
                const int64_t* __restrict__ ce, int64_t n_parent,
                const double* __restrict__ Sparent, double* __restrict__ S) {
    constexpr int J = 2 * NB, ES = 2 * J * J;
    __shared__ FutWarpSmem<J> s;
    const int64_t q = blockIdx.x;
    const int lane = threadIdx.x;
    if (q >= n_parent) return;
    wcopy<J>(s.Gam, Sparent + q * J * J, J * J, lane);
    for (int64_t r = cb[q]; r < ce[q]; ++r) {
        for (int e = lane; e < J * J; e += 32) S[r * J * J + e] = s.Gam[e];
        fut_load<J>(s.ePsi, s.eGam, E + r * ES, lane);
        fut_apply_w<J>(s, lane);
    }
}

template <int NB>
__global__ void __launch_bounds__(32)
k_fut_top_warp(const double* __restrict__ E, const int64_t* __restrict__ tb,
               const int64_t* __restrict__ te, int n_seg, double* __restrict__ S) {
    constexpr int J = 2 * NB, ES = 2 * J * J;
    __shared__ FutWarpSmem<J> s;
    const int g = blockIdx.x;
    const int lane = threadIdx.x;
    if (g >= n_seg) return;
    for (int e = lane; e < J * J; e += 32) s.Gam[e] = 0.0;
    __syncwarp();
    for (int64_t i = tb[g]; i < te[g]; ++i) {
        for (int e = lane; e < J * J; e += 32) S[i * J * J + e] = s.Gam[e];
        fut_load<J>(s.ePsi, s.eGam, E + i * ES, lane);
        fut_apply_w<J>(s, lane);
    }
}

// Narrow levels of these scans run one warp per group (as the Riccati tree).
#define NU_WARP_TREE_OVERLOADS(OP, COMBINE, DOWN, TOP, ...)                               \
    template <int NB>                                                                      \
    inline void scan_combine(const OP<NB>& op, const typename OP<NB>::Elem* Ein,           \
                             const int64_t* cb, const int64_t* ce, int64_t n,              \
                             typename OP<NB>::Elem* Eout, cudaStream_t st) {               \
        if (n <= RIC_WARP_TREE_MAX)                                                        \
            COMBINE<NB><<<(unsigned)n, 32, 0, st>>>((const double*)Ein, cb, ce, n,          \
                                                     (double*)Eout __VA_ARGS__);                 \
        else                                                                               \
            scan_combine_threads(op, Ein, cb, ce, n, Eout, st);                            \
    }                                                                                      \
    template <int NB>                                                                      \
    inline void scan_down(const OP<NB>& op, const typename OP<NB>::Elem* E,                \
                          const int64_t* cb, const int64_t* ce, int64_t n,                 \
                          const typename OP<NB>::State* Sp, typename OP<NB>::State* S,     \
                          cudaStream_t st) {                                               \
        if (n <= RIC_WARP_TREE_MAX)                                                        \
            DOWN<NB><<<(unsigned)n, 32, 0, st>>>((const double*)E, cb, ce, n,               \
                                                  (const double*)Sp, (double*)S __VA_ARGS__);    \
        else                                                                               \
            scan_down_threads(op, E, cb, ce, n, Sp, S, st);                                \
    }                                                                                      \
    template <int NB>                                                                      \
    inline void scan_top(const OP<NB>& op, const typename OP<NB>::Elem* E,                 \
                         const int64_t* tb, const int64_t* te, int n_seg,                  \
                         typename OP<NB>::State* S, cudaStream_t st) {                     \
        if (n_seg <= RIC_WARP_TREE_MAX)                                                    \
            TOP<NB><<<(unsigned)n_seg, 32, 0, st>>>((const double*)E, tb, te, n_seg,        \
                                                     (double*)S __VA_ARGS__);                    \
        else                                                                               \
            scan_top_threads(op, E, tb, te, n_seg, S, st);                                 \
    }

NU_WARP_TREE_OVERLOADS(ForwardOp, k_aff_combine_warp, k_aff_down_warp, k_aff_top_warp,
                       , op.k + 1)
NU_WARP_TREE_OVERLOADS(BackwardOp, k_aff_combine_warp, k_aff_down_warp, k_aff_top_warp,
                       , op.nr)
NU_WARP_TREE_OVERLOADS(FutureOp, k_fut_combine_warp, k_fut_down_warp, k_fut_top_warp, )
#undef NU_WARP_TREE_OVERLOADS

}  // namespace nu

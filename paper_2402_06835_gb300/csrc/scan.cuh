// Multi-level chunked scan for the sequential recursions of the factor.
//
// A recursion x_{n+1} = f_n(x_n) over n samples is cut into chunks of B
// samples.  An Op supplies, for one chunk c, an element E_c that represents
// the chunk's composite map (elem), the composition of two neighbouring
// elements (combine, earlier one first in scan order), the application of an
// element to an incoming state (apply), and the exact re-run of the chunk
// from its incoming state that writes the per-sample results (final).
//
//   level 0: one thread per chunk builds E_c            (k_scan_elem)
//   level l: one thread per group of G elements composes them (k_scan_combine)
//   top:     one thread applies the top elements in order and records the
//            state entering each (k_scan_top)
//   down:    one thread per group re-applies its G children from the group's
//            incoming state (k_scan_down), level by level back to level 0
//   final:   one thread per chunk re-runs its samples (k_scan_final)
//
// The sequential depth is B + (levels) * G + (top count) element operations
// instead of n recursion steps.  Each Op is a plain struct with device member
// functions; Elem and State are plain structs.
#pragma once

#include "nu_internal.cuh"

namespace nu {

template <class Op>
__global__ void k_scan_elem(Op op, int64_t n_chunks, typename Op::Elem* __restrict__ E) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= n_chunks) return;
    op.elem(c, E[c]);
}

template <class Op>
__global__ void k_scan_combine(Op op, const typename Op::Elem* __restrict__ Ein, int64_t n_in,
                               int G, typename Op::Elem* __restrict__ Eout) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t q0 = g * G;
    if (q0 >= n_in) return;
    typename Op::Elem acc = Ein[q0];
    const int64_t q1 = q0 + G < n_in ? q0 + G : n_in;
    for (int64_t q = q0 + 1; q < q1; ++q) op.combine(acc, Ein[q]);
    Eout[g] = acc;
}

template <class Op>
__global__ void k_scan_top(Op op, const typename Op::Elem* __restrict__ E, int64_t n,
                           typename Op::State* __restrict__ S) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    typename Op::State s;
    op.init_state(s);
    for (int64_t i = 0; i < n; ++i) {
        S[i] = s;
        op.apply(E[i], s);
    }
}

template <class Op>
__global__ void k_scan_down(Op op, const typename Op::Elem* __restrict__ E, int64_t n, int G,
                            const typename Op::State* __restrict__ Sparent,
                            typename Op::State* __restrict__ S) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t q0 = g * G;
    if (q0 >= n) return;
    typename Op::State s = Sparent[g];
    const int64_t q1 = q0 + G < n ? q0 + G : n;
    for (int64_t q = q0; q < q1; ++q) {
        S[q] = s;
        op.apply(E[q], s);
    }
}

template <class Op>
__global__ void k_scan_final(Op op, int64_t n_chunks, const typename Op::State* __restrict__ S) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= n_chunks) return;
    op.final(c, S[c]);
}

// Workspace layout of one scan (byte sizes, 256-aligned).
struct ScanPlan {
    int64_t n_chunks;
    int G;
    int levels;              // number of combine levels
    int64_t count[16];       // elements per level (level 0 = chunks)
    size_t elem_off[16];
    size_t state_off[16];
    size_t bytes;
};

template <class Op>
inline ScanPlan plan_scan(int64_t n_chunks, int G, int top) {
    ScanPlan p{};
    p.n_chunks = n_chunks;
    p.G = G;
    p.count[0] = n_chunks;
    int l = 0;
    while (p.count[l] > top && l < 14) {
        p.count[l + 1] = (p.count[l] + G - 1) / G;
        ++l;
    }
    p.levels = l;
    size_t off = 0;
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    for (int i = 0; i <= l; ++i) {
        p.elem_off[i] = off;
        off += al((size_t)p.count[i] * sizeof(typename Op::Elem));
        p.state_off[i] = off;
        off += al((size_t)p.count[i] * sizeof(typename Op::State));
    }
    p.bytes = off;
    return p;
}

// Enqueue the whole scan on `st`; returns the number of kernel launches.
template <class Op>
inline int run_scan(const Op& op, const ScanPlan& p, char* ws, cudaStream_t st) {
    using E = typename Op::Elem;
    using S = typename Op::State;
    const int TH = 64;
    int launches = 0;
    k_scan_elem<Op><<<div_up(p.n_chunks, TH), TH, 0, st>>>(op, p.n_chunks, (E*)(ws + p.elem_off[0]));
    ++launches;
    for (int l = 0; l < p.levels; ++l) {
        k_scan_combine<Op><<<div_up(p.count[l + 1], TH), TH, 0, st>>>(
            op, (const E*)(ws + p.elem_off[l]), p.count[l], p.G, (E*)(ws + p.elem_off[l + 1]));
        ++launches;
    }
    k_scan_top<Op><<<1, 32, 0, st>>>(op, (const E*)(ws + p.elem_off[p.levels]),
                                     p.count[p.levels], (S*)(ws + p.state_off[p.levels]));
    ++launches;
    for (int l = p.levels - 1; l >= 0; --l) {
        k_scan_down<Op><<<div_up(p.count[l + 1], TH), TH, 0, st>>>(
            op, (const E*)(ws + p.elem_off[l]), p.count[l], p.G,
            (const S*)(ws + p.state_off[l + 1]), (S*)(ws + p.state_off[l]));
        ++launches;
    }
    k_scan_final<Op><<<div_up(p.n_chunks, TH), TH, 0, st>>>(op, p.n_chunks,
                                                          (const S*)(ws + p.state_off[0]));
    ++launches;
    return launches;
}

// ------------------------------------------------------ small dense algebra
template <int J>
struct Mat {
    double a[J * J];
    __device__ __forceinline__ double& operator()(int r, int c) { return a[r * J + c]; }
    __device__ __forceinline__ double operator()(int r, int c) const { return a[r * J + c]; }
};

template <int J>
__device__ __forceinline__ void mat_eye(Mat<J>& m) {
#pragma unroll
    for (int r = 0; r < J; ++r)
#pragma unroll
        for (int c = 0; c < J; ++c) m(r, c) = r == c ? 1.0 : 0.0;
}

template <int J>
__device__ __forceinline__ void mat_zero(Mat<J>& m) {
#pragma unroll
    for (int i = 0; i < J * J; ++i) m.a[i] = 0.0;
}

// C = A B
template <int J>
__device__ __forceinline__ void mat_mul(const Mat<J>& A, const Mat<J>& B, Mat<J>& C) {
#pragma unroll
    for (int r = 0; r < J; ++r)
#pragma unroll
        for (int c = 0; c < J; ++c) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < J; ++k) s = fma(A(r, k), B(k, c), s);
            C(r, c) = s;
        }
}

// C = A^T B
template <int J>
__device__ __forceinline__ void mat_tmul(const Mat<J>& A, const Mat<J>& B, Mat<J>& C) {
#pragma unroll
    for (int r = 0; r < J; ++r)
#pragma unroll
        for (int c = 0; c < J; ++c) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < J; ++k) s = fma(A(k, r), B(k, c), s);
            C(r, c) = s;
        }
}

// C = A B^T
template <int J>
__device__ __forceinline__ void mat_mult(const Mat<J>& A, const Mat<J>& B, Mat<J>& C) {
#pragma unroll
    for (int r = 0; r < J; ++r)
#pragma unroll
        for (int c = 0; c < J; ++c) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < J; ++k) s = fma(A(r, k), B(c, k), s);
            C(r, c) = s;
        }
}

template <int J>
__device__ __forceinline__ void mat_symmetrize(Mat<J>& m) {
#pragma unroll
    for (int r = 0; r < J; ++r)
#pragma unroll
        for (int c = r + 1; c < J; ++c) {
            const double s = 0.5 * (m(r, c) + m(c, r));
            m(r, c) = s;
            m(c, r) = s;
        }
}

// X = M^-1 [B1 B2] (Gauss-Jordan with partial pivoting, static indexing);
// M is overwritten, B1 and B2 receive the solutions.
template <int J, int NRHS>
__device__ __forceinline__ void mat_solve(Mat<J>& M, Mat<J>* B[NRHS]) {
#pragma unroll
    for (int c = 0; c < J; ++c) {
        int piv = c;
        double best = fabs(M(c, c));
#pragma unroll
        for (int r = c + 1; r < J; ++r) {
            const double v = fabs(M(r, c));
            if (v > best) {
                best = v;
                piv = r;
            }
        }
#pragma unroll
        for (int r = c + 1; r < J; ++r) {
            if (r == piv) {
#pragma unroll
                for (int k = 0; k < J; ++k) {
                    double t = M(c, k); M(c, k) = M(r, k); M(r, k) = t;
#pragma unroll
                    for (int q = 0; q < NRHS; ++q) {
                        t = (*B[q])(c, k); (*B[q])(c, k) = (*B[q])(r, k); (*B[q])(r, k) = t;
                    }
                }
            }
        }
        const double inv = 1.0 / M(c, c);
#pragma unroll
        for (int k = 0; k < J; ++k) {
            M(c, k) *= inv;
#pragma unroll
            for (int q = 0; q < NRHS; ++q) (*B[q])(c, k) *= inv;
        }
#pragma unroll
        for (int r = 0; r < J; ++r) {
            if (r == c) continue;
            const double f = M(r, c);
#pragma unroll
            for (int k = 0; k < J; ++k) {
                M(r, k) = fma(-f, M(c, k), M(r, k));
#pragma unroll
                for (int q = 0; q < NRHS; ++q) (*B[q])(r, k) = fma(-f, (*B[q])(c, k), (*B[q])(r, k));
            }
        }
    }
}

}  // namespace nu

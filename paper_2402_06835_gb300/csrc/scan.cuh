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

#include <algorithm>
#include <vector>

#include "nu_internal.cuh"

namespace nu {

// Segments: several independent recursions (light curves) share one scan.
// Level-0 elements are the chunks of all segments, segment after segment;
// level l+1 element q composes the level-l elements [child_begin, child_end)
// of the same segment; the top level holds, per segment, the elements
// [top_begin, top_end).  A single light curve is one segment.
// Work item of a thread when each warp uses only its first L lanes: the
// scan's work per item is a sequential FP64 recursion, and this GPU issues
// one FP64 warp instruction per 64 cycles per sub-partition however many
// lanes are active, so a scan with few items spreads them over many warps
// (L = 1 puts one item on each sub-partition) and a large one packs them.
__device__ __forceinline__ int64_t spread_item(int L) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int lane = (int)(t & 31);
    return lane < L ? (t >> 5) * L + lane : -1;
}

template <class Op>
__global__ void k_scan_elem(Op op, int64_t n_chunks, typename Op::Elem* __restrict__ E,
                            int L) {
    const int64_t c = spread_item(L);
    if (c < 0 || c >= n_chunks) return;
    op.elem(c, E[c]);
}

template <class Op>
__global__ void k_scan_combine(Op op, const typename Op::Elem* __restrict__ Ein,
                               const int64_t* __restrict__ cb, const int64_t* __restrict__ ce,
                               int64_t n_out, typename Op::Elem* __restrict__ Eout,
                               int L) {
    const int64_t q = spread_item(L);
    if (q < 0 || q >= n_out) return;
    typename Op::Elem acc = Ein[cb[q]];
    for (int64_t r = cb[q] + 1; r < ce[q]; ++r) op.combine(acc, Ein[r]);
    Eout[q] = acc;
}

template <class Op>
__global__ void k_scan_top(Op op, const typename Op::Elem* __restrict__ E,
                           const int64_t* __restrict__ tb, const int64_t* __restrict__ te,
                           int n_seg, typename Op::State* __restrict__ S) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_seg) return;
    typename Op::State s;
    op.init_state(s);
    for (int64_t i = tb[g]; i < te[g]; ++i) {
        S[i] = s;
        op.apply(E[i], s);
    }
}

template <class Op>
__global__ void k_scan_down(Op op, const typename Op::Elem* __restrict__ E,
                            const int64_t* __restrict__ cb, const int64_t* __restrict__ ce,
                            int64_t n_parent, const typename Op::State* __restrict__ Sparent,
                            typename Op::State* __restrict__ S, int L) {
    const int64_t q = spread_item(L);
    if (q < 0 || q >= n_parent) return;
    typename Op::State s = Sparent[q];
    for (int64_t r = cb[q]; r < ce[q]; ++r) {
        S[r] = s;
        op.apply(E[r], s);
    }
}

template <class Op>
__global__ void k_scan_final(Op op, int64_t n_chunks, const typename Op::State* __restrict__ S,
                             int L) {
    const int64_t c = spread_item(L);
    if (c < 0 || c >= n_chunks) return;
    op.final(c, S[c]);
}

// Host-side construction of the level structure for segments with nc[l]
// chunks each.  idx receives the int64 index arrays (child ranges per level,
// then top ranges); the caller uploads them and fills the pointers.
struct ScanShape {
    int levels;
    int n_seg;
    int64_t count[16];
    size_t child_off[16];      // offset (in int64 entries) of child_begin of level l
    size_t top_off;            // offset of top_begin; top_end follows
    size_t n_index;            // total int64 entries
};

inline ScanShape build_scan_shape(const int64_t* nc, int n_seg, int G, int top,
                                  int64_t* idx /* null: only size the arrays */) {
    ScanShape sh{};
    sh.n_seg = n_seg;
    std::vector<int64_t> cnt(nc, nc + n_seg);       // per-segment count, current level
    int64_t total = 0, cur_max = 0;
    for (int g = 0; g < n_seg; ++g) {
        total += cnt[g];
        cur_max = std::max(cur_max, cnt[g]);
    }
    sh.count[0] = total;
    size_t pos = 0;
    int levels = 0;
    while (cur_max > top && levels < 14) {
        const int l = ++levels;
        int64_t out_total = 0;
        for (int g = 0; g < n_seg; ++g) out_total += (cnt[g] + G - 1) / G;
        sh.child_off[l] = pos;
        sh.count[l] = out_total;
        int64_t q_out = 0, in_off = 0;
        for (int g = 0; g < n_seg; ++g) {
            const int64_t nout = (cnt[g] + G - 1) / G;
            for (int64_t q = 0; q < nout; ++q, ++q_out) {
                if (idx) {
                    idx[pos + q_out] = in_off + q * G;                           // begin
                    idx[pos + out_total + q_out] = in_off + std::min((q + 1) * G, cnt[g]);
                }
            }
            in_off += cnt[g];
            cnt[g] = nout;
        }
        pos += 2 * (size_t)out_total;
        cur_max = 0;
        for (int g = 0; g < n_seg; ++g) cur_max = std::max(cur_max, cnt[g]);
    }
    sh.levels = levels;
    sh.top_off = pos;
    int64_t off = 0;
    for (int g = 0; g < n_seg; ++g) {
        if (idx) {
            idx[pos + g] = off;
            idx[pos + n_seg + g] = off + cnt[g];
        }
        off += cnt[g];
    }
    sh.n_index = pos + 2 * (size_t)n_seg;
    return sh;
}

// Device workspace of one scan: elements and states of every level.
template <class Op>
inline size_t scan_bytes(const ScanShape& sh) {
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    size_t off = 0;
    for (int l = 0; l <= sh.levels; ++l) {
        off += al((size_t)sh.count[l] * sizeof(typename Op::Elem));
        off += al((size_t)sh.count[l] * sizeof(typename Op::State));
    }
    return off;
}

// Lanes per warp for n thread-level work items: at most one warp per
// sub-partition (608 on 152 SMs) -- more warps would share a sub-partition's
// FP64 pipe -- with as few lanes per warp as that allows.
inline int scan_lanes(int64_t n) {
    int L = 1;
    while (L < 32 && n > (int64_t)L * 608) L *= 2;
    return L;
}
inline int scan_grid(int64_t n, int L, int th) { return div_up(div_up(n, L) * 32, th); }

// Tree steps, one thread per group.  An Op may overload scan_combine /
// scan_down / scan_top for its own type (found by argument-dependent lookup
// when run_scan is instantiated) to run some levels another way.
template <class Op>
inline void scan_combine_threads(const Op& op, const typename Op::Elem* Ein,
                                 const int64_t* cb, const int64_t* ce, int64_t n,
                                 typename Op::Elem* Eout, cudaStream_t st) {
    const int L = scan_lanes(n);
    k_scan_combine<Op><<<scan_grid(n, L, 128), 128, 0, st>>>(op, Ein, cb, ce, n, Eout, L);
}
template <class Op>
inline void scan_down_threads(const Op& op, const typename Op::Elem* E, const int64_t* cb,
                              const int64_t* ce, int64_t n, const typename Op::State* Sp,
                              typename Op::State* S, cudaStream_t st) {
    const int L = scan_lanes(n);
    k_scan_down<Op><<<scan_grid(n, L, 128), 128, 0, st>>>(op, E, cb, ce, n, Sp, S, L);
}
template <class Op>
inline void scan_top_threads(const Op& op, const typename Op::Elem* E, const int64_t* tb,
                             const int64_t* te, int n_seg, typename Op::State* S,
                             cudaStream_t st) {
    k_scan_top<Op><<<div_up(n_seg, 32), 32, 0, st>>>(op, E, tb, te, n_seg, S);
}
template <class Op>
inline void scan_combine(const Op& op, const typename Op::Elem* Ein, const int64_t* cb,
                         const int64_t* ce, int64_t n, typename Op::Elem* Eout,
                         cudaStream_t st) {
    scan_combine_threads(op, Ein, cb, ce, n, Eout, st);
}
template <class Op>
inline void scan_down(const Op& op, const typename Op::Elem* E, const int64_t* cb,
                      const int64_t* ce, int64_t n, const typename Op::State* Sp,
                      typename Op::State* S, cudaStream_t st) {
    scan_down_threads(op, E, cb, ce, n, Sp, S, st);
}
template <class Op>
inline void scan_top(const Op& op, const typename Op::Elem* E, const int64_t* tb,
                     const int64_t* te, int n_seg, typename Op::State* S, cudaStream_t st) {
    scan_top_threads(op, E, tb, te, n_seg, S, st);
}

// Enqueue the whole scan on `st`; idx_dev holds the uploaded index arrays.
// Returns the number of kernel launches.
template <class Op>
inline int run_scan(const Op& op, const ScanShape& sh, const int64_t* idx_dev, char* ws,
                    cudaStream_t st) {
    using E = typename Op::Elem;
    using S = typename Op::State;
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    E* Ep[16];
    S* Sp[16];
    size_t off = 0;
    for (int l = 0; l <= sh.levels; ++l) {
        Ep[l] = (E*)(ws + off);
        off += al((size_t)sh.count[l] * sizeof(E));
        Sp[l] = (S*)(ws + off);
        off += al((size_t)sh.count[l] * sizeof(S));
    }
    const int TH = 128;
    int launches = 0;
    {
        const int L = scan_lanes(sh.count[0]);
        k_scan_elem<Op><<<scan_grid(sh.count[0], L, TH), TH, 0, st>>>(op, sh.count[0], Ep[0],
                                                                    L);
        ++launches;
    }
    for (int l = 1; l <= sh.levels; ++l) {
        const int64_t* cb = idx_dev + sh.child_off[l];
        const int64_t* ce = cb + sh.count[l];
        scan_combine(op, Ep[l - 1], cb, ce, sh.count[l], Ep[l], st);
        ++launches;
    }
    const int64_t* tb = idx_dev + sh.top_off;
    scan_top(op, Ep[sh.levels], tb, tb + sh.n_seg, sh.n_seg, Sp[sh.levels], st);
    ++launches;
    for (int l = sh.levels; l >= 1; --l) {
        const int64_t* cb = idx_dev + sh.child_off[l];
        const int64_t* ce = cb + sh.count[l];
        scan_down(op, Ep[l - 1], cb, ce, sh.count[l], Sp[l], Sp[l - 1], st);
        ++launches;
    }
    {
        const int L = scan_lanes(sh.count[0]);
        k_scan_final<Op><<<scan_grid(sh.count[0], L, TH), TH, 0, st>>>(op, sh.count[0], Sp[0],
                                                                     L);
        ++launches;
    }
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

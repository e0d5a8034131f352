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
#include <vector>

#include "factor_core.cuh"
#include "factor_ops.cuh"
#include "nu_internal.cuh"
#include "ss.cuh"

namespace nu {

enum { ST_OK = 0, ST_EINVAL = 1, ST_ENOTPD = 2 };

__device__ inline void flag_bad(long long* ds, int code, long long idx) {
    // keep the smallest failing local index; the code that claims it wins
    const unsigned long long old = atomicMin((unsigned long long*)&ds[1], (unsigned long long)idx);
    if ((long long)old > idx) atomicExch((unsigned long long*)&ds[0], (unsigned long long)code);
}

// segment of packed sample i: s_off[g] <= i < s_off[g + 1]
__device__ __forceinline__ int seg_of(const int64_t* __restrict__ s_off, int n_seg, int64_t i) {
    int lo = 0, hi = n_seg;                  // find the last g with s_off[g] <= i
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s_off[mid] <= i) lo = mid; else hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------- transitions
template <int NB>
__global__ void k_transitions(const double* __restrict__ t, int64_t n,
                              const int64_t* __restrict__ s_off, int n_seg,
                              const Blocks* __restrict__ blocks, double* __restrict__ F,
                              long long* dstat) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int g = seg_of(s_off, n_seg, i);
    const int64_t loc = i - s_off[g];
    double* Fi = F + i * NB * 4;
    if (!isfinite(t[i])) flag_bad(dstat + 2 * g, ST_EINVAL, loc);
    if (loc == 0) {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            Fi[4 * b] = 1.0; Fi[4 * b + 1] = 0.0; Fi[4 * b + 2] = 0.0; Fi[4 * b + 3] = 1.0;
        }
        return;
    }
    const double tau = t[i] - t[i - 1];
    if (!(tau > 0.0)) flag_bad(dstat + 2 * g, ST_EINVAL, loc);
    const Blocks bl = blocks[g];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        double f[4];
        block_transition(bl.b[b], tau, f);
        Fi[4 * b] = f[0]; Fi[4 * b + 1] = f[1]; Fi[4 * b + 2] = f[2]; Fi[4 * b + 3] = f[3];
    }
}

// ------------------------------------------------- cross products per segment
// cross[g][a][b] = sum over the segment's chunks of partial[c][a][b]
__global__ void k_reduce_cross(const double* __restrict__ partial, const SegInfo* __restrict__ segs,
                               int nr, double* __restrict__ cross) {
    __shared__ double sh[128];
    const int g = blockIdx.x / (nr * nr);
    const int ab = blockIdx.x % (nr * nr);
    const int a = ab / nr, b = ab % nr;
    const SegInfo sg = segs[g];
    double s = 0.0;
    for (int64_t c = threadIdx.x; c < sg.n_c; c += blockDim.x)
        s += partial[(sg.c_off + c) * NRMAX * NRMAX + a * NRMAX + b];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) cross[(int64_t)g * NRMAX * NRMAX + a * nr + b] = sh[0];
}

// ------------------------------------------------------------------ null GLS
// One thread per segment: A = X^T Sigma^-1 X = R^T R, w = A^-1 X^T Sigma^-1 y,
// Rinv = R^-1.  wR[g]: [0..k) w, [k .. k+k*k) Rinv row-major.
__global__ void k_null_gls(int k, int n_seg, const double* __restrict__ cross_all,
                           double* __restrict__ wR_all, long long* dstat) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_seg) return;
    long long* ds = dstat + 2 * g;
    if (ds[0] != 0) return;       // the factor of this segment already failed
    const double* cross = cross_all + (int64_t)g * NRMAX * NRMAX;
    double* wR = wR_all + (int64_t)g * 32;
    const int nr = k + 1;
    double R[NU_MAX_K][NU_MAX_K] = {};
    for (int i = 0; i < k; ++i) {
        for (int j = i; j < k; ++j) {
            double s = cross[i * nr + j];
            for (int p = 0; p < i; ++p) s -= R[p][i] * R[p][j];
            if (i == j) {
                if (!(s > 0.0)) {          // X rank deficient under Sigma
                    flag_bad(ds, ST_EINVAL, 0);
                    return;
                }
                R[i][i] = sqrt(s);
            } else {
                R[i][j] = s / R[i][i];
            }
        }
    }
    double Ri[NU_MAX_K][NU_MAX_K] = {};
    for (int j = 0; j < k; ++j) {
        Ri[j][j] = 1.0 / R[j][j];
        for (int i = j - 1; i >= 0; --i) {
            double s = 0.0;
            for (int p = i + 1; p <= j; ++p) s += R[i][p] * Ri[p][j];
            Ri[i][j] = -s / R[i][i];
        }
    }
    double z[NU_MAX_K];
    for (int i = 0; i < k; ++i) {          // R^T z = u, u_a = X_a^T Sigma^-1 y
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
// square, ln D, and the backward right-hand sides U[i][0] = e0 / D,
// U[i][1+a] = (sum_c e_c Rinv[c][a]) / D.
__global__ void k_rhs(int64_t n, int k, const int64_t* __restrict__ s_off, int n_seg,
                      const double* __restrict__ E, const double* __restrict__ invD,
                      const double* __restrict__ wR_all, const double* __restrict__ Dpiv,
                      double* __restrict__ U, double* __restrict__ chi_terms,
                      double* __restrict__ logD) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* wR = wR_all + (int64_t)seg_of(s_off, n_seg, i) * 32;
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

// ------------------------------------------------ per-segment scalars
// One block per segment: ln|Sigma| = sum ln D, chi2 of the null fit, and the
// null log-likelihood of Eq. linear_search_ll (deterministic tree sums).
__global__ void k_seg_scalars(const double* __restrict__ chi_terms,
                              const double* __restrict__ logD, const SegInfo* __restrict__ segs,
                              double* __restrict__ scal) {
    __shared__ double sc[256], sl[256];
    const SegInfo sg = segs[blockIdx.x];
    double a = 0.0, b = 0.0;
    for (int64_t i = threadIdx.x; i < sg.n; i += blockDim.x) {
        a += chi_terms[sg.s_off + i];
        b += logD[sg.s_off + i];
    }
    sc[threadIdx.x] = a;
    sl[threadIdx.x] = b;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sc[threadIdx.x] += sc[threadIdx.x + w];
            sl[threadIdx.x] += sl[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double* s = scal + 4 * blockIdx.x;
        s[0] = sl[0];
        s[2] = sc[0];
        s[1] = -0.5 * sc[0] - 0.5 * sl[0] - 0.5 * (double)sg.n * log(2.0 * M_PI);
    }
}

// ------------------------------------------------------------- FP32 copies
// Up to six arrays in one launch: element i of the concatenation.
struct F32Copies {
    const double* src[6];
    float* dst[6];
    int64_t end[6];          // running element counts
};
__global__ void k_to_f32(F32Copies c, int64_t total) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= total) return;
    int a = 0;
    while (i >= c.end[a]) ++a;
    const int64_t j = i - (a > 0 ? c.end[a - 1] : 0);
    c.dst[a][j] = (float)c.src[a][j];
}

// ------------------------------------------------------------------ plan
// workspace of the scans that run one after another on the main stream
template <int NB>
static size_t scan_workspace(const ScanShape& sh) {
    size_t m = scan_bytes<RiccatiOp<NB>>(sh);
    m = std::max(m, scan_bytes<ForwardOp<NB>>(sh));
    m = std::max(m, scan_bytes<BackwardOp<NB>>(sh));
    return m;
}

FactorPlan plan_factor(const int64_t* n_per_seg, const Blocks* blocks, int n_seg, int k) {
    FactorPlan p{};
    p.nb = blocks[0].nb;
    p.k = k;
    p.n_seg = n_seg;
    std::vector<int64_t> nc(n_seg);
    int64_t n_all = 0;
    for (int g = 0; g < n_seg; ++g) n_all += n_per_seg[g];
    p.B = scan_chunk_len(n_all);
    p.G = scan_group(p.B);
    p.s_off.assign(n_seg + 1, 0);
    p.segs.resize(n_seg);
    p.blocks.assign(blocks, blocks + n_seg);
    for (int g = 0; g < n_seg; ++g) {
        nc[g] = (n_per_seg[g] + p.B - 1) / p.B;
        SegInfo& sg = p.segs[g];
        sg.s_off = p.n_total;
        sg.n = n_per_seg[g];
        sg.c_off = p.n_chunks;
        sg.n_c = nc[g];
        for (int j = 0; j < 2 * NU_MAX_BLOCKS; ++j) sg.pinf[j] = 0.0;
        for (int b = 0; b < blocks[g].nb; ++b) {
            sg.pinf[2 * b] = blocks[g].b[b].sigma2;
            sg.pinf[2 * b + 1] = blocks[g].b[b].type == 0 ? blocks[g].b[b].sigma2 : 0.0;
        }
        p.n_total += n_per_seg[g];
        p.n_chunks += nc[g];
        p.s_off[g + 1] = p.n_total;
    }
    p.shape = build_scan_shape(nc.data(), n_seg, p.G, SCAN_TOP, nullptr);
    p.index.assign(p.shape.n_index, 0);
    build_scan_shape(nc.data(), n_seg, p.G, SCAN_TOP, p.index.data());
    p.chunk_seg.resize(p.n_chunks);
    int64_t c = 0;
    for (int g = 0; g < n_seg; ++g)
        for (int64_t q = 0; q < nc[g]; ++q) p.chunk_seg[c++] = g;
    size_t scan = 0, scan_fu = 0;
    switch (p.nb) {
        case 1: scan = scan_workspace<1>(p.shape); scan_fu = scan_bytes<FutureOp<1>>(p.shape); break;
        case 2: scan = scan_workspace<2>(p.shape); scan_fu = scan_bytes<FutureOp<2>>(p.shape); break;
        case 3: scan = scan_workspace<3>(p.shape); scan_fu = scan_bytes<FutureOp<3>>(p.shape); break;
        default: scan = scan_workspace<4>(p.shape); scan_fu = scan_bytes<FutureOp<4>>(p.shape); break;
    }
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const int nr = k + 1;
    size_t off = 0;
    p.off_scan = off;       off += al(scan);
    p.off_scan_fu = off;    off += al(scan_fu);
    p.off_partial = off;    off += al((size_t)p.n_chunks * NRMAX * NRMAX * 8);
    p.off_idx = off;        off += al(p.index.size() * 8);
    p.off_chunk_seg = off;  off += al(p.chunk_seg.size() * 4);
    p.off_segs = off;       off += al((size_t)n_seg * sizeof(SegInfo));
    p.off_blocks = off;     off += al((size_t)n_seg * sizeof(Blocks));
    p.off_s_off = off;      off += al((size_t)(n_seg + 1) * 8);
    p.off_cross = off;      off += al((size_t)n_seg * NRMAX * NRMAX * 8);
    p.off_wR = off;         off += al((size_t)n_seg * 32 * 8);
    p.off_Dpiv = off;       off += al((size_t)p.n_total * 8);
    p.off_U = off;          off += al((size_t)p.n_total * nr * 8);
    p.off_chi = off;        off += al((size_t)p.n_total * 8);
    p.off_logD = off;       off += al((size_t)p.n_total * 8);
    p.bytes = off;
    return p;
}

nu_status upload_factor_plan(const FactorPlan& p, char* ws, cudaStream_t st) {
    cudaError_t e = cudaMemcpyAsync(ws + p.off_idx, p.index.data(), p.index.size() * 8,
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ws + p.off_chunk_seg, p.chunk_seg.data(), p.chunk_seg.size() * 4,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ws + p.off_segs, p.segs.data(), p.segs.size() * sizeof(SegInfo),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ws + p.off_blocks, p.blocks.data(), p.blocks.size() * sizeof(Blocks),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ws + p.off_s_off, p.s_off.data(), p.s_off.size() * 8,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // host sources are temporaries
    if (e != cudaSuccess) return cuda_fail(e, "factor plan upload");
    return NU_OK;
}

template <int NB>
static int launch_factor_nb(const FactorPlan& p, const FactorBuffers& b, char* ws,
                            const double* dv, const double* X, int64_t ldx, const double* y,
                            cudaStream_t st, cudaStream_t side) {
    constexpr int J = Dims<NB>::J;
    constexpr int JJ = Dims<NB>::JJ;
    const int64_t n = p.n_total;
    const int k = p.k;
    const int nr = k + 1;
    const int nblk = div_up(n, 256);
    char* scan_ws = ws + p.off_scan;
    double* partial = (double*)(ws + p.off_partial);
    const int64_t* idx = (const int64_t*)(ws + p.off_idx);
    const int* chunk_seg = (const int*)(ws + p.off_chunk_seg);
    const SegInfo* segs = (const SegInfo*)(ws + p.off_segs);
    const Blocks* blocks = (const Blocks*)(ws + p.off_blocks);
    const int64_t* s_off = (const int64_t*)(ws + p.off_s_off);
    double* cross = (double*)(ws + p.off_cross);
    double* wR = (double*)(ws + p.off_wR);
    double* Dpiv = (double*)(ws + p.off_Dpiv);
    double* U = (double*)(ws + p.off_U);
    double* chi = (double*)(ws + p.off_chi);
    double* logD = (double*)(ws + p.off_logD);
    int launched = 0;
    k_transitions<NB><<<nblk, 256, 0, st>>>(b.t, n, s_off, p.n_seg, blocks, b.F, b.dstat);
    ++launched;
    // 1. pivots and gains
    RiccatiOp<NB> ric{segs, chunk_seg, b.F, dv, p.B, b.kg, b.invD, Dpiv, b.dstat};
    launched += run_scan(ric, p.shape, idx, scan_ws, st);
    // 4. future information: needs only the pivots and gains, so it runs on the
    //    side stream (when there is one) beside steps 2 and 3
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool forked = false;
    if (side && side != st &&
        cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming) == cudaSuccess &&
        cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming) == cudaSuccess &&
        cudaEventRecord(ev_fork, st) == cudaSuccess &&
        cudaStreamWaitEvent(side, ev_fork, 0) == cudaSuccess)
        forked = true;
    FutureOp<NB> fu{segs, chunk_seg, b.F, b.kg, b.invD, p.B, b.G};
    if (forked) {
        launched += run_scan(fu, p.shape, idx, ws + p.off_scan_fu, side);
        if (cudaEventRecord(ev_join, side) != cudaSuccess) forked = false;
    }
    // 2. forward solves of X and y, cross products
    ForwardOp<NB> fw{segs, chunk_seg, b.F, b.kg, b.invD, X, ldx, b.t, y, k, p.B, b.work,
                     partial};
    launched += run_scan(fw, p.shape, idx, scan_ws, st);
    k_reduce_cross<<<p.n_seg * nr * nr, 128, 0, st>>>(partial, segs, nr, cross);
    ++launched;
    // 3. null fit, right-hand sides, backward solves
    if (k > 0) {
        k_null_gls<<<div_up(p.n_seg, 64), 64, 0, st>>>(k, p.n_seg, cross, wR, b.dstat);
        ++launched;
    }
    k_rhs<<<nblk, 256, 0, st>>>(n, k, s_off, p.n_seg, b.work, b.invD, wR, Dpiv, U, chi, logD);
    ++launched;
    BackwardOp<NB> bw{segs, chunk_seg, b.F, b.kg, U, nr, k, p.B, b.z0, b.Zt};
    launched += run_scan(bw, p.shape, idx, scan_ws, st);
    if (forked) {
        cudaStreamWaitEvent(st, ev_join, 0);
    } else {
        launched += run_scan(fu, p.shape, idx, ws + p.off_scan_fu, st);
    }
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    k_seg_scalars<<<p.n_seg, 256, 0, st>>>(chi, logD, segs, b.scal);
    ++launched;
    if (b.F32) {
        const int64_t sizes[6] = {n * NB * 4, n * (int64_t)J, n, n * (int64_t)JJ, n,
                                  n * (int64_t)k};
        const double* src[6] = {b.F, b.kg, b.invD, b.G, b.z0, b.Zt};
        float* dst[6] = {b.F32, b.kg32, b.invD32, b.G32, b.z032, b.Zt32};
        F32Copies c;
        int64_t total = 0;
        for (int a = 0; a < 6; ++a) {
            c.src[a] = src[a];
            c.dst[a] = dst[a];
            total += sizes[a];
            c.end[a] = total;
        }
        k_to_f32<<<div_up(total, 256), 256, 0, st>>>(c, total);
        ++launched;
    }
    return launched;
}

nu_status launch_factor(const FactorPlan& p, const FactorBuffers& b, char* ws,
                        const double* dv, const double* X, int64_t ldx, const double* y,
                        cudaStream_t st, cudaStream_t side, int* launched) {
    int l = 0;
    switch (p.nb) {
        case 1: l = launch_factor_nb<1>(p, b, ws, dv, X, ldx, y, st, side); break;
        case 2: l = launch_factor_nb<2>(p, b, ws, dv, X, ldx, y, st, side); break;
        case 3: l = launch_factor_nb<3>(p, b, ws, dv, X, ldx, y, st, side); break;
        default: l = launch_factor_nb<4>(p, b, ws, dv, X, ldx, y, st, side); break;
    }
    if (launched) *launched += l;
    count_launches(l);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "factor launch");
    return NU_OK;
}

cudaStream_t thread_side_stream() {
    constexpr int MAXDEV = 64;
    thread_local cudaStream_t side[MAXDEV] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAXDEV) return nullptr;
    if (!side[dev] && cudaStreamCreateWithFlags(&side[dev], cudaStreamNonBlocking) != cudaSuccess)
        side[dev] = nullptr;
    return side[dev];
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
    const FactorPlan plan = plan_factor(&n, &bl, 1, k);
    // persistent arrays (8-byte words)
    const int64_t w_t = n, w_F = n * nb * 4, w_kg = n * J, w_iD = n, w_G = n * JJ,
                  w_z0 = n, w_Zt = n * k, w_work = n * (k + 1), w_scal = 8, w_stat = 2;
    const int64_t w_f32 = (w_F + w_kg + w_iD + w_G + w_z0 + w_Zt + 8) / 2 + 8;
    const int64_t words = w_t + w_F + w_kg + w_iD + w_G + w_z0 + w_Zt + w_work + w_scal +
                          w_stat + w_f32 + 64;
    nu_factor* f = new nu_factor();
    f->n = n;
    f->nb = nb;
    f->k = k;
    f->blocks = bl;
    f->stream = (cudaStream_t)stream;
    f->mem_bytes = (size_t)words * 8;
    cudaStream_t st = f->stream;
    pool_keep_memory();
    cudaError_t e = cudaMallocAsync(&f->mem, f->mem_bytes, st);
    if (e != cudaSuccess) {
        delete f;
        return cuda_fail(e, "nu_gp_factor: cudaMallocAsync");
    }
    char* ws = nullptr;
    e = cudaMallocAsync((void**)&ws, plan.bytes, st);
    if (e != cudaSuccess) {
        cudaFreeAsync(f->mem, st);
        delete f;
        return cuda_fail(e, "nu_gp_factor: workspace");
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
    float* q = (float*)p;
    f->F32 = q; q += w_F;
    f->kg32 = q; q += w_kg;
    f->invD32 = q; q += w_iD;
    f->G32 = q; q += w_G;
    f->z032 = q; q += w_z0;
    f->Zt32 = q; q += w_Zt;
    long long init[2] = {0, (long long)n};
    e = cudaMemsetAsync(f->mem, 0, f->mem_bytes, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(f->dstat, init, sizeof(init), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(f->t, t_dev, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) {
        cudaFreeAsync(ws, st);
        cudaFreeAsync(f->mem, st);
        delete f;
        return cuda_fail(e, "nu_gp_factor: copy");
    }
    s = upload_factor_plan(plan, ws, st);            // synchronises: init is a temporary
    if (s == NU_OK) {
        FactorBuffers b{f->t, f->F, f->kg, f->invD, f->G, f->z0, f->Zt, f->work, f->scal,
                        f->dstat, f->F32, f->kg32, f->invD32, f->G32, f->z032, f->Zt32};
        s = launch_factor(plan, b, ws, diag_var_dev, X_dev, n, y_dev, st,
                          thread_side_stream(), nullptr);
    }
    cudaFreeAsync(ws, st);
    if (s == NU_OK) {
        e = cudaEventCreateWithFlags(&f->ready, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            f->ready = nullptr;
            s = cuda_fail(e, "nu_gp_factor: event");
        }
    }
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
    if (f->ready) cudaEventDestroy(f->ready);
    delete f;
}

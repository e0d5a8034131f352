// nu_batch_search: a survey of light curves of uneven length in one graph.
//
// The curves are packed back to back.  Every stage treats them as segments
// of one problem: the factor scans run over the chunks of all curves (a
// chunk never crosses a curve), the linear search covers every curve's
// (D, t0) grid with t0 = its samples, and the fold is a persistent kernel
// that takes (curve, period) work items from a device counter, which
// balances curves of different spans.  Host work (validation, layout, a
// regularity test of each curve's cadence, uploads of the small tables)
// happens before capture; the kernels are captured into one CUDA graph and
// launched once.  The instantiated graph of a configuration is kept and, on
// later calls, updated in place with the new call's parameters
// (cudaGraphExecUpdate) instead of being instantiated again.  The launch
// shapes of the fold (threads per block, resident blocks per SM) and of the
// linear search's window-start kernel (window starts per block, staged chunk)
// are chosen by a small autotuner the first time a configuration is seen:
// the candidates are timed on a slice of the batch and the fastest are
// cached for the process.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "factor_core.cuh"
#include "fold.cuh"
#include "nu_internal.cuh"

namespace nu {

// n_out periods spread evenly over the grid (the autotuner's slice)
__global__ void k_sample_periods(const double* __restrict__ periods, int64_t n_P, int n_out,
                                 double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_out) return;
    out[i] = periods[(int64_t)((double)i * (double)n_P / (double)n_out)];
}

__global__ void k_init_dstat(long long* dstat, const int64_t* __restrict__ s_off, int n_seg) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_seg) return;
    dstat[2 * g] = 0;
    dstat[2 * g + 1] = s_off[g + 1] - s_off[g];
}

__global__ void k_gather_ends(const double* __restrict__ t, const int64_t* __restrict__ s_off,
                              int n_seg, double* __restrict__ ends) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_seg) return;
    ends[2 * g] = t[s_off[g]];
    ends[2 * g + 1] = t[s_off[g + 1] - 1];
}

struct TuneKey {
    int nb, k, prec, n_D;
    bool operator<(const TuneKey& o) const {
        return std::tie(nb, k, prec, n_D) < std::tie(o.nb, o.k, o.prec, o.n_D);
    }
};
struct TuneVal {
    int blocks_per_sm, threads;     // fold
    WindowShape win;                // linear search
};

std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;

// Instantiated graphs by configuration (device, state size, k, precision,
// grid sizes, batch shape and tuned launch shapes).  A call takes its entry
// out of the cache while it uses it, so two threads never launch one
// executable graph at once.
struct GraphKey {
    int dev, nb, k, prec, n_D, n_lc, bps, threads, tlo, ch;
    int64_t N, n_P;
    bool operator<(const GraphKey& o) const {
        return std::tie(dev, nb, k, prec, n_D, n_lc, bps, threads, tlo, ch, N, n_P) <
               std::tie(o.dev, o.nb, o.k, o.prec, o.n_D, o.n_lc, o.bps, o.threads, o.tlo, o.ch,
                        o.N, o.n_P);
    }
};
std::mutex g_graph_mu;
std::map<GraphKey, cudaGraphExec_t> g_graphs;
constexpr size_t GRAPH_CACHE_MAX = 8;

cudaGraphExec_t take_graph(const GraphKey& key) {
    std::lock_guard<std::mutex> lock(g_graph_mu);
    auto it = g_graphs.find(key);
    if (it == g_graphs.end()) return nullptr;
    cudaGraphExec_t e = it->second;
    g_graphs.erase(it);
    return e;
}
void put_graph(const GraphKey& key, cudaGraphExec_t exec) {
    std::lock_guard<std::mutex> lock(g_graph_mu);
    if (g_graphs.count(key) || g_graphs.size() >= GRAPH_CACHE_MAX) {
        cudaGraphExecDestroy(exec);
        return;
    }
    g_graphs[key] = exec;
}

}  // namespace nu

using namespace nu;

extern "C" nu_status nu_batch_search(int n_lc, const int64_t* offsets_host,
                                     const double* t_dev, const double* y_dev,
                                     const double* diag_var_dev, const nu_term* terms_host,
                                     const int* n_terms_host, int k, const double* Ds_host,
                                     int n_D, const double* periods_dev, int64_t n_P,
                                     double phase_step, nu_precision prec, void* stream,
                                     double* Q_dev, double* T0_dev, int32_t* D_idx_dev,
                                     double* depth_out_dev, double* sigma_out_dev,
                                     double* lnP_dev, int* status_host) {
    // ------------------------------------------------------------ checks
    if (n_lc < 1 || !offsets_host || !t_dev || !y_dev || !diag_var_dev || !terms_host ||
        !n_terms_host || !Ds_host || !periods_dev || !Q_dev || !T0_dev || !D_idx_dev ||
        !depth_out_dev || !sigma_out_dev || !lnP_dev || !status_host)
        return fail(NU_EINVAL, "nu_batch_search: null argument or n_lc < 1");
    if (k < 0 || k > 2) return fail(NU_EINVAL, "nu_batch_search: k must be 0, 1 or 2");
    if (n_D < 1 || n_P < 1) return fail(NU_EINVAL, "nu_batch_search: empty grid");
    if (!(phase_step >= 0.0) || !std::isfinite(phase_step))
        return fail(NU_EINVAL, "nu_batch_search: phase_step must be >= 0");
    if (prec != NU_FP64 && prec != NU_MIXED)
        return fail(NU_EINVAL, "nu_batch_search: unknown precision");
    if (offsets_host[0] != 0) return fail(NU_EINVAL, "nu_batch_search: offsets[0] must be 0");
    for (int g = 0; g < n_lc; ++g)
        if (offsets_host[g + 1] - offsets_host[g] < 2)
            return fail(NU_EINVAL, "nu_batch_search: curve %d has fewer than 2 samples", g);
    for (int j = 0; j < n_D; ++j)
        if (!(Ds_host[j] > 0.0) || !std::isfinite(Ds_host[j]))
            return fail(NU_EINVAL, "nu_batch_search: durations must be finite and > 0");
    std::vector<Blocks> blocks(n_lc);
    {
        int tb = 0;
        for (int g = 0; g < n_lc; ++g) {
            const nu_status s = expand_terms(terms_host + tb, n_terms_host[g], &blocks[g]);
            if (s != NU_OK) return s;
            tb += n_terms_host[g];
            if (blocks[g].nb != blocks[0].nb)
                return fail(NU_EINVAL, "nu_batch_search: every curve must have the same "
                                       "state dimension (curve %d differs)", g);
        }
    }
    const int nb = blocks[0].nb, J = 2 * nb, JJ = J * (J + 1) / 2;
    const bool fp64 = prec == NU_FP64;
    const double gap_factor = 1.5;
    const int64_t N = offsets_host[n_lc];
    std::vector<int64_t> n_per(n_lc);
    for (int g = 0; g < n_lc; ++g) n_per[g] = offsets_host[g + 1] - offsets_host[g];
    const FactorPlan plan = plan_factor(n_per.data(), blocks.data(), n_lc, k);
    cudaStream_t st = (cudaStream_t)stream;
    if (phase_step == 0.0) {
        // default phase step: the median sample spacing of the first curve
        // (a host copy of its times; this synchronises the stream)
        const int64_t n0 = offsets_host[1];
        std::vector<double> h(n0);
        cudaError_t ec = cudaMemcpyAsync(h.data(), t_dev, n0 * sizeof(double),
                                         cudaMemcpyDeviceToHost, st);
        if (ec == cudaSuccess) ec = cudaStreamSynchronize(st);
        if (ec != cudaSuccess) return cuda_fail(ec, "nu_batch_search: copy of curve 0");
        std::vector<double> d(n0 - 1);
        for (int64_t i = 0; i + 1 < n0; ++i) d[i] = h[i + 1] - h[i];
        std::sort(d.begin(), d.end());
        const size_t m = d.size();
        phase_step = (m % 2) ? d[m / 2] : 0.5 * (d[m / 2 - 1] + d[m / 2]);
        if (!(phase_step > 0.0) || !std::isfinite(phase_step))
            return fail(NU_EINVAL, "nu_batch_search: curve 0 gives no positive median spacing");
    }
    pool_keep_memory();
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    // ------------------------------------------------------- factor memory
    const size_t esz = fp64 ? 8 : 4;
    size_t off = 0;
    const size_t o_F = off;     off += al((size_t)N * nb * 4 * 8);
    const size_t o_kg = off;    off += al((size_t)N * J * 8);
    const size_t o_iD = off;    off += al((size_t)N * 8);
    const size_t o_G = off;     off += al((size_t)N * JJ * 8);
    const size_t o_z0 = off;    off += al((size_t)N * 8);
    const size_t o_Zt = off;    off += al((size_t)N * (k > 0 ? k : 1) * 8);
    const size_t o_work = off;  off += al((size_t)N * (k + 1) * 8);
    const size_t o_scal = off;  off += al((size_t)n_lc * 4 * 8);
    const size_t o_dstat = off; off += al((size_t)n_lc * 2 * 8);
    const size_t o_f32 = off;   off += fp64 ? 0 : al((size_t)N * (nb * 4 + J + 1 + JJ + 1 + k) * 4 + 1024);
    const size_t o_ws = off;    off += al(plan.bytes);
    const size_t o_lin = off;   off += al((size_t)N * n_D * esz) * 3;
    const size_t o_ends = off;  off += al((size_t)n_lc * 2 * 8);
    const size_t o_irr = off;   off += al((size_t)n_lc * 4);
    const size_t o_Ds = off;    off += al((size_t)n_D * 8);
    const size_t o_ctr = off;   off += 256;
    const size_t o_tune = off;  off += al(512 * 8);
    const bool win_lo = n_D <= 4096;            // window-start recursion of the box search
    const size_t o_wplan = off; off += win_lo ? al((size_t)n_lc * window_plan_ints(n_D) * 4) : 0;
    const size_t base_bytes = off;
    char* mem = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&mem, base_bytes, st);
    if (e != cudaSuccess) return cuda_fail(e, "nu_batch_search: cudaMallocAsync");
    char* fold_mem = nullptr;
    auto cleanup = [&]() {
        if (fold_mem) cudaFreeAsync(fold_mem, st);
        cudaFreeAsync(mem, st);
    };
    FactorBuffers fb{t_dev,
                     (double*)(mem + o_F), (double*)(mem + o_kg), (double*)(mem + o_iD),
                     (double*)(mem + o_G), (double*)(mem + o_z0), (double*)(mem + o_Zt),
                     (double*)(mem + o_work), (double*)(mem + o_scal),
                     (long long*)(mem + o_dstat), nullptr, nullptr, nullptr, nullptr,
                     nullptr, nullptr};
    if (!fp64) {
        float* q = (float*)(mem + o_f32);
        fb.F32 = q;    q += N * nb * 4;
        fb.kg32 = q;   q += N * J;
        fb.invD32 = q; q += N;
        fb.G32 = q;    q += N * JJ;
        fb.z032 = q;   q += N;
        fb.Zt32 = q;
    }
    char* ws = mem + o_ws;
    void* lin_d = mem + o_lin;
    void* lin_v = mem + o_lin + al((size_t)N * n_D * esz);
    void* lin_l = mem + o_lin + 2 * al((size_t)N * n_D * esz);
    const int64_t* s_off_dev = (const int64_t*)(ws + plan.off_s_off);
    // ------------------------------------------------------ pre-capture work
    nu_status s = upload_factor_plan(plan, ws, st);
    if (s != NU_OK) {
        cleanup();
        return s;
    }
    std::vector<double> ends(2 * (size_t)n_lc);
    std::vector<int> irregular(n_lc, 0);
    int launched = 0;
    k_gather_ends<<<div_up(n_lc, 128), 128, 0, st>>>(t_dev, s_off_dev, n_lc,
                                                     (double*)(mem + o_ends));
    ++launched;
    e = cudaMemsetAsync(mem + o_irr, 0, (size_t)n_lc * 4, st);
    if (!fp64 && e == cudaSuccess)
        launched += launch_slots_test(t_dev, s_off_dev, n_lc, N, phase_step,
                                      (int*)(mem + o_irr), st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ends.data(), mem + o_ends, ends.size() * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(irregular.data(), mem + o_irr, (size_t)n_lc * 4,
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(mem + o_Ds, Ds_host, (size_t)n_D * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    count_launches(launched);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "nu_batch_search: setup");
    }
    std::vector<double> t_first(n_lc), t_last(n_lc);
    for (int g = 0; g < n_lc; ++g) {
        t_first[g] = ends[2 * g];
        t_last[g] = ends[2 * g + 1];
        if (!(t_last[g] >= t_first[g]) || (t_last[g] - t_first[g]) / phase_step > 1.0e9) {
            cleanup();
            return fail(NU_EINVAL, "nu_batch_search: curve %d: times unsorted or span too "
                                   "long for the phase step", g);
        }
    }
    FoldBatch fbat;
    plan_fold_batch(plan.s_off, t_first, t_last, irregular, fp64, phase_step, gap_factor, n_D,
                    fbat);
    size_t foff = 0;
    const size_t f_segs = foff;  foff += al(fbat.segs.size() * sizeof(FoldSeg));
    const size_t f_nodes = foff; foff += fbat.any_exact ? exact_layout(N, n_D, fp64).total : 0;
    const size_t f_buck = foff;  foff += al((size_t)(fbat.n_bucket_total + 1) * 4);
    const size_t f_rec = foff;   foff += al((size_t)(fbat.n_rec_total + 1) * sizeof(Node4<float>));
    const size_t f_lgm = foff;   foff += al((size_t)((fp64 ? 0 : fbat.n_gain_total) + 1) * sizeof(float));
    const size_t f_srec = foff;  foff += al((size_t)(fbat.n_srec_total + 1) * sizeof(ScreenRec));
    const size_t f_slot = foff;  foff += fp64 ? al((size_t)N * sizeof(int)) : 0;
    const size_t f_reg = foff;   foff += al((size_t)n_lc * 2 * sizeof(unsigned));
    const size_t f_lint = foff;  foff += al((size_t)(fbat.n_srec_total + 1) * sizeof(float));
    const size_t f_lm3 = foff;   foff += al((size_t)((fp64 ? fbat.n_gain_total : 0) + 1) * sizeof(float));
    const size_t f_peak = foff;  foff += al((size_t)n_lc * sizeof(unsigned long long));
    const size_t f_ptab = foff;  foff += al((size_t)n_P * period_const_bytes());
    e = cudaMallocAsync((void**)&fold_mem, foff, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(fold_mem + f_segs, fbat.segs.data(), fbat.segs.size() * sizeof(FoldSeg),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "nu_batch_search: fold setup");
    }
    const FoldSeg* fsegs = (const FoldSeg*)(fold_mem + f_segs);
    const FoldScratch fsc{fold_mem + f_nodes, (int*)(fold_mem + f_buck),
                          (Node4<float>*)(fold_mem + f_rec), (float*)(fold_mem + f_lgm),
                          (ScreenRec*)(fold_mem + f_srec),
                          (int*)(fold_mem + f_slot), (unsigned*)(fold_mem + f_reg),
                          (float*)(fold_mem + f_lint), (float*)(fold_mem + f_lm3),
                          (unsigned long long*)(fold_mem + f_peak),
                          (PeriodConst*)(fold_mem + f_ptab)};
    unsigned long long* ctr = (unsigned long long*)(mem + o_ctr);
    const double* Ds_dev = (const double*)(mem + o_Ds);
    int dev = 0, n_sm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    // the enqueue of everything after setup (graph body)
    cudaStream_t side = thread_side_stream();
    cudaError_t enq_err = cudaSuccess;      // first failed enqueue of a memset
    WindowShape win_shape = default_window_shape(N);
    auto enqueue = [&](int grid, int threads, int64_t nP_run, int n_run,
                       cudaStream_t st) -> int {
        int l = 0;
        k_init_dstat<<<div_up(n_lc, 128), 128, 0, st>>>(fb.dstat, s_off_dev, n_lc);
        ++l;
        int lf = 0;
        launch_factor(plan, fb, ws, diag_var_dev, nullptr, 0, y_dev, st, side, &lf);
        l += lf;
        int* wplan = win_lo ? (int*)(mem + o_wplan) : nullptr;
        const WindowShape wsh = win_shape;
        if (fp64) {
            FactorView<double> fv{fb.F, fb.kg, fb.invD, fb.G, fb.z0, fb.Zt};
            l += launch_window_batch(nb, true, t_dev, k, &fv, s_off_dev, n_lc, N, Ds_dev, n_D,
                                     wplan, wsh, lin_d, lin_v, lin_l, st);
        } else {
            FactorView<float> fv{fb.F32, fb.kg32, fb.invD32, fb.G32, fb.z032, fb.Zt32};
            l += launch_window_batch(nb, false, t_dev, k, &fv, s_off_dev, n_lc, N, Ds_dev, n_D,
                                     wplan, wsh, lin_d, lin_v, lin_l, st);
        }
        int lp = 0;
        const cudaError_t ep = launch_fold_prep(fbat, fsegs, s_off_dev, n_lc, N, fp64, t_dev,
                                                lin_d, lin_v, lin_l, n_D, phase_step, gap_factor,
                                                fsc, st, &lp);
        l += lp;
        if (ep != cudaSuccess && enq_err == cudaSuccess) enq_err = ep;
        const cudaError_t ec = cudaMemsetAsync(ctr, 0, 16, st);
        if (ec != cudaSuccess && enq_err == cudaSuccess) enq_err = ec;
        l += launch_fold_batch(fbat, fsegs, n_run, N, fp64, t_dev, fsc, n_D,
                               phase_step, gap_factor, periods_dev, nP_run, ctr, grid, threads,
                               Q_dev, T0_dev, D_idx_dev, depth_out_dev, sigma_out_dev,
                               lnP_dev, st);
        count_launches(l - lf);      // launch_factor counted its own
        return l;
    };
    // ------------------------------------------------------- autotuning
    const TuneKey key{nb, k, (int)prec, n_D};
    TuneVal tv{0, 0, win_shape};
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) tv = it->second;
    }
    if (tv.threads == 0) {
        // time the fold on a slice (the first curves, periods spread over the
        // whole grid) for each shape; the slice holds several times more
        // (curve, period) items than the largest grid has blocks, so that it
        // measures throughput rather than the latency of single items
        const int n_run = n_lc < 64 ? n_lc : 64;
        const int64_t nP_run = n_P < 512 ? n_P : 512;
        double* tune_periods = (double*)(mem + o_tune);
        k_sample_periods<<<2, 256, 0, st>>>(periods_dev, n_P, (int)nP_run, tune_periods);
        count_launches(1);
        ++launched;
        // blocks per SM x threads; small blocks suit short curves, whose
        // (curve, period) items hold few cells (each warp seeds its item)
        const int cand[6][2] = {{2, 256}, {4, 256}, {4, 128}, {8, 128}, {8, 64}, {16, 64}};
        float best_ms = 1e30f;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        launched += enqueue(n_sm * 2, 256, nP_run, n_run, st);    // warm the caches
        if (enq_err != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            cleanup();
            return cuda_fail(enq_err, "nu_batch_search: memset");
        }
        for (int c = 0; c < 6; ++c) {
            cudaMemsetAsync(ctr, 0, 16, st);
            cudaEventRecord(e0, st);
            const int lt = launch_fold_batch(fbat, fsegs, n_run, N, fp64, t_dev, fsc,
                                             n_D, phase_step, gap_factor, tune_periods,
                                             nP_run, ctr, n_sm * cand[c][0], cand[c][1], Q_dev,
                                             T0_dev, D_idx_dev, depth_out_dev, sigma_out_dev,
                                             lnP_dev, st);
            count_launches(lt);
            launched += lt;
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms) {
                best_ms = ms;
                tv.blocks_per_sm = cand[c][0];
                tv.threads = cand[c][1];
            }
        }
        // the linear search's window-start kernel on the same curves: window
        // starts per block x samples per staged chunk
        if (win_lo) {
            const WindowShape wc[6] = {{32, 64}, {64, 64}, {64, 32}, {128, 64}, {128, 128},
                                       {256, 64}};
            const int64_t n_part = offsets_host[n_run];
            float best_lin = 1e30f;
            for (int c = 0; c < 6; ++c) {
                cudaEventRecord(e0, st);
                int lt;
                if (fp64) {
                    FactorView<double> fv{fb.F, fb.kg, fb.invD, fb.G, fb.z0, fb.Zt};
                    lt = launch_window_batch(nb, true, t_dev, k, &fv, s_off_dev, n_run, n_part,
                                             Ds_dev, n_D, (int*)(mem + o_wplan), wc[c], lin_d,
                                             lin_v, lin_l, st);
                } else {
                    FactorView<float> fv{fb.F32, fb.kg32, fb.invD32, fb.G32, fb.z032, fb.Zt32};
                    lt = launch_window_batch(nb, false, t_dev, k, &fv, s_off_dev, n_run, n_part,
                                             Ds_dev, n_D, (int*)(mem + o_wplan), wc[c], lin_d,
                                             lin_v, lin_l, st);
                }
                count_launches(lt);
                launched += lt;
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best_lin) {
                    best_lin = ms;
                    tv.win = wc[c];
                }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune[key] = tv;
    }
    win_shape = tv.win;
    // ------------------------------------------------ capture and launch
    // capture on a private stream (the caller's may be the legacy default
    // stream, which cannot be captured), launch on the caller's stream
    // the executable graph of this configuration, when a previous call left
    // one, takes this call's parameters (buffers, outputs) by an update
    cudaGraph_t graph = nullptr;
    const GraphKey gkey{dev, nb, k, (int)prec, n_D, n_lc, tv.blocks_per_sm, tv.threads,
                        win_shape.tlo, win_shape.ch, N, n_P};
    cudaGraphExec_t exec = take_graph(gkey);
    cudaStream_t cs = nullptr;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    int in_graph = 0;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        in_graph = enqueue(n_sm * tv.blocks_per_sm, tv.threads, n_P, n_lc, cs);
        e = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess && enq_err != cudaSuccess) e = enq_err;
    }
    if (e == cudaSuccess && exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(exec, graph, &info) != cudaSuccess) {
            cudaGetLastError();                 // clear the failed update
            cudaGraphExecDestroy(exec);
            exec = nullptr;
        }
    }
    if (e == cudaSuccess && !exec) e = cudaGraphInstantiate(&exec, graph, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (exec) {
        if (e == cudaSuccess) put_graph(gkey, exec); else cudaGraphExecDestroy(exec);
    }
    if (graph) cudaGraphDestroy(graph);
    if (cs) cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "nu_batch_search: graph");
    }
    launched += in_graph;
    std::vector<long long> ds(2 * (size_t)n_lc);
    e = cudaMemcpyAsync(ds.data(), fb.dstat, ds.size() * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) return cuda_fail(e, "nu_batch_search: status");
    for (int g = 0; g < n_lc; ++g) status_host[g] = (int)ds[2 * g];
    (void)launched;
    return NU_OK;
}

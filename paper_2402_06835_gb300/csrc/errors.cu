// Error reporting of the C ABI and the host-side expansion of covariance
// terms (Appendix A SHO, Sect. 3.2 rotation map and exponential terms).
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "nu_internal.cuh"

namespace {
thread_local char g_msg[512] = "";
std::atomic<unsigned long long> g_launches{0};
}

namespace nu {

void pool_keep_memory() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    static thread_local int done_mask = 0;
    if (dev < 31 && (done_mask & (1 << dev))) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    if (dev < 31) done_mask |= (1 << dev);
}

void count_launches(int k) { g_launches.fetch_add((unsigned long long)k); }

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
}

nu_status fail(nu_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    return s;
}

nu_status cuda_fail(cudaError_t e, const char* where) {
    snprintf(g_msg, sizeof(g_msg), "%s: %s", where, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? NU_ENOMEM : NU_ECUDA;
}

static bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

// SHO in the Appendix A parametrisation (sigma, omega, Q).
static nu_status push_sho(Blocks* out, double sigma, double omega, double Q) {
    if (out->nb >= NU_MAX_BLOCKS)
        return fail(NU_EINVAL, "state dimension exceeds %d", 2 * NU_MAX_BLOCKS);
    if (!std::isfinite(sigma) || sigma < 0.0 || !finite_pos(omega) || !finite_pos(Q))
        return fail(NU_EINVAL, "SHO term needs sigma >= 0, omega > 0, Q > 0 "
                               "(got %g, %g, %g)", sigma, omega, Q);
    BlockParams& b = out->b[out->nb++];
    b.type = 0;
    b.sigma2 = sigma * sigma;
    b.omega = omega;
    b.Q = Q;
    b.ell = 0.0;
    return NU_OK;
}

nu_status expand_terms(const nu_term* terms, int n_terms, Blocks* out) {
    out->nb = 0;
    if (n_terms < 0 || (n_terms > 0 && terms == nullptr))
        return fail(NU_EINVAL, "terms: null pointer or negative count");
    for (int i = 0; i < n_terms; ++i) {
        const nu_term& tm = terms[i];
        nu_status s = NU_OK;
        if (tm.kind == NU_TERM_SHO) {
            s = push_sho(out, tm.p[0], tm.p[1], tm.p[2]);
        } else if (tm.kind == NU_TERM_EXP) {
            if (out->nb >= NU_MAX_BLOCKS)
                return fail(NU_EINVAL, "state dimension exceeds %d", 2 * NU_MAX_BLOCKS);
            if (!std::isfinite(tm.p[0]) || tm.p[0] < 0.0 || !finite_pos(tm.p[1]))
                return fail(NU_EINVAL, "EXP term needs sigma >= 0, ell > 0");
            BlockParams& b = out->b[out->nb++];
            b.type = 1;
            b.sigma2 = tm.p[0] * tm.p[0];
            b.omega = 0.0;
            b.Q = 0.0;
            b.ell = tm.p[1];
        } else if (tm.kind == NU_TERM_ROTATION) {
            // Sect. 3.2: two SHO modes at P and P/2
            const double sigma = tm.p[0], P = tm.p[1], Q0 = tm.p[2], dQ = tm.p[3],
                         f = tm.p[4];
            if (!std::isfinite(sigma) || sigma < 0.0 || !finite_pos(P) ||
                !std::isfinite(Q0) || !std::isfinite(dQ) || !std::isfinite(f) ||
                f < 0.0)
                return fail(NU_EINVAL, "ROTATION term needs sigma >= 0, period > 0, "
                                       "finite Q0, dQ and f >= 0");
            const double Q1 = 0.5 + Q0 + dQ;
            const double Q2 = 0.5 + Q0;
            if (!(Q1 > 0.5) || !(Q2 > 0.0))
                return fail(NU_EINVAL, "ROTATION term needs 1/2 + Q0 + dQ > 1/2 "
                                       "and 1/2 + Q0 > 0");
            const double w1 = 4.0 * M_PI * Q1 / (P * std::sqrt(4.0 * Q1 * Q1 - 1.0));
            const double S1 = sigma * sigma / ((1.0 + f) * w1 * Q1);
            const double w2 = 2.0 * w1;
            const double S2 = f * sigma * sigma / ((1.0 + f) * w2 * Q2);
            s = push_sho(out, std::sqrt(S1 * w1 * Q1), w1, Q1);
            if (s == NU_OK) s = push_sho(out, std::sqrt(S2 * w2 * Q2), w2, Q2);
        } else {
            return fail(NU_EINVAL, "unknown term kind %d", tm.kind);
        }
        if (s != NU_OK) return s;
    }
    if (out->nb == 0) {
        // white noise only: one inert block with zero variance keeps the
        // recursions uniform (its state stays zero)
        BlockParams& b = out->b[out->nb++];
        b.type = 1;
        b.sigma2 = 0.0;
        b.omega = 0.0;
        b.Q = 0.0;
        b.ell = 1.0;
    }
    return NU_OK;
}

}  // namespace nu

extern "C" const char* nu_last_error(void) { return g_msg; }

extern "C" uint64_t nu_launch_count(void) { return g_launches.load(); }

extern "C" const char* nu_version(void) { return "nuance-gb300 0.1 (sm_103a)"; }

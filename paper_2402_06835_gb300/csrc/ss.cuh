// State-space building blocks of the quasiseparable covariance.
//
// Appendix A's SHO covariance k(tau) = sigma^2 e^{-omega tau/2Q} {...} is the
// autocovariance of x'' + (omega/Q) x' + omega^2 x = white noise.  With the
// state (x, x'/omega) the stationary covariance is sigma^2 I and the
// transition over a lag tau is
//   F(tau) = e^{-c tau} [[C + c S, omega S], [-omega S, C - c S]],
//   c = omega / (2Q),
//   Q > 1/2: d = omega sqrt(1 - 1/(4Q^2)), C = cos(d tau),  S = sin(d tau)/d
//   Q < 1/2: d = omega sqrt(1/(4Q^2) - 1), C = cosh(d tau), S = sinh(d tau)/d
//   Q = 1/2: C = 1, S = tau,
// so that h^T F(tau) P_inf h = k(tau) with h = (1, 0) reproduces the three
// branches of Appendix A.  The exponential term of Sect. 3.2 is the scalar
// process with F = e^{-tau/ell}, embedded in a 2x2 block whose second
// component stays zero.
#pragma once

#include "nu_internal.cuh"

namespace nu {

template <int NB>
struct Dims {
    static constexpr int J = 2 * NB;
    static constexpr int JJ = J * (J + 1) / 2;
};

// packed upper-triangular index, i <= j
__host__ __device__ constexpr int pk(int i, int j, int J) {
    return i * J - (i * (i - 1)) / 2 + (j - i);
}

__device__ inline void block_transition(const BlockParams& p, double tau,
                                        double f[4]) {
    if (p.type == 1) {
        f[0] = exp(-tau / p.ell);
        f[1] = 0.0;
        f[2] = 0.0;
        f[3] = 0.0;
        return;
    }
    const double w = p.omega;
    const double Q = p.Q;
    const double c = w / (2.0 * Q);
    double eC, eS;   // e^{-c tau} C and e^{-c tau} S
    if (Q > 0.5) {
        const double d = w * sqrt(1.0 - 1.0 / (4.0 * Q * Q));
        double sn, cs;
        sincos(d * tau, &sn, &cs);
        const double e = exp(-c * tau);
        eC = e * cs;
        eS = e * (sn / d);
    } else if (Q < 0.5) {
        // overdamped: write cosh / sinh with the envelope folded in so that
        // long lags neither overflow nor cancel
        const double d = w * sqrt(1.0 / (4.0 * Q * Q) - 1.0);
        const double slow = exp(-(c - d) * tau);
        const double fast = exp(-(c + d) * tau);
        eC = 0.5 * (slow + fast);
        eS = 0.5 * slow * (-expm1(-2.0 * d * tau)) / d;
    } else {
        const double e = exp(-c * tau);
        eC = e;
        eS = e * tau;
    }
    f[0] = eC + c * eS;
    f[1] = w * eS;
    f[2] = -w * eS;
    f[3] = eC - c * eS;
}

// y = F x for block-diagonal F (NB blocks of 2x2, row-major per block)
template <int NB, typename T>
__device__ __forceinline__ void apply_F(const T* __restrict__ F, const T* x, T* y) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const T x0 = x[2 * b], x1 = x[2 * b + 1];
        y[2 * b] = F[4 * b] * x0 + F[4 * b + 1] * x1;
        y[2 * b + 1] = F[4 * b + 2] * x0 + F[4 * b + 3] * x1;
    }
}

// y = F^T x
template <int NB, typename T>
__device__ __forceinline__ void apply_FT(const T* __restrict__ F, const T* x, T* y) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const T x0 = x[2 * b], x1 = x[2 * b + 1];
        y[2 * b] = F[4 * b] * x0 + F[4 * b + 2] * x1;
        y[2 * b + 1] = F[4 * b + 1] * x0 + F[4 * b + 3] * x1;
    }
}

// h^T x: sum of the first component of every block
template <int NB, typename T>
__device__ __forceinline__ T hdot(const T* x) {
    T s = x[0];
#pragma unroll
    for (int b = 1; b < NB; ++b) s += x[2 * b];
    return s;
}

}  // namespace nu

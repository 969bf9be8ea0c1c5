// Device physics for the flux-differencing DGSEM: Burgers and Euler fluxes,
// two-point EC fluxes, Rusanov dissipation, the paper's entropy
// s = -rho log(p rho^-gamma) (eq. EntropyMathematical) and entropy variables
// (eq. EntropyVariables), plus compensated reduction helpers.
#pragma once

#include <cstdint>

#include "perrk_internal.h"

namespace perrk {

enum { EQ_BURGERS = 0, EQ_EULER = 1 };

template <typename Real> struct Lit;
template <> struct Lit<double> {
    static constexpr double series_u = 1e-4;     // |(y-x)/(y+x)|^2 below this: series branch
};
template <> struct Lit<float> {
    static constexpr float series_u = 1e-2f;
};

// float64 path: IEEE operations.  FP32 path (mixed form): the single MUFU
// approximations (reciprocal and square root within ~2 ulp, log2 within
// ~2^-22 absolute); the logarithms only enter the logarithmic means away
// from the series branch, where |log y - log x| >= 0.2.
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double dlog(double x) { return log(x); }
__device__ __forceinline__ float dlog(float x) { return __logf(x); }
__device__ __forceinline__ double dsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float dsqrt(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double dfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float dfma(float a, float b, float c) { return fmaf(a, b, c); }

// Logarithmic mean (y - x) / (log y - log x) with precomputed logs.  For close
// arguments (u = f^2, f = (y - x)/(y + x)) the identity
// (log y - log x) = 2 atanh f gives ln_mean = (x + y) / (2 atanh(f)/f) and
// f / atanh(f) = 1 - u/3 - 4u^2/45 - 44u^3/945 - ... (series of x/atanh x).
template <typename Real>
__device__ __forceinline__ Real ln_mean(Real x, Real y, Real lx, Real ly) {
    Real d = y - x, s = y + x;
    Real f = d * rcp(s);
    Real u = f * f;
    if (u < Lit<Real>::series_u) {
        Real poly = dfma(u, dfma(u, dfma(u, Real(-44.0 / 945.0), Real(-4.0 / 45.0)), Real(-1.0 / 3.0)), Real(1.0));
        return Real(0.5) * s * poly;
    }
    return d * rcp(ly - lx);
}

// FP32 (mixed form): both branches are computed and one is selected, so the
// warp does not diverge on the branch test (the unused direct quotient may be
// inf or NaN when x == y; it is discarded).
template <>
__device__ __forceinline__ float ln_mean<float>(float x, float y, float lx, float ly) {
    const float d = y - x, s = y + x;
    const float f = d * rcp(s);
    const float u = f * f;
    const float poly = fmaf(u, fmaf(u, fmaf(u, -44.0f / 945.0f, -4.0f / 45.0f), -1.0f / 3.0f), 1.0f);
    const float series = 0.5f * s * poly;
    const float direct = d * rcp(ly - lx);
    return u < Lit<float>::series_u ? series : direct;
}

// 1 / ln_mean(x, y): (x + y)^-1 * 2 atanh(f)/f = 2/(x+y) (1 + u/3 + u^2/5 + u^3/7 + ...)
template <typename Real>
__device__ __forceinline__ Real inv_ln_mean(Real x, Real y, Real lx, Real ly) {
    Real d = y - x, s = y + x;
    Real rs = rcp(s);
    Real f = d * rs;
    Real u = f * f;
    if (u < Lit<Real>::series_u) {
        Real poly = dfma(u, dfma(u, dfma(u, Real(1.0 / 7.0), Real(1.0 / 5.0)), Real(1.0 / 3.0)), Real(1.0));
        return Real(2.0) * rs * poly;
    }
    return (ly - lx) * rcp(d);
}

template <>
__device__ __forceinline__ float inv_ln_mean<float>(float x, float y, float lx, float ly) {
    const float d = y - x, s = y + x;
    const float rs = rcp(s);
    const float f = d * rs;
    const float u = f * f;
    const float poly = fmaf(u, fmaf(u, fmaf(u, 1.0f / 7.0f, 1.0f / 5.0f), 1.0f / 3.0f), 1.0f);
    const float series = 2.0f * rs * poly;
    const float direct = (ly - lx) * rcp(d);
    return u < Lit<float>::series_u ? series : direct;
}

// Per-node primitive bundle used by Ranocha's flux.
template <typename Real, int DIM>
struct Prim {
    Real rho, v[DIM], p, beta, lrho, lbeta;   // beta = rho / p
};

template <typename Real, int DIM>
__device__ __forceinline__ Prim<Real, DIM> make_prim(const Real *u, Real gm1, uint32_t &bad) {
    Prim<Real, DIM> P;
    P.rho = u[0];
    Real ir = rcp(P.rho);
    Real ke = 0;
    for (int a = 0; a < DIM; ++a) {
        P.v[a] = u[1 + a] * ir;
        ke = dfma(P.v[a], u[1 + a], ke);
    }
    P.p = gm1 * (u[DIM + 1] - Real(0.5) * ke);
    if (!(P.rho > Real(0)) || !(P.p > Real(0))) bad |= PERRK_FLAG_NONPHYSICAL;
    P.beta = P.rho * rcp(P.p);
    P.lrho = dlog(P.rho);
    P.lbeta = dlog(P.beta);
    return P;
}

// Ranocha's EC/KEP two-point flux in direction n (AX >= 0: n = n0 e_AX).
//   f_rho = ln(rho) avg(v.n), f_m = f_rho avg(v) + avg(p) n,
//   f_E = f_rho (v_L.v_R / 2 + 1/((gamma-1) ln(beta))) + (p_L v_R.n + p_R v_L.n) / 2
template <typename Real, int DIM, int AX>
__device__ __forceinline__ void ranocha(const Prim<Real, DIM> &L, const Prim<Real, DIM> &R, const Real *n, Real inv_gm1,
                                        Real *f) {
    Real rho_m = ln_mean(L.rho, R.rho, L.lrho, R.lrho);
    Real ibeta_m = inv_ln_mean(L.beta, R.beta, L.lbeta, R.lbeta);
    Real vnl, vnr;
    if (AX >= 0) {
        vnl = L.v[AX] * n[0];
        vnr = R.v[AX] * n[0];
    } else {
        vnl = 0;
        vnr = 0;
        for (int a = 0; a < DIM; ++a) {
            vnl = dfma(L.v[a], n[a], vnl);
            vnr = dfma(R.v[a], n[a], vnr);
        }
    }
    Real p_avg = Real(0.5) * (L.p + R.p);
    Real f0 = rho_m * Real(0.5) * (vnl + vnr);
    f[0] = f0;
    Real vv = 0;
    for (int a = 0; a < DIM; ++a) {
        Real va = Real(0.5) * (L.v[a] + R.v[a]);
        Real pn = (AX >= 0) ? (a == AX ? p_avg * n[0] : Real(0)) : p_avg * n[a];
        f[1 + a] = dfma(f0, va, pn);
        vv = dfma(L.v[a], R.v[a], vv);
    }
    f[DIM + 1] = dfma(f0, dfma(Real(0.5), vv, ibeta_m * inv_gm1), Real(0.5) * (L.p * vnr + R.p * vnl));
}

// physical flux f(u).n
template <typename Real, int DIM, int AX>
__device__ __forceinline__ void euler_flux(const Real *u, const Prim<Real, DIM> &P, const Real *n, Real *f) {
    Real vn;
    if (AX >= 0) {
        vn = P.v[AX] * n[0];
    } else {
        vn = 0;
        for (int a = 0; a < DIM; ++a) vn = dfma(P.v[a], n[a], vn);
    }
    f[0] = u[0] * vn;
    for (int a = 0; a < DIM; ++a) {
        Real pn = (AX >= 0) ? (a == AX ? P.p * n[0] : Real(0)) : P.p * n[a];
        f[1 + a] = dfma(u[1 + a], vn, pn);
    }
    f[DIM + 1] = (u[DIM + 1] + P.p) * vn;
}

// max wave speed |v.n| + c |n| over both states (Rusanov / LLF)
template <typename Real, int DIM, int AX>
__device__ __forceinline__ Real max_speed(const Prim<Real, DIM> &L, const Prim<Real, DIM> &R, const Real *n, Real gam) {
    Real vnl, vnr, nn;
    if (AX >= 0) {
        vnl = L.v[AX] * n[0];
        vnr = R.v[AX] * n[0];
        nn = fabs(n[0]);
    } else {
        vnl = 0;
        vnr = 0;
        nn = 0;
        for (int a = 0; a < DIM; ++a) {
            vnl = dfma(L.v[a], n[a], vnl);
            vnr = dfma(R.v[a], n[a], vnr);
            nn = dfma(n[a], n[a], nn);
        }
        nn = dsqrt(nn);
    }
    Real cl = dsqrt(gam * L.p * rcp(L.rho)), cr = dsqrt(gam * R.p * rcp(R.rho));
    Real a = dfma(cl, nn, fabs(vnl)), b = dfma(cr, nn, fabs(vnr));
    return a > b ? a : b;
}

// max wave speed with the normal's length given (box elements: |n| is the
// metric factor itself, no square root)
template <typename Real, int DIM>
__device__ __forceinline__ Real max_speed_nn(const Prim<Real, DIM> &L, const Prim<Real, DIM> &R, const Real *n, Real nn,
                                             Real gam) {
    Real vnl = 0, vnr = 0;
    for (int a = 0; a < DIM; ++a) {
        vnl = dfma(L.v[a], n[a], vnl);
        vnr = dfma(R.v[a], n[a], vnr);
    }
    Real cl = dsqrt(gam * L.p * rcp(L.rho)), cr = dsqrt(gam * R.p * rcp(R.rho));
    Real a = dfma(cl, nn, fabs(vnl)), b = dfma(cr, nn, fabs(vnr));
    return a > b ? a : b;
}

// ---------------------------------------------------------------- entropy (FP64)

template <int DIM>
__device__ __forceinline__ void euler_entropy(const double *u, double gam, double &s, double *w, uint32_t &bad) {
    double rho = u[0], ir = 1.0 / rho, m2 = 0.0;
    for (int a = 0; a < DIM; ++a) m2 = fma(u[1 + a], u[1 + a], m2);
    double p = (gam - 1.0) * (u[DIM + 1] - 0.5 * m2 * ir);
    if (!(rho > 0.0) || !(p > 0.0)) bad |= PERRK_FLAG_NONPHYSICAL;
    double S = log(p) - gam * log(rho);
    s = -rho * S;
    if (w) {
        double ip = 1.0 / p;
        w[0] = gam - S - (gam - 1.0) * 0.5 * m2 * ir * ip;
        for (int a = 0; a < DIM; ++a) w[1 + a] = (gam - 1.0) * u[1 + a] * ip;
        w[DIM + 1] = -(gam - 1.0) * rho * ip;
    }
}

// ---------------------------------------------------------------- reductions

// Error-free transformation a + b = s + e (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e) {
    s = a + b;
    double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Neumaier-compensated accumulation of x into (s, c).
__device__ __forceinline__ void comp_add(double &s, double &c, double x) {
    double t, e;
    two_sum(s, x, t, e);
    s = t;
    c += e;
}

// Block-wide compensated sum of NQ values; result valid in thread 0 (hi + lo).
template <int NQ>
__device__ __forceinline__ void block_sum(double (&s)[NQ], double (&c)[NQ], double *smem /*[2*NQ*32]*/) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
        for (int off = 16; off > 0; off >>= 1) {
            double os = __shfl_down_sync(0xffffffffu, s[k], off);
            double oc = __shfl_down_sync(0xffffffffu, c[k], off);
            double t, e;
            two_sum(s[k], os, t, e);
            s[k] = t;
            c[k] += oc + e;
        }
    }
    if (lane == 0)
        for (int k = 0; k < NQ; ++k) {
            smem[(2 * k) * 32 + warp] = s[k];
            smem[(2 * k + 1) * 32 + warp] = c[k];
        }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < NQ; ++k) {
            double ss = 0.0, cc = 0.0;
            for (int w = 0; w < nw; ++w) {
                comp_add(ss, cc, smem[(2 * k) * 32 + w]);
                cc += smem[(2 * k + 1) * 32 + w];
            }
            s[k] = ss;
            c[k] = cc;
        }
    __syncthreads();
}

}  // namespace perrk

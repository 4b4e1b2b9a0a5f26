// Time-averaged wave fluxes of one UGKWP-LTS step (a9), one thread per face.
//
//  F = F^eq + F^fr,wave through face j with unit normal n from L to R (Eqs. 47-50):
//   F^eq: the interface equilibrium g_0 from the half-range moments of the Maxwellians of W_L and W_R
//     (Eq. 17); its normal slopes a^L = (W_0 - W_L)/d_L on u.n > 0 and a^R = (W_R - W_0)/d_R on u.n < 0
//     (Eq. 20 with the Prandtl fix of Sec. III A), and A from the compatibility condition (Eq. 22); each half
//     weighted with its own cell's normalised coefficients dbar_{a,b,c} (Eq. 48).
//   F^fr,wave: the hydrodynamic wave of each side over its half (Eq. 50), read as in Sec. III B: rho^h times
//     the side's local distribution (the Maxwellian of the total W, which the new particles are sampled
//     from), weighted with dbar_d - e^{-dt/tau} where this step's particles carry e^{-x} of it (else
//     dbar_d), plus the massless remainder W^h - (rho^h / rho) W, represented to first order about the same
//     Maxwellian (Eq. 20 form) and never sampled, weighted with dbar_d. First order by default; with the
//     second-order reconstruction (Eq. 12, order 2) the states at the face are reconstructed from limited
//     cell gradients and the wave adds the normal slope term of W^h about the same Maxwellian, weighted with
//     dbar_e + dt e^{-x} / 2.
//  Boundary faces (n points out of the fluid cell L): a diffuse wall returns a wall Maxwellian at T_w with
//  the density that zeroes the wave mass flux (first order); far-field / fixed ghosts are virtual cells of
//  the ghost state with the fluid cell's time step on both halves (Sec. IV B), whose collisionless part
//  enters as particles, so their wave keeps dbar_d - e^{-x}; a symmetry face mirrors L (first order).
//  The moment algebra is a dense 4x4 closed form per face, so it runs on the FP32/FP64 pipes. In production
//  mode the velocity moments are FP32; the faces of wall cells (flag face_f64) weight them with their FP64
//  time integrals and sum in FP64.
// Included by the core unit (compiled with -fmad=false), so that the step's kernels and the batched persistent
// kernel evaluate the same individually rounded operations.
#pragma once
#include <cuda_runtime.h>
#include <cmath>
#include "ugkwp_internal.h"
#include "ugkwp_detmath.cuh"

namespace ugk {
namespace wf {

template <typename R> struct Prim { R rho, U, V, lam, th; };   // th = R T = 1 / (2 lambda)
template <typename R> struct Mom { R up[9], um[9], v[7], xi2, xi4, g0; };   // g0: density at u = 0

// FP32 (R = float) trades divisions for one reciprocal and multiplications (a few ulps, far inside the
// production tolerance); FP64 keeps the divisions of the CPU definition
template <typename R> __device__ __forceinline__ bool frame_prim(const R W[4], Prim<R>& p)
{
    p.rho = W[0];
    if (!(W[0] > R(0))) return false;
    R e;
    if constexpr (sizeof(R) == 4) {
        const R r = R(1) / W[0];
        p.U = W[1] * r;
        p.V = W[2] * r;
        e = W[3] * r - R(0.5) * (p.U * p.U + p.V * p.V);
    } else {
        p.U = W[1] / W[0];
        p.V = W[2] / W[0];
        e = W[3] / W[0] - R(0.5) * (p.U * p.U + p.V * p.V);
    }
    if (!(e > R(0))) return false;
    p.lam = R(0.75) / e;
    p.th = sizeof(R) == 4 ? e * R(2.0 / 3.0) : R(0.5) / p.lam;
    return true;
}

// kDet (FP64 only, the all-FP64 mode): e^x and erfc from IEEE operations (dexp, derfc) instead of CUDA's
// library functions, so that the moments do not depend on a math library's last bits
template <typename R, bool kDet = false> __device__ __forceinline__ void moments(const Prim<R>& p, Mom<R>& M)
{
    const R U = p.U, V = p.V, lam = p.lam, th = p.th;
    const R sl = sqrt(lam);
    R ex, small;
    // one erfc per Maxwellian: the smaller half-range mass from erfc(sqrt(lambda)|U|), the other as 1 - it
    if constexpr (sizeof(R) == 4) {
        ex = expf(-lam * U * U) * (0.5f * rsqrtf(3.14159265358979323846f * lam));
        small = R(0.5) * erfc(sl * fabs(U));
    } else if constexpr (kDet) {
        ex = dexp(-lam * U * U) / (R(2) * sqrt(R(3.14159265358979323846) * lam));
        small = R(0.5) * derfc(sl * fabs(U));
    } else {
        ex = exp(-lam * U * U) / (R(2) * sqrt(R(3.14159265358979323846) * lam));
        small = R(0.5) * erfc(sl * fabs(U));
    }
    M.up[0] = U >= R(0) ? R(1) - small : small;
    M.um[0] = U >= R(0) ? small : R(1) - small;
    M.up[1] = U * M.up[0] + ex;
    M.um[1] = U * M.um[0] - ex;
#pragma unroll
    for (int k = 2; k < 9; ++k) {
        M.up[k] = U * M.up[k - 1] + R(k - 1) * th * M.up[k - 2];
        M.um[k] = U * M.um[k - 1] + R(k - 1) * th * M.um[k - 2];
    }
    M.v[0] = R(1);
    M.v[1] = V;
#pragma unroll
    for (int k = 2; k < 7; ++k) M.v[k] = V * M.v[k - 1] + R(k - 1) * th * M.v[k - 2];
    M.xi2 = th;
    M.xi4 = R(3) * th * th;
    M.g0 = sizeof(R) == 4 ? ex * (R(2) * lam) : ex / th;
}

// <psi u^a v^b w^(2c)>, psi = (1, u, v, |u|^2/2)
template <typename R>
__device__ __forceinline__ void psi_mom(const R* Mu, const Mom<R>& M, int a, int b, int c, R o[4])
{
    const R w0 = c == 0 ? R(1) : M.xi2, w2 = c == 0 ? M.xi2 : M.xi4;
    o[0] = Mu[a] * M.v[b] * w0;
    o[1] = Mu[a + 1] * M.v[b] * w0;
    o[2] = Mu[a] * M.v[b + 1] * w0;
    o[3] = R(0.5) * (Mu[a + 2] * M.v[b] * w0 + Mu[a] * M.v[b + 2] * w0 + Mu[a] * M.v[b] * w2);
}

template <typename R>
__device__ __forceinline__ void psi_poly(const R* Mu, const Mom<R>& M, int a, int b, const R cf[4], R o[4])
{
    R t0[4], t1[4], t2[4], t3[4], t4[4], t5[4];
    psi_mom(Mu, M, a, b, 0, t0);
    psi_mom(Mu, M, a + 1, b, 0, t1);
    psi_mom(Mu, M, a, b + 1, 0, t2);
    psi_mom(Mu, M, a + 2, b, 0, t3);
    psi_mom(Mu, M, a, b + 2, 0, t4);
    psi_mom(Mu, M, a, b, 1, t5);
#pragma unroll
    for (int k = 0; k < 4; ++k)
        o[k] = cf[0] * t0[k] + cf[1] * t1[k] + cf[2] * t2[k] + cf[3] * R(0.5) * (t3[k] + t4[k] + t5[k]);
}

template <typename R> __device__ __forceinline__ void slope(const Prim<R>& p, const R dw[4], R a[4])
{
    const R U = p.U, V = p.V, lam = p.lam;
    // 1.5 / lambda = 3 th and 0.75 / lambda = 1.5 th in FP32
    const R i15 = sizeof(R) == 4 ? R(3) * p.th : R(1.5) / lam;
    const R R4 = R(2) * dw[3] - R(2) * U * dw[1] - R(2) * V * dw[2] + (U * U + V * V) * dw[0] - i15 * dw[0];
    a[3] = (R(4) * lam * lam / R(3)) * R4;
    a[1] = R(2) * lam * (dw[1] - U * dw[0]) - a[3] * U;
    a[2] = R(2) * lam * (dw[2] - V * dw[0]) - a[3] * V;
    const R q = sizeof(R) == 4 ? a[3] * (R(1.5) * p.th) : a[3] * R(0.75) / lam;
    a[0] = dw[0] - q - a[1] * U - a[2] * V - a[3] * R(0.5) * (U * U + V * V);
}

template <typename R> __device__ __forceinline__ void pr_fix(const Prim<R>& p, R a[4], R Pr)
{
    if (Pr == R(1)) return;
    const R U = p.U, V = p.V, lam = p.lam;
    const R dlam = R(-0.5) * a[3];
    const R dU = (a[1] + U * a[3]) / (R(2) * lam), dV = (a[2] + V * a[3]) / (R(2) * lam);
    const R drho = a[0] - R(1.5) * dlam / lam + dlam * (U * U + V * V) + R(2) * lam * (U * dU + V * dV);
    const R dl = dlam / Pr;
    a[3] = R(-2) * dl;
    a[1] = R(2) * lam * dU + R(2) * U * dl;
    a[2] = R(2) * lam * dV + R(2) * V * dl;
    a[0] = drho + R(1.5) * dl / lam - dl * (U * U + V * V) - R(2) * lam * (U * dU + V * dV);
}

// equilibrium part of Eq. 49 given the interface state W_0 (primitive p0); c[0..2] = dbar_a, dbar_b,
// dbar_c of each side. Moments in precision R; the time-integration weights and the weighted sum in
// precision C (C = double for the faces of wall cells in production mode: FP64 time integrals).
template <typename R, typename C, bool kDet = false>
__device__ void equilibrium_part(const R W0[4], const R WL[4], const R WR[4], const Prim<R>& p0, const C cL[3],
                                 const C cR[3], R dL, R dR, R Pr, C F[4])
{
    Mom<R> m0;
    moments<R, kDet>(p0, m0);
    R t1[4], t2[4];
    R dw[4], aL[4], aR[4], A[4];
    if constexpr (sizeof(R) == 4) {
        const R rl = R(1) / (dL * p0.rho), rr = R(1) / (dR * p0.rho);
#pragma unroll
        for (int k = 0; k < 4; ++k) dw[k] = (W0[k] - WL[k]) * rl;
        slope(p0, dw, aL);
#pragma unroll
        for (int k = 0; k < 4; ++k) dw[k] = (WR[k] - W0[k]) * rr;
        slope(p0, dw, aR);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) dw[k] = (W0[k] - WL[k]) / (dL * p0.rho);
        slope(p0, dw, aL);
#pragma unroll
        for (int k = 0; k < 4; ++k) dw[k] = (WR[k] - W0[k]) / (dR * p0.rho);
        slope(p0, dw, aR);
    }
    pr_fix(p0, aL, Pr);
    pr_fix(p0, aR, Pr);
    psi_poly(m0.up, m0, 1, 0, aL, t1);
    psi_poly(m0.um, m0, 1, 0, aR, t2);
#pragma unroll
    for (int k = 0; k < 4; ++k) dw[k] = -(t1[k] + t2[k]);
    slope(p0, dw, A);
    R f[4];
    psi_mom(m0.up, m0, 1, 0, 0, f);
#pragma unroll
    for (int k = 0; k < 4; ++k) F[k] = cL[0] * C(f[k]);
    psi_mom(m0.um, m0, 1, 0, 0, f);
#pragma unroll
    for (int k = 0; k < 4; ++k) F[k] += cR[0] * C(f[k]);
    psi_poly(m0.up, m0, 2, 0, aL, f);
#pragma unroll
    for (int k = 0; k < 4; ++k) F[k] += cL[1] * C(f[k]);
    psi_poly(m0.um, m0, 2, 0, aR, f);
#pragma unroll
    for (int k = 0; k < 4; ++k) F[k] += cR[1] * C(f[k]);
    psi_poly(m0.up, m0, 1, 0, A, f);
#pragma unroll
    for (int k = 0; k < 4; ++k) F[k] += cL[2] * C(f[k]);
    psi_poly(m0.um, m0, 1, 0, A, f);
#pragma unroll
    for (int k = 0; k < 4; ++k) F[k] = C(p0.rho) * (F[k] + cR[2] * C(f[k]));
}

// Free transport of one side's hydrodynamic wave over its half (Eq. 50) about the Maxwellian p (moments m) of
// the side's state W: rho^h <psi u_n>_half weighted with fr (the part the new particles are sampled from),
// the remainder dW = W^h - (rho^h / rho) W as rho <psi u_n (a . psi)>_half with <psi g (a . psi)> = dW / rho,
// weighted with fd, and with order 2 the normal slope dh of W^h as rho <psi u_n^2 (a . psi)>_half, weighted
// with cs. Linear in W^h, so the noise of W^h = W - W^p biases nothing.
// g (a . psi) is the derivative of the Maxwellian in the direction dW, so the remainder's flux is the
// directional derivative of the half-range flux rho <psi u_n>_half. With FP32 moments (R = float) it is
// evaluated in that form, from the primitive perturbation dp = (d rho, dU, dV, d theta), theta = R T, formed in
// FP64 once per cell (prim_perturbation, k_flux_prep) and rotated into the face frame: the moment solve in the
// absolute frame cancels terms of order |U|^2 / RT (about 300 at Ma 20), which FP32 cannot afford. The half-range moments M_k = <u^k>_half obey dM_k/dU = k M_{k-1} and
// dM_k/dtheta = k (k - 1) / 2 M_{k-2} (k >= 1, 2), dM_1/dtheta = +-g(0) / 2 (+ for u > 0).
template <typename R, typename C>
__device__ __forceinline__ void wave_part(const Prim<R>& p, const Mom<R>& m, bool up, const R W[4], const R Wh[4],
                                          const R dp[4], C fr, C fd, const R* dh, C cs, C F[4])
{
    const R* Mu = up ? m.up : m.um;
    R t[4], dw[4], a[4];
    psi_mom(Mu, m, 1, 0, 0, t);
#pragma unroll
    for (int k = 0; k < 4; ++k) F[k] += fr * C(Wh[0] * t[k]);
    if (sizeof(R) == 4) {
        const R dr = dp[0], dU = dp[1], dV = dp[2], dth = dp[3];
        const R th = m.xi2, V = p.V, s = V * V + R(2) * th, hg = (up ? R(0.5) : R(-0.5)) * m.g0;
        t[0] = dr * Mu[1] + p.rho * (Mu[0] * dU + hg * dth);
        t[1] = dr * Mu[2] + p.rho * (R(2) * Mu[1] * dU + Mu[0] * dth);
        t[2] = dr * Mu[1] * V + p.rho * ((Mu[0] * V) * dU + Mu[1] * dV + (hg * V) * dth);
        t[3] = R(0.5) * (dr * (Mu[3] + Mu[1] * s) +
                         p.rho * ((R(3) * Mu[2] + Mu[0] * s) * dU + (R(2) * V * Mu[1]) * dV + (R(5) * Mu[1] + hg * s) * dth));
#pragma unroll
        for (int k = 0; k < 4; ++k) F[k] += fd * C(t[k]);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) dw[k] = (Wh[k] - (Wh[0] / p.rho) * W[k]) / p.rho;
        slope(p, dw, a);
        psi_poly(Mu, m, 1, 0, a, t);
#pragma unroll
        for (int k = 0; k < 4; ++k) F[k] += fd * C(p.rho * t[k]);
    }
    if (dh) {
#pragma unroll
        for (int k = 0; k < 4; ++k) dw[k] = dh[k] / p.rho;
        slope(p, dw, a);
        psi_poly(Mu, m, 2, 0, a, t);
#pragma unroll
        for (int k = 0; k < 4; ++k) F[k] += cs * C(p.rho * t[k]);
    }
}

// The primitive perturbation (d rho, dU, dV, d theta) of the Maxwellian of W (face frame, FP64) that carries the
// remainder dW = W^h - (rho^h / rho) W of the hydrodynamic wave: W = (rho, rho U, rho V, rho (|U|^2 + 3 theta) / 2)
__device__ __forceinline__ void prim_perturbation(const double W[4], const double Wh[4], double dp[4])
{
    const double rho = W[0], U = W[1] / rho, V = W[2] / rho, q = Wh[0] / rho;
    const double th = (W[3] / rho - 0.5 * (U * U + V * V)) / 1.5;
    double dW[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) dW[k] = Wh[k] - q * W[k];
    dp[0] = dW[0];
    dp[1] = (dW[1] - U * dW[0]) / rho;
    dp[2] = (dW[2] - V * dW[0]) / rho;
    dp[3] = ((dW[3] - dW[0] * (0.5 * (U * U + V * V) + 1.5 * th)) - rho * (U * dp[1] + V * dp[2])) / (1.5 * rho);
}

// interior-type face; frL/frR weight each side's sampled-from wave part, fdL/fdR its remainder. WL, WR: the
// states at the face (the cell states in first order), WLc, WRc: the cell states the normal slopes of g_0 are
// taken against; dhL, dhR (nullable): normal derivatives of W^h for the slope term of the free-transport wave,
// weighted with csL, csR (order 2). Returns false if a side state is not a valid Maxwellian in precision R
// (the caller then uses FP64).
template <typename R, typename C, bool kDet = false>
__device__ bool face_flux(const R WL[4], const R WR[4], const R WhL[4], const R WhR[4], const R dpL[4],
                          const R dpR[4], C fdL, C fdR, const C cL[3], const C cR[3], C frL, C frR, R dL, R dR,
                          R Pr, const R WLc[4], const R WRc[4], const R* dhL, const R* dhR, C csL, C csR, C F[4])
{
    Prim<R> pL, pR, p0;
    Mom<R> mL, mR;
#pragma unroll
    for (int k = 0; k < 4; ++k) F[k] = C(0);
    if (!frame_prim(WL, pL) || !frame_prim(WR, pR)) return false;
    moments<R, kDet>(pL, mL);
    moments<R, kDet>(pR, mR);
    R t1[4], t2[4], W0[4];
    psi_mom(mL.up, mL, 0, 0, 0, t1);
    psi_mom(mR.um, mR, 0, 0, 0, t2);
#pragma unroll
    for (int k = 0; k < 4; ++k) W0[k] = pL.rho * t1[k] + pR.rho * t2[k];
    // vacuum interface: no molecule of either side reaches the face, no equilibrium flux
    if (frame_prim(W0, p0)) equilibrium_part<R, C, kDet>(W0, WLc, WRc, p0, cL, cR, dL, dR, Pr, F);
    wave_part<R, C>(pL, mL, true, WL, WhL, dpL, frL, fdL, dhL, csL, F);
    wave_part<R, C>(pR, mR, false, WR, WhR, dpR, frR, fdR, dhR, csR, F);
    return true;
}

// diffuse (or Maxwell) isothermal wall: the incoming half of the fluid cell's g and of its hydrodynamic wave
// (as in face_flux: weights frL and fdL), the outgoing wall Maxwellian at T_w with the density that makes the
// wave mass flux zero
template <typename R, typename C, bool kDet = false>
__device__ bool wall_flux(const R WL[4], const R WhL[4], const R dpL[4], C fdL, C caL, C frL, R lam_w, C ws,
                          C F[4])
{
    Prim<R> p;
    Mom<R> m;
    R t[4];
    if (!frame_prim(WL, p)) return false;
    moments<R, kDet>(p, m);
    psi_mom(m.up, m, 1, 0, 0, t);
#pragma unroll
    for (int k = 0; k < 4; ++k) F[k] = caL * C(p.rho * t[k]);
    wave_part<R, C>(p, m, true, WL, WhL, dpL, frL, fdL, nullptr, C(0), F);
    p.rho = R(1); p.U = R(0); p.V = R(0); p.lam = lam_w; p.th = R(0.5) / lam_w;
    moments<R, kDet>(p, m);
    psi_mom(m.um, m, 1, 0, 0, t);
    const C rw = -F[0] / C(t[0]);
    if (ws == C(0)) {
#pragma unroll
        for (int k = 0; k < 4; ++k) F[k] += rw * C(t[k]);
        return true;
    }
    // Maxwell wall: the fraction ws of the incoming half reflected specularly (in the face frame the mass,
    // tangential momentum and energy fluxes change sign, the normal momentum flux keeps it), the rest
    // re-emitted diffusely at T_w with zero net mass
    const C sg[4] = {C(-1), C(1), C(-1), C(-1)}, a = C(1) - ws;
#pragma unroll
    for (int k = 0; k < 4; ++k) F[k] = (F[k] + ws * (sg[k] * F[k])) + a * (rw * C(t[k]));
    return true;
}

// Taylor weights of phi1, psi2, psi3, beta, chi (see the cell decomposition), k = 0..19
constexpr int kSeriesF = 20;
__constant__ double c_series_f[5][kSeriesF];

// normalised coefficients (dbar_a, dbar_b, dbar_c, dbar_d, dbar_d - e^{-x}) of a ghost side (Eq. 48), FP64
__device__ void ghost_coeffs(double dt, double tau, double c[5])
{
    const double x = dt / tau;
    const double e = dexp(-x);
    double phi1, psi2, psi3, beta, chi;
    if (x < 1.0) {
        const double mx = -x;
        phi1 = psi2 = psi3 = beta = chi = 0.0;
#pragma unroll
        for (int k = kSeriesF - 1; k >= 0; --k) {
            phi1 = fma(mx, phi1, c_series_f[0][k]);
            psi2 = fma(mx, psi2, c_series_f[1][k]);
            psi3 = fma(mx, psi3, c_series_f[2][k]);
            beta = fma(mx, beta, c_series_f[3][k]);
            chi = fma(mx, chi, c_series_f[4][k]);
        }
    } else {
        phi1 = (1.0 - e) / x;
        psi2 = (e - 1.0 + x) / (x * x);
        psi3 = (0.5 * x * x - x + 1.0 - e) / (x * x * x);
        beta = (1.0 + e - 2.0 * phi1) / (x * x);
        chi = (phi1 - e) / x;
    }
    c[0] = x * psi2;
    c[1] = -dt * x * beta;
    c[2] = dt * x * psi3;
    c[3] = phi1;
    c[4] = x * chi;
}

__device__ double tau_of(const StepConsts& K, const double W[4])
{
    const double rho = W[0], r = 1.0 / rho, U = W[1] * r, V = W[2] * r;
    const double RT = (W[3] * r - 0.5 * (U * U + V * V)) * (2.0 / 3.0);
    const double mu = K.mu_inf * dpow(RT / kR, K.omega);
    return mu / (rho * RT);
}

// Order 2: the state of cell cc's W (which = 0) or W^h (which = 1) at face f, W_c + grad . (x_f - x_c) with x_f
// the face point (1-D: the cell end of its local face) or midpoint (2-D), and the normal derivative n . grad, in
// the global frame; false (first order for this side) when the reconstructed state is not a positive density
// and internal energy.
__device__ bool face_side(const StepConsts& K, const Dev& c, int cc, int f, int which, double nx, double ny,
                          double Wf[4], double dn[4])
{
    const double* g = c.grad + 16 * (size_t)cc + 8 * which;
    const double* Wc = (which ? c.Wh : c.W) + 4 * cc;
    // individually rounded operations (no fused multiply-add), as in the cell gradients: the face states feed
    // differences against the cell states that amplify any last-bit change
    double ddx, ddy;
    if (K.dim == 1) {
        const int k = (c.cf64[cc].meta[0] & 0xffffff) == f ? 0 : 1;   // local face 0: left end, 1: right end
        ddx = __dsub_rn(c.cvx[4 * cc + k], c.xc[cc]);
        ddy = 0.0;
    } else {
        ddx = __dsub_rn(__dadd_rn(c.fax[f], __dmul_rn(0.5, c.fex[f])), c.xc[cc]);
        ddy = __dsub_rn(__dadd_rn(c.fay[f], __dmul_rn(0.5, c.fey[f])), c.yc[cc]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        Wf[q] = __dadd_rn(Wc[q], __dadd_rn(__dmul_rn(g[2 * q], ddx), __dmul_rn(g[2 * q + 1], ddy)));
        dn[q] = __dadd_rn(__dmul_rn(g[2 * q], nx), __dmul_rn(g[2 * q + 1], ny));
    }
    const double ke = __dmul_rn(0.5, __dadd_rn(__dmul_rn(Wf[1], Wf[1]), __dmul_rn(Wf[2], Wf[2])));
    return Wf[0] > 0.0 && __dsub_rn(Wf[3], __ddiv_rn(ke, Wf[0])) > 0.0;
}

template <typename R, typename C, bool kDet = false>
__device__ bool one_face(const StepConsts& K, const Dev& c, int f, double out[4])
{
    constexpr bool f32 = sizeof(R) == 4;   // FP32 moments: the per-cell FP32 copies of k_flux_prep
    const int L = c.fL[f], Rc = c.fR[f], bc = c.fbc[f];
    const double nx = c.fnx[f], ny = c.fny[f];
    const R nxr = R(nx), nyr = R(ny);
    auto rot = [&](const double* W, R o[4]) {
        const R a = R(W[1]), b = R(W[2]);
        o[0] = R(W[0]);
        o[1] = a * nxr + b * nyr;
        o[2] = -a * nyr + b * nxr;
        o[3] = R(W[3]);
    };
    auto rot4 = [&](const float4 w, R o[4]) {
        o[0] = R(w.x);
        o[1] = R(w.y) * nxr + R(w.z) * nyr;
        o[2] = -R(w.y) * nyr + R(w.z) * nxr;
        o[3] = R(w.w);
    };
    // a cell's W and W^h in the face frame, precision R
    auto state = [&](int cc, R W[4], R Wh[4]) {
        if constexpr (f32) {
            rot4(c.w32[cc], W);
            rot4(c.wh32[cc], Wh);
        } else {
            rot(c.W + 4 * cc, W);
            rot(c.Wh + 4 * cc, Wh);
        }
    };
    // normalised coefficient k of cell cc in the precision C of the time integrals (production mode: the FP32
    // cells of the decomposition hold theirs in FP32 only)
    auto coef = [&](int cc, int k) -> C {
        if constexpr (sizeof(C) == 4) {
            return c.co32[8 * cc + k];
        } else {
            if (K.prec == 0 && K.order != 2 && !c.wallcell[cc]) return C(c.co32[8 * cc + k]);
            return C(c.co[7 * cc + k]);
        }
    };
    // FP32 moments: the primitive perturbation carrying a side's wave remainder, in the face frame (d rho and
    // d theta are invariant, (dU, dV) rotate like the velocity); unused in FP64
    auto prim_pert = [&](int cc, R o[4]) {
        if constexpr (f32) {
            const float4 g = c.dp32[cc];
            o[0] = R(g.x);
            o[1] = R(g.y) * nxr + R(g.z) * nyr;
            o[2] = -R(g.y) * nyr + R(g.z) * nxr;
            o[3] = R(g.w);
        }
    };
    R WL[4], WhL[4], WR[4], WhR[4], WLc[4], WRc[4], dhL[4], dhR[4];
    R dpL[4] = {R(0), R(0), R(0), R(0)}, dpR[4] = {R(0), R(0), R(0), R(0)};
    C F[4];
    bool ok;
    state(L, WL, WhL);
    prim_pert(L, dpL);
#pragma unroll
    for (int q = 0; q < 4; ++q) WLc[q] = WL[q];
    const C cL[3] = {coef(L, 0), coef(L, 1), coef(L, 2)};
    // the sampled-from part of a side's wave keeps dbar_d - e^{-x} where this step's particles carry e^{-x} of
    // it; its remainder keeps dbar_d
    const C frL = (K.wave_only || c.nhp[L] == 0) ? coef(L, 3) : coef(L, 5);
    const C fdL = coef(L, 3);
    // order 2: reconstructed face states of W (equilibrium part) and W^h (free-transport wave with its normal
    // slope term, weighted with dbar_e, or dbar_e + dt e^{-x} / 2 when the collisionless part is carried by
    // particles, Eq. 50) on interior, periodic and far-field / fixed faces; W and W^h are reconstructed
    // together, and a side whose reconstructed W is not a positive density and internal energy stays first
    // order
    const bool o2 = K.order == 2 && (bc == 0 || bc == UGKWP_BC_PERIODIC || bc == UGKWP_BC_FARFIELD ||
                                     bc == UGKWP_BC_FIXED);
    bool sL = false, sR = false;
    const C csL = K.wave_only ? coef(L, 4) : coef(L, 6);
    if (o2) {
        double Wf[4], dn[4];
        if (face_side(K, c, L, f, 0, nx, ny, Wf, dn)) {
            rot(Wf, WL);
            face_side(K, c, L, f, 1, nx, ny, Wf, dn);
            rot(Wf, WhL);
            rot(dn, dhL);
            sL = true;
        }
    }
    if (bc == 0 || bc == UGKWP_BC_PERIODIC) {
        state(Rc, WR, WhR);
        prim_pert(Rc, dpR);
#pragma unroll
        for (int q = 0; q < 4; ++q) WRc[q] = WR[q];
        const C cR[3] = {coef(Rc, 0), coef(Rc, 1), coef(Rc, 2)};
        const C frR = (K.wave_only || c.nhp[Rc] == 0) ? coef(Rc, 3) : coef(Rc, 5);
        if (o2) {
            double Wf[4], dn[4];
            if (face_side(K, c, Rc, f, 0, nx, ny, Wf, dn)) {
                rot(Wf, WR);
                face_side(K, c, Rc, f, 1, nx, ny, Wf, dn);
                rot(Wf, WhR);
                rot(dn, dhR);
                sR = true;
            }
        }
        ok = face_flux<R, C, kDet>(WL, WR, WhL, WhR, dpL, dpR, fdL, coef(Rc, 3), cL, cR, frL, frR, R(c.fdL[f]), R(c.fdR[f]),
                             R(K.Pr), WLc, WRc, sL ? dhL : nullptr, sR ? dhR : nullptr, csL,
                             K.wave_only ? coef(Rc, 4) : coef(Rc, 6), F);
    } else if (bc == UGKWP_BC_WALL) {
        ok = wall_flux<R, C, kDet>(WL, WhL, dpL, fdL, cL[0], frL, R(0.5 / (kR * K.Tw)), C(K.wall_specular), F);
    } else if (bc == UGKWP_BC_SYMMETRY) {
        const R Wm[4] = {WL[0], -WL[1], WL[2], WL[3]}, Whm[4] = {WhL[0], -WhL[1], WhL[2], WhL[3]};
        dpR[0] = dpL[0]; dpR[1] = -dpL[1]; dpR[2] = dpL[2]; dpR[3] = dpL[3];
        ok = face_flux<R, C, kDet>(WL, Wm, WhL, Whm, dpL, dpR, fdL, fdL, cL, cL, frL, frL, R(c.fdL[f]), R(c.fdL[f]), R(K.Pr), WL, Wm,
                             nullptr, nullptr, C(0), C(0), F);
    } else {
        double Wg[4];
        if (bc == UGKWP_BC_FIXED) {
            for (int k = 0; k < 4; ++k) Wg[k] = K.W_fix[k];
        } else {
            const double un = K.W_inf[1] * nx + K.W_inf[2] * ny;
            const double* src = un < 0.0 ? K.W_inf : c.W + 4 * L;
            for (int k = 0; k < 4; ++k) Wg[k] = src[k];
        }
        rot(Wg, WR);
        // the ghost's collisionless part e^{-x} enters as particles (ghost sources), so its wave
        // free-transport weight is dbar_d - e^{-x}; in the particle-free mode the wave keeps all of it
        double cg[5];
        ghost_coeffs(c.dt[L], tau_of(K, Wg), cg);
        const C cR[3] = {C(cg[0]), C(cg[1]), C(cg[2])};
        // the ghost's wave is its whole state (no remainder: dpR = 0)
        ok = face_flux<R, C, kDet>(WL, WR, WhL, WR, dpL, dpR, fdL, C(cg[3]), cL, cR, frL, C(K.wave_only ? cg[3] : cg[4]), R(c.fdL[f]),
                             R(c.fdL[f]), R(K.Pr), WLc, WR, sL ? dhL : nullptr, nullptr, csL, C(0), F);
    }
    const C nxc = C(nx), nyc = C(ny);
    out[0] = double(F[0]);
    out[1] = double(F[1] * nxc - F[2] * nyc);
    out[2] = double(F[1] * nyc + F[2] * nxc);
    out[3] = double(F[3]);
    return ok && isfinite(out[0]) && isfinite(out[1]) && isfinite(out[2]) && isfinite(out[3]);
}

__device__ __forceinline__ void store_flux(const Dev& c, int f, const double out[4])
{
    double2* o = reinterpret_cast<double2*>(c.flux + 4 * (size_t)f);
    o[0] = make_double2(out[0], out[1]);
    o[1] = make_double2(out[2], out[3]);
}

// production mode, once per cell before the faces: FP32 copies of W and W^h and the primitive perturbation that
// carries W^h's remainder (FP64, rounded once), so that the FP32 faces read 16-byte FP32 loads and run no FP64
// work (B300's FP64 pipe is narrow); the decomposition wrote the FP32 coefficients
__device__ __forceinline__ void flux_prep_body(const VB vb, const StepConsts& K, const Dev& c)
{
    const int cc = vb.b * blockDim.x + threadIdx.x;
    if (cc >= K.C) return;
    const double* W = c.W + 4 * cc;
    const double* Wh = c.Wh + 4 * cc;
    c.w32[cc] = make_float4(float(W[0]), float(W[1]), float(W[2]), float(W[3]));
    c.wh32[cc] = make_float4(float(Wh[0]), float(Wh[1]), float(Wh[2]), float(Wh[3]));
    double dp[4];
    prim_perturbation(W, Wh, dp);
    c.dp32[cc] = make_float4(float(dp[0]), float(dp[1]), float(dp[2]), float(dp[3]));
}

// production mode: every face with FP32 velocity moments; the faces of wall cells apply their time
// integrals (the normalised coefficients, computed in FP64 in the decomposition) and sum the weighted
// moments in FP64. A face whose FP32 evaluation under- or overflows (near-vacuum neighbours with extreme
// moments) is queued for the FP64 kernel.
__device__ __forceinline__ void flux32_body(const VB vb, const StepConsts& K, const Dev& c)
{
    const int f = vb.b * blockDim.x + threadIdx.x;
    if (f >= K.F || c.face_f64[f]) return;
    double out[4];
    if (one_face<float, float>(K, c, f, out)) store_flux(c, f, out);
    else c.retry[atomicAdd(c.nretry, 1)] = f;
}
__global__ void __launch_bounds__(256) k_flux_prep(const StepConsts K, const Dev c) { flux_prep_body(UGKWP_VB_LAUNCH, K, c); }
__global__ void __launch_bounds__(128) k_wave_flux32(const StepConsts K, const Dev c) { flux32_body(UGKWP_VB_LAUNCH, K, c); }

// the faces of wall cells in production mode: FP32 moments weighted with their FP64 time integrals
__device__ __forceinline__ void fluxmix_body(const VB vb, const StepConsts& K, const Dev& c)
{
    const int j = vb.b * blockDim.x + threadIdx.x;
    if (j >= K.n_mix) return;
    const int f = c.mixlist[j];
    double out[4];
    if (one_face<float, double>(K, c, f, out)) store_flux(c, f, out);
    else c.retry[atomicAdd(c.nretry, 1)] = f;
}
__global__ void __launch_bounds__(128) k_wave_flux_mixed(const StepConsts K, const Dev c) { fluxmix_body(UGKWP_VB_LAUNCH, K, c); }

// FP64 faces: the static list (every face in the FP64 mode, none in production mode), then the faces
// queued by the FP32 kernel. In the all-FP64 mode the moments take e^x and erfc from IEEE operations (dexp,
// derfc); production-mode faces (second order, FP32 failures) keep CUDA's exp and erfc. The FP64 pipe's cost grows with the active lanes of a warp, so in production
// mode the (rare) queued faces are spread one per warp (lane 0); in the all-FP64 mode every lane takes a
// face.
// (the body: lane tx of the 32-thread block vb of nvb)
__device__ __forceinline__ void flux64_body(const StepConsts& K, const Dev& c, int tx, int vb, int nvb, int lanes,
                                            int all_faces)
{
    if (tx >= lanes) return;
    const int n = all_faces ? K.F : K.n_f64 + *c.nretry;
    for (int j = tx * nvb + vb; j < n; j += nvb * lanes) {
        const int f = all_faces ? j : j < K.n_f64 ? c.f64list[j] : c.retry[j - K.n_f64];
        double out[4];
        if (K.prec == 1) one_face<double, double, true>(K, c, f, out);
        else one_face<double, double, false>(K, c, f, out);
        // a non-finite flux (near-vacuum neighbours: the interface density underflows against theirs and the
        // slopes overflow) carries nothing through the face
        if (!isfinite(out[0]) || !isfinite(out[1]) || !isfinite(out[2]) || !isfinite(out[3]))
            out[0] = out[1] = out[2] = out[3] = 0.0;
        store_flux(c, f, out);
    }
}
__global__ void __launch_bounds__(32) k_wave_flux64(const StepConsts K, const Dev c, int lanes, int all_faces)
{
    flux64_body(K, c, (int)threadIdx.x, (int)blockIdx.x, (int)gridDim.x, lanes, all_faces);
}

}  // namespace wf

inline void launch_wave_flux(const StepConsts& k, const Dev& d, int sms, cudaStream_t s)
{
    // second-order reconstruction: every face in FP64 (reconstructed states near the edge of the realizable
    // set and the slope terms lose too many digits in FP32 moments)
    if (k.order == 2) {
        wf::k_wave_flux64<<<(k.F + 31) / 32, 32, 0, s>>>(k, d, 32, 1);
        return;
    }
    if (k.prec == 0) {
        wf::k_flux_prep<<<(k.C + 255) / 256, 256, 0, s>>>(k, d);
        if (k.n_mix) wf::k_wave_flux_mixed<<<(k.n_mix + 127) / 128, 128, 0, s>>>(k, d);
        wf::k_wave_flux32<<<(k.F + 127) / 128, 128, 0, s>>>(k, d);
    }
    if (k.prec == 0) wf::k_wave_flux64<<<4 * sms, 32, 0, s>>>(k, d, 1, 0);
    else wf::k_wave_flux64<<<(k.F + 31) / 32, 32, 0, s>>>(k, d, 32, 0);
}

inline cudaError_t flux_set_tables(const double* tab, cudaStream_t s)
{
    return cudaMemcpyToSymbolAsync(wf::c_series_f, tab, sizeof(double) * 5 * wf::kSeriesF, 0, cudaMemcpyHostToDevice, s);
}

}  // namespace ugk

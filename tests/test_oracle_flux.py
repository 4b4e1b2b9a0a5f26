"""Pins of the oracle's wave-flux machinery by direct numerical quadrature over velocity space.

The oracle evaluates half-range Maxwellian moments in closed form (erfc/exp recursions) and solves the slope
systems in closed form. Here every integral is taken numerically instead: quadrature in the normal
velocity u (composite Gauss-Legendre over the half line or the whole line), Gauss-Hermite in the tangential
v and the out-of-plane w.
"""
import math

import numpy as np
import pytest

from oracle import binding as ob

R = 0.5
GH_X, GH_W = np.polynomial.hermite.hermgauss(24)


def prim(W):
    rho, U, V = W[0], W[1] / W[0], W[2] / W[0]
    RT = (W[3] / rho - 0.5 * (U * U + V * V)) * 2.0 / 3.0
    return rho, U, V, RT


GL_X, GL_W = np.polynomial.legendre.leggauss(20)


def integral_vec(W, fn, side):
    """int over u (side: +1 u>0, -1 u<0, 0 all) and v, w of fn(u, v, w) * Maxwellian(W); fn returns a
    (k, ...) array. Composite Gauss-Legendre panels of width sigma/2 in u, Gauss-Hermite in v and w."""
    rho, U, V, RT = prim(W)
    sig = math.sqrt(RT)
    lo, hi = U - 40 * sig, U + 40 * sig
    if side > 0:
        lo = max(lo, 0.0)
    elif side < 0:
        hi = min(hi, 0.0)
    if hi <= lo:
        return 0.0
    npan = int(math.ceil((hi - lo) / (0.5 * sig)))
    edges = np.linspace(lo, hi, npan + 1)
    half = 0.5 * (edges[1:] - edges[:-1])
    mid = 0.5 * (edges[1:] + edges[:-1])
    u = (mid[:, None] + half[:, None] * GL_X[None, :]).reshape(-1)
    wu = (half[:, None] * GL_W[None, :]).reshape(-1)
    gu = rho * np.exp(-(u - U) ** 2 / (2 * RT)) / math.sqrt(2 * math.pi * RT) * wu
    s = math.sqrt(2.0 * RT)
    v = V + s * GH_X
    w = s * GH_X
    wt = GH_W / math.sqrt(math.pi)
    uu, vv, ww = np.meshgrid(u, v, w, indexing="ij")
    wgt = gu[:, None, None] * wt[None, :, None] * wt[None, None, :]
    vals = np.asarray(fn(uu, vv, ww))
    return (vals * wgt).sum(axis=(-3, -2, -1))


def psi(u, v, w):
    return np.array([np.ones_like(u), u, v, 0.5 * (u * u + v * v + w * w)])


def vec_integral(W, fn, side):
    return integral_vec(W, fn, side)


def poly(a, u, v, w):
    return a[0] + a[1] * u + a[2] * v + a[3] * 0.5 * (u * u + v * v + w * w)


def cons(rho, U, V, T):
    return np.array([rho, rho * U, rho * V, rho * (0.5 * (U * U + V * V) + 1.5 * R * T)])


CASES = [
    (cons(1.0, 0.3, 0.1, 1.0), cons(1.2, 0.1, -0.2, 1.3)),
    (cons(1.0, 2.7, 0.0, 1.0), cons(3.0, 0.9, 0.0, 3.67)),
    (cons(0.5, -1.5, 0.7, 0.4), cons(0.4, -1.2, 0.5, 0.6)),
]


@pytest.mark.parametrize("WL,WR", CASES)
@pytest.mark.parametrize("Pr", [1.0, 2.0 / 3.0])
def test_face_flux_against_quadrature(WL, WR, Pr):
    cL = ob.coeffs(0.01, 0.004)
    cR = ob.coeffs(0.03, 0.02)
    WhL = WL * np.array([0.6, 0.6, 0.6, 0.6])
    WhR = cons(0.5, 0.2, 0.1, 1.1)
    dL, dR = 0.013, 0.021
    F, W0, aL, aR, A = ob.face_flux(WL, WR, WhL, WhR, cL, cR, dL, dR, Pr)
    # Eq. 17: W_0 from the half-range moments of g_L and g_R
    W0q = vec_integral(WL, psi, +1) + vec_integral(WR, psi, -1)
    np.testing.assert_allclose(W0, W0q, rtol=1e-11, atol=1e-13)
    if Pr == 1.0:
        # Eq. 20: int psi g_0 a = dW/dx on each half-slope
        np.testing.assert_allclose(vec_integral(W0, lambda u, v, w: psi(u, v, w) * poly(aL, u, v, w), 0),
                                   (W0 - WL) / dL, rtol=1e-10, atol=1e-10)
        np.testing.assert_allclose(vec_integral(W0, lambda u, v, w: psi(u, v, w) * poly(aR, u, v, w), 0),
                                   (WR - W0) / dR, rtol=1e-10, atol=1e-10)
    # Eq. 22: int psi g_0 A = -int psi g_0 (a . u) with the half slopes
    lhs = vec_integral(W0, lambda u, v, w: psi(u, v, w) * poly(A, u, v, w), 0)
    rhs = -(vec_integral(W0, lambda u, v, w: psi(u, v, w) * u * poly(aL, u, v, w), +1)
            + vec_integral(W0, lambda u, v, w: psi(u, v, w) * u * poly(aR, u, v, w), -1))
    np.testing.assert_allclose(lhs, rhs, rtol=1e-9, atol=1e-9)
    # Eqs. 49-50: the time-averaged flux, half space by half space
    Fq = np.zeros(4)
    for side, c, a in ((+1, cL, aL), (-1, cR, aR)):
        Fq += vec_integral(W0, lambda u, v, w: psi(u, v, w) * u * (c[0] + c[1] * u * poly(a, u, v, w)
                                                                   + c[2] * poly(A, u, v, w)), side)
    # Eq. 50 with the hydrodynamic wave of a side as rho^h times the side's local Maxwellian (weight
    # dbar_d - e^{-x}) plus the massless remainder W^h - (rho^h / rho) W as g (a . psi) about the same
    # Maxwellian (weight dbar_d); a from the moment system taken by quadrature
    for side, W, Wh, c in ((+1, WL, WhL, cL), (-1, WR, WhR, cR)):
        Fq += c[5] * (Wh[0] / W[0]) * vec_integral(W, lambda u, v, w: psi(u, v, w) * u, side)
        G = np.stack([vec_integral(W, lambda u, v, w, k=k: psi(u, v, w) * psi(u, v, w)[k], 0) for k in range(4)],
                     axis=1)
        a = np.linalg.solve(G, Wh - (Wh[0] / W[0]) * W)
        Fq += c[3] * vec_integral(W, lambda u, v, w: psi(u, v, w) * u * poly(a, u, v, w), side)
    np.testing.assert_allclose(F, Fq, rtol=1e-9, atol=1e-9 * np.abs(Fq).max())


def test_prandtl_fix_rescales_temperature_slope():
    """With Pr != 1 the slope is that of a Maxwellian whose d(lambda)/dx is divided by Pr (Sec. III A)."""
    WL, WR = CASES[0]
    cL = ob.coeffs(0.01, 0.004)
    _, W0, a1, _, _ = ob.face_flux(WL, WR, None, None, cL, cL, 0.01, 0.01, 1.0)
    Pr = 2.0 / 3.0
    _, _, aP, _, _ = ob.face_flux(WL, WR, None, None, cL, cL, 0.01, 0.01, Pr)
    rho, U, V, RT = prim(W0)
    lam = 1.0 / (2 * RT)
    # primitive derivatives from the Pr = 1 slope, by finite differences of ln g at sample velocities
    dlam = -0.5 * a1[3]
    dU = (a1[1] + U * a1[3]) / (2 * lam)
    dV = (a1[2] + V * a1[3]) / (2 * lam)
    drho = a1[0] - 1.5 * dlam / lam + dlam * (U * U + V * V) + 2 * lam * (U * dU + V * dV)

    def lng(x, u, v, w):
        r = rho * (1 + x * drho)
        l = lam + x * dlam / Pr
        return math.log(r) + 1.5 * math.log(l) - l * ((u - U - x * dU) ** 2 + (v - V - x * dV) ** 2 + w * w)

    h = 1e-6
    for (u, v, w) in [(0.3, -0.2, 0.4), (1.5, 0.7, -0.1), (-0.8, 0.0, 1.2), (0.0, 2.0, 0.0)]:
        fd = (lng(h, u, v, w) - lng(-h, u, v, w)) / (2 * h)
        assert fd == pytest.approx(poly(aP, u, v, w), rel=1e-6, abs=1e-6)


@pytest.mark.parametrize("x", [1e-4, 0.3, 5.0, 900.0])
def test_uniform_state_flux_is_euler_flux(x):
    """Uniform W with W^h = W (no particles yet): slopes vanish and the total wave flux is
    (dbar_a + dbar_d - e^{-x}) times the Euler flux = (1 - e^{-x}) F_Euler (Eqs. 16, 49, 50)."""
    rho, U, V, T = 1.3, 0.7, -0.4, 1.7
    W = cons(rho, U, V, T)
    dt = 0.02
    c = ob.coeffs(dt, dt / x)
    F, W0, aL, aR, A = ob.face_flux(W, W, W, W, c, c, 0.1, 0.1)
    p = rho * R * T
    E = W[3]
    euler = np.array([rho * U, rho * U * U + p, rho * U * V, U * (E + p)])
    np.testing.assert_allclose(W0, W, rtol=1e-13)
    np.testing.assert_allclose(aL, 0, atol=1e-12)
    np.testing.assert_allclose(F, (1 - math.exp(-x)) * euler, rtol=1e-12)


def test_mu_inf_hard_sphere_factor():
    """omega = 1/2 gives lambda = 16 mu / (5 rho sqrt(2 pi R T)), the hard-sphere mean free path."""
    mu = ob.lib().oracle_mu_inf(1.0, 0.5)
    assert 16.0 * mu / (5.0 * math.sqrt(2 * math.pi * R)) == pytest.approx(1.0, rel=1e-15)

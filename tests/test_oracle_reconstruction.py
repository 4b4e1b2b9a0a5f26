"""Second-order reconstruction of the wave fluxes (Eq. 12; order 2, S6 reading), pinned on the CPU oracle:
the limited gradients are exact for linear fields where the limiters must not act, vanish at an extremum,
leave a uniform state untouched, and the particle-free scheme converges at second order on a smooth advected
density wave where the first-order scheme converges at first order."""
import numpy as np
import pytest

from oracle import binding as ob
from paper_2607_09552_b300 import workloads as wl


def _one_wave_step(case, prim, order=2):
    case.init_prim = prim
    o = ob.Oracle(case, precision=1, wave_only=True, order=order)
    o.step(1)
    return o


def _linear_gradients(ratio):
    ni, nj = 12, 9
    m = wl.plate_mesh(ni=ni, nj=nj, h1=0.05, ratio=ratio)
    case = wl.Case("lin", m, Kn=0.05, Ma=2.0, Tw=1.0, cfl=0.5, n_ref=10)
    xv, yv = m.xv.reshape(nj + 1, ni + 1), m.yv.reshape(nj + 1, ni + 1)
    xc = 0.25 * (xv[:-1, :-1] + xv[:-1, 1:] + xv[1:, :-1] + xv[1:, 1:]).reshape(-1)
    yc = 0.25 * (yv[:-1, :-1] + yv[:-1, 1:] + yv[1:, :-1] + yv[1:, 1:]).reshape(-1)
    a, bx, by, U, V, T = 1.0, 0.3, -0.7, 0.4, -0.2, 1.3
    prim = np.zeros((ni * nj, 4))
    prim[:, 0] = a + bx * xc + by * yc
    prim[:, 1], prim[:, 2], prim[:, 3] = U, V, T
    G = _one_wave_step(case, prim).gradients()
    e = 1.5 * 0.5 * T + 0.5 * (U * U + V * V)            # E per unit density (R = 1/2)
    fac = np.array([1.0, U, V, e])
    interior = [i + ni * j for j in range(1, nj - 1) for i in range(1, ni - 1)]
    exact = np.array([[[bx * f, by * f] for f in fac]] * len(interior))
    return G[interior, :4, :], exact


def test_gradients_exact_for_linear_fields():
    """rho linear in (x, y) with U, V, T constant makes every conservative component linear; the
    least-squares gradient reproduces it, and on a uniform Cartesian mesh Venkatakrishnan's factor is 1 in
    interior cells (each face value lies half way to the neighbour's: Delta_1 = 2 Delta_2); on a stretched
    mesh the smooth limiter trims the gradient by a few percent at most."""
    G, exact = _linear_gradients(1.0)
    np.testing.assert_allclose(G, exact, rtol=1e-9, atol=1e-12)
    G, exact = _linear_gradients(1.2)
    nz = exact != 0.0
    ratio = G[nz] / exact[nz]
    assert np.all(ratio <= 1.0 + 1e-12) and np.all(ratio > 0.95)


def test_smooth_slopes_1d():
    """1-D: exact slope of a linear field on a stretched line (equal one-sided slopes); zero next to a boundary
    face; around an interior maximum the slopes change sign and stay below the larger one-sided slope."""
    ni = 20
    m = wl.line_mesh(ni, 0.0, 1.0, end_ratio=5.0, bc_left=wl.BC_FIXED, bc_right=wl.BC_FIXED)
    xs = m.xv[: ni + 1]
    xc = 0.5 * (xs[:-1] + xs[1:])
    case = wl.Case("lin1d", m, Kn=0.05, Ma=1.0, Tw=1.0, cfl=0.5, n_ref=10, ghost_state=(1.0, 0.5, 0.0, 1.0))
    prim = np.zeros((ni, 4))
    prim[:, 0] = 1.0 + 0.5 * xc
    prim[:, 1], prim[:, 3] = 0.5, 1.0
    G = _one_wave_step(case, prim).gradients()
    np.testing.assert_allclose(G[1:-1, 0, 0], 0.5, rtol=1e-10)
    assert np.all(G[[0, -1], :, :] == 0.0)
    prim[:, 0] = 1.0 + 0.3 * np.sin(np.pi * xc)
    G = _one_wave_step(case, prim).gradients()
    rho = prim[:, 0]
    k = int(np.argmax(rho))
    a = (rho[k] - rho[k - 1]) / (xc[k] - xc[k - 1])
    b = (rho[k + 1] - rho[k]) / (xc[k + 1] - xc[k])
    assert a > 0.0 > b and abs(G[k, 0, 0]) < max(abs(a), abs(b))
    assert np.all(G[1:k - 1, 0, 0] > 0.0) and np.all(G[k + 2:-1, 0, 0] < 0.0)


def test_second_order_steady_shock_converges():
    """The smooth limiter keeps the particle-free second-order scheme differentiable: the 1-D Ma 3 shock
    settles to a steady state (residual below 1e-10), as at first order; with van Leer's limiter the
    residual stalled near 5e-3."""
    case = wl.case_shock1d(ni=200, n_ref=20, Pr=1.0)
    o = ob.Oracle(case, precision=1, wave_only=True, order=2)
    o.step(12000)
    assert float(o.residual()[:4].max()) < 1e-10


def test_uniform_state_preserved_at_second_order():
    case = wl.case_cylinder(ni=10, nj=16, h1=2e-3, r_out=4.0, Kn=0.1, Ma=5.0, n_ref=10)
    o = ob.Oracle(case, precision=1, wave_only=True, order=2)
    W0 = o.field()[0].copy()
    o.step(1)
    assert np.all(o.gradients() == 0.0)
    # far from the cylinder the freestream is untouched; next to the wall the flow starts to change
    W1 = o.field()[0]
    outer = np.arange(case.mesh.ni * case.mesh.nj) % case.mesh.ni >= 3
    np.testing.assert_allclose(W1[outer], W0[outer], rtol=1e-13, atol=1e-13)


def _advection_error(ni, order):
    m = wl.line_mesh(ni, 0.0, 1.0, end_ratio=1.0, bc_left=wl.BC_PERIODIC, bc_right=wl.BC_PERIODIC)
    xs = m.xv[: ni + 1]
    xc = 0.5 * (xs[:-1] + xs[1:])
    U = 1.0
    rho = 1.0 + 0.2 * np.sin(2.0 * np.pi * xc)
    prim = np.zeros((ni, 4))
    prim[:, 0], prim[:, 1], prim[:, 3] = rho, U, 1.0 / rho      # uniform pressure: pure advection
    case = wl.Case("adv", m, Kn=1e-5, Ma=0.0, Tw=1.0, cfl=0.5, n_ref=10)
    case.init_prim = prim
    o = ob.Oracle(case, precision=1, wave_only=True, order=order)
    dt, _ = o.geometry()
    n = int(round(0.5 / dt[0]))
    o.step(n)
    t = n * dt[0]
    exact = 1.0 + 0.2 * (np.cos(2 * np.pi * (xs[:-1] - U * t)) - np.cos(2 * np.pi * (xs[1:] - U * t))) / (
        2 * np.pi * np.diff(xs))
    return float(np.abs(o.field()[0][:, 0] - exact).mean())


def test_second_order_convergence_of_a_smooth_advected_wave():
    """Particle-free (GKS limit, Kn 1e-5), CFL 0.5: halving the cells divides the mean error of the density by
    about 4 at order 2 (van Leer), about 2 at order 1."""
    e1 = [_advection_error(n, 1) for n in (32, 64, 128)]
    e2 = [_advection_error(n, 2) for n in (32, 64, 128)]
    r1 = [e1[k] / e1[k + 1] for k in range(2)]
    r2 = [e2[k] / e2[k + 1] for k in range(2)]
    assert all(1.6 < r < 2.3 for r in r1), r1
    assert all(r > 3.2 for r in r2), r2
    assert e2[-1] < 0.05 * e1[-1]

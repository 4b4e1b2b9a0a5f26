"""Maxwell wall (accommodation alpha = 1 - wall_specular; §8f f3 reading), pinned on the CPU oracle: specular
walls exchange neither mass nor energy with the gas (wave part: the reflected half mirrors the incoming one;
particles: u_n -> -u_n), diffuse walls at T_w != T do exchange energy, and alpha = 1 is the diffuse wall of
the default bit for bit."""
import numpy as np
import pytest

from oracle import binding as ob
from paper_2607_09552_b300 import workloads as wl


def _closed_box(ws, Tw=2.0, ni=24):
    m = wl.line_mesh(ni, 0.0, 1.0, end_ratio=1.0, bc_left=wl.BC_WALL, bc_right=wl.BC_WALL)
    xs = m.xv[: ni + 1]
    xc = 0.5 * (xs[:-1] + xs[1:])
    case = wl.Case("box_walls", m, Kn=0.05, Ma=0.5, Tw=Tw, cfl=0.5, n_ref=40, wall_specular=ws)
    prim = np.zeros((ni, 4))
    prim[:, 0] = 1.0 + 0.3 * np.cos(np.pi * xc)
    prim[:, 1] = 0.2 * np.sin(np.pi * xc)
    prim[:, 3] = 1.0
    case.init_prim = prim
    return case


def _totals(o):
    W, _ = o.field()
    _, vol = o.geometry()
    return np.array([np.sum(vol * W[:, 0]), np.sum(vol * W[:, 3])])


def test_specular_walls_conserve_mass_and_energy():
    o = ob.Oracle(_closed_box(1.0), precision=1)
    t0 = _totals(o)
    o.step(40)
    t1 = _totals(o)
    assert o.stats()[6] > 0                                   # particles did hit the walls
    np.testing.assert_allclose(t1, t0, rtol=1e-12)


def test_diffuse_walls_exchange_energy():
    o = ob.Oracle(_closed_box(0.0), precision=1)
    t0 = _totals(o)
    o.step(40)
    t1 = _totals(o)
    assert t1[0] == pytest.approx(t0[0], rel=1e-12)          # still no mass through a wall
    assert abs(t1[1] - t0[1]) > 1e-4 * t0[1]                  # heated by the T_w = 2 walls


def test_partial_accommodation_between_the_limits():
    """Energy gained from the hot walls grows with the accommodation alpha = 1 - wall_specular."""
    gains = []
    for ws in (1.0, 0.5, 0.0):
        o = ob.Oracle(_closed_box(ws), precision=1)
        t0 = _totals(o)
        o.step(40)
        gains.append(_totals(o)[1] - t0[1])
    assert abs(gains[0]) < 1e-10 * t0[1] < gains[1] < gains[2]


def test_invalid_specular_fraction_rejected():
    for bad in (-0.1, 1.5, float("nan")):
        with pytest.raises(ob.OracleError):
            ob.Oracle(_closed_box(bad), precision=1)


@pytest.mark.parametrize("ws", [0.0, 0.5, 1.0])
@pytest.mark.parametrize("geometry", ["stretched_line", "jittered_triangles"])
def test_gas_at_rest_at_wall_temperature_stays_in_equilibrium(geometry, ws):
    """A closed box of gas at rest at T = T_w: the wall wave flux (any accommodation) carries no mass, no
    tangential momentum and no energy, and its normal momentum is the gas pressure, so the particle-free step
    (Eq. 53 with the wall fluxes only) leaves every cell unchanged."""
    if geometry == "stretched_line":
        m = wl.line_mesh(20, 0.0, 1.0, end_ratio=3.0, bc_left=wl.BC_WALL, bc_right=wl.BC_WALL)
    else:
        m = wl.jitter_interior(wl.split_quads(wl.box_mesh(6, 5, tags=(wl.BC_WALL,) * 4), 0, "i"), 1, 0.2)
    case = wl.Case("rest", m, Kn=0.05, Ma=0.0, Tw=1.0, cfl=0.5, n_ref=30, wall_specular=ws)
    o = ob.Oracle(case, precision=1, wave_only=True)
    W0 = o.field()[0].copy()
    o.step(20)
    assert np.abs(o.field()[0] - W0).max() < 1e-14


# ---- wall wave flux away from equilibrium, by quadrature of its definition --------------------------------
# Reading of the wall face (Sec. IV B has both halves use the cell's own time step): molecules leaving the
# fluid cell towards the wall (u_n > 0 in the face frame) carry the cell's g with the weight dbar_a and its
# hydrodynamic wave: rho^h times the cell's local Maxwellian with the weight of the part the new particles are
# sampled from, plus the massless remainder W^h - (rho^h / rho) W as g (a . psi) about the same Maxwellian with
# the weight dbar_d; the outgoing half holds the fraction ws of the incoming distribution mirrored
# (u_n -> -u_n) plus 1 - ws of a wall Maxwellian at T_w whose density makes that diffuse part carry exactly the
# rest of the incoming mass. Here every integral is taken by quadrature, the remainder's a from its moment
# system by quadrature too.

def _maxwell(W):
    rho, U, V = W[0], W[1] / W[0], W[2] / W[0]
    RT = (W[3] / rho - 0.5 * (U * U + V * V)) * 2.0 / 3.0
    return rho, U, V, RT


def _half_moments(W, sign, mirror=False, n_u=400, n_v=40, poly=None):
    """int over u sign u > 0 (u the face-normal velocity; mirror: of the distribution reflected u -> -u),
    v, w of Psi(u, v, w) u f(u, v, w), f the Maxwellian of W times (a . psi) when poly = a is given (the
    polynomial taken at the unreflected velocity): tensor Gauss-Legendre in u (on [0, 14 sigma] from the mean
    outward) and Gauss-Hermite in v, w. sign = 0: the whole line, without the factor u."""
    rho, U, V, RT = _maxwell(W)
    sig = np.sqrt(RT)
    x, wx = np.polynomial.legendre.leggauss(n_u)
    Uc = -U if mirror else U
    if sign > 0:
        lo, hi = 0.0, max(Uc, 0.0) + 14 * sig
    elif sign < 0:
        lo, hi = min(Uc, 0.0) - 14 * sig, 0.0
    else:
        lo, hi = Uc - 14 * sig, Uc + 14 * sig
    u = 0.5 * (hi - lo) * x + 0.5 * (hi + lo)
    wu = 0.5 * (hi - lo) * wx
    gh, gw = np.polynomial.hermite.hermgauss(n_v)
    v = V + np.sqrt(2 * RT) * gh
    w = np.sqrt(2 * RT) * gh
    wv = gw / np.sqrt(np.pi)
    fu = rho * np.exp(-(u - Uc) ** 2 / (2 * RT)) / np.sqrt(2 * np.pi * RT) * wu
    uu, vv, ww = np.meshgrid(u, v, w, indexing="ij")
    wt = fu[:, None, None] * wv[None, :, None] * wv[None, None, :]
    psi = np.array([np.ones_like(uu), uu, vv, 0.5 * (uu * uu + vv * vv + ww * ww)])
    if poly is not None:
        us = -uu if mirror else uu
        wt = wt * (poly[0] + poly[1] * us + poly[2] * vv + poly[3] * 0.5 * (us * us + vv * vv + ww * ww))
    return (psi * (uu if sign != 0 else 1.0) * wt).sum(axis=(1, 2, 3))


def _remainder_slope(W, Wh):
    """a with int psi f_W (a . psi) = W^h - (rho^h / rho) W, by quadrature of the 4 x 4 moment system."""
    G = np.zeros((4, 4))
    for k in range(4):
        e = np.zeros(4)
        e[k] = 1.0
        G[:, k] = _half_moments(W, 0, poly=e)
    return np.linalg.solve(G, Wh - (Wh[0] / W[0]) * W)


def _cons(rho, U, V, T):
    return np.array([rho, rho * U, rho * V, rho * (0.5 * (U * U + V * V) + 0.75 * T)])


@pytest.mark.parametrize("ws", [0.0, 0.15, 1.0])
@pytest.mark.parametrize("WL,WhL", [
    (_cons(1.3, 0.7, -0.4, 2.1), _cons(0.4, 1.1, 0.3, 1.6)),     # moving into the wall, non-equilibrium wave
    (_cons(0.8, -0.5, 0.9, 0.7), _cons(0.2, -0.2, 0.6, 1.2)),    # moving away from the wall
    (_cons(2.0, 0.0, 0.0, 3.0), None),                           # no free-transport wave
])
def test_wall_flux_matches_quadrature_of_its_definition(WL, WhL, ws):
    Tw = 1.7
    c = ob.coeffs(0.013, 0.004)
    fr = c[3] - np.exp(-0.013 / 0.004)
    F = ob.wall_flux(Tw, ws, WL, WhL, c, fr)
    inc = c[0] * _half_moments(WL, +1)
    spec = c[0] * _half_moments(WL, -1, mirror=True)          # specular part: mirrored onto u_n < 0
    if WhL is not None:
        a = _remainder_slope(WL, WhL)
        inc = inc + fr * (WhL[0] / WL[0]) * _half_moments(WL, +1) + c[3] * _half_moments(WL, +1, poly=a)
        spec = (spec + fr * (WhL[0] / WL[0]) * _half_moments(WL, -1, mirror=True)
                + c[3] * _half_moments(WL, -1, mirror=True, poly=a))
    wall = _half_moments(_cons(1.0, 0.0, 0.0, Tw), -1)
    rho_w = -(1.0 - ws) * inc[0] / wall[0]
    Fq = inc + ws * spec + rho_w * wall
    scale = np.abs(inc).max()
    np.testing.assert_allclose(F, Fq, rtol=0, atol=1e-11 * scale)
    assert abs(F[0]) <= 1e-13 * scale                            # no net mass through the wall


def test_monitors_restate_the_wall_load_definitions():
    """Monitored loads of the oracle (Sec. V A, V B) against their definitions restated here from the
    per-face surface values and the wall geometry: C_d = sum_j s_j (p_j n_x - tau_j n_y) / (rho U^2 / 2),
    C_H = sum_j s_j q_j / (rho U^3 / 2), stagnation C_p and C_Q from the mean of the two wall faces facing the
    freestream most, and each EMA (alpha = 2/1001) from the first step; a flat plate has no stagnation point."""
    from paper_2607_09552_b300 import steady
    case = wl.case_cylinder(ni=12, nj=16, h1=2e-3, r_out=4.0, Kn=0.1, Ma=5.0, n_ref=20)
    o = ob.Oracle(case, precision=1)
    nx, ny, s = steady.wall_geometry(case)
    U = wl.freestream_speed(case.Ma)
    j = np.argsort(-nx, kind="stable")[:2]
    assert nx[j[0]] > 0.9
    ema = None
    for k in range(6):
        o.step(1)
        p, tau, q = o.surface(averaged=False)
        cd, ch = steady.loads(case, p, tau, q, (nx, ny, s))
        cp = (0.5 * (p[j[0]] + p[j[1]]) - 0.5) / (0.5 * U * U)
        cq = 0.5 * (q[j[0]] + q[j[1]]) / (0.5 * U ** 3)
        v = np.array([cd, ch, cp, cq])
        ema = v.copy() if ema is None else ema + (2.0 / 1001.0) * (v - ema)
        m = o.monitors()
        np.testing.assert_allclose(m[:4], v, rtol=1e-12)
        np.testing.assert_allclose(m[4:], ema, rtol=1e-12)
    plate = wl.Case("plate_small", wl.plate_mesh(ni=27, nj=13, h1=2e-3, ratio=1.25), Kn=0.05, Ma=5.0, Tw=2.0,
                    cfl=0.8, n_ref=29)
    o = ob.Oracle(plate, precision=1)
    o.step(2)
    m = o.monitors()
    assert np.isfinite(m[[0, 1, 4, 5]]).all() and np.isnan(m[[2, 3, 6, 7]]).all()


@pytest.mark.parametrize("gts", [False, True])
def test_gas_at_rest_between_diffuse_walls_keeps_the_wall_temperature_with_particles(gts):
    """Gas at rest at T_w between two diffuse walls at T_w (1-D, 16 cells stretched 10x, Kn 1: particles carry
    almost all of the gas) is the exact steady state: with the stochastic method its temperature (total energy
    over total mass, 30 samples over 600 steps after 200) averaged over 6 seeds stays within 5 standard errors
    of T_w. New particles drawn with per-cell moment matching (a lone particle at the thermal speed
    sqrt(3 R T)) carry too little energy to the walls per unit mass, and the walls then heat the gas to about
    1.13 T_w here (14 standard errors)."""
    means = []
    for seed in range(6):
        m = wl.line_mesh(16, 0.0, 1.0, end_ratio=10.0, bc_left=wl.BC_WALL, bc_right=wl.BC_WALL)
        c = wl.Case("wall_rest", m, Kn=1.0, Ma=0.0, Tw=1.0, cfl=0.5, n_ref=50, seed=seed)
        o = ob.Oracle(c, gts=gts, precision=0)
        o.step(200)
        _, vol = o.geometry()
        Ts = []
        for _ in range(30):
            o.step(20)
            W, _ = o.field()
            Ts.append((W[:, 3] * vol).sum() / (W[:, 0] * vol).sum() / 0.75)   # e = (3/2) R T, R = 1/2
        means.append(np.mean(Ts))
    means = np.array(means)
    se = means.std(ddof=1) / np.sqrt(len(means))
    assert abs(means.mean() - 1.0) <= 5.0 * se, (means, se)
    assert abs(means.mean() - 1.0) <= 0.03, means

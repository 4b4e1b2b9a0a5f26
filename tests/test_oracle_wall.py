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

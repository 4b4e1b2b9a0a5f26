"""Steady surfaces and fields against the oracle after averaging (the spec bar: 1 %).

Both sides start from the same seeded state and draw from the same Philox streams. In the all-FP64 mode the
two realisations stay identical (the wave fluxes differ only in the last bits), so the averaged quantities
agree far inside the bar; in production precision the FP32 wave-flux moments make the realisations part
after some hundred steps, and the comparison is statistical: the windows are long enough that the particle
noise of the averages (about 1 % between two seeds at N_ref 150 over 3,000 steps on the small cylinder) stays
below the bar. Metric (S28 reading of Sec. V A's averaging windows): ||X_gpu - X_oracle||_2 / ||X_oracle||_2
for p, q and each field component (momentum as a vector); tau_w, which changes sign at the stagnation point,
by its RMS difference over max |tau_w|.
"""
import numpy as np
import pytest

from oracle import binding as ob
from paper_2607_09552_b300 import workloads as wl

pytestmark = pytest.mark.gpu


def _run(sim, burn, navg, field_every=1):
    """Advance `burn` steps, restart the surface averages, then average the field over `navg` steps."""
    sim.step(burn)
    sim.reset_surface()
    W = 0.0
    n = 0
    for k in range(navg):
        sim.step(1)
        if k % field_every == 0:
            W = W + sim.field()[0]
            n += 1
    return sim.surface(True), W / n


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _compare(g, o, bar, tau_bar=None):
    (pg, tg, qg), Wg = g
    (po, to, qo), Wo = o
    out = {"p": _rel(pg, po), "q": _rel(qg, qo),
           "tau": float(np.sqrt(np.mean((tg - to) ** 2)) / np.abs(to).max()),
           "rho": _rel(Wg[:, 0], Wo[:, 0]), "momentum": _rel(Wg[:, 1:3], Wo[:, 1:3]), "energy": _rel(Wg[:, 3], Wo[:, 3])}
    for k, v in out.items():
        assert v <= (tau_bar if (k == "tau" and tau_bar) else bar), (k, out)
    return out


def test_normal_shock_full_length_fp64(cuda_lib):
    """The 1-D Ma 3 normal shock at full size (200 cells stretched 50x, N_ref 100, Shakhov Pr 2/3, CFL 0.5),
    2,000 LTS steps in the all-FP64 mode, seed 0: the field averaged over the last 1,000 steps agrees with the
    oracle's within 1 % per component (measured about 1e-12: the realisations stay identical)."""
    case = wl.case_shock1d()
    g = cuda_lib.Solver(case, precision=1)
    o = ob.Oracle(case, precision=1)
    res = []
    for sim in (g, o):
        sim.step(1000)
        W = 0.0
        for _ in range(1000):
            sim.step(1)
            W = W + sim.field()[0]
        res.append(W / 1000)
    Wg, Wo = res
    for c in (0, 1, 3):
        assert _rel(Wg[:, c], Wo[:, c]) <= 0.01, c
    assert int(g.stats()[0]) == int(o.stats()[0]) == 2000


def test_cylinder_steady_surfaces_fp64(cuda_lib):
    """A small Ma 5 cylinder (16 x 24 O-mesh to 3 D, Kn 0.1, N_ref 60), all-FP64: 1,500 steps, then p, tau_w
    and q averaged over 1,000 steps, and the averaged field, within 1 % of the oracle's."""
    case = wl.case_cylinder(ni=16, nj=24, h1=5e-3, r_out=3.0, Kn=0.1, Ma=5.0, n_ref=60)
    # capacity for the start-up transient (the particle count peaks near 6x its steady value)
    g = _run(cuda_lib.Solver(case, precision=1, capacity=16 * case.n_ref * case.mesh.ncells), 1500, 1000)
    o = _run(ob.Oracle(case, precision=1), 1500, 1000)
    _compare(g, o, 0.01)


def test_cylinder_steady_surfaces_production(cuda_lib):
    """The same cylinder with N_ref 150 in production precision: 1,500 steps, then 5,000 averaged steps; p, q
    and the averaged field within 1 % of the oracle's, tau_w (whose noise is the largest, about 1.1 % between
    two seeds over 3,000 steps) within 1.5 %."""
    case = wl.case_cylinder(ni=16, nj=24, h1=5e-3, r_out=3.0, Kn=0.1, Ma=5.0, n_ref=150)
    g = _run(cuda_lib.Solver(case, precision=0, use_graph=True, capacity=16 * case.n_ref * case.mesh.ncells), 1500,
             5000, field_every=5)
    o = _run(ob.Oracle(case, precision=0), 1500, 5000, field_every=5)
    _compare(g, o, 0.01, tau_bar=0.015)

"""The library's residual normalisation (no counterpart in the paper, which judges steady state by monitored
histories, Sec. V A): the raw residual sqrt(sum_i Omega_i ((W^{n+1} - W^n) / dt_i)^2) of each component over
a freestream scale that does not depend on the first step, so that starts whose first step leaves a component
(almost) unchanged keep a meaningful 1e-6 threshold."""
import math

import numpy as np

from oracle import binding as ob
from paper_2607_09552_b300 import workloads as wl


def _scale(case, vol):
    c = wl.freestream_speed(case.Ma) + math.sqrt(5.0 / 6.0)
    ra = math.sqrt(float(np.sum(vol)))
    return np.array([c, c * c, c * c, 0.5 * c ** 3]) * ra


def test_uniform_start_has_a_zero_finite_residual():
    """A uniform freestream between far-field ends does not move: the raw and the normalised residual are 0
    (a first-step normalisation would divide by zero here)."""
    m = wl.line_mesh(24, 0.0, 1.0, 4.0, bc_right=wl.BC_FARFIELD)
    case = wl.Case("uniform_line", m, Kn=0.1, Ma=5.0, Tw=1.0, cfl=0.8, n_ref=20)
    o = ob.Oracle(case, wave_only=True, precision=1)
    o.step(3)
    r = o.residual()
    assert np.all(np.isfinite(r))
    assert np.all(r == 0.0)


def test_plate_density_residual_is_not_blown_up_by_the_first_step():
    """Particle-free plate from the uniform freestream: the first step changes the density only through the
    rounding of the wall cells' fluxes, so a residual normalised by the first step reads about 1e10 later on.
    The freestream-scaled residual starts below 1e-6 in density, stays O(1) or less in every component, and
    the normalised values are the raw ones over the stated scale."""
    case = wl.case_plate(ni=24, nj=12, h1=1e-3, ratio=1.3)
    o = ob.Oracle(case, wave_only=True, precision=1)
    o.step(1)
    r1 = o.residual()
    S = _scale(case, o.geometry()[1])
    np.testing.assert_allclose(r1[:4] * S, r1[4:], rtol=1e-14, atol=0)
    assert r1[0] < 1e-6 * max(r1[1:4])
    hist = []
    for _ in range(20):
        o.step(5)
        hist.append(o.residual()[:4].copy())
    hist = np.array(hist)
    assert np.all(np.isfinite(hist))
    assert hist.max() < 10.0
    # the density residual grows from its first-step value as the flow develops, then stays O(1) at most
    assert hist[:, 0].max() > 1e3 * r1[0]


def test_normalised_residual_falls_on_the_particle_free_shock():
    """The particle-free 1-D shock settles under local time steps: the normalised residual falls by orders of
    magnitude."""
    case = wl.case_shock1d(ni=40, n_ref=20)
    o = ob.Oracle(case, wave_only=True, precision=1)
    o.step(1)
    r0 = float(o.residual()[:4].max())
    o.step(3000)
    r1 = float(o.residual()[:4].max())
    assert r1 < 1e-3 * r0

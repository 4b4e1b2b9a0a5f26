"""Pins of the Shakhov acceptance-rejection sampling (Eq. 4, Sec. III B) in the oracle.

With acceptance density proportional to phi(z) (1 + (a . z)(|z|^2 - 5)), phi the 3-D standard normal, the
heat-flux moment is E[z_x |z|^2 / 2] = a_x (E[z_x^2 |z|^4] - 5 E[z_x^2 |z|^2]) / 2 = a_x (35 - 25) / 2 = 5 a_x,
while the mean stays 0 and E[|z|^2] stays 3 (odd and orthogonal corrections): the sampled part carries the
Shakhov heat flux (1 - Pr) Q share the weights encode. a = 0 reproduces the Maxwellian proposals exactly."""
import numpy as np
import pytest

from oracle import binding as ob
from paper_2607_09552_b300 import workloads as wl


@pytest.mark.parametrize("prec", [0, 1])
def test_ar_heat_flux_moment(prec):
    n = 400000
    ax, ay = 0.012, -0.007
    M = 1.0 + 186.0 * np.hypot(ax, ay)
    z, fb = ob.ar_sample(prec, 11, 0, 3, 1 << 40, n, ax, ay, M)
    assert fb == 0
    s2 = np.sum(z * z, axis=1)
    hx, hy = np.mean(z[:, 0] * s2 / 2), np.mean(z[:, 1] * s2 / 2)
    se = np.std(z[:, 0] * s2 / 2) / np.sqrt(n)
    assert abs(hx - 5 * ax) < 5 * se and abs(hy - 5 * ay) < 5 * se, (hx, hy, se)
    assert np.all(np.abs(np.mean(z, axis=0)) < 5 / np.sqrt(n))
    assert abs(np.mean(s2) - 3.0) < 5 * np.std(s2) / np.sqrt(n)
    assert np.max(s2) <= 36.0


def test_ar_zero_weights_accept_every_first_proposal():
    z0, fb = ob.ar_sample(0, 5, 2, 7, 99, 1000, 0.0, 0.0, 1.0)
    z1, _ = ob.ar_sample(0, 5, 2, 7, 99, 1000, 0.0, 0.0, 1.0)
    assert fb == 0 and np.array_equal(z0, z1)
    # every accepted draw is a first-attempt proposal, unless truncated at |z| > 6
    assert np.all(np.sum(z0 * z0, axis=1) <= 36.0)


def test_ar_fallback_counted_when_rejection_is_certain():
    # psi <= -1 for every proposal in this direction band would reject; a huge M rejects almost all
    z, fb = ob.ar_sample(1, 1, 0, 0, 0, 200, 1e-3, 0.0, 1e12)
    assert fb == 200


def test_shakhov_shock_runs_and_counts():
    case = wl.case_shock1d(ni=40, n_ref=30)
    assert case.Pr != 1.0
    o = ob.Oracle(case, precision=1)
    o.step(5)
    st = o.stats()
    assert st[2] > 0 and 0 <= st[9] <= st[2] // 10
    W = o.field()[0]
    assert np.all(np.isfinite(W)) and np.all(W[:, 0] > 0)

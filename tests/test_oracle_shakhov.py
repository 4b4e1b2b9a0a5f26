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


def test_shakhov_weights_carry_the_heat_flux_of_the_retained_particles():
    """The weights of each sampling cell against Eq. 5 evaluated directly: Q = (1 / (2 Omega_i)) sum m c |c|^2
    over the particles retained in the cell at the start of the step, c = u - U_i with U_i the cell's (total)
    velocity; a = (1 - Pr) Q / (5 rho_i (R T^h)^(3/2)), M = 1 + 6 * 31 |a| (reading of Sec. III B). The
    oracle forms Q from fixed-point raw moments (sums of m, m u, m u u, m u |u|^2, ...) expanded about U_i; the
    expansion cancels digits of those sums (upstream U_i / sqrt(R T_i) is about 3), so the bar is 2e-9 of the
    largest weight (measured 4e-10)."""
    case = wl.case_shock1d(ni=40, n_ref=60)
    o = ob.Oracle(case, precision=1)
    o.step(30)
    W0, _ = o.field()
    P = o.particles()
    _, vol = o.geometry()
    o.step(1)
    hq = o.shakhov_weights()
    cd = o.cell_data()
    rho = W0[:, 0]
    U = W0[:, 1] / rho
    c = P["cell"]
    cu = P["u"] - U[c]
    c2 = cu * cu + P["v"] ** 2 + P["w"] ** 2
    Q = np.bincount(c, weights=P["m"] * cu * c2, minlength=o.C) / (2.0 * vol)
    RTh = cd[:, 7]
    sampled = cd[:, 3] > 0
    assert sampled.sum() > 30
    with np.errstate(divide="ignore", invalid="ignore"):
        ax = (1.0 - case.Pr) * Q / (5.0 * rho * RTh ** 1.5)
    scale = np.abs(ax[sampled]).max()
    assert scale > 1e-4                                           # a shock: heat flux present
    np.testing.assert_allclose(hq[sampled, 0], ax[sampled], rtol=1e-8, atol=2e-9 * scale)
    np.testing.assert_array_equal(hq[sampled, 1], 0.0)            # 1-D: no Q_y
    np.testing.assert_allclose(hq[sampled, 2], 1.0 + 186.0 * np.abs(ax[sampled]), rtol=1e-8)

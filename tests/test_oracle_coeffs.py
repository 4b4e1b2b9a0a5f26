"""Pins of the normalised time-integration coefficients (Eq. 16 divided by dt, Eq. 48) against a
50-digit evaluation of Eq. 16, their limits and the GTS identity dt * dbar = delta (Sec. IV B)."""
import mpmath
import numpy as np
import pytest

from oracle import binding as ob

mpmath.mp.dps = 50


def delta_exact(dt, tau):
    """Eq. 16 with (dt, tau), 50 digits."""
    dt, tau = mpmath.mpf(dt), mpmath.mpf(tau)
    e = mpmath.exp(-dt / tau)
    da = dt - tau * (1 - e)
    db = 2 * tau ** 2 * (1 - e) - tau * dt - tau * dt * e
    dc = dt ** 2 / 2 - tau * dt + tau ** 2 * (1 - e)
    dd = tau * (1 - e)
    de = tau * dt * e - tau ** 2 * (1 - e)
    return [da, db, dc, dd, de], e


@pytest.mark.parametrize("x", list(np.logspace(-8, 3, 45)) + [0.999, 1.0, 1.001])
@pytest.mark.parametrize("dt", [1e-4, 0.37])
def test_normalised_coefficients_match_50_digits(x, dt):
    tau = dt / x
    got = ob.coeffs(dt, tau)
    d, e = delta_exact(dt, tau)
    ref = [v / mpmath.mpf(dt) for v in d]
    ref += [ref[3] - e, ref[4] + mpmath.mpf(dt) / 2 * e]
    for k in range(7):
        r = float(ref[k])
        assert abs(got[k] - r) <= 1e-13 * abs(r) + 1e-300, (k, x, got[k], r)


def test_limits():
    dt = 0.01
    # dt/tau -> infinity (e^{-x} below the double range): the GKS coefficients of Eq. 16 with e = 0,
    # dbar_a = 1 - tau/dt, dbar_b = 2 tau^2/dt - tau, dbar_c = dt/2 - tau + tau^2/dt, dbar_d = tau/dt
    tau = dt / 2000.0
    c = ob.coeffs(dt, tau)
    assert c[0] == pytest.approx(1 - tau / dt, rel=1e-14)
    assert c[1] == pytest.approx(2 * tau ** 2 / dt - tau, rel=1e-14)
    assert c[2] == pytest.approx(dt / 2 - tau + tau ** 2 / dt, rel=1e-14)
    assert c[3] == pytest.approx(tau / dt, rel=1e-14)
    assert c[5] == pytest.approx(tau / dt, rel=1e-14)
    # dt/tau -> 0: free transport, dbar_a ~ x/2, dbar_d ~ 1 - x/2, dbar_d - e^-x ~ x/2
    x = 1e-7
    c = ob.coeffs(dt, dt / x)
    assert c[0] == pytest.approx(x / 2, rel=1e-6)
    assert c[3] == pytest.approx(1 - x / 2, rel=1e-12)
    assert c[5] == pytest.approx(x / 2, rel=1e-6)


def test_gts_identity():
    """With dt_L = dt_R = dt_G, dt_G * dbar = delta of Eq. 16 (the LTS form reduces to GTS)."""
    for x in (1e-3, 0.5, 3.0, 40.0):
        dt = 0.2
        tau = dt / x
        d, _ = delta_exact(dt, tau)
        c = ob.coeffs(dt, tau)
        for k in range(5):
            assert dt * c[k] == pytest.approx(float(d[k]), rel=1e-13, abs=1e-300)

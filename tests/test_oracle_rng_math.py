"""Pins of the oracle's Philox stream and its deterministic elementary functions (test infrastructure)."""
import math
import os

import numpy as np
import pytest

from oracle import binding as ob

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    for line in open(os.path.join(GOLD, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(t, 16) for t in line.split()]
        assert ob.philox(w[0:4], w[4:6]) == w[6:10]


def _ulp_err32(got, ref):
    got = np.asarray(got, dtype=np.float32)
    refr = np.asarray(ref, dtype=np.float64)
    return np.abs(got.astype(np.float64) - refr) / np.spacing(np.abs(refr).astype(np.float32)).astype(np.float64)


def test_logf_within_two_ulp():
    L = ob.lib()
    rng = np.random.default_rng(1)
    xs = np.concatenate([rng.uniform(0, 1, 20000), np.exp(rng.uniform(-80, 80, 20000)),
                         ((np.arange(2000) + 0.5) * 2.0 ** -23)]).astype(np.float32)
    got = np.array([L.oracle_logf(float(x)) for x in xs], dtype=np.float32)
    ref = np.log(xs.astype(np.float64))
    err = np.abs(got.astype(np.float64) - ref)
    tol = 2.0 * np.maximum(np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64), 2.0 ** -149)
    # near x = 1 the result is tiny; compare against the scale of the argument reduction error there
    tol = np.maximum(tol, 2.0 ** -24 * np.abs(xs.astype(np.float64) - 1.0))
    assert np.all(err <= tol), (xs[err > tol][:5], got[err > tol][:5], ref[err > tol][:5])


def test_logd_expd_within_two_ulp():
    L = ob.lib()
    rng = np.random.default_rng(2)
    xs = np.concatenate([rng.uniform(1e-300, 1, 5000), np.exp(rng.uniform(-700, 700, 5000))])
    for x in xs:
        r = math.log(x)
        g = L.oracle_logd(float(x))
        assert abs(g - r) <= 2 * math.ulp(r) + 2 ** -53 * abs(x - 1.0), (x, g, r)
    ys = np.concatenate([rng.uniform(-700, 700, 5000), rng.uniform(-1, 1, 5000)])
    for y in ys:
        r = math.exp(y)
        g = L.oracle_expd(float(y))
        assert abs(g - r) <= 2 * math.ulp(r), (y, g, r)
    assert L.oracle_expd(-709.0) == 0.0
    assert L.oracle_expd(0.0) == 1.0


def test_expf_within_two_ulp():
    """Float e^x (production decomposition: e^{-dt/tau} and T^omega) against the double-precision exponential,
    over the arguments the method meets (-87 .. 8), with 0 below -87."""
    L = ob.lib()
    rng = np.random.default_rng(4)
    xs = np.concatenate([rng.uniform(-87.0, 8.0, 20000), rng.uniform(-1.0, 1.0, 5000),
                         -np.exp(rng.uniform(-20.0, 0.0, 5000))]).astype(np.float32)
    got = np.array([L.oracle_expf(float(x)) for x in xs], dtype=np.float32)
    ref = np.exp(xs.astype(np.float64))
    err = np.abs(got.astype(np.float64) - ref)
    tol = 2.0 * np.maximum(np.spacing(ref.astype(np.float32)).astype(np.float64), 2.0 ** -149)
    assert np.all(err <= tol), (xs[err > tol][:5], got[err > tol][:5], ref[err > tol][:5])
    assert L.oracle_expf(-87.5) == 0.0 and L.oracle_expf(0.0) == 1.0


def test_sincos2pi_float_and_double():
    rng = np.random.default_rng(3)
    us = ((rng.integers(0, 2 ** 23, 20000) + 0.5) * 2.0 ** -23).astype(np.float32)
    for u in us[:5000]:
        s, c = ob.sincos2pif(float(u))
        assert abs(s - math.sin(2 * math.pi * float(u))) <= 3e-7
        assert abs(c - math.cos(2 * math.pi * float(u))) <= 3e-7
    import mpmath
    mpmath.mp.dps = 40
    for u in rng.uniform(0, 1, 3000):
        s, c = ob.sincos2pid(float(u))
        a = 2 * mpmath.pi * mpmath.mpf(float(u))
        assert abs(s - float(mpmath.sin(a))) <= 3e-16
        assert abs(c - float(mpmath.cos(a))) <= 3e-16




def test_erfcd_against_multiprecision():
    """FP64 erfc of the wave flux's half-range moments (series of A&S 7.1.6 below 3/2, Laplace's continued
    fraction A&S 7.1.14 above) against 40-digit mpmath over [-6, 27]: within 2e-14 relative where e^{-x^2} is
    at least 1e-30 (the rounding of x^2 sets a floor of about x^2 ulp beyond that, checked at 1e-13), with
    erfc(-x) = 2 - erfc(x), erfc(0) = 1 and 0 where e^{-x^2} is flushed (x^2 > 708, as the exponential)."""
    import mpmath
    mpmath.mp.dps = 40
    L = ob.lib()
    xs = np.concatenate([np.linspace(-6.0, 6.0, 2401), np.linspace(6.0, 27.0, 211), [1.5 - 2 ** -40, 1.5]])
    for x in xs:
        x = float(x)
        ref = float(mpmath.erfc(mpmath.mpf(x)))
        g = L.oracle_erfcd(x)
        if x * x > 708.0:
            assert g == 0.0, x
            continue
        bar = 2e-14 if x * x < 69.0 else 1e-13
        assert abs(g - ref) <= bar * ref, (x, g, ref)
        if x > 0:
            assert L.oracle_erfcd(-x) == 2.0 - g
    assert L.oracle_erfcd(0.0) == 1.0
    assert L.oracle_erfcd(30.0) == 0.0
    assert L.oracle_erfcd(-30.0) == 2.0

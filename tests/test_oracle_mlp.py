"""Pins of the warm-start network oracle (oracle/mlp.py) against things other than itself: central finite
differences in float64, torch's CPU autograd of the same network, closed forms of the feature map and of
Adam's first step, and the bfloat16 rounding of torch's own conversion."""
import numpy as np
import pytest
import torch

from oracle import mlp as om
from paper_2607_09552_b300 import workloads as wl

FMAP = dict(cx=0.0, cy=0.0, ell=0.5, ext=20.0, kn_lo=0.005, kn_hi=0.2, ma_lo=5.0, ma_hi=15.0, tw_lo=1.0, tw_hi=5.0)


def _small(seed=3, F=8, H=6, D=2, n=11):
    rng = np.random.default_rng(seed)
    p = rng.normal(0.0, 0.7, om.n_params(F, H, D))
    X = rng.normal(0.0, 1.0, (n, F))
    T = rng.normal(0.0, 1.0, (n, 4))
    return p, X, T, F, H, D


def test_gradient_matches_central_differences():
    p, X, T, F, H, D = _small()
    _, g = om.loss_and_grad(p, X, T, F, H, D, bf16=False)
    h = 1e-6
    fd = np.zeros_like(p)
    for i in range(p.size):
        a, b = p.copy(), p.copy()
        a[i] += h
        b[i] -= h
        fd[i] = (om.loss_and_grad(a, X, T, F, H, D, bf16=False)[0] - om.loss_and_grad(b, X, T, F, H, D, bf16=False)[0]) / (2 * h)
    assert np.max(np.abs(fd - g)) <= 1e-6 * max(1.0, np.max(np.abs(g)))


def test_gradient_matches_torch_autograd():
    p, X, T, F, H, D = _small(seed=5, F=40, H=16, D=3, n=23)
    loss, g = om.loss_and_grad(p, X, T, F, H, D, bf16=False)
    pt = torch.tensor(p, dtype=torch.float64, requires_grad=True)
    off = 0
    Ws, bs = [], []
    for i, o in om.layer_shapes(F, H, D):
        Ws.append(pt[off:off + i * o].reshape(o, i))
        off += i * o
    for i, o in om.layer_shapes(F, H, D):
        bs.append(pt[off:off + o])
        off += o
    a = torch.tensor(X)
    for l in range(D + 1):
        z = torch.nn.functional.linear(a, Ws[l], bs[l])
        a = torch.nn.functional.silu(z) if l < D else z
    lt = torch.mean((a - torch.tensor(T)) ** 2)
    lt.backward()
    assert abs(lt.item() - loss) <= 1e-14 * abs(loss)
    np.testing.assert_allclose(g, pt.grad.numpy(), rtol=1e-12, atol=1e-13 * np.max(np.abs(g)))


def test_bf16_rounding_matches_torch_and_ties_to_even():
    rng = np.random.default_rng(0)
    x = (rng.normal(size=4000) * 10.0 ** rng.uniform(-6, 6, 4000)).astype(np.float32)
    ref = torch.tensor(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(om.bf16_round(x), ref)
    # 1 + 2^-8 lies half-way between 1 and 1 + 2^-7: ties to the even mantissa (1); 1 + 3 * 2^-8 -> 1 + 2^-6
    assert om.bf16_round(np.float32(1.0 + 2.0 ** -8)) == 1.0
    assert om.bf16_round(np.float32(1.0 + 3 * 2.0 ** -8)) == 1.0 + 2.0 ** -6


def test_silu_derivative_closed_form():
    assert om.silu_grad(np.array([0.0]))[0] == 0.5
    z = np.linspace(-8, 8, 101)
    h = 1e-6
    np.testing.assert_allclose(om.silu_grad(z), (om.silu(z + h) - om.silu(z - h)) / (2 * h), atol=1e-8)


def test_adam_first_step_moves_by_lr_against_the_gradient_sign():
    rng = np.random.default_rng(1)
    p = rng.normal(size=50)
    g = rng.normal(size=50)
    p1, m, v = om.adam(p, g, np.zeros(50), np.zeros(50), 1, lr=1e-3, eps=0.0)
    np.testing.assert_allclose(p1, p - 1e-3 * np.sign(g), rtol=0, atol=1e-15)


def test_feature_map_closed_forms():
    # x = cx, y = cy: x^ = y^ = 0, so every sine is 0 and every cosine 1
    f = om.features(np.array([0.0]), np.array([0.0]), 0.005, 15.0, 3.0, FMAP)[0]
    assert np.all(f[0:8] == 0) and np.all(f[8:16] == 1) and np.all(f[16:24] == 0) and np.all(f[24:32] == 1)
    assert f[32] == 0 and f[33] == 0
    assert f[34] == -1.0 and f[35] == 1.0 and f[36] == 0.0
    assert np.all(f[37:] == 0)
    # x = cx + ext: x^ = 1, sin(2^k pi) = 0, cos(pi) = -1, cos(2^k pi) = 1 for k >= 1
    f = om.features(np.array([20.0]), np.array([-20.0]), 0.2, 5.0, 1.0, FMAP)[0]
    np.testing.assert_allclose(f[0:8], 0.0, atol=1e-12)
    np.testing.assert_allclose(f[8:16], [-1] + [1] * 7, atol=1e-12)
    np.testing.assert_allclose(f[32:37], [1.0, -1.0, 1.0, -1.0, -1.0], atol=1e-15)
    # the map is odd and monotone
    x = np.linspace(-20, 20, 41)
    xh = om.coord_map(x, 0.0, 0.5, 20.0)
    assert np.all(np.diff(xh) > 0)
    np.testing.assert_allclose(xh, -xh[::-1], atol=1e-15)


def test_targets_and_field_round_trip():
    rng = np.random.default_rng(2)
    n = 100
    rho = rng.uniform(0.1, 5, n)
    u, v = rng.uniform(-4, 4, n), rng.uniform(-4, 4, n)
    T = rng.uniform(0.5, 20, n)
    W = np.stack([rho, rho * u, rho * v, rho * (0.5 * (u * u + v * v) + 1.5 * 0.5 * T)], axis=1)
    Y = om.targets_from_W(W, U_inf=4.5644)
    prim = om.field_from_outputs(Y, 4.5644, 0.01, 100.0, 100.0)
    np.testing.assert_allclose(prim, np.stack([rho, u, v, T], axis=1), rtol=1e-12)


def test_loss_is_zero_on_exact_targets_and_init_layout():
    p = wl.mlp_init(0, 64, 32, 2)
    assert p.dtype == np.float32 and p.size == om.n_params(64, 32, 2)
    Ws, bs = om.unpack(p.astype(np.float64), 64, 32, 2)
    assert all(np.all(b == 0) for b in bs)
    assert np.max(np.abs(Ws[0])) <= np.sqrt(6 / 64)
    X = np.random.default_rng(0).normal(size=(9, 64))
    Y = om.forward(p, X, 64, 32, 2)
    loss, g = om.loss_and_grad(p, X, Y, 64, 32, 2)
    assert loss == 0.0 and np.all(g == 0)

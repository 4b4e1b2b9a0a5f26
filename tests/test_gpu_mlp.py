"""GPU parity of the warm-start network kernels against the float64 oracle (oracle/mlp.py), and the warm
start's effect on the steady iteration.

Tolerances: the GPU uses the same BF16-rounded weights as the oracle; its tensor-core products take each
FP32 activation or gradient as two BF16 terms (relative error below 2^-17) and accumulate in FP32 (at most
256-term dot products forward, up to 4096-point sums in the weight gradients), so outputs agree to about
1e-5 relative and gradients per tensor to about 1e-5; the bars below are 1e-4.
Features are computed in float64 and rounded once to float32 (1e-6 absolute bar)."""
import numpy as np
import pytest

from oracle import mlp as om
from paper_2607_09552_b300 import workloads as wl

pytestmark = pytest.mark.gpu

FMAP = dict(cx=0.0, cy=0.0, ell=0.5, ext=20.0, kn_lo=0.005, kn_hi=0.2, ma_lo=5.0, ma_hi=15.0, tw_lo=1.0, tw_hi=5.0)


def _torch():
    import torch
    return torch


def _centroids(mesh):
    """Area-weighted centroids of the quadrilaterals (split along the 0-2 diagonal)."""
    ni, nj = mesh.ni, mesh.nj
    xv, yv = mesh.xv.reshape(nj + 1, ni + 1), mesh.yv.reshape(nj + 1, ni + 1)
    X = [xv[:-1, :-1], xv[:-1, 1:], xv[1:, 1:], xv[1:, :-1]]
    Y = [yv[:-1, :-1], yv[:-1, 1:], yv[1:, 1:], yv[1:, :-1]]

    def area(a, b, c):
        return 0.5 * ((X[b] - X[a]) * (Y[c] - Y[a]) - (X[c] - X[a]) * (Y[b] - Y[a]))
    A1, A2 = area(0, 1, 2), area(0, 2, 3)
    xc = (A1 * (X[0] + X[1] + X[2]) + A2 * (X[0] + X[2] + X[3])) / (3 * (A1 + A2))
    yc = (A1 * (Y[0] + Y[1] + Y[2]) + A2 * (Y[0] + Y[2] + Y[3])) / (3 * (A1 + A2))
    return xc.reshape(-1), yc.reshape(-1)


def _close_by_column(a, b, rtol, col_atol):
    """|a - b| <= rtol |b| + col_atol * max |b[:, k]| in every column k."""
    for k in range(b.shape[1]):
        np.testing.assert_allclose(a[:, k], b[:, k], rtol=rtol, atol=col_atol * float(np.abs(b[:, k]).max()))


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_features_match_oracle(cuda_lib):
    torch = _torch()
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(-20, 20, 3000), rng.uniform(-0.6, 0.6, 1000), [0.0, 20.0, -20.0]])
    y = np.concatenate([rng.uniform(-20, 20, 3000), rng.uniform(-0.6, 0.6, 1000), [0.0, -20.0, 0.5]])
    f = cuda_lib.mlp_features(FMAP, torch.tensor(x, device="cuda"), torch.tensor(y, device="cuda"), 0.03, 7.5, 2.5)
    ref = om.features(x, y, 0.03, 7.5, 2.5, FMAP)
    assert np.max(np.abs(f.cpu().numpy() - ref)) <= 1e-6


@pytest.mark.parametrize("n", [1, 77, 4100])
def test_forward_matches_oracle(cuda_lib, n):
    torch = _torch()
    p = wl.mlp_init(3)
    net = cuda_lib.Mlp(params=p)
    X = np.random.default_rng(n).normal(size=(n, 64)).astype(np.float32)
    y = net.forward(torch.tensor(X, device="cuda")).cpu().numpy()
    ref = om.forward(p, X, 64, 256, 4)
    assert _rel(y, ref) <= 1e-4, _rel(y, ref)
    np.testing.assert_allclose(y, ref, atol=1e-4 * np.max(np.abs(ref)))


@pytest.mark.parametrize("n", [64, 1000, 4096])
def test_gradient_matches_oracle(cuda_lib, n):
    torch = _torch()
    rng = np.random.default_rng(7 + n)
    p = wl.mlp_init(5)
    # a non-zero bias state so that every bias gradient is exercised
    p[-(3 * 256 + 4 + 256):] = rng.normal(0, 0.1, 3 * 256 + 4 + 256).astype(np.float32)
    net = cuda_lib.Mlp(params=p)
    X = rng.normal(size=(n, 64)).astype(np.float32)
    T = rng.normal(size=(n, 4)).astype(np.float32)
    loss = net.loss_grad(torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda"))
    g = net.grad()
    lref, gref = om.loss_and_grad(p, X, T, 64, 256, 4)
    assert abs(loss - lref) <= 1e-5 * lref
    Ws, bs = om.unpack(g.astype(np.float64), 64, 256, 4)
    Wr, br = om.unpack(gref, 64, 256, 4)
    for a, b in zip(Ws + bs, Wr + br):
        assert _rel(a, b) <= 1e-4, _rel(a, b)


@pytest.mark.parametrize("shape,n", [((37, 48, 2, 4), 300), ((45, 72, 3, 4), 1031)])
def test_ragged_shapes_match_oracle(cuda_lib, shape, n):
    """Inputs, widths and point counts off the 16-deep contraction steps and the 64 x 64 output tiles: the
    zero padding of partial tiles and the guarded epilogues, forward and every gradient."""
    torch = _torch()
    nf, width, depth, n_out = shape
    rng = np.random.default_rng(n)
    p = wl.mlp_init(11, nf, width, depth, n_out)
    nb = depth * width + n_out
    p[-nb:] = rng.normal(0, 0.1, nb).astype(np.float32)
    net = cuda_lib.Mlp(nf, width, depth, n_out, params=p)
    X = rng.normal(size=(n, nf)).astype(np.float32)
    T = rng.normal(size=(n, n_out)).astype(np.float32)
    y = net.forward(torch.tensor(X, device="cuda")).cpu().numpy()
    ref = om.forward(p, X, nf, width, depth)
    assert y.shape == ref.shape
    assert _rel(y, ref) <= 1e-4, _rel(y, ref)
    loss = net.loss_grad(torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda"))
    lref, gref = om.loss_and_grad(p, X, T, nf, width, depth)
    assert abs(loss - lref) <= 1e-5 * lref
    Ws, bs = om.unpack(net.grad().astype(np.float64), nf, width, depth)
    Wr, br = om.unpack(gref, nf, width, depth)
    for a, b in zip(Ws + bs, Wr + br):
        assert _rel(a, b) <= 1e-4, _rel(a, b)


def test_row_indexed_gradient_equals_gathered_rows(cuda_lib):
    torch = _torch()
    rng = np.random.default_rng(11)
    p = wl.mlp_init(9)
    X = rng.normal(size=(3000, 64)).astype(np.float32)
    T = rng.normal(size=(3000, 4)).astype(np.float32)
    rows = rng.permutation(3000)[:1111].astype(np.int32)
    a = cuda_lib.Mlp(params=p)
    la = a.loss_grad(torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda"), torch.tensor(rows, device="cuda"))
    b = cuda_lib.Mlp(params=p)
    lb = b.loss_grad(torch.tensor(X[rows], device="cuda"), torch.tensor(T[rows], device="cuda"))
    assert la == lb
    assert np.array_equal(a.grad(), b.grad())


def test_adam_steps_match_oracle(cuda_lib):
    torch = _torch()
    rng = np.random.default_rng(4)
    p = wl.mlp_init(2)
    net = cuda_lib.Mlp(params=p)
    X = torch.tensor(rng.normal(size=(500, 64)).astype(np.float32), device="cuda")
    T = torch.tensor(rng.normal(size=(500, 4)).astype(np.float32), device="cuda")
    pr = p.astype(np.float64)
    m = np.zeros_like(pr)
    v = np.zeros_like(pr)
    for t in range(1, 4):
        net.loss_grad(X, T)
        g = net.grad().astype(np.float64)
        net.adam(1e-3)
        pr, m, v = om.adam(pr, g, m, v, t, 1e-3)
        got = net.params().astype(np.float64)
        # FP32 master weights: the step itself is exact to FP32 rounding of each parameter
        assert np.max(np.abs(got - pr)) <= 2e-6 * max(1.0, np.max(np.abs(pr)))
        pr = got  # continue from the GPU's rounded state


def test_training_lowers_the_loss(cuda_lib):
    torch = _torch()
    from paper_2607_09552_b300 import warmstart as ws
    rng = np.random.default_rng(8)
    x, y = rng.uniform(-3, 3, 20000), rng.uniform(-3, 3, 20000)
    r = np.sqrt(x * x + y * y)
    target = np.stack([np.log(1 + 3 * np.exp(-r)), np.tanh(x), 0.3 * np.sin(y), np.exp(-0.5 * r)], axis=1)
    feats = cuda_lib.mlp_features(FMAP, torch.tensor(x, device="cuda"), torch.tensor(y, device="cuda"), 0.05, 8, 2)
    targs = torch.tensor(target.astype(np.float32), device="cuda")
    net = ws.new_network(0)
    hist = ws.train(net, feats, targs, steps=600, batch=2048, lr=2e-3, log_every=100)
    assert hist[-1][1] < 0.05 * hist[0][1], hist


def test_dataset_rows_match_oracle(cuda_lib):
    torch = _torch()
    case = wl.case_cylinder(12, 16, 0.02, 6.0, Kn=0.05, Ma=6.0, Tw=2.0, n_ref=10)
    s = cuda_lib.Solver(case, precision=0, wave_only=True)
    s.step(5)
    W = s.field()[0]
    feat, targ = s.dataset(FMAP)
    xc, yc = _centroids(case.mesh)
    assert np.max(np.abs(feat.cpu().numpy() - om.features(xc, yc, 0.05, 6.0, 2.0, FMAP))) <= 1e-6
    U = wl.freestream_speed(6.0)
    np.testing.assert_allclose(targ.cpu().numpy(), om.targets_from_W(W, U), rtol=1e-6, atol=1e-6)
    # a time average accumulated on the device
    acc = torch.zeros(4 * s.C, dtype=torch.float64, device="cuda")
    snaps = []
    for k in range(3):
        s.step(1)
        s.field_accumulate(acc, reset=(k == 0))
        snaps.append(s.field()[0])
    np.testing.assert_allclose(acc.cpu().numpy().reshape(-1, 4), np.sum(snaps, axis=0), rtol=1e-15)
    _, targ2 = s.dataset(FMAP, acc, 1.0 / 3.0)
    np.testing.assert_allclose(targ2.cpu().numpy(), om.targets_from_W(np.mean(snaps, axis=0), U), rtol=1e-6, atol=1e-6)


def test_warm_start_sets_the_network_field(cuda_lib):
    case = wl.case_cylinder(12, 16, 0.02, 6.0, Kn=0.05, Ma=6.0, Tw=2.0, n_ref=10)
    p = wl.mlp_init(1)
    p[-4:] = np.array([0.3, 0.5, -0.1, 0.2], dtype=np.float32)   # output biases: a non-trivial field
    net = cuda_lib.Mlp(params=p)
    s = cuda_lib.Solver(case, precision=0)
    s.warm_start(net, FMAP)
    W, Wp = s.field()
    assert s.num_particles() == 0 and np.all(Wp == 0)
    xc, yc = _centroids(case.mesh)
    Y = om.forward(p, om.features(xc, yc, 0.05, 6.0, 2.0, FMAP), 64, 256, 4)
    U = wl.freestream_speed(6.0)
    T_cap = 10 * max(1 + 6.0 ** 2 / 3, 2.0, 1.0)
    T_min = 0.01 * min(1.0, 2.0, 1.0)
    U_cap = U + 10 * np.sqrt(0.5 * T_cap)
    prim = om.field_from_outputs(Y, U, 2 * T_min, T_cap / 2, U_cap / 2)
    Wref = np.stack([prim[:, 0], prim[:, 0] * prim[:, 1], prim[:, 0] * prim[:, 2],
                     prim[:, 0] * (0.5 * (prim[:, 1] ** 2 + prim[:, 2] ** 2) + 0.75 * prim[:, 3])], axis=1)
    _close_by_column(W, Wref, 2e-4, 2e-4)
    # clipping: a huge log T output is held at T_cap / 2
    p[-1] = 60.0
    net.set_params(p)
    s.warm_start(net, FMAP)
    W = s.field()[0]
    rho = W[:, 0]
    T = (W[:, 3] / rho - 0.5 * ((W[:, 1] / rho) ** 2 + (W[:, 2] / rho) ** 2)) / 0.75
    np.testing.assert_allclose(T, T_cap / 2, rtol=1e-12)
    s.step(3)   # the method runs from the warm field


def test_warm_start_leaves_the_converged_state_unchanged(cuda_lib):
    """Particle-free mode (deterministic, all FP64): from the freestream and from an (untrained, arbitrary)
    network field, the iteration converges to the same steady state."""
    from paper_2607_09552_b300 import steady
    case = wl.case_cylinder(16, 24, 0.02, 6.0, Kn=0.05, Ma=5.0, Tw=1.0, n_ref=10)
    ref = steady.first_residual(case, precision=1, wave_only=True)
    a = cuda_lib.Solver(case, precision=1, wave_only=True, use_graph=True)
    ra = steady.run_to_residual(a, 1e-9, 400000, 500, ref)
    p = wl.mlp_init(4)
    p[-4:] = np.array([0.2, 0.3, 0.05, 0.3], dtype=np.float32)
    b = cuda_lib.Solver(case, precision=1, wave_only=True, use_graph=True)
    b.warm_start(cuda_lib.Mlp(params=p), FMAP)
    rb = steady.run_to_residual(b, 1e-9, 400000, 500, ref)
    assert ra["converged"] and rb["converged"], (ra, rb)
    Wa, Wb = a.field()[0], b.field()[0]
    _close_by_column(Wb, Wa, 1e-6, 1e-8)


def test_trained_network_reaches_steady_state_in_fewer_steps(cuda_lib):
    """Train on the converged particle-free fields of four small-cylinder cases, then start a held-out case
    from the network: it reaches a 1e-6 residual (relative to the freestream start's first step; all FP64)
    in fewer steps than the freestream start, at the same converged state."""
    from paper_2607_09552_b300 import steady
    from paper_2607_09552_b300 import warmstart as ws
    train_conds = [(0.01, 6.0, 1.0), (0.1, 12.0, 3.0), (0.03, 9.0, 4.5), (0.15, 7.0, 2.0)]
    held = (0.05, 8.0, 2.5)
    mk = lambda kn, ma, tw: wl.case_cylinder(16, 24, 0.02, 6.0, Kn=kn, Ma=ma, Tw=tw, n_ref=10)
    ts = ws.TrainingSet()
    for kn, ma, tw in train_conds:
        s = cuda_lib.Solver(mk(kn, ma, tw), precision=1, wave_only=True, use_graph=True)
        steady.run_to_residual(s, 1e-7, 400000, 500)
        ts.add(s, FMAP)
    feats, targs = ts.tensors()
    net = ws.new_network(0)
    hist = ws.train(net, feats, targs, steps=1500, batch=512, lr=2e-3, log_every=500)
    case = mk(*held)
    ref = steady.first_residual(case, precision=1, wave_only=True)
    cold = cuda_lib.Solver(case, precision=1, wave_only=True, use_graph=True)
    rc = steady.run_to_residual(cold, 1e-6, 400000, 100, ref)
    warm = cuda_lib.Solver(case, precision=1, wave_only=True, use_graph=True)
    warm.warm_start(net, FMAP)
    rw = steady.run_to_residual(warm, 1e-6, 400000, 100, ref)
    assert rc["converged"] and rw["converged"], (rc, rw)
    assert rw["steps"] < rc["steps"], (rw, rc, hist)
    Wc, Ww = cold.field()[0], warm.field()[0]
    _close_by_column(Ww, Wc, 1e-3, 1e-5)

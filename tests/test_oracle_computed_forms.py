"""The oracle's computed forms of two per-particle decisions, pinned against their definitions.

Sec. III B / IV B (Eq. 27 with the local step): a retained particle's free-flight time is
t_f = min(-tau_i ln eps, dt_i), and it collides when t_f < dt_i. The oracle (and the kernels) decide the
collision as eps > e^{-dt_i/tau_i} in the particle precision and take the logarithm only for the colliding
particles. Eq. 28: a particle that does not collide moves x + u t_f; the oracle decides that it stays in its
cell by tr (n_k . u) <= d_k - n_k . x for the faces ahead, before any exit time is formed.

Here both decisions are taken again from their definitions, in float64 with libm's logarithm, for every
retained particle of 100 steps of a closed box of stretched rectangular cells (about 1e7 particle-steps),
and compared with what the oracle did (a collided particle is removed: the box has no exits; a particle that
stayed keeps its cell and velocity and sits at x + u dt_i). Disagreements are allowed only inside a stated
rounding band around the decision boundary, and their number is bounded."""
import numpy as np
import pytest

from oracle import binding as ob
from paper_2607_09552_b300 import workloads as wl

M0, M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
W0, W1 = np.uint32(0x9E3779B9), np.uint32(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)


def philox_np(c0, c1, c2, c3, k0, k1):
    """Philox4x32-10 (Salmon et al., SC'11) on arrays of counters, from its published definition."""
    c = [np.asarray(x, dtype=np.uint32).copy() for x in (c0, c1, c2, c3)]
    k0, k1 = np.uint32(k0), np.uint32(k1)
    for r in range(10):
        if r > 0:
            k0 = np.uint32((int(k0) + int(W0)) & 0xFFFFFFFF)
            k1 = np.uint32((int(k1) + int(W1)) & 0xFFFFFFFF)
        p0 = M0 * c[0].astype(np.uint64)
        p1 = M1 * c[2].astype(np.uint64)
        hi0, lo0 = (p0 >> np.uint64(32)).astype(np.uint32), (p0 & MASK).astype(np.uint32)
        hi1, lo1 = (p1 >> np.uint64(32)).astype(np.uint32), (p1 & MASK).astype(np.uint32)
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return c


def test_numpy_philox_matches_the_oracle():
    rng = np.random.default_rng(3)
    ctr = rng.integers(0, 2 ** 32, size=(20, 4), dtype=np.uint64).astype(np.uint32)
    key = (0x12345678, 0x9ABCDEF0)
    out = philox_np(ctr[:, 0], ctr[:, 1], ctr[:, 2], ctr[:, 3], *key)
    for i in range(20):
        assert [int(o[i]) for o in out] == ob.philox([int(v) for v in ctr[i]], list(key))


def _box_case():
    # closed box of rectangles, stretched in y (cell heights 0.004 ... 0.07): local steps vary about 17x
    m = wl.plate_mesh(ni=16, nj=24, h1=4e-3, ratio=1.13)
    for a in (m.bc_imin, m.bc_imax, m.bc_jmin, m.bc_jmax):
        a[:] = wl.BC_WALL
    return wl.Case("closed_box", m, Kn=0.02, Ma=0.0, Tw=1.0, cfl=0.8, n_ref=260)


@pytest.mark.slow
def test_collision_and_stay_decisions_match_their_definitions():
    case = _box_case()
    m = case.mesh
    o = ob.Oracle(case, precision=0)
    dt, vol = o.geometry()
    xs = m.xv.reshape(m.nj + 1, m.ni + 1)[0]
    ys = m.yv.reshape(m.nj + 1, m.ni + 1)[:, 0]
    ci = np.arange(m.ncells)
    xa, xb = xs[ci % m.ni], xs[ci % m.ni + 1]
    ya, yb = ys[ci // m.ni], ys[ci // m.ni + 1]
    o.step(5)
    n_draws = n_stay_checked = 0
    col_dis = col_band = stay_dis = stay_band = 0
    while n_draws < 10_000_000:
        step = int(o.stats()[0])
        P0 = o.particles()
        o.step(1)
        cd = o.cell_data()
        tau, emx = cd[:, 0], cd[:, 2]
        P1 = o.particles()
        # the collision decision
        pid = P0["pid"]
        w = philox_np(pid & 0xFFFFFFFF, pid >> np.uint64(32), np.full(pid.size, step, np.uint32),
                      np.full(pid.size, 5, np.uint32), case.seed & 0xFFFFFFFF, case.seed >> 32)[0]
        U = ((w >> np.uint32(9)).astype(np.float32) + np.float32(0.5)) * np.float32(2.0 ** -23)
        c0 = P0["cell"]
        tf = -tau[c0] * np.log(U.astype(np.float64))
        collide_def = tf < dt[c0]
        survived = np.isin(pid, P1["pid"])
        collide_or = ~survived
        dis = collide_def != collide_or
        band = np.abs(U.astype(np.float64) / np.exp(-dt[c0] / tau[c0]) - 1.0) <= 1e-6
        col_dis += int(np.count_nonzero(dis & ~band))
        col_band += int(np.count_nonzero(dis & band))
        n_draws += pid.size
        # the stay decision of the survivors (t_r = dt_i): definition in float64 on the float inputs
        s0 = np.nonzero(survived)[0]
        order1 = np.argsort(P1["pid"])
        j1 = order1[np.searchsorted(P1["pid"], pid[s0], sorter=order1)]
        cc = c0[s0]
        t = dt[cc].astype(np.float32).astype(np.float64)
        x0, y0 = P0["x"][s0], P0["y"][s0]
        u, v = P0["u"][s0], P0["v"][s0]
        xe, ye = x0 + u * t, y0 + v * t
        margin = np.minimum.reduce([xe - xa[cc], xb[cc] - xe, ye - ya[cc], yb[cc] - ye])
        stays_def = margin >= 0.0
        f32 = np.float32
        xs_or = (P0["x"][s0].astype(f32) + P0["u"][s0].astype(f32) * t.astype(f32)).astype(np.float64)
        ys_or = (P0["y"][s0].astype(f32) + P0["v"][s0].astype(f32) * t.astype(f32)).astype(np.float64)
        stays_or = ((P1["cell"][j1] == cc) & (P1["u"][j1] == u) & (P1["v"][j1] == v) & (P1["x"][j1] == xs_or)
                    & (P1["y"][j1] == ys_or))
        dis = stays_def != stays_or
        # float32 positions and face offsets round at 6e-8 of the box size; the band is 30 times that
        band = np.abs(margin) <= 2e-6
        stay_dis += int(np.count_nonzero(dis & ~band))
        stay_band += int(np.count_nonzero(dis & band))
        n_stay_checked += s0.size
    assert n_draws >= 10_000_000
    assert col_dis == 0
    assert col_band <= 1e-5 * n_draws
    assert stay_dis == 0
    assert stay_band <= 1e-5 * n_stay_checked
    # both decisions went both ways many times
    assert 0.05 * n_draws < n_draws - n_stay_checked < 0.9 * n_draws

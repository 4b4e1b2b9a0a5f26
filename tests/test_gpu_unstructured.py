"""GPU parity on unstructured meshes of triangles and convex quadrilaterals (§8f f1): the CUDA library
through ugkwp_create_unstructured against the CPU oracle on the same seeded inputs, to the bar of the
structured meshes (bit-exact cell decomposition, particles, integer tallies and crossings; cell conservatives
within 1e-12 of the per-component scale in the all-FP64 mode, 1e-5 in production precision)."""
import numpy as np
import pytest

from oracle import binding as ob
from paper_2607_09552_b300 import workloads as wl
from tests.parity import assert_field_close, assert_particles_equal, snapshot
from tests.test_gpu_parity import TOL, _compare_step

pytestmark = pytest.mark.gpu


def _cases():
    # hybrid cylinder: 4 quadrilateral layers at the wall, 7 triangulated layers (104 + 364 cells)
    hyb = wl.Case("hybrid_cylinder", wl.tri_omesh(4, 11, 26, 2e-3, 4.0), Kn=0.1, Ma=5.0, Tw=1.0, cfl=0.8, n_ref=33)
    # jittered triangles with all four boundary kinds: far field, fixed ghost, wall (T_w = 2), symmetry
    box = wl.jitter_interior(wl.split_quads(wl.box_mesh(13, 9, 0.0, 1.3, 0.0, 0.9, tags=(
        wl.BC_FARFIELD, wl.BC_FIXED, wl.BC_WALL, wl.BC_SYMMETRY)), 0, "i"), 7, 0.2)
    tri = wl.Case("tri_box", box, Kn=0.05, Ma=1.5, Tw=2.0, cfl=0.6, n_ref=29, ghost_state=(1.2, 0.8, 0.0, 1.1))
    return {"hybrid_cylinder": hyb, "tri_box": tri}


CASES = _cases()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("gts", [False, True])
def test_setup_bitwise(cuda_lib, name, gts):
    g = cuda_lib.Solver(CASES[name], gts=gts)
    o = ob.Oracle(CASES[name], gts=gts)
    dg, vg = g.geometry()
    do, vo = o.geometry()
    assert np.array_equal(vg, vo) and np.array_equal(dg, do)
    assert (g.F, g.nwall) == (o.F, o.nwall)
    assert g.fx == o.fx


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", [0, 1])
def test_first_step(cuda_lib, name, prec):
    g = cuda_lib.Solver(CASES[name], precision=prec, record_faces=True)
    o = ob.Oracle(CASES[name], precision=prec, record_faces=True)
    g.step(1)
    o.step(1)
    assert o.stats()[5] > 0
    _compare_step(g, o, prec)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec,gts", [(0, False), (1, False), (0, True)])
def test_step_from_identical_snapshot(cuda_lib, name, prec, gts):
    g = cuda_lib.Solver(CASES[name], gts=gts, precision=prec)
    o = ob.Oracle(CASES[name], gts=gts, precision=prec)
    o.step(6)
    step, W, wret, parts = snapshot(o)
    g.set_state(step, W, wret, parts)
    g.step(1)
    o.step(1)
    _compare_step(g, o, prec)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", [0, 1])
def test_second_order_step(cuda_lib, name, prec):
    """Least-squares gradients over triangle and quadrilateral neighbours (Eq. 12) with the same bar as the
    structured meshes' order-2 step."""
    g = cuda_lib.Solver(CASES[name], precision=prec, order=2)
    o = ob.Oracle(CASES[name], precision=prec, order=2)
    o.step(5)
    step, W, wret, parts = snapshot(o)
    g.set_state(step, W, wret, parts)
    g.step(1)
    o.step(1)
    assert np.any(o.gradients() != 0.0)
    assert np.array_equal(g.cell_data(), o.cell_data())
    assert_particles_equal(g.particles(), o.particles())
    assert_field_close(g.flux(), o.flux(), 1e-11 if prec == 1 else 1e-4)
    assert_field_close(g.field()[0], o.field()[0], TOL[prec])


def test_wave_only_trajectory(cuda_lib):
    g = cuda_lib.Solver(CASES["tri_box"], precision=1, wave_only=True)
    o = ob.Oracle(CASES["tri_box"], precision=1, wave_only=True)
    g.step(10)
    o.step(10)
    assert_field_close(g.field()[0], o.field()[0], 1e-12)


def test_graph_replay_equals_eager(cuda_lib):
    a = cuda_lib.Solver(CASES["hybrid_cylinder"], use_graph=True)
    b = cuda_lib.Solver(CASES["hybrid_cylinder"])
    a.step(4)
    b.step(4)
    assert np.array_equal(a.field()[0], b.field()[0])
    assert_particles_equal(a.particles(), b.particles())


def test_malformed_meshes_rejected(cuda_lib):
    good = wl.split_quads(wl.box_mesh(2, 2), 0, "i")
    cuda_lib.Solver(wl.Case("ok", good, Kn=0.1, Ma=1.0, Tw=1.0, cfl=0.5, n_ref=8)).close()
    cw = good.cells.copy()
    cw[0, :3] = cw[0, [0, 2, 1]]
    bad = [wl.UMesh(good.xv, good.yv, cw, good.boundary),
           wl.UMesh(good.xv, good.yv, good.cells, good.boundary[1:]),
           wl.UMesh(good.xv, good.yv, np.vstack([good.cells, good.cells[:1]]), good.boundary)]
    per = good.boundary.copy()
    per[0, 2] = wl.BC_PERIODIC
    bad.append(wl.UMesh(good.xv, good.yv, good.cells, per))
    for m in bad:
        with pytest.raises(cuda_lib.UgkwpError) as e:
            cuda_lib.Solver(wl.Case("bad", m, Kn=0.1, Ma=1.0, Tw=1.0, cfl=0.5, n_ref=8))
        assert e.value.status == 1

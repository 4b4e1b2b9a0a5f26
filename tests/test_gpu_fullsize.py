"""Parity at the full workload sizes, in the production launch configuration used by bench.py.

The oracle finishes one step of each full-size workload in seconds, so every output is compared, not a
sample: the first step from the uniform freestream, and one step from an oracle-generated snapshot (the
oracle's own state after a few steps, loaded into the GPU).
"""
import numpy as np
import pytest

from oracle import binding as ob
from paper_2607_09552_b300 import workloads as wl
from tests.parity import assert_field_close, assert_particles_equal, snapshot

pytestmark = pytest.mark.gpu

FULL = {
    "shock1d_200": lambda: wl.case_shock1d(),
    "cylinder_120x160_kn0.1_ma5": wl.case_cylinder_kn01,
    "cylinder_240x320_kn0.01_ma15": wl.case_cylinder_kn001,
    "cylinder_tri_7420_kn0.05_ma5": wl.case_cylinder_tri,
    "cylinder_tri_16100_kn0.005_ma5": wl.case_cylinder_tri_kn001,
    "plate_tri_5885_kn0.0169_ma20.2": wl.case_plate_tri,
}


def _compare(g, o):
    assert np.array_equal(g.cell_data(), o.cell_data())
    tg, to = g.tallies(), o.tallies()
    for k in ("wm", "wpl", "wret", "cross", "wall"):
        assert np.array_equal(tg[k], to[k]), k
    assert_particles_equal(g.particles(), o.particles())
    assert_field_close(g.field()[0], o.field()[0], 1e-5)


@pytest.mark.parametrize("name", list(FULL))
def test_full_size_first_step(cuda_lib, name):
    case = FULL[name]()
    g = cuda_lib.Solver(case, precision=0, use_graph=True)
    o = ob.Oracle(case, precision=0)
    g.step(1)
    o.step(1)
    _compare(g, o)


@pytest.mark.parametrize("name", list(FULL))
def test_full_size_step_from_oracle_snapshot(cuda_lib, name):
    case = FULL[name]()
    o = ob.Oracle(case, precision=0)
    o.step(3)
    step, W, wret, parts = snapshot(o)
    g = cuda_lib.Solver(case, precision=0, use_graph=True)
    g.set_state(step, W, wret, parts)
    g.step(1)
    o.step(1)
    _compare(g, o)

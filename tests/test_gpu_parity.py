"""GPU parity: the CUDA library through its C ABI against the CPU oracle on the same seeded inputs.

Bar (per step, from an identical snapshot): bit-exact cell decomposition outputs (tau, e^{-dt/tau}, N^hp,
new-particle mass and sampling moments), bit-exact particle sets (ids, cells, positions, velocities,
masses), bit-exact integer tallies and crossing counts; cell conservatives within 1e-12 of the per-component
scale in the all-FP64 mode and 1e-5 in production precision (FP32 interior wave fluxes).
"""
import numpy as np
import pytest

from oracle import binding as ob
from paper_2607_09552_b300 import workloads as wl
from tests.parity import assert_field_close, assert_particles_equal, small_cases, snapshot

pytestmark = pytest.mark.gpu

CASES = small_cases()
TOL = {0: 1e-5, 1: 1e-12}


def _pair(cuda_lib, case, prec, gts=False, wave_only=False, **kw):
    g = cuda_lib.Solver(case, gts=gts, precision=prec, wave_only=wave_only, **kw)
    o = ob.Oracle(case, gts=gts, precision=prec, wave_only=wave_only)
    return g, o


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("gts", [False, True])
def test_setup_geometry_and_time_steps_bitwise(cuda_lib, name, gts):
    g, o = _pair(cuda_lib, CASES[name], 0, gts=gts)
    dg, vg = g.geometry()
    do, vo = o.geometry()
    assert np.array_equal(vg, vo)
    assert np.array_equal(dg, do)
    assert (g.F, g.nwall) == (o.F, o.nwall)
    assert g.fx == o.fx


def _compare_step(g, o, prec):
    cg, co = g.cell_data(), o.cell_data()
    assert np.array_equal(cg, co), np.nonzero(cg != co)
    tg, to = g.tallies(), o.tallies()
    for k in ("wm", "wpl", "wret", "cross", "wall", "frec"):
        assert np.array_equal(tg[k], to[k]), (k, np.nonzero(tg[k] != to[k]))
    sg, so = g.stats(), o.stats()
    assert np.array_equal(sg[1:8], so[1:8]), (sg, so)
    assert sg[10] == so[8]
    assert sg[11] == so[9]
    assert sg[12] == so[10]
    assert_particles_equal(g.particles(), o.particles())
    Fg, Fo = g.flux(), o.flux()
    assert_field_close(Fg, Fo, 10 * TOL[prec])
    assert_field_close(g.field()[0], o.field()[0], TOL[prec])


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", [0, 1])
def test_first_step_from_freestream(cuda_lib, name, prec):
    g, o = _pair(cuda_lib, CASES[name], prec)
    g.step(1)
    o.step(1)
    _compare_step(g, o, prec)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec,gts", [(0, False), (1, False), (0, True)])
def test_step_from_identical_snapshot(cuda_lib, name, prec, gts):
    """Advance the oracle a few steps, load its state into the GPU, then compare one step."""
    g, o = _pair(cuda_lib, CASES[name], prec, gts=gts)
    o.step(6)
    step, W, wret, parts = snapshot(o)
    g.set_state(step, W, wret, parts)
    g.step(1)
    o.step(1)
    _compare_step(g, o, prec)


@pytest.mark.parametrize("name", ["box", "cylinder", "shock1d"])
@pytest.mark.parametrize("prec", [0, 1])
def test_side_recorded_crossings_bitwise(cuda_lib, name, prec):
    """Record mode (S33): the per-face crossing masses before and after the dt_R / dt_L scaling, from an
    identical snapshot, equal the oracle's bit for bit."""
    case = CASES[name]
    g = cuda_lib.Solver(case, precision=prec, record_faces=True)
    o = ob.Oracle(case, precision=prec, record_faces=True)
    o.step(5)
    step, W, wret, parts = snapshot(o)
    g.set_state(step, W, wret, parts)
    g.step(1)
    o.step(1)
    tg, to = g.tallies(), o.tallies()
    assert np.count_nonzero(to["frec"]) > 0
    assert np.array_equal(tg["frec"], to["frec"]), np.nonzero(tg["frec"] != to["frec"])
    assert np.array_equal(tg["cross"], to["cross"])
    _compare_step(g, o, prec)


def test_side_recorded_flux_balance_on_gpu(cuda_lib):
    """Sec. IV A, Eqs. 35-43 on the GPU: fixed local steps varying 50x over a periodic box, mass scaled by
    dt_R / dt_L at each crossing; over M steps the recorded sums satisfy sum(m_R) / dt_R = sum(m_L) / dt_L on
    every face and direction, up to the fixed-point rounding of each record (half a unit per side)."""
    case = wl.case_periodic_box(ni=10, end_ratio=50.0, n_ref=40, Kn=0.2)
    g = cuda_lib.Solver(case, precision=1, record_faces=True)
    dt, _ = g.geometry()
    M = 30
    acc = np.zeros((g.F, 4))
    ncr = np.zeros((g.F, 2))
    for _ in range(M):
        g.step(1)
        t = g.tallies()
        acc += t["frec"].astype(np.float64)
        ncr += t["cross"]
    ni = case.mesh.ni
    for f in range(g.F):
        L, R = (ni - 1, 0) if f == 0 else (f - 1, f)
        for d, (a, b) in enumerate(((L, R), (R, L))):
            mL, mR = acc[f, 2 * d], acc[f, 2 * d + 1]
            assert mL > 0 and ncr[f, d] > 0
            assert abs(mR / dt[b] - mL / dt[a]) <= ncr[f, d] * (0.5 / dt[a] + 0.5 / dt[b]) * (1 + 1e-9)


@pytest.mark.parametrize("prec", [0, 1])
def test_time_varying_steps_parity(cuda_lib, prec):
    """Replaced local steps (Sec. IV A study tool): from an identical snapshot, both sides given the same new
    steps (a factor 2 on half of a 50x-stretched periodic box) take the same step bit for bit, records
    included."""
    case = CASES["box"]
    g = cuda_lib.Solver(case, precision=prec, record_faces=True)
    o = ob.Oracle(case, precision=prec, record_faces=True)
    o.step(4)
    step, W, wret, parts = snapshot(o)
    g.set_state(step, W, wret, parts)
    d0, _ = o.geometry()
    dt = d0.copy()
    dt[: len(dt) // 2] *= 2.0
    g.set_time_steps(dt)
    o.set_time_steps(dt)
    assert np.array_equal(g.geometry()[0], o.geometry()[0])
    g.step(1)
    o.step(1)
    _compare_step(g, o, prec)


def test_time_varying_steps_break_the_balance_on_gpu(cuda_lib):
    """Sec. IV A, Eqs. 44-46 on the GPU: fixed steps keep the two sides' time-averaged particle fluxes equal to
    the records' rounding; the schedule dt_L = (1, 2, ...), dt_R = 2 does not (the per-step parity of the
    replaced steps is checked above)."""
    from tests.test_oracle_invariants import _time_averaged_ratio
    case = wl.case_periodic_box(ni=10, end_ratio=1.0, n_ref=60, Kn=0.05)
    g = cuda_lib.Solver(case, precision=1, record_faces=True)
    d0, _ = g.geometry()
    fixed = _time_averaged_ratio(g, lambda ell: np.concatenate([d0[:5], 2.0 * d0[5:]]), 20)
    assert abs(fixed - 1.0) < 1e-11
    sched = lambda ell: np.concatenate([d0[:5] * (1.0 if ell % 2 == 0 else 2.0), 2.0 * d0[5:]])
    g2 = cuda_lib.Solver(case, precision=1, record_faces=True)
    rg = _time_averaged_ratio(g2, sched, 40)
    assert abs(rg - 1.0) > 1e-2


@pytest.mark.parametrize("name", ["shock1d", "cylinder", "plate", "box"])
@pytest.mark.parametrize("prec", [0, 1])
def test_second_order_step_parity(cuda_lib, name, prec):
    """Order 2 (Eq. 12, S6): from an identical snapshot the reconstructed wave fluxes (FP64 in both modes) and
    the updated field agree within the step tolerances; the particles (untouched by the fluxes within a step)
    bit for bit."""
    case = CASES[name]
    g = cuda_lib.Solver(case, precision=prec, order=2)
    o = ob.Oracle(case, precision=prec, order=2)
    o.step(5)
    step, W, wret, parts = snapshot(o)
    g.set_state(step, W, wret, parts)
    g.step(1)
    o.step(1)
    assert np.any(o.gradients() != 0.0)
    # FP64 mode: the step bar (1e-12, fluxes 1e-11; measured 2e-14 per element); production mode keeps the step
    # bar (FP32 face moments are not used at order 2, but the FP64 face fluxes there take CUDA's exp and erfc)
    assert np.array_equal(g.cell_data(), o.cell_data())
    tg, to = g.tallies(), o.tallies()
    for k in ("wm", "wpl", "wret", "cross", "wall", "frec"):
        assert np.array_equal(tg[k], to[k]), k
    assert_particles_equal(g.particles(), o.particles())
    assert_field_close(g.flux(), o.flux(), 1e-11 if prec == 1 else 1e-4)
    assert_field_close(g.field()[0], o.field()[0], TOL[prec])


@pytest.mark.parametrize("name", ["shock1d", "cylinder", "plate", "box"])
def test_second_order_wave_only_mode(cuda_lib, name):
    g = cuda_lib.Solver(CASES[name], precision=1, wave_only=True, order=2)
    o = ob.Oracle(CASES[name], precision=1, wave_only=True, order=2)
    g.step(3)
    o.step(3)
    assert_field_close(g.field()[0], o.field()[0], 1e-12)


@pytest.mark.parametrize("prec", [0, 1])
def test_maxwell_wall_step_parity(cuda_lib, prec):
    """Maxwell wall with accommodation 0.85 (the paper's plate value): from an identical snapshot the
    specular/diffuse choice per hit, the wall tallies and the particles agree bit for bit, the field within
    the step tolerance."""
    import dataclasses
    case = dataclasses.replace(CASES["plate"], wall_specular=0.15)
    g = cuda_lib.Solver(case, precision=prec)
    o = ob.Oracle(case, precision=prec)
    o.step(5)
    step, W, wret, parts = snapshot(o)
    g.set_state(step, W, wret, parts)
    g.step(1)
    o.step(1)
    assert o.stats()[6] > 0
    _compare_step(g, o, prec)


def test_specular_walls_conserve_energy_on_gpu(cuda_lib):
    from tests.test_oracle_wall import _closed_box, _totals
    g = cuda_lib.Solver(_closed_box(1.0), precision=1)
    t0 = _totals(g)
    g.step(40)
    np.testing.assert_allclose(_totals(g), t0, rtol=1e-12)


@pytest.mark.parametrize("name", ["shock1d", "cylinder", "plate"])
def test_short_trajectory_fp64(cuda_lib, name):
    """Whole trajectories from the same freestream start in the all-FP64 mode. Both sides take e^x and erfc of
    the wave fluxes from their own IEEE-operation implementations of the same definitions, so a step agrees to
    a few ulp (measured 1e-15 of the component scales); over 4 steps particle ids and cells stay identical,
    particle values agree to 1e-12 relative and the field to 1e-12 per element (against max(|W|, 0.1 x the
    component's scale): low-density wake cells amplify the last-bit differences, measured 4e-14)."""
    from tests.parity import sort_particles
    g, o = _pair(cuda_lib, CASES[name], 1)
    for _ in range(4):
        g.step(1)
        o.step(1)
    a, b = sort_particles(g.particles()), sort_particles(o.particles())
    assert np.array_equal(a["pid"], b["pid"])
    assert np.array_equal(a["cell"], b["cell"])
    for k in ("x", "y", "u", "v", "w", "m"):
        np.testing.assert_allclose(a[k], b[k], rtol=1e-12, atol=1e-14)
    assert_field_close(g.field()[0], o.field()[0], 1e-12, floor=0.1)


@pytest.mark.parametrize("name", ["shock1d", "cylinder", "plate", "box"])
def test_wave_only_mode(cuda_lib, name):
    """No particles (the GKS limit): a deterministic FP64 field update."""
    g, o = _pair(cuda_lib, CASES[name], 1, wave_only=True)
    g.step(3)
    o.step(3)
    assert g.num_particles() == 0
    assert_field_close(g.field()[0], o.field()[0], 1e-12)
    np.testing.assert_allclose(g.residual()[4:], o.residual()[4:], rtol=1e-12)


def test_gks_limit_no_particles(cuda_lib):
    """Tiny Kn: e^{-dt/tau} underflows, nothing is sampled, kernels run with zero particles."""
    case = wl.case_shock1d(ni=40, n_ref=20)
    case.Kn = 1e-6
    g, o = _pair(cuda_lib, case, 0)
    g.step(3)
    o.step(3)
    assert g.num_particles() == 0 and g.stats()[2] == 0
    assert_field_close(g.field()[0], o.field()[0], 1e-5)


def test_surface_quantities(cuda_lib):
    case = CASES["cylinder"]
    g, o = _pair(cuda_lib, case, 1)
    g.step(5)
    o.step(5)
    for av in (False, True):
        pg, tg, qg = g.surface(av)
        po, to, qo = o.surface(av)
        for a, b in ((pg, po), (tg, to), (qg, qo)):
            np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-14 * np.abs(b).max())


@pytest.mark.parametrize("name", ["cylinder", "plate"])
@pytest.mark.parametrize("prec", [0, 1])
def test_monitors(cuda_lib, name, prec):
    """The device's monitored wall loads (C_d, C_H, stagnation C_p, C_Q and their EMAs, ugkwp_monitors)
    against the oracle's step by step: 1e-12 in the all-FP64 mode, 1e-4 in production precision (FP32 wave-flux
    moments in the wall pressure of interior-facing sums); the plate has no stagnation point on either side."""
    g, o = _pair(cuda_lib, CASES[name], prec)
    assert np.isnan(g.monitors()).all()
    for _ in range(5):
        g.step(1)
        o.step(1)
        mg, mo = g.monitors(), o.monitors()
        assert np.array_equal(np.isnan(mg), np.isnan(mo))
        ok = ~np.isnan(mo)
        np.testing.assert_allclose(mg[ok], mo[ok], rtol=1e-12 if prec == 1 else 1e-4)
    assert (name == "cylinder") == bool(np.isfinite(mg[2]))


def test_residual(cuda_lib):
    g, o = _pair(cuda_lib, CASES["plate"], 1)
    g.step(3)
    o.step(3)
    np.testing.assert_allclose(g.residual(), o.residual(), rtol=1e-12)


def test_determinism_and_graph_replay(cuda_lib):
    case = CASES["cylinder"]
    a = cuda_lib.Solver(case, precision=0)
    b = cuda_lib.Solver(case, precision=0, use_graph=True)
    a.step(7)
    b.step(3)
    b.step(4)
    assert np.array_equal(a.field()[0], b.field()[0])
    assert_particles_equal(a.particles(), b.particles())
    assert np.array_equal(a.stats(), b.stats())


def test_capacity_limit_reports_error(cuda_lib):
    case = CASES["box"]
    g = cuda_lib.Solver(case, precision=0, capacity=100)
    g.step(1)
    with pytest.raises(cuda_lib.UgkwpError) as e:
        g.field()
    assert e.value.status == 4


@pytest.mark.parametrize("prec", [0, 1])
def test_capacity_limit_with_ghost_sources_reports_error(cuda_lib, prec):
    """Far-field ghost sources that enter more particles than the capacity holds: the slots past it are
    neither written nor counted, so the following steps (several, in one graph launch each) stay within the
    buffers, and the error is reported (ELIMIT, status 4)."""
    case = CASES["cylinder"]
    g = cuda_lib.Solver(case, precision=prec, capacity=300, use_graph=True)
    g.step(6)
    with pytest.raises(cuda_lib.UgkwpError) as e:
        g.field()
    assert e.value.status == 4


def test_option_validation(cuda_lib):
    """Bad options are refused with EINVAL (status 1): a reconstruction order other than 1 or 2, a specular
    wall fraction outside [0, 1], a particle cutoff outside [0, 1), a non-positive or non-finite replacement time step (which leaves the
    steps unchanged)."""
    import dataclasses
    with pytest.raises(cuda_lib.UgkwpError) as e:
        cuda_lib.Solver(CASES["box"], precision=1, order=3)
    assert e.value.status == 1
    with pytest.raises(cuda_lib.UgkwpError) as e:
        cuda_lib.Solver(dataclasses.replace(CASES["plate"], wall_specular=1.5), precision=1)
    assert e.value.status == 1
    for bad in (-0.1, 1.0, np.nan):
        with pytest.raises(cuda_lib.UgkwpError) as e:
            cuda_lib.Solver(CASES["box"], precision=1, emx_cutoff=bad)
        assert e.value.status == 1
    g = cuda_lib.Solver(CASES["box"], precision=1)
    d0, _ = g.geometry()
    for bad in (0.0, -1.0, np.inf, np.nan):
        dt = d0.copy()
        dt[3] = bad
        with pytest.raises(cuda_lib.UgkwpError) as e:
            g.set_time_steps(dt)
        assert e.value.status == 1
    assert np.array_equal(g.geometry()[0], d0)


def test_empty_and_single_particle_cells(cuda_lib):
    """N^hp = 1 cells (the sampled particle takes the mean velocity) and cells without new particles, over
    several steps, each compared from an identical snapshot."""
    case = wl.case_periodic_box(ni=9, end_ratio=3.0, n_ref=1, Kn=0.05)
    g, o = _pair(cuda_lib, case, 0)
    for _ in range(3):
        step, W, wret, parts = snapshot(o)
        g.set_state(step, W, wret, parts)
        g.step(1)
        o.step(1)
        _compare_step(g, o, 0)


def test_checkpoint_resume_is_bit_identical(cuda_lib, tmp_path):
    """A run saved after 9 steps and resumed in a fresh context for 6 more steps equals the uninterrupted
    15-step run (particle draws are keyed by particle id and step; sort steps follow the step counter)."""
    case = CASES["cylinder"]
    a = cuda_lib.Solver(case, precision=0)
    a.step(9)
    path = str(tmp_path / "ckpt.bin")
    a.save(path)
    a.step(6)
    b = cuda_lib.Solver(case, precision=0)
    b.load_checkpoint(path)
    b.step(6)
    assert np.array_equal(a.field()[0], b.field()[0])
    assert_particles_equal(a.particles(), b.particles())
    ta, tb = a.tallies(), b.tallies()
    for k in ("wm", "wpl", "wret", "cross"):
        assert np.array_equal(ta[k], tb[k])
    assert np.array_equal(a.residual(), b.residual())
    for x, y in zip(a.surface(True), b.surface(True)):
        np.testing.assert_allclose(x, y, rtol=1e-14, atol=0)


def test_batched_graph_equals_individual_runs(cuda_lib):
    """One graph launch per step for several uneven cases gives each case exactly its own trajectory."""
    names = ["cylinder", "plate", "shock1d"]
    solo = [cuda_lib.Solver(CASES[n], precision=0) for n in names]
    for s in solo:
        s.step(6)
    grouped = [cuda_lib.Solver(CASES[n], precision=0) for n in names]
    b = cuda_lib.Batch(grouped)
    b.step(2)
    b.step(4)
    for a, g in zip(solo, grouped):
        assert np.array_equal(a.field()[0], g.field()[0])
        assert_particles_equal(a.particles(), g.particles())
        assert np.array_equal(a.stats()[:8], g.stats()[:8])
    b.close()


@pytest.mark.parametrize("ctas_per_sm", [4, 6])
def test_persistent_batch_equals_individual_runs(cuda_lib, ctas_per_sm):
    """The batched persistent kernel (one launch per step for all cases, work items taken from a device counter,
    each waiting for its case's previous stage) gives each case exactly its own trajectory: cell states bit for
    bit, particles as sets, tallies, counters, residual and monitors."""
    names = ["cylinder", "plate", "shock1d", "box", "cylinder_dense"]
    solo = [cuda_lib.Solver(CASES[n], precision=0) for n in names]
    for s in solo:
        s.step(7)
    grouped = [cuda_lib.Solver(CASES[n], precision=0) for n in names]
    grouped[0].step(1)     # uneven start: the cases need not be at the same step
    b = cuda_lib.Batch(grouped[1:] + grouped[:1], persistent=True, ctas_per_sm=ctas_per_sm)
    plan = b.plan()
    assert plan[0] == 1 and plan[1] > 0 and plan[3] == ctas_per_sm and plan[2] % ctas_per_sm == 0
    b.step(3)
    b.step(3)
    assert b.status() == (0, -1)
    b.close()
    for g in grouped[1:]:
        g.step(1)          # the contexts keep stepping on their own after batched steps
    for a, g in zip(solo, grouped):
        assert int(a.stats()[0]) == int(g.stats()[0])
        assert np.array_equal(a.field()[0], g.field()[0])
        assert_particles_equal(a.particles(), g.particles())
        assert np.array_equal(a.stats()[:8], g.stats()[:8])
        ta, tg = a.tallies(), g.tallies()
        for k in ("wm", "wpl", "wret", "cross", "wall"):
            assert np.array_equal(ta[k], tg[k]), k
        assert np.array_equal(a.residual(), g.residual())
        assert np.array_equal(a.monitors(), g.monitors(), equal_nan=True)


def test_persistent_batch_scope_and_wait_limit(cuda_lib):
    """Cases outside the persistent kernel's scope are refused (EINVAL); a stage wait that runs out stops the
    batch with ELIMIT (the test hook makes the step's last item wait for an item that does not exist), flags every
    case, and leaves the device usable."""
    with pytest.raises(cuda_lib.UgkwpError) as e:
        cuda_lib.Batch([cuda_lib.Solver(CASES["box"], precision=1)], persistent=True)
    assert e.value.status == 1
    names = ["cylinder", "plate", "shock1d"]
    grouped = [cuda_lib.Solver(CASES[n], precision=0) for n in names]
    b = cuda_lib.Batch(grouped, persistent=True)
    b.step(1)
    assert b.status() == (0, -1)
    b.set_wait_limit(2_000_000, stall=True)   # 2 ms
    b.step(1)
    st, where = b.status()
    assert st == 4 and where == (len(names) - 1) * 20 + 19   # the last case's update stage
    for g in grouped:
        with pytest.raises(cuda_lib.UgkwpError) as e:
            g.field()
        assert e.value.status == 4
    b.step(1)                                  # a stopped batch does nothing
    assert b.status()[0] == 4
    b.close()
    fresh = cuda_lib.Solver(CASES["cylinder"], precision=0)
    fresh.step(2)
    assert np.all(np.isfinite(fresh.field()[0]))


def test_launch_parameters_and_autotuner_leave_results_unchanged(cuda_lib):
    """The transport kernel (warp-staged, the production default, against warp-chunked), chunk size, blocks per
    SM and the sort interval reorder work and particles only: the state is the same bit for bit (particles
    compared as sets), also across an autotuning pass that steps the run."""
    case = CASES["cylinder"]
    # the autotuning pass steps through the start-up transient (particle count up to about 6x the steady one,
    # 8.5 N_ref per cell near step 400 on this mesh)
    cap = 16 * case.n_ref * case.mesh.ncells
    a = cuda_lib.Solver(case, precision=0, use_graph=True, capacity=cap)
    b = cuda_lib.Solver(case, precision=0, use_graph=True, capacity=cap)
    assert a.launch() == [128, 8, 8, 2]
    b.set_launch(128, 2, 16, 1)
    assert b.launch() == [128, 2, 16, 1]
    a.step(21)
    b.step(21)
    assert np.array_equal(a.field()[0], b.field()[0])
    assert_particles_equal(a.particles(), b.particles())
    ta, tb = a.tallies(), b.tallies()
    for k in ("wm", "wpl", "wret", "cross", "wall"):
        assert np.array_equal(ta[k], tb[k]), k
    assert np.array_equal(a.stats()[:8], b.stats()[:8])
    best, ms = b.autotune(4)
    assert best[3] in (1, 2) and best[2] in (8, 16, 32) and ms > 0
    if best[3] == 1:
        assert best[0] in (128, 256) and best[1] in (4, 6, 8)
    n = int(b.stats()[0]) - int(a.stats()[0])
    a.step(n)
    b.step(5)
    a.step(5)
    assert np.array_equal(a.field()[0], b.field()[0])
    assert_particles_equal(a.particles(), b.particles())
    ta, tb = a.tallies(), b.tallies()
    for k in ("wm", "wpl", "wret", "cross"):
        assert np.array_equal(ta[k], tb[k])
    with pytest.raises(cuda_lib.UgkwpError):
        b.set_launch(100, 0, 0)
    with pytest.raises(cuda_lib.UgkwpError):
        b.set_launch(0, 0, 0, 3)
    # the FP64 mode runs the warp-chunked kernel only
    f = cuda_lib.Solver(case, precision=1, use_graph=False)
    assert f.launch()[3] == 1
    with pytest.raises(cuda_lib.UgkwpError):
        f.set_launch(0, 0, 0, 2)
    f.close()


@pytest.mark.parametrize("name", ["cylinder", "plate", "shock1d", "cylinder_dense"])
@pytest.mark.parametrize("tile,bps,sort", [(64, 6, 8), (64, 8, 16), (128, 4, 8), (128, 8, 32)])
def test_warp_staged_transport_equals_warp_chunked(cuda_lib, name, tile, bps, sort):
    """The warp-staged transport kernel (per-warp bulk-copied tiles, crossing particles queued and flown 32 at a
    time, records updated in place) gives the state of the warp-chunked kernel bit for bit (particles compared as
    sets) over steps that include counting-sort steps, with and without graph replay."""
    case = CASES[name]
    a = cuda_lib.Solver(case, precision=0, use_graph=True)
    a.set_launch(256, 4, 8, 1)
    b = cuda_lib.Solver(case, precision=0, use_graph=(bps == 8))
    b.set_launch(tile, bps, sort, 2)
    assert b.launch() == [tile, bps, sort, 2]
    a.step(19)
    b.step(19)
    assert np.array_equal(a.field()[0], b.field()[0])
    assert_particles_equal(a.particles(), b.particles())
    ta, tb = a.tallies(), b.tallies()
    for k in ("wm", "wpl", "wret", "cross", "wall"):
        assert np.array_equal(ta[k], tb[k]), k
    assert np.array_equal(a.stats()[:8], b.stats()[:8])
    a.close()
    b.close()


def test_device_memory_from_torch_allocator(cuda_lib):
    """ugkwp_opts.dev_alloc / dev_free: a context whose device memory comes from torch's caching allocator
    (the binding's default) holds it there (torch counts it) and steps to the same state, bit for bit, as one
    whose memory the library allocates itself; the temporaries of the read-back calls go through it too."""
    import torch
    case = CASES["cylinder"]
    before = torch.cuda.memory_allocated()
    a = cuda_lib.Solver(case, precision=0, use_graph=True, torch_memory=True)
    held = torch.cuda.memory_allocated() - before
    assert held > 0
    b = cuda_lib.Solver(case, precision=0, use_graph=True, torch_memory=False)
    assert torch.cuda.memory_allocated() - before == held
    a.step(12)
    b.step(12)
    assert np.array_equal(a.field()[0], b.field()[0])
    assert np.array_equal(a.field()[1], b.field()[1])
    assert_particles_equal(a.particles(), b.particles())
    assert np.array_equal(a.cell_data(), b.cell_data())
    assert torch.cuda.memory_allocated() - before == held
    a.close()
    assert torch.cuda.memory_allocated() == before
    b.close()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("gts", [False, True])
def test_particle_cutoff_step_parity(cuda_lib, prec, gts):
    """Particle cutoff (opts.emx_cutoff 0.05) on a 1-D shock at Kn 0.05 whose coarse cells are wave-dominated:
    the same cells sample nothing on both sides (the decision e^{-x} < cutoff in FP64 on the same value), and
    the step from an identical snapshot keeps the step bar."""
    case = wl.case_shock1d(ni=60, n_ref=30)
    case.Kn = 0.05
    g = cuda_lib.Solver(case, gts=gts, precision=prec, emx_cutoff=0.05)
    o = ob.Oracle(case, gts=gts, precision=prec, emx_cutoff=0.05)
    o.step(20)
    step, W, wret, parts = snapshot(o)
    g.set_state(step, W, wret, parts)
    g.step(1)
    o.step(1)
    cd = o.cell_data()
    cut = cd[:, 2] < 0.05
    assert gts or cut.sum() >= 3
    assert np.all(cd[cut, 3] == 0)
    _compare_step(g, o, prec)

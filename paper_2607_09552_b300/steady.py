"""Steady-state monitoring of the UGKWP-LTS iteration: residual-driven runs, integrated wall loads and the
EMA criterion for "steady" in the stochastic method.

The paper judges steady state by exponential-moving-average histories (alpha = 2/1001) of wall quantities
(Sec. V A) and defines no residual. Two yardsticks are provided here:
- `run_to_residual`: the deterministic particle-free mode (the GKS limit of the method) stepped until every
  conservative component of the residual sqrt(sum_i Omega_i ((W^{n+1} - W^n) / dt_i)^2) falls below a
  threshold, relative to a reference (by default the library's freestream scale of each component);
- `steady_step`: the first step after which the EMA of a monitored history stays within a tolerance of
  the mean of the run's final window; the monitors are integrated wall loads (drag and heat load, `loads`),
  whose particle noise is far below that of any single wall face.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import workloads as wl


def wall_geometry(case):
    """Outward normals (nx, ny) of the fluid cells and lengths s of the wall faces, in the library's
    wall-face order: on a structured mesh i-faces (vertex rows i = const) before j-faces, each in increasing
    face index; on an unstructured one in order of the cells and their edges."""
    m = case.mesh
    if m.dim != 2:
        return np.zeros(0), np.zeros(0), np.zeros(0)
    if hasattr(m, "cells"):
        # unstructured: a boundary edge belongs to one cell, so face order puts it at (cell, local edge)
        walls = {tuple(sorted((int(a), int(b)))) for a, b, t in m.boundary if t == wl.BC_WALL}
        out = []
        for q in m.cells:
            vs = [int(v) for v in q if v >= 0]
            for a, b in zip(vs, vs[1:] + vs[:1]):
                if tuple(sorted((a, b))) in walls:
                    dx, dy = m.xv[b] - m.xv[a], m.yv[b] - m.yv[a]
                    s = math.hypot(dx, dy)
                    out.append((dy / s, -dx / s, s))
        a = np.array(out).reshape(-1, 3)
        return a[:, 0], a[:, 1], a[:, 2]
    ni, nj = m.ni, m.nj
    xv, yv = m.xv.reshape(nj + 1, ni + 1), m.yv.reshape(nj + 1, ni + 1)
    out = []
    # i-faces: face between vertices (i, j) and (i, j + 1); the fluid cell is (0, j) at i = 0 (normal -i side)
    for j in range(nj):
        for i, tag in ((0, m.bc_imin[j]), (ni, m.bc_imax[j])):
            if tag != wl.BC_WALL:
                continue
            dx, dy = xv[j + 1, i] - xv[j, i], yv[j + 1, i] - yv[j, i]
            s = math.hypot(dx, dy)
            n = (-dy / s, dx / s) if i == 0 else (dy / s, -dx / s)
            out.append((j * (ni + 1) + i, n[0], n[1], s))
    # j-faces: between vertices (i, j) and (i + 1, j); the fluid cell is (i, 0) at j = 0
    if not m.periodic_j:
        base = (ni + 1) * nj
        for i in range(ni):
            for j, tag in ((0, m.bc_jmin[i]), (nj, m.bc_jmax[i])):
                if tag != wl.BC_WALL:
                    continue
                dx, dy = xv[j, i + 1] - xv[j, i], yv[j, i + 1] - yv[j, i]
                s = math.hypot(dx, dy)
                n = (dy / s, -dx / s) if j == 0 else (-dy / s, dx / s)
                out.append((base + j * ni + i, n[0], n[1], s))
    out.sort()
    a = np.array([o[1:] for o in out]).reshape(-1, 3)
    return a[:, 0], a[:, 1], a[:, 2]


def loads(case, p, tau, q, geom=None):
    """(drag coefficient, heat-load coefficient): F_x / (rho U^2 / 2 L) and Q / (rho U^3 / 2 L) with
    F = sum_j s_j (p_j n_j + tau_j t_j), t = (-n_y, n_x), Q = sum_j s_j q_j, L = 1."""
    nx, ny, s = geom if geom is not None else wall_geometry(case)
    U = wl.freestream_speed(case.Ma)
    fx = float(np.sum(s * (p * nx - tau * ny)))
    Q = float(np.sum(s * q))
    return fx / (0.5 * U * U), Q / (0.5 * U ** 3)


def steady_step(hist, alpha: float = 2.0 / 1001.0, tol: float = 0.01, window: float = 0.2):
    """First step after which the EMA of `hist` stays within a band around the mean of its final window (the
    last `window` fraction of the run); len(hist) if it never settles. The band is the larger of tol times
    that mean and three standard deviations of the EMA over the final window (the particle noise the EMA
    keeps at steady state). Returns (step, ema)."""
    h = np.asarray(hist, dtype=np.float64)
    ema = np.empty_like(h)
    e = h[0]
    for k, v in enumerate(h):
        e = e + alpha * (v - e) if k else v
        ema[k] = e
    tail = ema[int(len(h) * (1 - window)):]
    ref = tail.mean()
    band = max(tol * abs(ref), 3.0 * float(tail.std()))
    bad = np.nonzero(np.abs(ema - ref) > band)[0]
    return (int(bad[-1] + 1) if bad.size else 0), ema


def run_to_residual(solver, tol: float = 1e-6, max_steps: int = 200000, chunk: int = 200, ref=None,
                    marks=(1e-3, 1e-4, 1e-5, 1e-6)):
    """Step until every conservative component of the residual is below tol; the residual is the raw one
    divided by `ref` (4 values, e.g. the freestream start's first-step residual, so that runs from different
    starting fields share one yardstick) or, without ref, the library's freestream-normalised residual.
    Returns dict(steps, residual, seconds, marks={threshold: (steps, seconds)} for the thresholds crossed)."""
    t0 = time.perf_counter()
    steps, res = 0, math.inf
    crossed = {}
    while steps < max_steps:
        solver.step(chunk)
        steps += chunk
        r = solver.residual()
        res = float(np.max(r[4:] / ref)) if ref is not None else float(np.max(r[:4]))
        for m in marks:
            if res < m and m not in crossed:
                crossed[m] = (steps, time.perf_counter() - t0)
        if res < tol:
            break
    return dict(steps=steps, residual=res, seconds=time.perf_counter() - t0, converged=res < tol, marks=crossed)


def first_residual(case, **solver_kw):
    """Raw first-step residual (4 values) of a fresh context started from the freestream."""
    from . import ugkwp
    s = ugkwp.Solver(case, **solver_kw)
    s.step(1)
    r = s.residual()[4:].copy()
    s.close()
    # a component that does not move in the first step (e.g. by symmetry) is measured against the largest
    return np.where(r > 0.0, r, max(float(r.max()), 1e-300))

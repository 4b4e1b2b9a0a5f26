"""ORACLE (test infrastructure only): ctypes binding of the plain-C oracle.

Only tests, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py` may import this module.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


class OracleMesh(C.Structure):
    _fields_ = [("ni", C.c_int32), ("nj", C.c_int32), ("dim", C.c_int32), ("periodic_j", C.c_int32),
                ("xv", C.POINTER(C.c_double)), ("yv", C.POINTER(C.c_double)),
                ("bc_imin", C.POINTER(C.c_int32)), ("bc_imax", C.POINTER(C.c_int32)),
                ("bc_jmin", C.POINTER(C.c_int32)), ("bc_jmax", C.POINTER(C.c_int32))]


class OracleUMesh(C.Structure):
    _fields_ = [("n_vertices", C.c_int32), ("n_cells", C.c_int32), ("xv", C.POINTER(C.c_double)),
                ("yv", C.POINTER(C.c_double)), ("cells", C.POINTER(C.c_int32)), ("n_boundary", C.c_int32),
                ("boundary", C.POINTER(C.c_int32))]


class OracleGas(C.Structure):
    _fields_ = [("omega", C.c_double), ("Pr", C.c_double), ("wall_specular", C.c_double)]


class OracleOpts(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("case_id", C.c_uint32), ("n_ref", C.c_int32), ("precision", C.c_int32),
                ("wave_only", C.c_int32), ("record_faces", C.c_int32), ("capacity", C.c_int32),
                ("ghost_state", C.c_double * 4), ("order", C.c_int32), ("emx_cutoff", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = C.CDLL(path)
        _lib.oracle_create.restype = C.c_int
        _lib.oracle_last_error.restype = C.c_char_p
        _lib.oracle_num_particles.restype = C.c_int64
        _lib.oracle_logf.restype = C.c_float
        _lib.oracle_logf.argtypes = [C.c_float]
        _lib.oracle_logd.restype = C.c_double
        _lib.oracle_logd.argtypes = [C.c_double]
        _lib.oracle_expd.restype = C.c_double
        _lib.oracle_expd.argtypes = [C.c_double]
        _lib.oracle_erfcd.restype = C.c_double
        _lib.oracle_erfcd.argtypes = [C.c_double]
        _lib.oracle_expf.restype = C.c_float
        _lib.oracle_expf.argtypes = [C.c_float]
        _lib.oracle_sincos2pif.argtypes = [C.c_float, C.POINTER(C.c_float), C.POINTER(C.c_float)]
        _lib.oracle_sincos2pid.argtypes = [C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        _lib.oracle_mu_inf.restype = C.c_double
        _lib.oracle_mu_inf.argtypes = [C.c_double, C.c_double]
        _lib.oracle_coeffs.argtypes = [C.c_double, C.c_double, C.POINTER(C.c_double)]
    return _lib


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t))


def dptr(a):
    return _p(a, C.c_double)


def philox(ctr, key):
    out = (C.c_uint32 * 4)()
    lib().oracle_philox4x32_10((C.c_uint32 * 4)(*ctr), (C.c_uint32 * 2)(*key), out)
    return list(out)


def coeffs(dt, tau):
    out = (C.c_double * 7)()
    lib().oracle_coeffs(dt, tau, out)
    return np.array(out[:])


def sincos2pif(u):
    s, c = C.c_float(), C.c_float()
    lib().oracle_sincos2pif(u, C.byref(s), C.byref(c))
    return s.value, c.value


def sincos2pid(u):
    s, c = C.c_double(), C.c_double()
    lib().oracle_sincos2pid(u, C.byref(s), C.byref(c))
    return s.value, c.value


def face_flux(WL, WR, WhL, WhR, cL, cR, dL, dR, Pr=1.0):
    """Interior-face flux in the face frame (normal = +x). Returns F, W0, aL, aR, A."""
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (WL, WR)]
    hL = None if WhL is None else np.ascontiguousarray(WhL, dtype=np.float64)
    hR = None if WhR is None else np.ascontiguousarray(WhR, dtype=np.float64)
    cLa = np.ascontiguousarray(cL, dtype=np.float64)
    cRa = np.ascontiguousarray(cR, dtype=np.float64)
    outs = [np.zeros(4) for _ in range(5)]
    lib().oracle_face_flux_test(dptr(arrs[0]), dptr(arrs[1]), None if hL is None else dptr(hL),
                                None if hR is None else dptr(hR), dptr(cLa), dptr(cRa), C.c_double(dL),
                                C.c_double(dR), C.c_double(Pr), *[dptr(o) for o in outs])
    return outs


def wall_flux(Tw, ws, WL, WhL, cL, frL):
    """Wall-face flux in the face frame (normal from the fluid cell into the wall): incoming half of the cell's
    g (weight cL[0]) and g^h (weight frL), outgoing wall part with specular fraction ws."""
    a = np.ascontiguousarray(WL, dtype=np.float64)
    h = None if WhL is None else np.ascontiguousarray(WhL, dtype=np.float64)
    c = np.ascontiguousarray(cL, dtype=np.float64)
    F = np.zeros(4)
    lib().oracle_wall_flux_test(C.c_double(Tw), C.c_double(ws), dptr(a), None if h is None else dptr(h), dptr(c),
                                C.c_double(frL), dptr(F))
    return F


class OracleError(RuntimeError):
    pass


class Oracle:
    """One oracle context for a workload `Case` (see paper_2607_09552_b300.workloads)."""

    def __init__(self, case, gts: bool = False, precision: int = 0, wave_only: bool = False,
                 record_faces: bool = False, seed: int | None = None, case_id: int = 0, order: int = 1,
                 emx_cutoff: float = 0.0):
        L = lib()
        m = case.mesh
        self._keep = [np.ascontiguousarray(a, dtype=np.float64) for a in (m.xv, m.yv)]
        unstructured = hasattr(m, "cells")
        if unstructured:
            self._keep += [np.ascontiguousarray(a, dtype=np.int32) for a in (m.cells, m.boundary)]
            mesh = OracleUMesh(len(m.xv), m.ncells, dptr(self._keep[0]), dptr(self._keep[1]),
                               _p(self._keep[2], C.c_int32), len(m.boundary), _p(self._keep[3], C.c_int32))
        else:
            self._keep += [np.ascontiguousarray(a, dtype=np.int32)
                           for a in (m.bc_imin, m.bc_imax, m.bc_jmin, m.bc_jmax)]
            mesh = OracleMesh(m.ni, m.nj, m.dim, m.periodic_j, dptr(self._keep[0]), dptr(self._keep[1]),
                              *[_p(a, C.c_int32) for a in self._keep[2:]])
        gas = OracleGas(case.omega, case.Pr, getattr(case, "wall_specular", 0.0))
        opts = OracleOpts(case.seed if seed is None else seed, case_id, case.n_ref, precision, int(wave_only),
                          int(record_faces), 0, (C.c_double * 4)(*case.ghost_state), int(order),
                          float(emx_cutoff))
        self.ctx = C.c_void_p()
        create = L.oracle_create_unstructured if unstructured else L.oracle_create
        st = create(C.byref(mesh), C.byref(gas), C.c_double(case.Kn), C.c_double(case.Ma),
                             C.c_double(case.Tw), C.c_double(case.cfl), C.c_int32(int(gts)), C.byref(opts),
                             C.byref(self.ctx))
        if st != 0:
            raise OracleError(f"oracle_create failed with status {st}")
        self.C = m.ncells
        nf, nw = C.c_int32(), C.c_int32()
        L.oracle_get_geometry(self.ctx, None, None, C.byref(nf), C.byref(nw))
        self.F, self.nwall = nf.value, nw.value
        fx = (C.c_int32 * 3)()
        L.oracle_fixed_exponents(self.ctx, fx)
        self.fx = list(fx)
        if case.init_prim is not None:
            self.set_field(case.init_prim)

    def __del__(self):
        if getattr(self, "ctx", None):
            lib().oracle_destroy(self.ctx)
            self.ctx = None

    def _check(self, st):
        if st != 0:
            raise OracleError(f"oracle status {st}: {lib().oracle_last_error(self.ctx).decode()}")

    def step(self, n: int = 1):
        self._check(lib().oracle_step(self.ctx, C.c_int32(n)))

    def set_time_steps(self, dt):
        """Replace the local time steps (C values > 0) from the next step on (time-varying study, Sec. IV A)."""
        a = np.ascontiguousarray(dt, dtype=np.float64)
        self._check(lib().oracle_set_time_steps(self.ctx, dptr(a)))

    def set_field(self, prim):
        a = np.ascontiguousarray(prim, dtype=np.float64).reshape(-1)
        self._check(lib().oracle_set_field(self.ctx, dptr(a)))

    def field(self):
        W = np.zeros(4 * self.C)
        Wp = np.zeros(4 * self.C)
        lib().oracle_get_field(self.ctx, dptr(W), dptr(Wp))
        return W.reshape(self.C, 4), Wp.reshape(self.C, 4)

    def residual(self):
        out = np.zeros(8)
        lib().oracle_residual(self.ctx, dptr(out))
        return out

    def surface(self, averaged: bool = True):
        p, t, q = (np.zeros(self.nwall) for _ in range(3))
        self._check(lib().oracle_surface(self.ctx, dptr(p), dptr(t), dptr(q), C.c_int32(self.nwall),
                                         C.c_int32(int(averaged))))
        return p, t, q

    def reset_surface(self):
        self._check(lib().oracle_reset_surface(self.ctx))

    def monitors(self):
        """[C_d, C_H, stagnation C_p, C_Q, then their EMAs] of the last step"""
        out = np.zeros(8)
        self._check(lib().oracle_monitors(self.ctx, dptr(out)))
        return out

    def stats(self):
        """[steps, particles, new, removed, left, crossings, wall hits, max iterations, floored cells,
        A-R fallbacks, particles entering from ghosts]"""
        out = np.zeros(11, dtype=np.int64)
        lib().oracle_stats(self.ctx, _p(out, C.c_int64))
        return out

    def geometry(self):
        dt = np.zeros(self.C)
        vol = np.zeros(self.C)
        lib().oracle_get_geometry(self.ctx, dptr(dt), dptr(vol), None, None)
        return dt, vol

    def mesh_tables(self):
        """Cells (x_c, y_c, area) [C, 3]; faces (L, R, tag) [F, 3] and (n_x, n_y, length, d_L, d_R) [F, 5]."""
        cells = np.zeros((self.C, 3))
        faces = np.zeros((self.F, 3), dtype=np.int32)
        fgeo = np.zeros((self.F, 5))
        self._check(lib().oracle_get_mesh(self.ctx, dptr(cells), _p(faces, C.c_int32), dptr(fgeo)))
        return cells, faces, fgeo

    def particles(self):
        n = lib().oracle_num_particles(self.ctx)
        pid = np.zeros(n, dtype=np.uint64)
        cell = np.zeros(n, dtype=np.int32)
        f = [np.zeros(n) for _ in range(6)]
        lib().oracle_get_particles(self.ctx, C.c_int64(n), _p(pid, C.c_uint64), _p(cell, C.c_int32),
                                   *[dptr(a) for a in f])
        return dict(pid=pid, cell=cell, x=f[0], y=f[1], u=f[2], v=f[3], w=f[4], m=f[5])

    def set_state(self, step, W, wret, parts):
        W = np.ascontiguousarray(W, dtype=np.float64).reshape(-1)
        wret = np.ascontiguousarray(wret, dtype=np.int64).reshape(-1)
        n = len(parts["pid"])
        arrs = [np.ascontiguousarray(parts[k], dtype=np.float64) for k in ("x", "y", "u", "v", "w", "m")]
        pid = np.ascontiguousarray(parts["pid"], dtype=np.uint64)
        cell = np.ascontiguousarray(parts["cell"], dtype=np.int32)
        self._check(lib().oracle_set_state(self.ctx, C.c_int64(step), dptr(W), _p(wret, C.c_int64), C.c_int64(n),
                                           _p(pid, C.c_uint64), _p(cell, C.c_int32), *[dptr(a) for a in arrs]))

    def tallies(self):
        wm, wpl, wret = (np.zeros(5 * self.C, dtype=np.int64) for _ in range(3))
        cross = np.zeros(2 * self.F, dtype=np.int64)
        wall = np.zeros(max(3 * self.nwall, 1), dtype=np.int64)
        frec = np.zeros(4 * self.F, dtype=np.int64)
        lib().oracle_get_tallies(self.ctx, _p(wm, C.c_int64), _p(wpl, C.c_int64), _p(wret, C.c_int64),
                                 _p(cross, C.c_int64), _p(wall, C.c_int64), _p(frec, C.c_int64))
        return dict(wm=wm.reshape(self.C, 5), wpl=wpl.reshape(self.C, 5), wret=wret.reshape(self.C, 5),
                    cross=cross.reshape(self.F, 2), wall=wall[:3 * self.nwall].reshape(self.nwall, 3),
                    frec=frec.reshape(self.F, 4))

    def cell_data(self):
        out = np.zeros(8 * self.C)
        lib().oracle_get_cell_data(self.ctx, dptr(out))
        return out.reshape(self.C, 8)

    def shakhov_weights(self):
        """Pr != 1: per cell the acceptance-rejection weights (a_x, a_y, M) of the last step's sampling (C x 3)."""
        out = np.zeros(3 * self.C)
        self._check(lib().oracle_get_shakhov(self.ctx, dptr(out)))
        return out.reshape(self.C, 3)

    def gradients(self):
        """Order 2: per cell the limited gradients (d/dx, d/dy) of the 4 components of W then of W^h, from the
        last step's decomposition (C x 8 x 2)."""
        out = np.zeros(16 * self.C)
        self._check(lib().oracle_get_gradients(self.ctx, dptr(out)))
        return out.reshape(self.C, 8, 2)

    def flux(self):
        out = np.zeros(4 * self.F)
        lib().oracle_get_flux(self.ctx, dptr(out))
        return out.reshape(self.F, 4)


def ar_sample(precision, seed, case_id, step, pid0, n, ax, ay, M):
    """n Shakhov acceptance-rejection normal triples (n x 3) and the fallback count (oracle_ar_sample)."""
    L = lib()
    L.oracle_ar_sample.restype = C.c_int64
    z = np.zeros(3 * n)
    fb = L.oracle_ar_sample(C.c_int32(precision), C.c_uint64(seed), C.c_uint32(case_id), C.c_int64(step),
                            C.c_uint64(pid0), C.c_int32(n), C.c_double(ax), C.c_double(ay), C.c_double(M), dptr(z))
    return z.reshape(n, 3), int(fb)


def balance_condition(dtL, dtR):
    a = np.ascontiguousarray(dtL, dtype=np.float64)
    b = np.ascontiguousarray(dtR, dtype=np.float64)
    out = np.zeros(2)
    lib().oracle_balance_condition(C.c_int32(len(a)), dptr(a), dptr(b), dptr(out))
    return out

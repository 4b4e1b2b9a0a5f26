"""Thin ctypes binding of libugkwp.so (include/ugkwp.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels; this module only converts numpy arrays and
Python scalars to the C ABI. Importing it loads the in-tree library and raises if it is missing or was
built without a usable CUDA device; there is no CPU fallback.
"""
from __future__ import annotations

import atexit
import ctypes as C
import os
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libugkwp.so")

STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ELIMIT", 5: "ENONPHYS", 6: "EOVERFLOW"}
LTS, GTS = 0, 1

# every entry point declared in include/ugkwp.h
EXPORTS = ["ugkwp_create", "ugkwp_create_unstructured", "ugkwp_destroy", "ugkwp_step", "ugkwp_residual", "ugkwp_surface", "ugkwp_reset_surface", "ugkwp_monitors",
           "ugkwp_set_field", "ugkwp_set_time_steps", "ugkwp_get_field", "ugkwp_stats", "ugkwp_num_particles", "ugkwp_get_particles",
           "ugkwp_set_state", "ugkwp_get_tallies", "ugkwp_get_cell_data", "ugkwp_get_flux", "ugkwp_get_geometry",
           "ugkwp_fixed_exponents", "ugkwp_save", "ugkwp_load", "ugkwp_batch_create", "ugkwp_batch_step",
           "ugkwp_batch_create_persistent", "ugkwp_batch_set_wait_limit", "ugkwp_batch_status", "ugkwp_batch_plan",
           "ugkwp_batch_destroy", "ugkwp_set_profiling", "ugkwp_profile", "ugkwp_mlp_create", "ugkwp_mlp_destroy",
           "ugkwp_mlp_num_params", "ugkwp_mlp_get_params", "ugkwp_mlp_set_params", "ugkwp_mlp_forward",
           "ugkwp_mlp_grad", "ugkwp_mlp_adam", "ugkwp_mlp_features", "ugkwp_field_accumulate", "ugkwp_mlp_dataset",
           "ugkwp_warm_start", "ugkwp_get_field_noalloc", "ugkwp_set_launch", "ugkwp_get_launch", "ugkwp_autotune",
           "ugkwp_last_error"]
STAGES = ["decompose", "sample", "particles", "wave_flux", "sort", "update"]   # wave_flux: ghost sources + wave fluxes


class UgkwpMesh(C.Structure):
    _fields_ = [("ni", C.c_int32), ("nj", C.c_int32), ("dim", C.c_int32), ("periodic_j", C.c_int32),
                ("xv", C.POINTER(C.c_double)), ("yv", C.POINTER(C.c_double)),
                ("bc_imin", C.POINTER(C.c_int32)), ("bc_imax", C.POINTER(C.c_int32)),
                ("bc_jmin", C.POINTER(C.c_int32)), ("bc_jmax", C.POINTER(C.c_int32))]


class UgkwpUMesh(C.Structure):
    _fields_ = [("n_vertices", C.c_int32), ("n_cells", C.c_int32), ("xv", C.POINTER(C.c_double)),
                ("yv", C.POINTER(C.c_double)), ("cells", C.POINTER(C.c_int32)), ("n_boundary", C.c_int32),
                ("boundary", C.POINTER(C.c_int32))]


class UgkwpGas(C.Structure):
    _fields_ = [("omega", C.c_double), ("Pr", C.c_double), ("wall_specular", C.c_double)]


class UgkwpOpts(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("case_id", C.c_uint32), ("n_ref", C.c_int32), ("precision", C.c_int32),
                ("wave_only", C.c_int32), ("record_faces", C.c_int32), ("capacity", C.c_int32),
                ("ghost_state", C.c_double * 4), ("stream", C.c_void_p), ("use_graph", C.c_int32),
                ("order", C.c_int32), ("dev_alloc", C.c_void_p), ("dev_free", C.c_void_p),
                ("alloc_user", C.c_void_p), ("emx_cutoff", C.c_double)]


# Device memory of the contexts from torch's caching allocator (ugkwp_opts.dev_alloc / dev_free)
_ALLOC_T = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE_T = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


def _torch_alloc(nbytes, stream, user):
    import torch
    s = torch.cuda.ExternalStream(stream) if stream else None
    try:
        return torch.cuda.caching_allocator_alloc(int(nbytes), stream=s)
    except RuntimeError:
        return None


def _torch_free(ptr, user):
    import torch
    torch.cuda.caching_allocator_delete(ptr)


_TORCH_ALLOC = _ALLOC_T(_torch_alloc)
_TORCH_FREE = _FREE_T(_torch_free)
_LIVE = weakref.WeakSet()   # contexts to destroy before the interpreter tears torch down


@atexit.register
def _close_all():
    for s in list(_LIVE):
        s.close()


_lib = None


def load():
    """Load libugkwp.so from the package directory (raises if it is absent)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2607_09552_b300.build`")
        lib = C.CDLL(LIB_PATH)
        lib.ugkwp_last_error.restype = C.c_char_p
        lib.ugkwp_num_particles.restype = C.c_int64
        lib.ugkwp_destroy.restype = None
        lib.ugkwp_batch_destroy.restype = None
        lib.ugkwp_mlp_destroy.restype = None
        lib.ugkwp_mlp_num_params.restype = C.c_int64
        _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t))


def _d(a):
    return _p(a, C.c_double)


class UgkwpFeatureMap(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("cx", "cy", "ell", "ext", "kn_lo", "kn_hi", "ma_lo", "ma_hi", "tw_lo",
                                          "tw_hi")]


def feature_map(fm: dict) -> UgkwpFeatureMap:
    return UgkwpFeatureMap(*[float(fm[k]) for k, _ in UgkwpFeatureMap._fields_])


def _dev(t):
    """Device pointer of a contiguous CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


class UgkwpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Solver:
    """One UGKWP-LTS context on the current CUDA device for a workload `Case`."""

    def __init__(self, case, gts: bool = False, precision: int = 0, wave_only: bool = False, seed: int | None = None,
                 case_id: int = 0, capacity: int = 0, use_graph: bool = False, stream=None,
                 record_faces: bool = False, order: int = 1, torch_memory: bool = True, emx_cutoff: float = 0.0):
        """torch_memory: the context's device memory from torch's caching allocator (else the library calls
        cudaMalloc itself). emx_cutoff: cells with e^{-dt/tau} below it sample no new particles (0: off)."""
        L = load()
        m = case.mesh
        self._keep = [np.ascontiguousarray(m.xv, dtype=np.float64), np.ascontiguousarray(m.yv, dtype=np.float64)]
        unstructured = hasattr(m, "cells")
        if unstructured:
            self._keep += [np.ascontiguousarray(a, dtype=np.int32) for a in (m.cells, m.boundary)]
            mesh = UgkwpUMesh(len(m.xv), m.ncells, _d(self._keep[0]), _d(self._keep[1]),
                              _p(self._keep[2], C.c_int32), len(m.boundary), _p(self._keep[3], C.c_int32))
        else:
            self._keep += [np.ascontiguousarray(a, dtype=np.int32)
                           for a in (m.bc_imin, m.bc_imax, m.bc_jmin, m.bc_jmax)]
            mesh = UgkwpMesh(m.ni, m.nj, m.dim, m.periodic_j, _d(self._keep[0]), _d(self._keep[1]),
                             *[_p(a, C.c_int32) for a in self._keep[2:]])
        gas = UgkwpGas(case.omega, case.Pr, getattr(case, "wall_specular", 0.0))
        opts = UgkwpOpts(case.seed if seed is None else seed, case_id, case.n_ref, precision, int(wave_only),
                         int(record_faces), capacity, (C.c_double * 4)(*case.ghost_state), C.c_void_p(stream),
                         int(use_graph), int(order))
        opts.emx_cutoff = float(emx_cutoff)
        if torch_memory:
            opts.dev_alloc = C.cast(_TORCH_ALLOC, C.c_void_p)
            opts.dev_free = C.cast(_TORCH_FREE, C.c_void_p)
        self.ctx = C.c_void_p()
        create = L.ugkwp_create_unstructured if unstructured else L.ugkwp_create
        st = create(C.byref(mesh), C.byref(gas), C.c_double(case.Kn), C.c_double(case.Ma),
                            C.c_double(case.Tw), C.c_double(case.cfl), C.c_int32(GTS if gts else LTS), C.byref(opts),
                            C.byref(self.ctx))
        if st != 0:
            msg = L.ugkwp_last_error(self.ctx).decode() if self.ctx else ""
            if self.ctx:
                L.ugkwp_destroy(self.ctx)
                self.ctx = None
            raise UgkwpError(st, f"ugkwp_create: {msg}")
        _LIVE.add(self)
        self.C = m.ncells
        nf, nw = C.c_int32(), C.c_int32()
        self._check(L.ugkwp_get_geometry(self.ctx, None, None, C.byref(nf), C.byref(nw)))
        self.F, self.nwall = nf.value, nw.value
        fx = (C.c_int32 * 3)()
        self._check(L.ugkwp_fixed_exponents(self.ctx, fx))
        self.fx = list(fx)
        if case.init_prim is not None:
            self.set_field(case.init_prim)

    def close(self):
        if getattr(self, "ctx", None):
            load().ugkwp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        self.close()

    def _check(self, st):
        if st != 0:
            raise UgkwpError(st, load().ugkwp_last_error(self.ctx).decode())

    def step(self, n: int = 1):
        self._check(load().ugkwp_step(self.ctx, C.c_int32(n)))

    def set_field(self, prim):
        a = np.ascontiguousarray(prim, dtype=np.float64).reshape(-1)
        self._check(load().ugkwp_set_field(self.ctx, _d(a)))

    def set_time_steps(self, dt):
        """Replace the local time steps (C values > 0) from the next step on (time-varying study, Sec. IV A)."""
        a = np.ascontiguousarray(dt, dtype=np.float64)
        self._check(load().ugkwp_set_time_steps(self.ctx, _d(a)))

    def field(self):
        W = np.zeros(4 * self.C)
        Wp = np.zeros(4 * self.C)
        self._check(load().ugkwp_get_field(self.ctx, _d(W), _d(Wp)))
        return W.reshape(self.C, 4), Wp.reshape(self.C, 4)

    def field_noalloc(self, with_wp: bool = True):
        """As field(), through ugkwp_get_field_noalloc (no device allocation; meshes up to 98304 cells)."""
        W = np.zeros(4 * self.C)
        Wp = np.zeros(4 * self.C) if with_wp else None
        self._check(load().ugkwp_get_field_noalloc(self.ctx, _d(W), None if Wp is None else _d(Wp)))
        return W.reshape(self.C, 4), (None if Wp is None else Wp.reshape(self.C, 4))

    def residual(self):
        out = np.zeros(8)
        self._check(load().ugkwp_residual(self.ctx, _d(out)))
        return out

    def surface(self, averaged: bool = True):
        p, t, q = (np.zeros(max(self.nwall, 1)) for _ in range(3))
        self._check(load().ugkwp_surface(self.ctx, _d(p), _d(t), _d(q), C.c_int32(self.nwall), C.c_int32(int(averaged))))
        return p[:self.nwall], t[:self.nwall], q[:self.nwall]

    def reset_surface(self):
        self._check(load().ugkwp_reset_surface(self.ctx))

    def monitors(self):
        """[C_d, C_H, stagnation C_p, C_Q (NaN without a stagnation point), then their EMAs] of the last step"""
        out = np.zeros(8)
        self._check(load().ugkwp_monitors(self.ctx, _d(out)))
        return out

    def stats(self):
        """[steps, particles, new, removed, left, crossings, wall hits, max iterations, cumulative
        particle-steps, cumulative new particles, cells floored in the last step, A-R fallbacks,
        particles entered from ghost sources]"""
        out = np.zeros(13, dtype=np.int64)
        self._check(load().ugkwp_stats(self.ctx, _p(out, C.c_int64)))
        return out

    def save(self, path: str):
        self._check(load().ugkwp_save(self.ctx, os.fsencode(path)))

    def load_checkpoint(self, path: str):
        self._check(load().ugkwp_load(self.ctx, os.fsencode(path)))

    def set_launch(self, chunk: int = 0, blocks_per_sm: int = 0, sort_every: int = 0, transport: int = 0):
        """Transport kernel 1: warp-chunked, 2: warp-staged (production precision; chunk 64 or 128 is its warp tile,
        4, 6 or 8 CTAs per SM); 0 keeps a value."""
        self._check(load().ugkwp_set_launch(self.ctx, C.c_int32(chunk), C.c_int32(blocks_per_sm), C.c_int32(sort_every),
                                            C.c_int32(transport)))

    def launch(self):
        """[chunk, blocks_per_sm, sort_every, transport kernel]"""
        out = (C.c_int32 * 4)()
        self._check(load().ugkwp_get_launch(self.ctx, out))
        return list(out)

    def autotune(self, steps: int = 16):
        """(best [chunk, blocks_per_sm, sort_every, transport], ms per step) after timing the candidates on real
        steps."""
        out = (C.c_int32 * 4)()
        ms = C.c_double()
        self._check(load().ugkwp_autotune(self.ctx, C.c_int32(steps), out, C.byref(ms)))
        return list(out), ms.value

    def set_profiling(self, on: bool):
        self._check(load().ugkwp_set_profiling(self.ctx, C.c_int32(int(on))))

    def profile(self):
        """(per-stage milliseconds summed over the profiled steps, number of profiled steps)"""
        ms = np.zeros(8)
        n = C.c_int64()
        self._check(load().ugkwp_profile(self.ctx, _d(ms), C.byref(n)))
        return dict(zip(STAGES, ms[:6])), n.value

    def num_particles(self) -> int:
        return int(load().ugkwp_num_particles(self.ctx))

    def geometry(self):
        dt = np.zeros(self.C)
        vol = np.zeros(self.C)
        self._check(load().ugkwp_get_geometry(self.ctx, _d(dt), _d(vol), None, None))
        return dt, vol

    def particles(self):
        n = self.num_particles()
        pid = np.zeros(max(n, 1), dtype=np.uint64)
        cell = np.zeros(max(n, 1), dtype=np.int32)
        f = [np.zeros(max(n, 1)) for _ in range(6)]
        self._check(load().ugkwp_get_particles(self.ctx, C.c_int64(n), _p(pid, C.c_uint64), _p(cell, C.c_int32),
                                               *[_d(a) for a in f]))
        return dict(pid=pid[:n], cell=cell[:n], x=f[0][:n], y=f[1][:n], u=f[2][:n], v=f[3][:n], w=f[4][:n],
                    m=f[5][:n])

    def set_state(self, step, W, wret, parts):
        W = np.ascontiguousarray(W, dtype=np.float64).reshape(-1)
        wret = np.ascontiguousarray(wret, dtype=np.int64).reshape(-1)
        n = len(parts["pid"])
        arrs = [np.ascontiguousarray(parts[k], dtype=np.float64) for k in ("x", "y", "u", "v", "w", "m")]
        pid = np.ascontiguousarray(parts["pid"], dtype=np.uint64)
        cell = np.ascontiguousarray(parts["cell"], dtype=np.int32)
        self._check(load().ugkwp_set_state(self.ctx, C.c_int64(step), _d(W), _p(wret, C.c_int64), C.c_int64(n),
                                           _p(pid, C.c_uint64), _p(cell, C.c_int32), *[_d(a) for a in arrs]))

    def tallies(self):
        wm, wpl, wret = (np.zeros(5 * self.C, dtype=np.int64) for _ in range(3))
        cross = np.zeros(2 * self.F, dtype=np.int64)
        wall = np.zeros(max(3 * self.nwall, 1), dtype=np.int64)
        frec = np.zeros(4 * self.F, dtype=np.int64)
        self._check(load().ugkwp_get_tallies(self.ctx, _p(wm, C.c_int64), _p(wpl, C.c_int64), _p(wret, C.c_int64),
                                             _p(cross, C.c_int64), _p(wall, C.c_int64), _p(frec, C.c_int64)))
        return dict(wm=wm.reshape(self.C, 5), wpl=wpl.reshape(self.C, 5), wret=wret.reshape(self.C, 5),
                    cross=cross.reshape(self.F, 2), wall=wall[:3 * self.nwall].reshape(self.nwall, 3),
                    frec=frec.reshape(self.F, 4))

    def cell_data(self):
        out = np.zeros(8 * self.C)
        self._check(load().ugkwp_get_cell_data(self.ctx, _d(out)))
        return out.reshape(self.C, 8)

    def flux(self):
        out = np.zeros(4 * self.F)
        self._check(load().ugkwp_get_flux(self.ctx, _d(out)))
        return out.reshape(self.F, 4)

    def field_accumulate(self, acc, reset: bool = False):
        """acc (float64 CUDA tensor of 4 C values) = W or acc + W."""
        if acc.dtype.itemsize != 8 or acc.numel() != 4 * self.C:
            raise ValueError("acc must hold 4 C float64 values")
        self._check(load().ugkwp_field_accumulate(self.ctx, _dev(acc), C.c_int32(int(reset))))

    def dataset(self, fmap: dict, W=None, scale: float = 1.0, n_features: int = 64):
        """(features [C][n_features], targets [C][4]) float32 CUDA tensors of the current field or of W * scale."""
        import torch
        feat = torch.empty((self.C, n_features), dtype=torch.float32, device="cuda")
        targ = torch.empty((self.C, 4), dtype=torch.float32, device="cuda")
        fm = feature_map(fmap)
        self._check(load().ugkwp_mlp_dataset(self.ctx, C.byref(fm), _dev(W), C.c_double(scale),
                                             C.c_int32(n_features), _dev(feat), _dev(targ)))
        return feat, targ

    def warm_start(self, mlp, fmap: dict):
        fm = feature_map(fmap)
        self._check(load().ugkwp_warm_start(self.ctx, mlp.h, C.byref(fm)))


class Batch:
    """Several Solver contexts advanced together by one graph launch per step (ugkwp_batch_*): per-case streams
    of the step kernels, or (persistent=True) the batched persistent kernel with `ctas_per_sm` CTAs per SM."""

    def __init__(self, solvers, stream=None, persistent: bool = False, ctas_per_sm: int = 0):
        L = load()
        self.solvers = list(solvers)
        arr = (C.c_void_p * len(self.solvers))(*[s.ctx.value for s in self.solvers])
        self.h = C.c_void_p()
        if persistent:
            st = L.ugkwp_batch_create_persistent(arr, C.c_int32(len(self.solvers)), C.c_void_p(stream),
                                                 C.c_int32(ctas_per_sm), C.byref(self.h))
        else:
            st = L.ugkwp_batch_create(arr, C.c_int32(len(self.solvers)), C.c_void_p(stream), C.byref(self.h))
        if st != 0:
            raise UgkwpError(st, "ugkwp_batch_create_persistent" if persistent else "ugkwp_batch_create")

    def step(self, n: int = 1):
        st = load().ugkwp_batch_step(self.h, C.c_int32(n))
        if st != 0:
            raise UgkwpError(st, "ugkwp_batch_step")

    def set_wait_limit(self, limit_ns: int, stall: bool = False):
        st = load().ugkwp_batch_set_wait_limit(self.h, C.c_int64(limit_ns), C.c_int32(int(stall)))
        if st != 0:
            raise UgkwpError(st, "ugkwp_batch_set_wait_limit")

    def status(self):
        """(status, where): 0 or ELIMIT (4) once a persistent batch stopped; where = case * 20 + stage."""
        w = C.c_int32(-1)
        st = load().ugkwp_batch_status(self.h, C.byref(w))
        return st, w.value

    def plan(self):
        """[persistent, items per step, CTAs per launch, CTAs per SM]"""
        out = (C.c_int32 * 4)()
        st = load().ugkwp_batch_plan(self.h, out)
        if st != 0:
            raise UgkwpError(st, "ugkwp_batch_plan")
        return list(out)

    def close(self):
        if getattr(self, "h", None):
            load().ugkwp_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


class Mlp:
    """The warm-start network (ugkwp_mlp_*): parameters, forward, gradient and Adam on the device."""

    def __init__(self, n_features: int = 64, width: int = 256, depth: int = 4, n_out: int = 4, params=None,
                 stream=None):
        L = load()
        self.shape = (n_features, width, depth, n_out)
        self.h = C.c_void_p()
        p = None
        if params is not None:
            p = np.ascontiguousarray(params, dtype=np.float32)
        st = L.ugkwp_mlp_create(C.c_int32(n_features), C.c_int32(width), C.c_int32(depth), C.c_int32(n_out),
                                None if p is None else _p(p, C.c_float), C.c_void_p(stream), C.byref(self.h))
        if st != 0:
            raise UgkwpError(st, "ugkwp_mlp_create")
        self.n = int(L.ugkwp_mlp_num_params(self.h))
        if p is not None and p.size != self.n:
            self.close()
            raise ValueError(f"expected {self.n} parameters, got {p.size}")

    def close(self):
        if getattr(self, "h", None):
            load().ugkwp_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    @staticmethod
    def _check(st, what):
        if st != 0:
            raise UgkwpError(st, what)

    def params(self):
        out = np.zeros(self.n, dtype=np.float32)
        self._check(load().ugkwp_mlp_get_params(self.h, _p(out, C.c_float), None), "ugkwp_mlp_get_params")
        return out

    def grad(self):
        out = np.zeros(self.n, dtype=np.float32)
        self._check(load().ugkwp_mlp_get_params(self.h, None, _p(out, C.c_float)), "ugkwp_mlp_get_params")
        return out

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != self.n:
            raise ValueError(f"expected {self.n} parameters, got {p.size}")
        self._check(load().ugkwp_mlp_set_params(self.h, _p(p, C.c_float)), "ugkwp_mlp_set_params")

    def forward(self, x):
        import torch
        y = torch.empty((x.shape[0], self.shape[3]), dtype=torch.float32, device=x.device)
        self._check(load().ugkwp_mlp_forward(self.h, _dev(x), C.c_int32(x.shape[0]), _dev(y)), "ugkwp_mlp_forward")
        return y

    def loss_grad(self, x, t, rows=None, want_loss: bool = True):
        n = x.shape[0] if rows is None else rows.shape[0]
        loss = C.c_float()
        self._check(load().ugkwp_mlp_grad(self.h, _dev(x), _dev(t), _dev(rows), C.c_int32(n),
                                          C.byref(loss) if want_loss else None), "ugkwp_mlp_grad")
        return loss.value if want_loss else None

    def adam(self, lr: float):
        self._check(load().ugkwp_mlp_adam(self.h, C.c_float(lr)), "ugkwp_mlp_adam")


def mlp_features(fmap: dict, x, y, Kn: float, Ma: float, Tw: float, n_features: int = 64, stream=None):
    """Feature rows (float32 CUDA tensor [n][n_features]) of the points of float64 CUDA tensors x, y."""
    import torch
    feat = torch.empty((x.shape[0], n_features), dtype=torch.float32, device=x.device)
    fm = feature_map(fmap)
    st = load().ugkwp_mlp_features(C.byref(fm), _dev(x), _dev(y), C.c_int32(x.shape[0]), C.c_double(Kn),
                                   C.c_double(Ma), C.c_double(Tw), C.c_int32(n_features), _dev(feat),
                                   C.c_void_p(stream))
    if st != 0:
        raise UgkwpError(st, "ugkwp_mlp_features")
    return feat

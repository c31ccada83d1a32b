"""Thin ctypes binding of ``libcswdg.so`` (include/cswdg.h).

Argument marshalling only: every step of the method runs in the CUDA
library.  The functions keep the C names; ``Solver`` wraps one solver handle
with numpy in/out arrays.  Importing this module loads the library and raises
if it is missing or cannot be loaded -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcswdg.so")

OK, EINVAL, ECUDA, EMESH, ENONPHYS, ELSQ, ETIMEOUT, ENOMEM = range(8)
STATUS_NAMES = ["OK", "EINVAL", "ECUDA", "EMESH", "ENONPHYS", "ELSQ", "ETIMEOUT", "ENOMEM"]
BURGERS, EULER = 0, 1
FP64, FP32_BULK, FP32 = 0, 1, 2
LIMITER_OFF, LIMITER_KXRCF, LIMITER_ALL = 0, 1, 2


class cswdg_config(C.Structure):
    _fields_ = [("equation", C.c_int32), ("degree", C.c_int32), ("precision", C.c_int32),
                ("limiter", C.c_int32), ("c_k", C.c_double), ("cfl", C.c_double),
                ("gamma", C.c_double), ("stream", C.c_void_p)]


class CswdgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} (run paper_2106_06280_gb300/build.py)")
    L = C.CDLL(LIB_PATH)
    vp, dp, i32, i64 = C.c_void_p, C.POINTER(C.c_double), C.c_int32, C.c_int64
    sig = {
        "cswdg_create": ([C.POINTER(cswdg_config), C.POINTER(vp)], C.c_int),
        "cswdg_destroy": ([vp], None),
        "cswdg_last_error": ([vp], C.c_char_p),
        "cswdg_set_boundary": ([vp, i32, i32, dp, i32], C.c_int),
        "cswdg_mesh_upload": ([vp, i64, dp, i64, C.POINTER(i32), i64, C.POINTER(i32), dp], C.c_int),
        "cswdg_num_ic_points": ([vp], i32),
        "cswdg_ic_points": ([vp, dp], C.c_int),
        "cswdg_project_ic": ([vp, dp, i32], C.c_int),
        "cswdg_step": ([vp, C.c_double, i64, C.c_double, dp], C.c_int),
        "cswdg_profile_step": ([vp, C.c_double, i64, C.c_double, dp, C.POINTER(i64)], C.c_int),
        "cswdg_launches_per_step": ([vp, i32], i32),
        "cswdg_get_time": ([vp, dp], C.c_int),
        "cswdg_set_time": ([vp, C.c_double], C.c_int),
        "cswdg_read_modes": ([vp, dp], C.c_int),
        "cswdg_write_modes": ([vp, dp], C.c_int),
        "cswdg_read_flags": ([vp, C.POINTER(C.c_uint8)], C.c_int),
        "cswdg_num_flagged": ([vp, C.POINTER(i64)], C.c_int),
        "cswdg_conservation": ([vp, dp], C.c_int),
        "cswdg_eval_rhs": ([vp, C.c_double, dp, dp], C.c_int),
        "cswdg_limit": ([vp, C.c_double, dp, dp, C.POINTER(C.c_uint8)], C.c_int),
        "cswdg_cfl_dt": ([vp, dp], C.c_int),
        "cswdg_stage_dev": ([vp, vp, vp, vp, C.c_double, C.c_double, C.c_double, C.c_double], C.c_int),
        "cswdg_internal_layout": ([vp, C.POINTER(i64), C.POINTER(i32)], C.c_int),
        "cswdg_stencil_operator": ([vp, i64, dp, C.POINTER(i32)], C.c_int),
        "cswdg_conservation_noalloc": ([vp, vp, vp], C.c_int),
        "cswdg_selftest_timeout": ([vp, i32], C.c_int),
        "cswdg_host_mesh": ([i32, C.POINTER(i32), i64, dp, i64, C.POINTER(i32), i64, C.POINTER(i32), dp, dp,
                             C.POINTER(i32), C.POINTER(C.c_uint8), C.POINTER(i32)], C.c_int),
        "cswdg_autotune": ([vp, dp, C.POINTER(i32)], C.c_int),
        "cswdg_rhs_adjoint": ([vp, C.c_double, dp, dp, dp], C.c_int),
        "cswdg_adjoint_steps": ([vp, C.c_double, i64, i32, dp, dp, dp, dp, dp], C.c_int),
        "cswdg_limit_adjoint": ([vp, C.c_double, dp, dp, dp, C.POINTER(C.c_uint8)], C.c_int),
        "cswdg_set_stage_shape": ([vp, i32, i32, i32], C.c_int),
        "cswdg_probe_fp64_fma": ([vp, dp], C.c_int),
        "cswdg_read_modes_f32": ([vp, C.POINTER(C.c_float)], C.c_int),
        "cswdg_write_modes_f32": ([vp, C.POINTER(C.c_float)], C.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    return L


lib = _load()
EXPORTED = ["cswdg_create", "cswdg_destroy", "cswdg_last_error", "cswdg_set_boundary", "cswdg_mesh_upload",
            "cswdg_num_ic_points", "cswdg_ic_points", "cswdg_project_ic", "cswdg_step", "cswdg_profile_step",
            "cswdg_launches_per_step", "cswdg_get_time",
            "cswdg_set_time", "cswdg_read_modes", "cswdg_write_modes", "cswdg_read_flags", "cswdg_num_flagged",
            "cswdg_conservation", "cswdg_eval_rhs", "cswdg_limit", "cswdg_cfl_dt", "cswdg_stage_dev",
            "cswdg_internal_layout", "cswdg_stencil_operator", "cswdg_conservation_noalloc", "cswdg_selftest_timeout",
            "cswdg_autotune", "cswdg_rhs_adjoint", "cswdg_adjoint_steps", "cswdg_limit_adjoint",
            "cswdg_set_stage_shape", "cswdg_host_mesh", "cswdg_probe_fp64_fma",
            "cswdg_read_modes_f32", "cswdg_write_modes_f32"]
TUNE_CANDIDATES = 11


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def probe_fp64_fma(stream=None):
    """Measured FP64 FMA throughput of the current device in GFLOP/s."""
    g = np.zeros(1)
    st = lib.cswdg_probe_fp64_fma(C.c_void_p(stream or 0), _p(g))
    if st != 0:
        raise CswdgError(st, "cswdg_probe_fp64_fma failed")
    return float(g[0])


def host_mesh(problem, degree):
    """Connectivity, locality order and geometry of a workloads.Problem as the
    library builds them on the host (no device): dict of geo (14, nc), nbr
    (3, nc), nbf (nc,), perm (nc,), all in the internal cell order."""
    m = problem.mesh
    kinds = np.zeros(16, dtype=np.int32)
    for tag, (kind, _) in problem.boundaries.items():
        kinds[tag] = kind
    xy = _d(m.xy)
    tri = np.ascontiguousarray(m.tri, dtype=np.int32)
    bface = np.ascontiguousarray(m.bface, dtype=np.int32)
    per = None if m.period is None else _d(m.period)
    nc = tri.shape[0]
    geo = np.zeros((14, nc))
    nbr = np.zeros((3, nc), dtype=np.int32)
    nbf = np.zeros(nc, dtype=np.uint8)
    perm = np.zeros(nc, dtype=np.int32)
    st = lib.cswdg_host_mesh(degree, _p(kinds, C.c_int32), xy.shape[0], _p(xy), nc, _p(tri, C.c_int32), bface.shape[0],
                             _p(bface, C.c_int32), None if per is None else _p(per), _p(geo), _p(nbr, C.c_int32),
                             _p(nbf, C.c_uint8), _p(perm, C.c_int32))
    if st != OK:
        raise CswdgError(st, "host mesh processing failed")
    return {"geo": geo, "nbr": nbr, "nbf": nbf, "perm": perm}


def _p(a, ctype=C.c_double):
    return a.ctypes.data_as(C.POINTER(ctype))


class Solver:
    """One solver handle.  equation: BURGERS/EULER, degree 1/2, precision
    FP64/FP32_BULK/FP32, limiter LIMITER_*; stream: a cudaStream_t as int (e.g.
    torch.cuda.current_stream().cuda_stream) or None."""

    def __init__(self, equation, degree, precision=FP64, limiter=LIMITER_KXRCF, c_k=1.0, cfl=0.1,
                 gamma=1.4, stream=None):
        cfg = cswdg_config(equation, degree, precision, limiter, c_k, cfl, gamma, stream)
        h = C.c_void_p()
        st = lib.cswdg_create(C.byref(cfg), C.byref(h))
        if st != OK:
            raise CswdgError(st, "cswdg_create failed")
        self.h = h
        self.nvar = 1 if equation == BURGERS else 4
        self.np = (degree + 1) * (degree + 2) // 2
        self.nc = 0

    def _chk(self, st):
        if st != OK:
            raise CswdgError(st, lib.cswdg_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            lib.cswdg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_boundary(self, tag, kind, params=()):
        p = _d(list(params) + [0.0])
        self._chk(lib.cswdg_set_boundary(self.h, tag, kind, _p(p), len(params)))

    def mesh_upload(self, xy, tri, bface, period=None):
        xy = _d(xy)
        tri = np.ascontiguousarray(tri, dtype=np.int32)
        bface = np.ascontiguousarray(bface, dtype=np.int32)
        per = None if period is None else _d(period)
        self._chk(lib.cswdg_mesh_upload(self.h, xy.shape[0], _p(xy), tri.shape[0], _p(tri, C.c_int32),
                                        bface.shape[0], _p(bface, C.c_int32), None if per is None else _p(per)))
        self.nc = tri.shape[0]

    def setup(self, problem):
        """Boundary table and mesh of a workloads.Problem."""
        for tag, (kind, par) in problem.boundaries.items():
            self.set_boundary(tag, kind, par)
        m = problem.mesh
        self.mesh_upload(m.xy, m.tri, m.bface, m.period)

    def ic_points(self):
        q = lib.cswdg_num_ic_points(self.h)
        xy = np.zeros((self.nc, q, 2))
        self._chk(lib.cswdg_ic_points(self.h, _p(xy)))
        return xy

    def project_ic(self, fn, apply_limiter=1):
        """apply_limiter: 0 none, 1 configured limiter once, 2 every cell once."""
        xy = self.ic_points()
        vals = _d(fn(xy[..., 0].ravel(), xy[..., 1].ravel())).reshape(self.nc, -1, self.nvar)
        vals = _d(vals)
        self._chk(lib.cswdg_project_ic(self.h, _p(vals), int(apply_limiter)))

    def step(self, dt=0.0, nsteps=1, t_end=1e300):
        t = np.zeros(1)
        self._chk(lib.cswdg_step(self.h, dt, nsteps, t_end, _p(t)))
        return float(t[0])

    def profile_step(self, dt=0.0, nsteps=1, t_end=1e300):
        ms = np.zeros(5)
        nl = C.c_int64()
        self._chk(lib.cswdg_profile_step(self.h, dt, nsteps, t_end, _p(ms), C.byref(nl)))
        return dict(cfl=ms[0], stage=ms[1], detect=ms[2], limit=ms[3], scatter=ms[4]), int(nl.value)

    def autotune(self):
        """Pick the stage kernel's launch shape on the current state; returns
        (cells per block, grid or 0, tile_faces 0/1, per-candidate ms)."""
        ms = np.zeros(TUNE_CANDIDATES)
        ch = np.zeros(3, dtype=np.int32)
        self._chk(lib.cswdg_autotune(self.h, _p(ms), ch.ctypes.data_as(C.POINTER(C.c_int32))))
        return int(ch[0]), int(ch[1]), int(ch[2]), ms

    def set_stage_shape(self, cells_per_block, grid=0, tile_faces=0):
        self._chk(lib.cswdg_set_stage_shape(self.h, cells_per_block, grid, tile_faces))

    def launches_per_step(self, use_cfl=True):
        return int(lib.cswdg_launches_per_step(self.h, int(use_cfl)))

    def get_time(self):
        t = np.zeros(1)
        self._chk(lib.cswdg_get_time(self.h, _p(t)))
        return float(t[0])

    def set_time(self, t):
        self._chk(lib.cswdg_set_time(self.h, t))

    def read_modes(self, out=None):
        if out is None:
            out = np.zeros((self.nc, self.nvar, self.np))
        self._chk(lib.cswdg_read_modes(self.h, _p(out)))
        return out

    def write_modes(self, modes):
        modes = _d(modes)
        self._chk(lib.cswdg_write_modes(self.h, _p(modes)))

    def read_modes_f32(self, out=None):
        """The modal state as float32 (same layout as read_modes)."""
        if out is None:
            out = np.zeros((self.nc, self.nvar, self.np), dtype=np.float32)
        assert out.dtype == np.float32 and out.flags.c_contiguous
        self._chk(lib.cswdg_read_modes_f32(self.h, _p(out, C.c_float)))
        return out

    def write_modes_f32(self, modes):
        modes = np.ascontiguousarray(modes, dtype=np.float32)
        self._chk(lib.cswdg_write_modes_f32(self.h, _p(modes, C.c_float)))

    def read_flags(self):
        f = np.zeros(self.nc, dtype=np.uint8)
        self._chk(lib.cswdg_read_flags(self.h, _p(f, C.c_uint8)))
        return f

    def num_flagged(self):
        n = C.c_int64()
        self._chk(lib.cswdg_num_flagged(self.h, C.byref(n)))
        return int(n.value)

    def conservation(self):
        s = np.zeros(self.nvar)
        self._chk(lib.cswdg_conservation(self.h, _p(s)))
        return s

    def eval_rhs(self, modes, t=0.0):
        modes = _d(modes)
        out = np.zeros_like(modes)
        self._chk(lib.cswdg_eval_rhs(self.h, t, _p(modes), _p(out)))
        return out

    def rhs_adjoint(self, modes, lam, t=0.0):
        """(dL_h/du)^T lam at the state modes (user basis and cell order)."""
        modes, lam = _d(modes), _d(lam)
        out = np.zeros_like(modes)
        self._chk(lib.cswdg_rhs_adjoint(self.h, t, _p(modes), _p(lam), _p(out)))
        return out

    def adjoint_steps(self, u0, gT, dt, nsteps, checkpoint_every=20, return_dts=False):
        """Run nsteps steps from u0 (size dt, or the CFL rule when dt <= 0, the
        sizes then held fixed backwards) and return (u_N, (du_N/du_0)^T gT),
        plus the step sizes when return_dts."""
        u0, gT = _d(u0), _d(gT)
        uT = np.zeros_like(u0)
        g0 = np.zeros_like(u0)
        dts = np.zeros(int(nsteps))
        self._chk(lib.cswdg_adjoint_steps(self.h, dt, nsteps, checkpoint_every, _p(u0), _p(gT), _p(uT), _p(g0), _p(dts)))
        return (uT, g0, dts) if return_dts else (uT, g0)

    def selftest_timeout(self, polls=4096):
        """Run the bounded-wait self-test; raises CswdgError (ETIMEOUT) as designed."""
        self._chk(lib.cswdg_selftest_timeout(self.h, polls))

    def limit_adjoint(self, modes, lam, t=0.0):
        """(dLim/du)^T lam at the state modes with the flags frozen; returns (grad, flags)."""
        modes, lam = _d(modes), _d(lam)
        out = np.zeros_like(modes)
        fl = np.zeros(self.nc, dtype=np.uint8)
        self._chk(lib.cswdg_limit_adjoint(self.h, t, _p(modes), _p(lam), _p(out), _p(fl, C.c_uint8)))
        return out, fl

    def limit(self, modes, t=0.0):
        modes = _d(modes)
        out = np.zeros_like(modes)
        fl = np.zeros(self.nc, dtype=np.uint8)
        self._chk(lib.cswdg_limit(self.h, t, _p(modes), _p(out), _p(fl, C.c_uint8)))
        return out, fl

    def cfl_dt(self):
        d = np.zeros(1)
        self._chk(lib.cswdg_cfl_dt(self.h, _p(d)))
        return float(d[0])

    def stage_dev(self, un_ptr, uprev_ptr, out_ptr, a, b, dt, t_rhs):
        self._chk(lib.cswdg_stage_dev(self.h, un_ptr, uprev_ptr, out_ptr, a, b, dt, t_rhs))

    def conservation_noalloc(self, modes_dev_ptr, sums_dev_ptr):
        """Queue the allocation-free conservation sums of a device state in the
        internal layout into a device buffer of nvar doubles (no allocation)."""
        self._chk(lib.cswdg_conservation_noalloc(self.h, modes_dev_ptr, sums_dev_ptr))

    def stencil_operator(self, cell):
        n = C.c_int32()
        self._chk(lib.cswdg_stencil_operator(self.h, cell, None, C.byref(n)))
        out = np.zeros(max(n.value, 1))
        self._chk(lib.cswdg_stencil_operator(self.h, cell, _p(out), C.byref(n)))
        return out[: n.value]

    def internal_layout(self):
        ld = C.c_int64()
        perm = np.zeros(self.nc, dtype=np.int32)
        self._chk(lib.cswdg_internal_layout(self.h, C.byref(ld), _p(perm, C.c_int32)))
        return int(ld.value), perm

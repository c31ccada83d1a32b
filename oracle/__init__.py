"""ctypes front end of the FP64 CPU oracle (``cswdg_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and
the benchmark's CPU-baseline leg, never by the product path.  It shares no
code with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cswdg_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_bp = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction: same bits on x86 and Arm).

    OpenMP spreads the independent per-cell loops (operator, detection,
    reconstruction) over the host cores; every cell is computed by one thread
    from read-only inputs, so the results do not depend on the thread count.
    """
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-D_GNU_SOURCE", "-fPIC", "-shared",
                               "-ffp-contract=off", "-fopenmp", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        vp = C.c_void_p
        L.or_create.restype = vp
        L.or_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double]
        L.or_destroy.argtypes = [vp]
        L.or_error.argtypes = [vp]
        L.or_nvol.argtypes = [vp]
        L.or_nscp.argtypes = [vp]
        L.or_set_boundary.argtypes = [vp, C.c_int, C.c_int, _dp, C.c_int]
        L.or_mesh.argtypes = [vp, C.c_int, _dp, C.c_int, _ip, C.c_int, _ip, C.c_void_p]
        L.or_rhs.argtypes = [vp, _dp, C.c_double, _dp]
        L.or_rhs_cells.argtypes = [vp, _dp, C.c_double, C.c_int, _ip, _dp]
        L.or_detect.argtypes = [vp, _dp, C.c_double, _bp, _dp]
        L.or_detect_cells.argtypes = [vp, _dp, C.c_double, C.c_int, _ip, _bp, _dp]
        L.or_limit.argtypes = [vp, _dp, C.c_double, _dp, _bp]
        L.or_limit_cells.argtypes = [vp, _dp, C.c_double, C.c_int, _ip, _dp]
        L.or_cfl_dt.restype = C.c_double
        L.or_cfl_dt.argtypes = [vp, _dp, C.c_double]
        L.or_step.argtypes = [vp, _dp, C.c_double, C.c_double, C.c_void_p]
        L.or_run.argtypes = [vp, _dp, C.c_double, C.c_double, C.c_double, C.c_int, _dp]
        L.or_volume_points.argtypes = [vp, _dp]
        L.or_project.argtypes = [vp, _dp, _dp]
        L.or_conservation.argtypes = [vp, _dp, _dp]
        L.or_project_cells.argtypes = [vp, C.c_int, _ip, _dp, _dp]
        L.or_eval_points.argtypes = [vp, _dp, C.c_int, _ip, _dp, _dp]
        L.or_error_rule.argtypes = [vp, _dp, _dp]
        L.or_connectivity.argtypes = [vp, _ip, _ip, _dp]
        L.or_hook_gauss_legendre.argtypes = [C.c_int, _dp, _dp]
        L.or_hook_rule.argtypes = [C.c_int, C.c_int, _dp, _dp]
        L.or_hook_psi.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, _dp]
        L.or_hook_lsq.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp]
        L.or_hook_stencil.argtypes = [vp, C.c_int, _dp, _ip]
        L.or_hook_subcell_means.argtypes = [vp, _dp, C.c_int, C.c_double, _dp]
        L.or_hook_weno.argtypes = [vp, C.c_int, C.c_double, _dp, C.c_void_p, C.c_int, _dp, _dp]
        L.or_hook_beta.restype = C.c_double
        L.or_hook_beta.argtypes = [vp, C.c_int, C.c_int, _dp, C.c_int]
        L.or_hook_frame.argtypes = [vp, C.c_int, _dp]
        L.or_hook_flux.argtypes = [vp, _dp, _dp, C.c_double, C.c_double, _dp]
        L.or_hook_limit_cell.argtypes = [vp, _dp, C.c_double, C.c_int, _dp]
        L.or_hook_limit_cell_linear.argtypes = [vp, _dp, C.c_double, C.c_int, _dp]
        L.or_euler_eigen.argtypes = [C.c_double, _dp, C.c_double, C.c_double, _dp, _dp]
        _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


class Oracle:
    """One problem on one mesh: eq 0 Burgers / 1 Euler, degree k in {1,2},
    limiter 0 off / 1 KXRCF / 2 every cell."""

    def __init__(self, problem=None, k=1, limiter=1, ck=1.0, gamma=1.4, *, equation=None, mesh=None,
                 boundaries=None):
        L = lib()
        if problem is not None:
            equation, mesh, boundaries = problem.equation, problem.mesh, problem.boundaries
        self.eq, self.k, self.limiter = equation, k, limiter
        self.nvar = 1 if equation == 0 else 4
        self.np = (k + 1) * (k + 2) // 2
        self.mesh = mesh
        self.h = L.or_create(equation, k, limiter, ck, gamma)
        if L.or_error(self.h):
            raise RuntimeError("oracle quadrature set-up failed")
        for tag, (kind, par) in (boundaries or {}).items():
            par = _f64(list(par) + [0.0])
            L.or_set_boundary(self.h, int(tag), int(kind), par, len(par) - 1)
        self._period = None if mesh.period is None else _f64(mesh.period)
        st = L.or_mesh(self.h, mesh.nv, _f64(mesh.xy), mesh.nc, _i32(mesh.tri), len(mesh.bface),
                       _i32(mesh.bface),
                       None if self._period is None else self._period.ctypes.data)
        if st != 0:
            raise RuntimeError(f"oracle mesh set-up failed ({st})")
        self.nc = mesh.nc

    def __del__(self):
        try:
            lib().or_destroy(self.h)
        except Exception:
            pass

    def shape(self):
        return (self.nc, self.nvar, self.np)

    def zeros(self):
        return np.zeros(self.shape())

    # --- initial data ---
    def volume_points(self):
        q = lib().or_nvol(self.h)
        xy = np.zeros((self.nc, q, 2))
        lib().or_volume_points(self.h, xy)
        return xy

    def project(self, fn):
        xy = self.volume_points()
        vals = _f64(fn(xy[..., 0].ravel(), xy[..., 1].ravel())).reshape(self.nc, -1, self.nvar)
        u = self.zeros()
        lib().or_project(self.h, _f64(vals), u)
        return u

    def project_cells(self, fn, cells, u):
        """Project fn onto the modes of the listed cells of u (in place)."""
        cells = _i32(cells)
        xy = self.volume_points()[cells]
        vals = _f64(fn(xy[..., 0].ravel(), xy[..., 1].ravel())).reshape(len(cells), -1, self.nvar)
        lib().or_project_cells(self.h, len(cells), cells, _f64(vals), u)
        return u

    # --- operator pieces ---
    def rhs(self, u, t=0.0):
        out = self.zeros()
        lib().or_rhs(self.h, _f64(u), t, out)
        return out

    def rhs_cells(self, u, cells, t=0.0):
        cells = _i32(cells)
        out = np.zeros((len(cells), self.nvar, self.np))
        lib().or_rhs_cells(self.h, _f64(u), t, len(cells), cells, out)
        return out

    def detect(self, u, t=0.0):
        fl = np.zeros(self.nc, dtype=np.uint8)
        R = np.zeros(self.nc)
        lib().or_detect(self.h, _f64(u), t, fl, R)
        return fl, R

    def detect_cells(self, u, cells, t=0.0):
        cells = _i32(cells)
        fl = np.zeros(len(cells), dtype=np.uint8)
        R = np.zeros(len(cells))
        lib().or_detect_cells(self.h, _f64(u), t, len(cells), cells, fl, R)
        return fl, R

    def limit(self, u, t=0.0):
        out = self.zeros()
        fl = np.zeros(self.nc, dtype=np.uint8)
        st = lib().or_limit(self.h, _f64(u), t, out, fl)
        return out, fl, st

    def limit_cells(self, u, cells, t=0.0):
        cells = _i32(cells)
        out = np.zeros((len(cells), self.nvar, self.np))
        st = lib().or_limit_cells(self.h, _f64(u), t, len(cells), cells, out)
        return out, st

    def cfl_dt(self, u, cfl):
        return lib().or_cfl_dt(self.h, _f64(u), cfl)

    def step(self, u, t, dt):
        u = _f64(u).copy()
        fl = np.zeros(self.nc, dtype=np.uint8)
        st = lib().or_step(self.h, u, t, dt, fl.ctypes.data)
        return u, fl, st

    def run(self, u, t0, t_end, cfl, max_steps=10 ** 9):
        u = _f64(u).copy()
        tout = np.zeros(1)
        n = lib().or_run(self.h, u, t0, t_end, cfl, max_steps, tout)
        if n < 0:
            raise RuntimeError("oracle limiter failure")
        return u, n, float(tout[0])

    def conservation(self, u):
        s = np.zeros(self.nvar)
        lib().or_conservation(self.h, _f64(u), s)
        return s

    def error_rule(self):
        n = 36
        xy = np.zeros((self.nc, n, 2))
        w = np.zeros((self.nc, n))
        lib().or_error_rule(self.h, xy, w)
        return xy, w

    def eval_points(self, u, cells, xy):
        cells = _i32(cells)
        out = np.zeros((len(cells), self.nvar))
        lib().or_eval_points(self.h, _f64(u), len(cells), cells, _f64(xy), out)
        return out

    def connectivity(self):
        nb = np.zeros(3 * self.nc, dtype=np.int32)
        nbf = np.zeros(3 * self.nc, dtype=np.int32)
        sh = np.zeros(6 * self.nc)
        lib().or_connectivity(self.h, nb, nbf, sh)
        return nb.reshape(-1, 3), nbf.reshape(-1, 3), sh.reshape(-1, 3, 2)

    def l1_error(self, u, exact_fn, t, var=0):
        """Domain-averaged L1 error of variable var against exact_fn(x, y, t)."""
        xy, w = self.error_rule()
        cells = np.repeat(np.arange(self.nc), xy.shape[1])
        uh = self.eval_points(u, cells, xy.reshape(-1, 2))[:, var]
        ex = exact_fn(xy[..., 0].ravel(), xy[..., 1].ravel(), t)[:, var]
        err = np.abs(uh - ex)
        return float(np.sum(w.ravel() * err) / np.sum(w)), float(np.max(err))

    # --- hooks for the pins ---
    def stencil(self, c):
        tri = np.zeros(3 * 7 * 6)
        gh = np.zeros(3, dtype=np.int32)
        lib().or_hook_stencil(self.h, c, tri, gh)
        return tri.reshape(3, 7, 3, 2), gh

    def subcell_means(self, u, c, t=0.0):
        out = np.zeros(3 * 7 * self.nvar)
        lib().or_hook_subcell_means(self.h, _f64(u), c, t, out)
        return out.reshape(3, 7, self.nvar)

    def weno(self, c, ubar0, thirds, halves=None, force_linear=False):
        info = np.zeros(40)
        modes = np.zeros(self.np)
        hf = None if halves is None else _f64(halves).ravel()
        st = lib().or_hook_weno(self.h, c, ubar0, _f64(thirds).ravel(), None if hf is None else hf.ctypes.data,
                                int(force_linear), info, modes)
        return dict(q2=info[0:2], q3=info[2:7], q4=info[7:16], gamma=info[21:25], beta=info[25:29],
                    omega=info[29:33], beta1l=info[33:36], sigma=info[36:39], tau=info[39], modes=modes, status=st)

    def beta(self, c, coef, deg):
        coef = _f64(coef)
        return lib().or_hook_beta(self.h, c, len(coef), coef, deg)

    def frame(self, c):
        out = np.zeros(19)
        lib().or_hook_frame(self.h, c, out)
        return dict(x0=out[0], y0=out[1], h0=out[2], area=out[3], hbar=out[4], m0=out[5:])

    def flux(self, UL, UR, nx, ny):
        F = np.zeros(self.nvar)
        lib().or_hook_flux(self.h, _f64(UL), _f64(UR), nx, ny, F)
        return F

    def limit_cell(self, u, c, t=0.0):
        out = np.zeros(self.nvar * self.np)
        st = lib().or_hook_limit_cell(self.h, _f64(u), t, c, out)
        return out.reshape(self.nvar, self.np), st

    def limit_cell_linear(self, u, c, t=0.0):
        """limit_cell with the linear weights (omega = gamma) in every field."""
        out = np.zeros(self.nvar * self.np)
        st = lib().or_hook_limit_cell_linear(self.h, _f64(u), t, c, out)
        return out.reshape(self.nvar, self.np), st


def gauss_legendre(n):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().or_hook_gauss_legendre(n, x, w)
    return x, w


def tri_rule(which, param):
    """which 0: symmetric rule of the given degree; 1: Duffy rule with param^2 points."""
    b = np.zeros(3 * 64)
    w = np.zeros(64)
    n = lib().or_hook_rule(which, param, b, w)
    if n < 0:
        raise RuntimeError("rule failed")
    return b[: 3 * n].reshape(n, 3), w[:n]


def psi(k, m, r, s):
    out = np.zeros(3)
    lib().or_hook_psi(k, m, r, s, out)
    return out


def lsq(A, b):
    A = _f64(A)
    c = np.zeros(A.shape[1])
    st = lib().or_hook_lsq(A.shape[0], A.shape[1], A, _f64(b), c)
    return c, st


def euler_eigen(U, nx, ny, gamma=1.4):
    R = np.zeros(16)
    L = np.zeros(16)
    lib().or_euler_eigen(gamma, _f64(U), nx, ny, R, L)
    return R.reshape(4, 4), L.reshape(4, 4)

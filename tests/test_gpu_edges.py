"""Edge cases on the GPU: the smallest meshes (2 and 8 cells on a periodic
square, where every neighbour of a cell is the same cell across different
faces; 2 cells with transmissive boundaries), and argument errors that the C
interface must report as statuses."""
import numpy as np
import pytest

import oracle
from paper_2106_06280_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("n,k", [(1, 1), (1, 2), (2, 1), (2, 2)])
def test_tiny_periodic_burgers_fp64(csw, cuda_stream, n, k):
    pb = W.burgers_sine(n, seed=11)
    s = csw.Solver(0, k, csw.FP64, csw.LIMITER_ALL, stream=cuda_stream)
    s.setup(pb)
    o = oracle.Oracle(pb, k=k, limiter=2)
    u = o.project(pb.u0)
    ug, fg = s.limit(u, 0.0)
    uo, fo, st = o.limit(u, 0.0)
    assert st == 0 and np.array_equal(fg, fo)
    assert rel(ug, uo) < 1e-11
    dt = 0.5 * o.cfl_dt(u, 0.1)
    for i in range(3):
        u, _, st = o.step(u, i * dt, dt)
    s.write_modes(o.project(pb.u0))
    s.set_time(0.0)
    s.step(dt, 3, 1e9)
    assert rel(s.read_modes(), u) < 1e-11


def test_two_cell_euler_transmissive_fp64(csw, cuda_stream):
    pb = W.riemann_quadrants(1, seed=14)
    assert pb.mesh.nc == 2
    s = csw.Solver(1, 2, csw.FP64, csw.LIMITER_KXRCF, stream=cuda_stream)
    s.setup(pb)
    o = oracle.Oracle(pb, k=2, limiter=1)
    u = W.random_modes(pb.mesh, 4, 6, 5)
    assert rel(s.eval_rhs(u, 0.0), o.rhs(u, 0.0)) < 1e-11
    ug, fg = s.limit(u, 0.0)
    uo, fo, st = o.limit(u, 0.0)
    assert st == 0 and np.array_equal(fg, fo)
    assert rel(ug, uo) < 1e-11


def test_argument_errors_are_statuses(csw, cuda_stream):
    s = csw.Solver(1, 2, csw.FP64, csw.LIMITER_KXRCF, stream=cuda_stream)
    with pytest.raises(csw.CswdgError, match="EINVAL"):
        s.step(0.0, 1, 1.0)  # no mesh yet
    pb = W.riemann_quadrants(3, seed=14)
    with pytest.raises(csw.CswdgError, match="EINVAL"):
        s.mesh_upload(pb.mesh.xy, pb.mesh.tri[:0], pb.mesh.bface, None)  # no triangles
    s.setup(pb)
    with pytest.raises(csw.CswdgError, match="EINVAL"):
        s.step(0.0, -1, 1.0)
    with pytest.raises(csw.CswdgError, match="EINVAL"):
        s.set_stage_shape(100, 0)
    u = W.random_modes(pb.mesh, 4, 6, 6)
    with pytest.raises(csw.CswdgError, match="EINVAL"):
        s.adjoint_steps(u, u, 0.1, 1, 0)  # no checkpoint interval
    s.close()
    s = csw.Solver(1, 2, csw.FP64, csw.LIMITER_OFF, stream=cuda_stream)
    s.setup(pb)
    with pytest.raises(csw.CswdgError, match="EINVAL"):
        s.limit_adjoint(u, u, 0.0)
    s.close()


def test_bounded_wait_timeout_is_a_status(csw, cuda_stream):
    """A device wait that runs out ends its kernel with an error bit that the host
    reports as ETIMEOUT (the self-test waits on a barrier phase that nothing
    completes, with a short poll limit); the solver stays usable: a step
    afterwards matches the oracle."""
    import time

    pb = W.burgers_sine(4, seed=11)
    s = csw.Solver(0, 2, csw.FP64, csw.LIMITER_KXRCF, stream=cuda_stream)
    s.setup(pb)
    t0 = time.perf_counter()
    with pytest.raises(csw.CswdgError, match="ETIMEOUT"):
        s.selftest_timeout(4096)
    assert time.perf_counter() - t0 < 5.0
    with pytest.raises(csw.CswdgError, match="EINVAL"):
        s.selftest_timeout(0)
    o = oracle.Oracle(pb, k=2, limiter=1)
    u = o.project(pb.u0)
    s.write_modes(u)
    s.set_time(0.0)
    dt = 0.5 * o.cfl_dt(u, 0.1)
    s.step(dt, 1, 1e9)
    uo, _, st = o.step(u, 0.0, dt)
    assert st == 0 and rel(s.read_modes(), uo) < 1e-11
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_positivity_trigger_matches_the_oracle(csw, cuda_stream, precision):
    """Reading R-pos as a detection trigger: a gas at rest (no inflow face, so
    KXRCF gives R = 0) with one cell whose polynomial is negative at some
    quadrature points.  The GPU flags exactly that cell, like the oracle, and
    reconstructs it to the oracle's modes (FP64: 1e-11; FP32-bulk: float
    rounding of the state)."""
    pb = W.euler_entropy_wave(6, seed=12)
    o = oracle.Oracle(pb, k=2, limiter=1)
    area = W.cell_areas(pb.mesh)
    base = W.prim_to_cons(np.array([1.0]), 0.0, 0.0, 1.0)[0]
    u = np.zeros((pb.mesh.nc, 4, 6))
    u[:, :, 0] = base[None, :] * np.sqrt(area)[:, None]
    c = 11
    u[c, 0, 1] = 2.0 * u[c, 0, 0]
    u[c, 3, 2] = -1.5 * u[c, 3, 0]
    fo, R = o.detect(u)
    assert fo[c] == 1 and R[c] == 0.0 and fo.sum() == 1
    lo, st = o.limit_cell(u, c)
    s = csw.Solver(csw.EULER, 2, precision, csw.LIMITER_KXRCF, stream=cuda_stream)
    s.setup(pb)
    ug, fg = s.limit(u, 0.0)
    assert np.array_equal(fg, fo)
    tol = 1e-11 if precision == 0 else 1e-6
    assert np.abs(ug[c] - lo).max() < tol * np.abs(lo).max()
    s.close()


def test_stage_dev_matches_the_operator_and_checks_alignment(csw, cuda_stream):
    """cswdg_stage_dev on caller-owned device buffers in the internal layout
    (cell i = perm[user cell], coefficients sqrt(2/|K|) times the user modes):
    out = uprev + dt L_h(uprev) equals the user-layout operator of cswdg_eval_rhs;
    a device pointer that is not 16-byte aligned is refused with a status before
    any launch (the kernels move cells in 16-byte vectors)."""
    torch = pytest.importorskip("torch")
    pb = W.double_mach(26, 7, seed=13)
    s = csw.Solver(csw.EULER, 2, csw.FP64, csw.LIMITER_OFF, stream=cuda_stream)
    s.setup(pb)
    ld, perm = s.internal_layout()
    nc = pb.mesh.nc
    u = W.random_modes(pb.mesh, 4, 6, 71, scale=0.05)
    scale = np.sqrt(2.0 / W.cell_areas(pb.mesh))[:, None, None]
    ui = np.zeros((nc, 4, 6))
    ui[perm] = u * scale
    dt, t = 1e-4, 0.013
    L = s.eval_rhs(u, t)
    dev = torch.device("cuda", 0)
    up = torch.tensor(ui.reshape(-1), dtype=torch.float64, device=dev)
    out = torch.zeros(nc * 4 * 6 + 2, dtype=torch.float64, device=dev)
    s.stage_dev(None, up.data_ptr(), out.data_ptr(), 0.0, 1.0, dt, t)
    torch.cuda.synchronize()
    got = out[: nc * 24].cpu().numpy().reshape(nc, 4, 6)[perm] / scale
    assert rel(got, u + dt * L) < 1e-13
    with pytest.raises(csw.CswdgError) as e:
        s.stage_dev(None, up.data_ptr(), out.data_ptr() + 8, 0.0, 1.0, dt, t)
    assert e.value.status == csw.EINVAL
    s.close()

"""GPU parity: every step of the hot path through the C interface against the
FP64 CPU oracle on the same seeded inputs.

FP64 mode: coefficients within 1e-11 relative L-infinity (relative to the
largest coefficient magnitude of the field compared), troubled-cell flags
bit-exact.  Meshes span several thread blocks with a ragged tail (cell counts
not multiples of 128).
"""
import numpy as np
import pytest

import oracle
from paper_2106_06280_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-11


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def make(csw, stream, problem, k, limiter, precision=0, ck=1.0, cfl=0.1):
    s = csw.Solver(problem.equation, k, precision, limiter, c_k=ck, cfl=cfl, stream=stream)
    s.setup(problem)
    o = oracle.Oracle(problem, k=k, limiter=limiter, ck=ck)
    return s, o


def problems():
    return {
        "burgers": W.burgers_sine(9, seed=11),              # 162 cells, periodic
        "entropy": W.euler_entropy_wave(7, seed=12),         # 98 cells, periodic
        "dmr": W.double_mach(26, 7, seed=13),                # 364 cells, inflow/wall/outflow/shock boundaries
        "riemann": W.riemann_quadrants(9, seed=14),          # 162 cells, transmissive
    }


def random_state(problem, k, seed):
    np_ = (k + 1) * (k + 2) // 2
    return W.random_modes(problem.mesh, problem.nvar, np_, seed)


@pytest.mark.parametrize("name", ["burgers", "entropy", "dmr", "riemann"])
@pytest.mark.parametrize("k", [1, 2])
def test_rhs_fp64(csw, cuda_stream, name, k):
    pb = problems()[name]
    s, o = make(csw, cuda_stream, pb, k, 0)
    u = random_state(pb, k, 100 + k)
    t = 0.013
    L_g = s.eval_rhs(u, t)
    L_o = o.rhs(u, t)
    for v in range(pb.nvar):
        assert rel(L_g[:, v], L_o[:, v]) < TOL64, (name, k, v, rel(L_g[:, v], L_o[:, v]))


@pytest.mark.parametrize("name", ["burgers", "entropy", "dmr", "riemann"])
@pytest.mark.parametrize("k", [1, 2])
def test_limiter_all_cells_fp64(csw, cuda_stream, name, k):
    pb = problems()[name]
    s, o = make(csw, cuda_stream, pb, k, 2)
    u = random_state(pb, k, 200 + k)
    t = 0.021
    ug, fg = s.limit(u, t)
    uo, fo, st = o.limit(u, t)
    assert st == 0
    assert np.array_equal(fg, fo)
    assert np.all(fg == 1)
    for v in range(pb.nvar):
        assert rel(ug[:, v], uo[:, v]) < TOL64, (name, k, v, rel(ug[:, v], uo[:, v]))
    # cell means untouched (up to the rounding of the basis rescaling on upload and read-back)
    assert np.abs(ug[:, :, 0] - u[:, :, 0]).max() <= 8e-16 * np.abs(u[:, :, 0]).max()


@pytest.mark.parametrize("name", ["burgers", "entropy", "dmr", "riemann"])
@pytest.mark.parametrize("k", [1, 2])
def test_kxrcf_flags_and_limit_fp64(csw, cuda_stream, name, k):
    pb = problems()[name]
    s, o = make(csw, cuda_stream, pb, k, 1)
    u = random_state(pb, k, 300 + k)
    t = 0.0
    ug, fg = s.limit(u, t)
    uo, fo, st = o.limit(u, t)
    assert st == 0
    assert 0 < fo.sum() < len(fo)  # a mix of flagged and clean cells
    assert np.array_equal(fg, fo)
    for v in range(pb.nvar):
        assert rel(ug[:, v], uo[:, v]) < TOL64


@pytest.mark.parametrize("name,k,limiter,nsteps", [("burgers", 2, 1, 6), ("burgers", 1, 2, 4), ("entropy", 2, 2, 3),
                                                     ("dmr", 2, 1, 6), ("dmr", 1, 1, 6), ("riemann", 1, 1, 6)])
def test_steps_fp64(csw, cuda_stream, name, k, limiter, nsteps):
    pb = problems()[name]
    s, o = make(csw, cuda_stream, pb, k, limiter)
    u0 = o.project(pb.u0)
    # discontinuous initial data: every cell reconstructed once
    uo, _, _ = (oracle.Oracle(pb, k=k, limiter=2) if pb.equation == 1 else o).limit(u0, 0.0)
    dt = 0.5 * o.cfl_dt(uo, 0.1)
    s.write_modes(uo)
    s.set_time(0.0)
    flo = None
    for n in range(nsteps):
        uo, flo, st = o.step(uo, n * dt, dt)
        assert st == 0
    t = s.step(dt, nsteps, 1e9)
    assert abs(t - nsteps * dt) < 1e-13
    ug = s.read_modes()
    fg = s.read_flags()
    if limiter == 1:
        assert np.array_equal(fg, flo)
    for v in range(pb.nvar):
        assert rel(ug[:, v], uo[:, v]) < TOL64, (name, v, rel(ug[:, v], uo[:, v]))


def test_cfl_dt_and_clip(csw, cuda_stream):
    pb = problems()["entropy"]
    s, o = make(csw, cuda_stream, pb, 2, 1)
    u = o.project(pb.u0)
    s.write_modes(u)
    assert abs(s.cfl_dt() - o.cfl_dt(u, 0.1)) < 1e-14 * o.cfl_dt(u, 0.1)
    s.set_time(0.0)
    t_end = 2.5 * o.cfl_dt(u, 0.1)
    t = s.step(0.0, 10, t_end)  # clipped at t_end, extra steps are no-ops
    assert t == t_end


@pytest.mark.parametrize("name", ["burgers", "dmr"])
def test_project_ic_and_conservation(csw, cuda_stream, name):
    pb = problems()[name]
    s, o = make(csw, cuda_stream, pb, 2, 0)
    s.project_ic(pb.u0, apply_limiter=0)
    ug = s.read_modes()
    uo = o.project(pb.u0)
    assert rel(ug, uo) < TOL64
    assert np.allclose(s.conservation(), o.conservation(uo), rtol=1e-13, atol=1e-13)


def test_project_ic_all_cells_limited(csw, cuda_stream):
    pb = problems()["dmr"]
    s, o = make(csw, cuda_stream, pb, 2, 1)
    s.project_ic(pb.u0, apply_limiter=2)
    ug = s.read_modes()
    oa = oracle.Oracle(pb, k=2, limiter=2)
    uo, fo, st = oa.limit(oa.project(pb.u0), 0.0)
    for v in range(pb.nvar):
        assert rel(ug[:, v], uo[:, v]) < TOL64


@pytest.mark.parametrize("shape", [(64, 0), (128, 0), (256, 0), (64, 3), (128, 2), (256, 1),
                                   (128, 0, 1), (256, 0, 1), (128, 2, 1), (256, 1, 1)])
def test_stage_shapes_fp64(csw, cuda_stream, shape):
    """Every launch shape of the stage kernel (tiles of 64/128/256 cells, one
    block per tile or a small persistent grid looping over several tiles) gives
    the oracle's operator (DMR boundaries, random state) and its CFL steps (the
    wave-speed maximum of the next step is folded into the last stage), on a
    338-cell periodic Euler mesh: 2 to 6 tiles per launch, ragged last tile."""
    pb = problems()["dmr"]
    s, o = make(csw, cuda_stream, pb, 2, 1)
    s.set_stage_shape(*shape)
    u = random_state(pb, 2, 500)
    assert rel(s.eval_rhs(u, 0.011), o.rhs(u, 0.011)) < TOL64
    s.close()
    pb = W.euler_entropy_wave(13, seed=41)
    s, o = make(csw, cuda_stream, pb, 2, 1)
    s.set_stage_shape(*shape)
    u = o.project(pb.u0)
    s.write_modes(u)
    s.set_time(0.0)
    t, uo = 0.0, u
    for n in range(3):
        dt = o.cfl_dt(uo, 0.1)
        uo, _, st = o.step(uo, t, dt)
        assert st == 0
        t += dt
    tg = s.step(0.0, 3, 1e9)
    assert abs(tg - t) < 1e-13 * t
    assert rel(s.read_modes(), uo) < TOL64


def test_autotune_keeps_results(csw, cuda_stream):
    pb = problems()["riemann"]
    s, o = make(csw, cuda_stream, pb, 2, 1)
    u = random_state(pb, 2, 501)
    s.write_modes(u)
    blk, grid, tile_faces, ms = s.autotune()
    assert blk in (64, 128, 256) and grid >= 0 and tile_faces in (0, 1) and np.all(ms > 0)
    assert not (tile_faces and blk == 64)
    assert np.allclose(s.read_modes(), u, rtol=0, atol=1e-15 * np.abs(u).max())  # state untouched
    s.set_time(0.0)
    dt = 0.5 * o.cfl_dt(u, 0.1)
    uo, _, _ = o.step(u, 0.0, dt)
    s.step(dt, 1, 1e9)
    assert rel(s.read_modes(), uo) < TOL64

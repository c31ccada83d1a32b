"""The tile-shared stage kernel (k_stage_tiles) against the per-cell stage
kernel (k_stage) and the oracle.

k_stage_tiles computes each face between two cells of a tile once and hands
the neighbour -F; the local Lax-Friedrichs flux is evaluated so that
llf2(U_b, U_a, -n) = -llf2(U_a, U_b, n) bit for bit, the traces are formed by
the same fused sums, and every cell takes its fluxes off its residual in the
per-cell kernel's order.  So the two kernels agree bit for bit on every mesh
(periodic faces whose two stored normals are not exact negatives are computed
from each side's own normal): the tests compare with np.array_equal.

Meshes: periodic (Burgers sine, Euler entropy wave), the DMR boundaries
(Dirichlet inflow, wall, outflow, moving shock line) and transmissive
quadrants, with cell counts that leave a ragged last tile for 128- and
256-cell tiles, one block per tile and persistent grids looping over tiles.
"""
import numpy as np
import pytest

import oracle
from paper_2106_06280_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TILE_SHAPES = [(128, 0, 1), (256, 0, 1), (128, 3, 1), (256, 2, 1)]


def meshes():
    return {
        "burgers": W.burgers_sine(23, seed=21),             # 1,058 cells, periodic
        "entropy": W.euler_entropy_wave(17, seed=22),        # 578 cells, periodic
        "dmr": W.double_mach(72, 18, seed=23),               # 2,592 cells
        "riemann": W.riemann_quadrants(20, seed=24),         # 800 cells, transmissive
    }


def state(pb, k, seed):
    nv = 1 if pb.equation == 0 else 4
    np_ = (k + 1) * (k + 2) // 2
    return W.random_modes(pb.mesh, nv, np_, seed, scale=0.05 if nv == 4 else 0.3)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("name", ["burgers", "entropy", "dmr", "riemann"])
def test_tile_operator_bitwise(csw, cuda_stream, name, k, precision):
    pb = meshes()[name]
    s = csw.Solver(pb.equation, k, precision, csw.LIMITER_OFF, stream=cuda_stream)
    s.setup(pb)
    u = state(pb, k, 600 + k)
    s.set_stage_shape(128, 0, 0)
    ref = s.eval_rhs(u, 0.021)
    for shape in TILE_SHAPES:
        s.set_stage_shape(*shape)
        got = s.eval_rhs(u, 0.021)
        assert np.array_equal(got, ref), (shape, float(np.abs(got - ref).max()))
    s.close()


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("name", ["entropy", "dmr"])
def test_tile_operator_fp64_vs_oracle(csw, cuda_stream, name, k):
    """FP64: the tile kernel's operator against the oracle's rhs at 1e-11."""
    pb = meshes()[name]
    s = csw.Solver(pb.equation, k, csw.FP64, csw.LIMITER_OFF, stream=cuda_stream)
    s.setup(pb)
    o = oracle.Oracle(pb, k=k, limiter=0)
    u = state(pb, k, 610 + k)
    s.set_stage_shape(256, 0, 1)
    got = s.eval_rhs(u, 0.013)
    want = o.rhs(u, 0.013)
    assert float(np.abs(got - want).max() / np.abs(want).max()) < 1e-11
    s.close()


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_tile_steps_bitwise(csw, cuda_stream, precision):
    """Whole SSP-RK3 steps with the KXRCF limiter on the projected DMR state
    (stages 2 and 3 combine with u^n, the last stage folds the next step's wave
    speed, the detection reads the kernel's KXRCF records): modes and flags of
    the tile shapes equal the per-cell kernel's bit for bit after 10 CFL steps."""
    pb = meshes()["dmr"]
    out = {}
    for shape in [(128, 0, 0)] + TILE_SHAPES:
        s = csw.Solver(csw.EULER, 2, precision, csw.LIMITER_KXRCF, stream=cuda_stream)
        s.setup(pb)
        s.set_stage_shape(*shape)
        s.project_ic(pb.u0, apply_limiter=2)
        s.set_time(0.0)
        t = s.step(0.0, 10, 1e300)
        out[shape] = (s.read_modes(), s.read_flags(), t)
        s.close()
    ud, fd, td = out[(128, 0, 0)]
    assert fd.sum() > 0
    for shape in TILE_SHAPES:
        ug, fg, tg = out[shape]
        assert tg == td, shape
        assert np.array_equal(ug, ud), (shape, float(np.abs(ug - ud).max()))
        assert np.array_equal(fg, fd), shape


def test_tile_shape_rejects_64(csw, cuda_stream):
    pb = meshes()["riemann"]
    s = csw.Solver(pb.equation, 1, csw.FP64, csw.LIMITER_OFF, stream=cuda_stream)
    s.setup(pb)
    with pytest.raises(RuntimeError):
        s.set_stage_shape(64, 0, 1)
    s.close()


@pytest.mark.parametrize("n,k", [(1, 1), (1, 2), (2, 2)])
def test_tile_tiny_periodic_meshes_bitwise(csw, cuda_stream, n, k):
    """2 and 8 cells on a periodic square: a cell meets the same neighbour
    across several faces (and itself across none), the periodic images give
    normals that need not be exact negatives, and the whole mesh is one ragged
    tile."""
    for pb in (W.burgers_sine(n, seed=31), W.euler_entropy_wave(n, seed=32)):
        s = csw.Solver(pb.equation, k, csw.FP64, csw.LIMITER_OFF, stream=cuda_stream)
        s.setup(pb)
        u = state(pb, k, 620 + n)
        s.set_stage_shape(128, 0, 0)
        ref = s.eval_rhs(u, 0.0)
        for shape in TILE_SHAPES:
            s.set_stage_shape(*shape)
            assert np.array_equal(s.eval_rhs(u, 0.0), ref), shape
        s.close()


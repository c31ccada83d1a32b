"""GPU checks on the benchmark-family configurations at full size.

* Burgers P1, 20x20 split squares (800 cells), FP64, KXRCF C_K = 1, to t = 0.1:
  whole run against the oracle (coefficients 1e-11, flags bit-exact at the end).
* Burgers P2, 160x160 (51,200 cells): 12 steps against the oracle in FP64
  (1e-11, flags) and in FP32-bulk mode (L1 error relative to the mean |u|
  below 2e-6); then the GPU alone through shock formation (t = 2/pi) to the
  configuration's t = 1.0 in both precisions: cell-mean conservation, limited
  cells present, cell means within the exact solution's range [0.25, 0.75]
  up to a stated excursion, and the FP32-bulk L1 difference from FP64 there.
* Burgers P2, 20x20, through the shock to t = 1.0: the whole run against the
  oracle in FP64.
* Double Mach reflection, Euler P2, 960x240 (460,800 cells): one operator
  evaluation and one limiter pass on a seeded random state, compared with the
  oracle on 600 sampled cells (FP64: 1e-11 and identical flags).
"""
import numpy as np
import pytest

import oracle
from paper_2106_06280_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def l1(a, b, area):
    return float(np.sum(area * np.abs(a[:, 0, 0] - b[:, 0, 0]) / np.sqrt(area)) / np.sum(area))


def test_config1_full_run_fp64(csw, cuda_stream):
    pb = W.burgers_sine(20, seed=1)
    o = oracle.Oracle(pb, k=1, limiter=1, ck=1.0)
    s = csw.Solver(0, 1, csw.FP64, csw.LIMITER_KXRCF, c_k=1.0, cfl=0.1, stream=cuda_stream)
    s.setup(pb)
    u0 = o.project(pb.u0)
    uo, _, _ = o.limit(u0, 0.0)
    s.write_modes(uo)
    s.set_time(0.0)
    t = 0.0
    n = 0
    fl = None
    while t < 0.1:
        dt = min(o.cfl_dt(uo, 0.1), 0.1 - t)
        uo, fl, st = o.step(uo, t, dt)
        t += dt
        n += 1
    tg = s.step(0.0, n + 5, 0.1)  # extra steps beyond t_end do nothing
    assert abs(tg - 0.1) < 1e-15
    ug = s.read_modes()
    assert np.array_equal(s.read_flags(), fl)
    assert np.abs(ug - uo).max() / np.abs(uo).max() < 1e-11


@pytest.mark.parametrize("precision", [0, 1])
def test_config2_steps_vs_oracle(csw, cuda_stream, precision):
    pb = W.burgers_sine(160, seed=2)
    o = oracle.Oracle(pb, k=2, limiter=1)
    s = csw.Solver(0, 2, precision, csw.LIMITER_KXRCF, c_k=1.0, cfl=0.1, stream=cuda_stream)
    s.setup(pb)
    uo = o.project(pb.u0)
    uo, _, _ = o.limit(uo, 0.0)
    s.write_modes(uo)
    s.set_time(0.0)
    dt = o.cfl_dt(uo, 0.1)
    for i in range(12):
        uo, flo, st = o.step(uo, i * dt, dt)
    s.step(dt, 12, 1e9)
    ug = s.read_modes()
    area = W.cell_areas(pb.mesh)
    if precision == 0:
        assert np.abs(ug - uo).max() / np.abs(uo).max() < 1e-11
        assert np.array_equal(s.read_flags(), flo)
    else:
        err = l1(ug, uo, area) / 0.5  # mean |u| is 0.5
        assert err < 2e-6, err


def test_config2_to_t1_fp32_vs_fp64(csw, cuda_stream):
    """Config 2 to its end time: the shock forms at t = 2/pi and the limiter
    holds every cell mean within [0.25, 0.75] up to the excursion stated in the
    bound (the oracle's on 20x20 / 40x40 / 80x80: 7e-4 / 2e-5 / 1.2e-3); checked
    at 10 times through the run.  The FP32-bulk run is compared with the FP64
    run (which the 12-step test ties to the oracle) by the area-weighted L1
    difference of the cell means relative to the mean |u| = 0.5.  Measured on
    the GB300: excursions above / below the range 5.4e-4 / 9.8e-4 (FP64) and
    2.2e-3 / 1.6e-3 (FP32-bulk); FP32-bulk against FP64 L1 1.7e-4."""
    pb = W.burgers_sine(160, seed=2)
    area = W.cell_areas(pb.mesh)
    out, ext = {}, {}
    for prec in (0, 1):
        s = csw.Solver(0, 2, prec, csw.LIMITER_KXRCF, c_k=1.0, cfl=0.1, stream=cuda_stream)
        s.setup(pb)
        s.project_ic(pb.u0, apply_limiter=1)
        c0 = s.conservation()[0]
        hi, lo = 0.0, 1.0
        for tk in np.linspace(0.1, 1.0, 10):
            t = s.step(0.0, 1000000, float(tk))
            assert t == float(tk)
            m = s.read_modes()[:, 0, 0] / np.sqrt(area)
            assert np.all(np.isfinite(m))
            hi, lo = max(hi, m.max()), min(lo, m.min())
        # FP32-bulk: the two sides of a face use geometry factors |n~| = 2|e|/|K| rounded
        # separately to float, a drift of about 6e-9 of the total per step
        assert abs(s.conservation()[0] - c0) < (1e-11 if prec == 0 else 2e-4) * abs(c0)
        assert s.num_flagged() > 0
        ext[prec] = (hi - 0.75, 0.25 - lo)
        assert hi < 0.75 + 3e-3 and lo > 0.25 - 3e-3, ext
        out[prec] = s.read_modes()
        s.close()
    err = l1(out[1], out[0], area) / 0.5
    print(f"config 2 at t = 1: excursions FP64 {ext[0]}, FP32-bulk {ext[1]}; FP32-bulk vs FP64 L1 {err:.3e}")
    assert err < 1e-3, err


def test_burgers_p2_through_the_shock_vs_oracle(csw, cuda_stream):
    """Burgers P2 on 20x20 to t = 1.0 (the shock forms at 2/pi), whole run in
    FP64 against the oracle: at the end the flags match and the coefficients
    agree within 1e-11 of the largest (measured on the GB300: 708 steps,
    2.6e-14, no flag differs)."""
    pb = W.burgers_sine(20, seed=2)
    o = oracle.Oracle(pb, k=2, limiter=1)
    uo = o.limit(o.project(pb.u0), 0.0)[0]
    s = csw.Solver(0, 2, csw.FP64, csw.LIMITER_KXRCF, c_k=1.0, cfl=0.1, stream=cuda_stream)
    s.setup(pb)
    s.write_modes(uo)
    s.set_time(0.0)
    t, n, flo = 0.0, 0, None
    while t < 1.0:
        dt = min(o.cfl_dt(uo, 0.1), 1.0 - t)
        uo, flo, st = o.step(uo, t, dt)
        t += dt
        n += 1
    assert abs(s.step(0.0, n + 5, 1.0) - 1.0) < 1e-15
    ug = s.read_modes()
    err = np.abs(ug - uo).max() / np.abs(uo).max()
    nflip = int(np.sum(s.read_flags() != flo))
    print(f"20x20 P2 to t = 1: {n} steps, max relative coefficient difference {err:.3e}, flags differing {nflip}")
    assert nflip == 0 and flo.sum() > 0
    assert err < 1e-11, err


def test_config3_full_size_sampled_fp64(csw, cuda_stream):
    pb = W.double_mach(960, 240, seed=3)
    o = oracle.Oracle(pb, k=2, limiter=1)
    u = W.random_modes(pb.mesh, 4, 6, 33, scale=0.02)
    rng = np.random.default_rng(7)
    cells = np.sort(rng.choice(pb.mesh.nc, 600, replace=False)).astype(np.int32)
    s = csw.Solver(1, 2, csw.FP64, csw.LIMITER_OFF, stream=cuda_stream)
    s.setup(pb)
    Lg = s.eval_rhs(u, 0.05)
    Lo = o.rhs_cells(u, cells, 0.05)
    assert np.abs(Lg[cells] - Lo).max() / np.abs(Lo).max() < 1e-11
    s.close()
    s = csw.Solver(1, 2, csw.FP64, csw.LIMITER_KXRCF, stream=cuda_stream)
    s.setup(pb)
    ug, fg = s.limit(u, 0.05)
    fo, _ = o.detect_cells(u, cells, 0.05)
    assert np.array_equal(fg[cells], fo)
    flagged = cells[fo.astype(bool)]
    assert len(flagged) > 10
    lo, st = o.limit_cells(u, flagged, 0.05)
    assert np.abs(ug[flagged] - lo).max() / np.abs(lo).max() < 1e-11


def test_config4_small_ensemble_fp64(csw, cuda_stream):
    """Independent Riemann problems advanced as one disconnected mesh (the
    ensemble workload's structure, 5 meshes of uneven sizes): 4 steps against
    the oracle with KXRCF limiting.

    The reconstruction amplifies rounding-level differences on this flow (a
    limiter pass multiplies an input difference by up to about 100 in the
    low-density cells; over 4 steps the oracle turns a relative input
    perturbation of 1e-13 into 1.7e-9), so a fixed 1e-11 after 4 steps is not
    a property of the method.  The tolerance is the oracle's own response to a
    relative perturbation of 1e-12 of every input coefficient, ten times below
    the 1e-11 that single operator and limiter passes are held to.  Flags stay
    bit-exact."""
    pb = W.riemann_ensemble(5, total=3000, seed=2000, lo=200, hi=1200)
    o = oracle.Oracle(pb, k=2, limiter=1)
    oa = oracle.Oracle(pb, k=2, limiter=2)
    s = csw.Solver(1, 2, csw.FP64, csw.LIMITER_KXRCF, stream=cuda_stream)
    s.setup(pb)
    u0 = oa.limit(oa.project(pb.u0), 0.0)[0]
    s.project_ic(pb.u0, apply_limiter=2)
    assert np.abs(s.read_modes() - u0).max() / np.abs(u0).max() < 1e-11
    dt = 0.5 * o.cfl_dt(u0, 0.1)

    def run(u):
        fl = None
        for i in range(4):
            u, fl, st = o.step(u, i * dt, dt)
            assert st == 0
        return u, fl

    uo, flo = run(u0)
    sign = np.where(W.uniform01(99, np.arange(u0.size)).reshape(u0.shape) < 0.5, -1.0, 1.0)
    up, _ = run(u0 * (1.0 + 1e-12 * sign))
    sens = np.abs(up - uo).max() / np.abs(uo).max()
    s.step(dt, 4, 1e9)
    ug = s.read_modes()
    assert np.array_equal(s.read_flags(), flo) and flo.sum() > 0
    err = np.abs(ug - uo).max() / np.abs(uo).max()
    assert err < max(1e-11, sens), (err, sens)


def test_config4_full_size_sampled(csw, cuda_stream):
    """The full ensemble (256 Riemann problems, 4,984,396 triangles in one
    disconnected mesh, the bench's ensemble workload): operator and KXRCF +
    CSWENO in FP64 against the oracle on 600 sampled cells (identical flags),
    and one FP32-bulk step of the projected, every-cell-limited initial state
    staying finite with positive means.  The coefficients are held to 1e-10
    here instead of 1e-11: the meshes sit on a 16 x 16 grid of unit squares 1.5
    apart (coordinates up to 24 against cells of 1/250), so the geometry that
    the GPU and the oracle derive from the vertices in different orders already
    differs by about eps64 x 24 x 250 = 1.3e-12 relative, and the operator (of
    order 1/h) carries that into its coefficients (measured 1.7e-11)."""
    pb = W.riemann_ensemble(256, seed=1000)
    assert pb.mesh.nc > 4_900_000
    o = oracle.Oracle(pb, k=2, limiter=1)
    u = W.random_modes(pb.mesh, 4, 6, 44, scale=0.02)
    cells = np.sort(np.random.default_rng(8).choice(pb.mesh.nc, 600, replace=False)).astype(np.int32)
    s = csw.Solver(1, 2, csw.FP64, csw.LIMITER_KXRCF, stream=cuda_stream)
    s.setup(pb)
    Lg = s.eval_rhs(u, 0.0)
    Lo = o.rhs_cells(u, cells, 0.0)
    assert np.abs(Lg[cells] - Lo).max() / np.abs(Lo).max() < 1e-10
    ug, fg = s.limit(u, 0.0)
    fo, _ = o.detect_cells(u, cells, 0.0)
    assert np.array_equal(fg[cells], fo)
    flagged = cells[fo.astype(bool)]
    assert len(flagged) > 10
    lo, st = o.limit_cells(u, flagged, 0.0)
    assert np.abs(ug[flagged] - lo).max() / np.abs(lo).max() < 1e-10
    s.close()
    s = csw.Solver(1, 2, csw.FP32_BULK, csw.LIMITER_KXRCF, stream=cuda_stream)
    s.setup(pb)
    s.project_ic(pb.u0, apply_limiter=2)
    s.step(0.0, 1, pb.t_end)
    means = s.read_modes()[:, :, 0]
    assert np.all(np.isfinite(means)) and means[:, 0].min() > 0.0
    s.close()

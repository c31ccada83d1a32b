"""The Euler configurations run to their stated end times on the GPU.

* Double Mach reflection (Sec. 4.2 Example 5), 960x240 (460,800 triangles),
  Euler P2, FP32-bulk, KXRCF + CSWENO, CFL 0.1, to t = 0.2: every cell mean
  finite with positive density and pressure; the undisturbed regions keep
  their states (pre-shock gas right of the incident shock, which meets the top
  boundary at x_s(0.2) = 1/6 + 5/sqrt(3) = 3.05; post-shock gas near the inflow
  corner); the flagged fraction is reported.
* The same set-up on a reduced 240x60 mesh in FP64 and FP32-bulk to t = 0.2:
  the FP32-bulk error against FP64 (which the parity tests tie to the oracle),
  the L1 difference of the density means relative to the L1 norm of FP64's.
* The ensemble (256 four-quadrant Riemann problems, 4,984,396 triangles) in
  FP32-bulk to t = 0.25: finite, positive density and pressure means.
"""
import numpy as np
import pytest

from paper_2106_06280_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _means(s, area):
    m = s.read_modes()[:, :, 0] / np.sqrt(area)[:, None]
    p = (W.GAMMA - 1.0) * (m[:, 3] - 0.5 * (m[:, 1] ** 2 + m[:, 2] ** 2) / m[:, 0])
    return m, p


def _centroids(mesh):
    return mesh.xy[mesh.tri].mean(axis=1)


def test_config3_dmr_to_t02_fp32_bulk(csw, cuda_stream):
    pb = W.double_mach(960, 240, seed=3)
    area = W.cell_areas(pb.mesh)
    s = csw.Solver(csw.EULER, 2, csw.FP32_BULK, csw.LIMITER_KXRCF, c_k=1.0, cfl=0.1, stream=cuda_stream)
    s.setup(pb)
    s.project_ic(pb.u0, apply_limiter=2)
    rows = []
    for tk in (0.05, 0.1, 0.15, 0.2):
        t = s.step(0.0, 10 ** 7, tk)
        assert t == tk
        m, p = _means(s, area)
        assert np.all(np.isfinite(m))
        rows.append((tk, float(m[:, 0].min()), float(p.min()), s.num_flagged()))
        assert m[:, 0].min() > 0.0 and p.min() > 0.0, rows
    print("double Mach reflection, FP32-bulk (t, min density mean, min pressure mean, flagged cells): "
          + "; ".join(f"{r[0]:.2f} {r[1]:.4f} {r[2]:.4f} {r[3]}" for r in rows))
    c = _centroids(pb.mesh)
    pre_state, post = W.dmr_states()
    ahead = (c[:, 0] > 3.3) & (c[:, 1] > 0.5)
    corner = (c[:, 0] < 0.3) & (c[:, 1] > 0.7)
    assert ahead.sum() > 100 and corner.sum() > 100
    assert np.abs(m[ahead] - pre_state).max() < 1e-4 * np.abs(pre_state).max()
    assert np.abs(m[corner] - post).max() < 1e-3 * np.abs(post).max()
    assert 0 < rows[-1][3] < 0.2 * pb.mesh.nc
    s.close()


def test_config3_reduced_fp32_bulk_vs_fp64_at_t02(csw, cuda_stream):
    """FP32-bulk against FP64 on the double Mach reflection at its end time,
    240x60 (28,800 triangles): the L1 difference of the density means relative
    to the L1 norm of the FP64 density means."""
    pb = W.double_mach(240, 60, seed=3)
    area = W.cell_areas(pb.mesh)
    rho = {}
    for prec in (csw.FP64, csw.FP32_BULK):
        s = csw.Solver(csw.EULER, 2, prec, csw.LIMITER_KXRCF, c_k=1.0, cfl=0.1, stream=cuda_stream)
        s.setup(pb)
        s.project_ic(pb.u0, apply_limiter=2)
        assert s.step(0.0, 10 ** 7, 0.2) == 0.2
        m, p = _means(s, area)
        assert np.all(np.isfinite(m)) and m[:, 0].min() > 0.0 and p.min() > 0.0
        rho[prec] = m[:, 0]
        s.close()
    l1 = float(np.sum(area * np.abs(rho[csw.FP32_BULK] - rho[csw.FP64])) / np.sum(area * np.abs(rho[csw.FP64])))
    print(f"double Mach reflection 240x60 at t = 0.2: FP32-bulk vs FP64 relative L1 of the density means {l1:.3e}")
    assert l1 < 1e-2, l1


def test_config4_ensemble_to_t025_fp32_bulk(csw, cuda_stream):
    pb = W.riemann_ensemble(256, seed=1000)
    area = W.cell_areas(pb.mesh)
    s = csw.Solver(csw.EULER, 2, csw.FP32_BULK, csw.LIMITER_KXRCF, c_k=1.0, cfl=0.1, stream=cuda_stream)
    s.setup(pb)
    s.project_ic(pb.u0, apply_limiter=2)
    rows = []
    for tk in (0.125, 0.25):
        assert s.step(0.0, 10 ** 7, tk) == tk
        m, p = _means(s, area)
        assert np.all(np.isfinite(m))
        rows.append((tk, float(m[:, 0].min()), float(p.min()), s.num_flagged()))
        assert m[:, 0].min() > 0.0 and p.min() > 0.0, rows
    print("ensemble, FP32-bulk (t, min density mean, min pressure mean, flagged cells): "
          + "; ".join(f"{r[0]:.3f} {r[1]:.4f} {r[2]:.4f} {r[3]}" for r in rows) + f" of {pb.mesh.nc}")
    s.close()

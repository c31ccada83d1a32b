"""The allocation-free conservation entry point (cswdg_conservation_noalloc)
gives the same sums as cswdg_conservation, on two calls in a row with
different states, in FP64 and FP32-bulk mode.  Collected last on purpose."""
import numpy as np
import pytest

from paper_2106_06280_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def internal_state(torch, s, modes, areas, dtype):
    """The library's internal device layout: cell-major [(i*nvar + v)*np + m],
    internal cell i = perm[user cell], coefficients scaled by sqrt(2/|K|)."""
    _, perm = s.internal_layout()
    nc, nv, np_ = modes.shape
    host = np.zeros((nc, nv, np_))
    host[perm] = modes * np.sqrt(2.0 / areas)[:, None, None]
    return torch.tensor(host.ravel(), dtype=dtype, device="cuda").contiguous()


@pytest.mark.parametrize("mesh,precision,rtol", [
    ("small", 0, 1e-13), ("small", 1, 1e-6), ("small", 2, 1e-6),
    ("dmr", 0, 1e-13), ("dmr", 1, 1e-6)])
def test_conservation_noalloc_matches_allocating_entry_point(csw, cuda_stream, mesh, precision, rtol):
    """small: 338 cells, two reduction blocks with a ragged tail; dmr: the
    460,800-cell double-Mach mesh, 1,800 blocks.  Precision modes 0 (FP64),
    1 (FP32 state, FP64 weights) and 2 (FP32 throughout)."""
    import torch

    if mesh == "small":
        pb = W.euler_entropy_wave(13, seed=41)
    else:
        pb = W.double_mach(960, 240, seed=3)
    s = csw.Solver(csw.EULER, 2, precision, csw.LIMITER_OFF, stream=cuda_stream)
    s.setup(pb)
    areas = W.cell_areas(pb.mesh)
    dtype = torch.float64 if precision == 0 else torch.float32
    sums_dev = torch.zeros(4, dtype=torch.float64, device="cuda")
    for seed in (42, 43):  # two calls in a row, different states
        modes = W.random_modes(pb.mesh, 4, 6, seed)
        s.write_modes(modes)
        ref = s.conservation()
        u_dev = internal_state(torch, s, modes, areas, dtype)
        sums_dev.fill_(-1.0)
        s.conservation_noalloc(u_dev.data_ptr(), sums_dev.data_ptr())
        torch.cuda.synchronize()
        got = sums_dev.cpu().numpy()
        assert np.allclose(got, ref, rtol=rtol, atol=rtol * np.abs(ref).max()), (seed, got, ref)
    s.close()

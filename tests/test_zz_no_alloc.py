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


@pytest.mark.parametrize("precision,rtol", [(0, 1e-13), (1, 1e-6)])
def test_conservation_noalloc_matches_allocating_entry_point(csw, cuda_stream, precision, rtol):
    import torch

    pb = W.euler_entropy_wave(13, seed=41)  # 338 cells: two reduction blocks, ragged tail
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

"""Host-side mesh processing of the library (cswdg_host_mesh: no device), on
the CPU: the properties the stage kernel relies on.

* Neighbour relations are mutual and the packed local-face indices point back.
* The two cells of an interior face carry exactly opposite unit normals (bit
  for bit): the stage kernel evaluates each face flux with its own trace first
  and its own normal, and the LLF evaluation is exactly antisymmetric, so the
  two cells obtain exact negatives only with exactly opposite normals.
* |n~| = 2 |e| / |K| describes one edge length from both sides.
* The internal order is a permutation of the caller's cells, and the cell
  geometry (inverse Jacobian, KXRCF scale) matches the caller's triangle it
  came from.
"""
import dataclasses

import numpy as np
import pytest

from paper_2106_06280_gb300 import build
from paper_2106_06280_gb300 import workloads as W

G_RX, G_RY, G_SX, G_SY, G_N0X, G_N0Y, G_N0L = range(7)


@pytest.fixture(scope="module")
def cswdg():
    build.build()
    from paper_2106_06280_gb300 import cswdg as m
    return m


def problems():
    return [
        ("burgers_periodic", W.burgers_sine(12, seed=1), 2),
        ("vortex_periodic", W.isentropic_vortex(10, seed=5, box=(0.0, 10.0, 0.0, 10.0)), 2),
        ("dmr_walls_shock", W.double_mach(24, 6, seed=3), 2),
        ("riemann_transmissive", W.riemann_quadrants(9, seed=14), 1),
    ]


@pytest.mark.parametrize("name,pb,k", problems(), ids=[p[0] for p in problems()])
def test_host_mesh_faces_and_normals(cswdg, name, pb, k):
    h = cswdg.host_mesh(pb, k)
    geo, nbr, nbf, perm = h["geo"], h["nbr"], h["nbf"], h["perm"]
    nc = pb.mesh.nc
    assert np.array_equal(np.sort(perm), np.arange(nc))
    a = pb.mesh.xy[pb.mesh.tri[perm, 1]] - pb.mesh.xy[pb.mesh.tri[perm, 0]]
    b = pb.mesh.xy[pb.mesh.tri[perm, 2]] - pb.mesh.xy[pb.mesh.tri[perm, 0]]
    area = 0.5 * np.abs(a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0])
    # the scaled inverse Jacobian of the caller's triangle the cell came from:
    # (2 dr/dx)(2 ds/dy) - (2 dr/dy)(2 ds/dx) = 4 / det(J) = 8 / |K| (reference area 2)
    jac = geo[G_RX] * geo[G_SY] - geo[G_RY] * geo[G_SX]
    assert np.allclose(jac, 8.0 / area, rtol=1e-12, atol=0)
    ninterior = 0
    for f in range(3):
        nx, ny, nl = geo[G_N0X + 3 * f], geo[G_N0Y + 3 * f], geo[G_N0L + 3 * f]
        assert np.allclose(nx * nx + ny * ny, 1.0, rtol=0, atol=1e-14)
        code = nbr[f]
        inner = np.flatnonzero(code >= 0)
        ninterior += len(inner)
        c2 = code[inner]
        f2 = (nbf[inner].astype(np.int64) >> (2 * f)) & 3
        # mutual neighbours, local faces pointing back
        assert np.array_equal(nbr[f2, c2], inner)
        # exactly opposite unit normals, bit for bit
        assert np.array_equal(geo[G_N0X + 3 * f2, c2], -nx[inner])
        assert np.array_equal(geo[G_N0Y + 3 * f2, c2], -ny[inner])
        # one edge length seen from both sides: |n~| |K| / 2
        e1 = nl[inner] * area[inner] / 2
        e2 = geo[G_N0L + 3 * f2, c2] * area[c2] / 2
        assert np.allclose(e1, e2, rtol=1e-13, atol=0)
    # KXRCF scale (Sec. 3.1 with h the circumradius, reading R-kxrcf): kappa = h^{(k+1)/2} / sqrt(2),
    # the stored coefficients being sqrt(2/|K|) times the orthonormal ones
    c = b - a
    la, lb, lc = np.hypot(*a.T), np.hypot(*b.T), np.hypot(*c.T)
    hc = la * lb * lc / (4.0 * area)
    assert np.allclose(geo[13], hc ** ((k + 1) / 2) / np.sqrt(2.0), rtol=1e-12, atol=0)
    # each interior face is seen twice; boundary faces have negative codes
    assert ninterior % 2 == 0
    assert (nbr < 0).sum() == len(pb.mesh.bface) or pb.mesh.period is not None


def test_host_mesh_rejects_bad_arguments(cswdg):
    pb = W.burgers_sine(4, seed=1)
    with pytest.raises(cswdg.CswdgError, match="EINVAL"):
        cswdg.host_mesh(pb, 3)  # no such degree
    # a clockwise triangle is a mesh error, reported as a status
    tri = pb.mesh.tri.copy()
    tri[0] = tri[0][[0, 2, 1]]
    mesh = dataclasses.replace(pb.mesh, tri=tri)
    bad = dataclasses.replace(pb, mesh=mesh)
    with pytest.raises(cswdg.CswdgError, match="EMESH"):
        cswdg.host_mesh(bad, 2)


def test_morton_order_keeps_neighbours_close(cswdg):
    """On the full 460,800-cell double-Mach mesh the internal (Morton) order puts
    91 % of the face neighbours in the same 256-cell block and the median index
    distance at 3, which is what lets the stage kernel find its neighbours'
    modes in L1/L2."""
    pb = W.double_mach(960, 240, seed=3)
    nbr = cswdg.host_mesh(pb, 2)["nbr"]
    c = np.arange(pb.mesh.nc)
    inner = [nbr[f] >= 0 for f in range(3)]
    same = np.concatenate([(nbr[f][m] // 256) == (c[m] // 256) for f, m in enumerate(inner)])
    dist = np.concatenate([np.abs(nbr[f][m] - c[m]) for f, m in enumerate(inner)])
    assert same.mean() > 0.85 and np.median(dist) <= 8, (same.mean(), np.median(dist))


def test_tile_face_counts_of_the_flop_model(cswdg):
    """The per-variant FP64 flop count of bench.py (host logic only): k_stage's
    fixed count; for k_stage_tiles a brute-force walk over the tiles' faces
    (each interior face once, each face to another tile or the boundary once
    per side) gives the same flux and outer-trace counts, and the count lies
    between its bounds (one flux per face pair at the least, k_stage's three at
    the most)."""
    import bench
    pb = W.double_mach(40, 10, seed=3)
    nbr = cswdg.host_mesh(pb, 2)["nbr"]
    nc = nbr.shape[1]
    assert bench.stage_flops_per_cell(cswdg, pb, (128, 0, 0)) == bench.STAGE_FLOPS_PER_CELL_EULER_P2
    for blk in (128, 256):
        flux = outer = 0
        for c in range(nc):
            for f in range(3):
                n = int(nbr[f, c])
                if n >= 0 and n // blk == c // blk and n != c:
                    flux += 1 if c < n else 0
                else:
                    flux += 1
                    outer += 1 if n >= 0 else 0
        want = 7 * 147 + 12 * (40 + 52) + 4 * (flux / nc) * 67 + 4 * (outer / nc) * 40 + 120 + 110
        got = bench.stage_flops_per_cell(cswdg, pb, (blk, 0, 1))
        assert abs(got - want) < 1e-9 * want
        lo = 7 * 147 + 12 * (40 + 52) + 4 * 1.5 * 67 + 230
        assert lo <= got < bench.STAGE_FLOPS_PER_CELL_EULER_P2

"""Seeded synthetic workloads: meshes, initial data and boundary set-ups.

This module holds no arithmetic of the method itself.  It only draws the
inputs both the CUDA path and the CPU oracle consume:

* ``split_square_mesh`` -- n_x x n_y squares, each cut along a diagonal
  chosen by a counter-based splitmix64 stream, interior vertices jittered
  uniformly by at most ``jitter * h`` per coordinate, boundary vertices left
  in place so that periodic faces pair exactly.  This replaces the paper's
  Gmsh meshes (Sec. 4, "meshes which contain some triangles of irregular
  size"), which are not available.
* initial conditions and boundary tables of the paper's test problems
  (Sec. 4.1 Examples 1-3, Sec. 4.2 Examples 5 and 7) and of the synthetic
  configurations built on them.

Boundary kinds (shared numbering with the C interface):
PERIODIC=0, DIRICHLET=1 (constant state), TRANSMISSIVE=2, WALL=3,
SHOCKLINE=4 (params x0, cot, speed, stateA, stateB: stateA where
x < x0 + y*cot + speed*t).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PERIODIC, DIRICHLET, TRANSMISSIVE, WALL, SHOCKLINE = 0, 1, 2, 3, 4
GAMMA = 1.4

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """Counter-based splitmix64: output n is mix(seed + (n+1)*golden)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (counters.astype(np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, counters: np.ndarray) -> np.ndarray:
    """Doubles in [0,1) from the top 53 bits of splitmix64."""
    return (splitmix64(seed, counters) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


@dataclass
class Mesh:
    xy: np.ndarray          # (nv, 2) float64
    tri: np.ndarray         # (nc, 3) int32, counter-clockwise
    bface: np.ndarray       # (nb, 3) int32: v0, v1, tag
    period: tuple | None    # (Lx, Ly) for periodic meshes
    bounds: tuple           # (x0, x1, y0, y1)
    nx: int = 0
    ny: int = 0

    @property
    def nc(self) -> int:
        return int(self.tri.shape[0])

    @property
    def nv(self) -> int:
        return int(self.xy.shape[0])


def split_square_mesh(nx: int, ny: int, x0: float, x1: float, y0: float, y1: float,
                      seed: int, jitter: float = 0.2, periodic: bool = False,
                      tag_fn=None) -> Mesh:
    """Jittered split-square triangulation with 2*nx*ny triangles.

    Draw order of the counter-based stream: counters 0 .. nx*ny-1 choose the
    diagonal of square (i, j) (index j*nx + i; low bit 0 -> diagonal
    (i,j)-(i+1,j+1), 1 -> (i+1,j)-(i,j+1)); counters nx*ny + 2*v and
    nx*ny + 2*v + 1 jitter vertex v = j*(nx+1) + i in x and y.
    ``tag_fn(side, xm, ym)`` returns the boundary tag of an edge with midpoint
    (xm, ym) on side 'left'|'right'|'bottom'|'top' (default: tag 0).
    """
    ii, jj = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="xy")
    ii = ii.ravel()
    jj = jj.ravel()
    hx = (x1 - x0) / nx
    hy = (y1 - y0) / ny
    x = x0 + (x1 - x0) * (ii / nx)
    y = y0 + (y1 - y0) * (jj / ny)
    x[ii == nx] = x1
    y[jj == ny] = y1
    nsq = nx * ny
    vid = np.arange((nx + 1) * (ny + 1))
    interior = (ii > 0) & (ii < nx) & (jj > 0) & (jj < ny)
    jx = (2.0 * uniform01(seed, nsq + 2 * vid) - 1.0) * jitter * hx
    jy = (2.0 * uniform01(seed, nsq + 2 * vid + 1) - 1.0) * jitter * hy
    x = np.where(interior, x + jx, x)
    y = np.where(interior, y + jy, y)
    xy = np.stack([x, y], axis=1)

    si, sj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    si = si.ravel()
    sj = sj.ravel()
    a = sj * (nx + 1) + si
    b = a + 1
    c = a + (nx + 1) + 1
    d = a + (nx + 1)
    diag = (splitmix64(seed, np.arange(nsq)) & np.uint64(1)).astype(bool)
    t1 = np.where(diag[:, None], np.stack([a, b, d], 1), np.stack([a, b, c], 1))
    t2 = np.where(diag[:, None], np.stack([b, c, d], 1), np.stack([a, c, d], 1))
    tri = np.empty((2 * nsq, 3), dtype=np.int32)
    tri[0::2] = t1
    tri[1::2] = t2

    if tag_fn is None:
        tag_fn = lambda side, xm, ym: 0  # noqa: E731
    bf = []
    for i in range(nx):  # bottom, left-to-right (interior on the left of v0->v1)
        v0, v1 = i, i + 1
        bf.append((v0, v1, tag_fn("bottom", 0.5 * (x[v0] + x[v1]), y0)))
    for i in range(nx):  # top
        v0, v1 = ny * (nx + 1) + i + 1, ny * (nx + 1) + i
        bf.append((v0, v1, tag_fn("top", 0.5 * (x[v0] + x[v1]), y1)))
    for j in range(ny):  # left
        v0, v1 = (j + 1) * (nx + 1), j * (nx + 1)
        bf.append((v0, v1, tag_fn("left", x0, 0.5 * (y[v0] + y[v1]))))
    for j in range(ny):  # right
        v0, v1 = j * (nx + 1) + nx, (j + 1) * (nx + 1) + nx
        bf.append((v0, v1, tag_fn("right", x1, 0.5 * (y[v0] + y[v1]))))
    bface = np.asarray(bf, dtype=np.int32)
    return Mesh(xy=np.ascontiguousarray(xy), tri=tri, bface=bface,
                period=(x1 - x0, y1 - y0) if periodic else None,
                bounds=(x0, x1, y0, y1), nx=nx, ny=ny)


# ---------------------------------------------------------------------------
# Problems
# ---------------------------------------------------------------------------

def prim_to_cons(rho, u, v, p, gamma=GAMMA):
    rho = np.asarray(rho, dtype=np.float64)
    u = np.broadcast_to(np.asarray(u, dtype=np.float64), rho.shape)
    v = np.broadcast_to(np.asarray(v, dtype=np.float64), rho.shape)
    p = np.broadcast_to(np.asarray(p, dtype=np.float64), rho.shape)
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return np.stack([rho, rho * u, rho * v, E], axis=-1)


@dataclass
class Problem:
    name: str
    equation: int                      # 0 Burgers, 1 Euler
    mesh: Mesh
    u0: object                         # callable (x, y) -> (n, nvar)
    boundaries: dict = field(default_factory=dict)  # tag -> (kind, params list)
    t_end: float = 0.0
    exact: object = None               # callable (x, y, t) -> (n, nvar) or None

    @property
    def nvar(self) -> int:
        return 1 if self.equation == 0 else 4


def burgers_sine(n: int, seed: int = 1) -> Problem:
    """u_t + (u^2/2)_x + (u^2/2)_y = 0 on periodic [0,2]^2 with
    u0 = 0.5 + 0.25 sin(pi (x+y)) (the paper's Example 1 family, Eq. 2dBurgers)."""
    mesh = split_square_mesh(n, n, 0.0, 2.0, 0.0, 2.0, seed, periodic=True)

    def u0(x, y):
        return (0.5 + 0.25 * np.sin(np.pi * (x + y)))[:, None]

    return Problem("burgers_sine", 0, mesh, u0, {0: (PERIODIC, [])}, 0.1, None)


def euler_entropy_wave(n: int, seed: int = 7) -> Problem:
    """Sec. 4.1 Example 2: rho = 1 + 0.2 sin(pi(x+y)), u=0.7, v=0.3, p=1 on
    periodic [0,2]^2; exact solution rho(x,y,t) = 1 + 0.2 sin(pi(x+y-t))."""
    mesh = split_square_mesh(n, n, 0.0, 2.0, 0.0, 2.0, seed, periodic=True)

    def exact(x, y, t):
        return prim_to_cons(1.0 + 0.2 * np.sin(np.pi * (x + y - t)), 0.7, 0.3, 1.0)

    return Problem("euler_entropy_wave", 1, mesh, lambda x, y: exact(x, y, 0.0),
                   {0: (PERIODIC, [])}, 2.0, exact)


def isentropic_vortex(n: int, seed: int = 5, eps: float | None = None,
                      centre: tuple | None = None, box=(0.0, 10.0, -5.0, 5.0)) -> Problem:
    """Sec. 4.1 Example 3 vortex in the paper's own form:
    rho = (1 - (gamma-1)/(16 gamma pi^2) eps^2 e^{2(1-r^2)})^{1/(gamma-1)},
    u = 1 - eps e^{1-r^2} (y-y0)/(2 pi), v = eps e^{1-r^2} (x-x0-t)/(2 pi), p = rho^gamma,
    advected with unit speed in x on a periodic box."""
    rng_u = uniform01(seed, np.arange(3))
    if eps is None:
        eps = 3.0 + 4.0 * rng_u[0]
    x0b, x1b, y0b, y1b = box
    if centre is None:
        centre = (x0b + (x1b - x0b) * (0.3 + 0.4 * rng_u[1]), y0b + (y1b - y0b) * (0.3 + 0.4 * rng_u[2]))
    xc, yc = centre
    Lx = x1b - x0b
    mesh = split_square_mesh(n, n, x0b, x1b, y0b, y1b, seed, periodic=True)

    def exact(x, y, t):
        dx = x - xc - t
        dx = dx - Lx * np.round(dx / Lx)
        dy = y - yc
        r2 = dx * dx + dy * dy
        g = GAMMA
        rho = (1.0 - (g - 1.0) / (16.0 * g * np.pi ** 2) * eps ** 2 * np.exp(2.0 * (1.0 - r2))) ** (1.0 / (g - 1.0))
        u = 1.0 - eps * np.exp(1.0 - r2) * dy / (2.0 * np.pi)
        v = eps * np.exp(1.0 - r2) * dx / (2.0 * np.pi)
        return prim_to_cons(rho, u, v, rho ** g)

    return Problem("isentropic_vortex", 1, mesh, lambda x, y: exact(x, y, 0.0),
                   {0: (PERIODIC, [])}, 2.0, exact)


DMR_X0 = 1.0 / 6.0
DMR_COT = 1.0 / math.sqrt(3.0)
DMR_SPEED = 20.0 / math.sqrt(3.0)


def dmr_states(gamma=GAMMA):
    pre = prim_to_cons(np.array([1.4]), 0.0, 0.0, 1.0, gamma)[0]
    post = prim_to_cons(np.array([8.0]), 8.25 * math.cos(math.pi / 6.0), -8.25 * math.sin(math.pi / 6.0), 116.5, gamma)[0]
    return pre, post


def double_mach(nx: int = 960, ny: int = 240, seed: int = 3) -> Problem:
    """Sec. 4.2 Example 5: Mach 10 shock through (1/6, 0) at 60 degrees on
    [0,4]x[0,1].  Tags: 1 post-shock inflow (left side and bottom x < 1/6),
    2 reflecting wall (bottom x >= 1/6), 3 right side: the undisturbed
    pre-shock state (the exact solution there up to t = 0.28, when the
    incident shock reaches x = 4; the paper leaves this side to the cited
    set-up), 4 top boundary following the exact shock position
    x_s(t) = 1/6 + (1 + 20 t)/sqrt(3)."""
    pre, post = dmr_states()

    def tag_fn(side, xm, ym):
        if side == "left":
            return 1
        if side == "right":
            return 3
        if side == "top":
            return 4
        return 1 if xm < DMR_X0 else 2

    mesh = split_square_mesh(nx, ny, 0.0, 4.0, 0.0, 1.0, seed, tag_fn=tag_fn)

    def u0(x, y):
        post_region = x < DMR_X0 + y * DMR_COT
        return np.where(post_region[:, None], post[None, :], pre[None, :])

    bnd = {1: (DIRICHLET, list(post)), 2: (WALL, []), 3: (DIRICHLET, list(pre)),
           4: (SHOCKLINE, [DMR_X0, DMR_COT, DMR_SPEED] + list(post) + list(pre))}
    return Problem("double_mach", 1, mesh, u0, bnd, 0.2, None)


def riemann_quadrants(n: int, seed: int) -> Problem:
    """Sec. 4.2 Example 7 family on [0,1]^2 with transmissive boundaries and
    four quadrant states drawn from the seed: rho in [0.1,1.5], p in
    [0.03,1.5], |u|,|v| <= 1.2."""
    r = uniform01(seed, np.arange(16)).reshape(4, 4)
    rho = 0.1 + 1.4 * r[:, 0]
    p = 0.03 + 1.47 * r[:, 1]
    u = -1.2 + 2.4 * r[:, 2]
    v = -1.2 + 2.4 * r[:, 3]
    states = prim_to_cons(rho, u, v, p)
    mesh = split_square_mesh(n, n, 0.0, 1.0, 0.0, 1.0, seed, tag_fn=lambda s, xm, ym: 2)

    def u0(x, y):
        q = np.where(x >= 0.5, np.where(y >= 0.5, 0, 3), np.where(y >= 0.5, 1, 2))
        return states[q]

    return Problem("riemann_quadrants", 1, mesh, u0, {2: (TRANSMISSIVE, [])}, 0.25, None)


def cell_areas(mesh: Mesh) -> np.ndarray:
    """Triangle areas (shoelace), used only to scale random modal data."""
    p = mesh.xy[mesh.tri]
    return 0.5 * ((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1])
                  - (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1]))


def random_modes(mesh: Mesh, nvar: int, np_: int, seed: int, scale: float = 0.3) -> np.ndarray:
    """Seeded random modal state (nc, nvar, np) in the physically orthonormal
    basis: cell means of order one plus random higher modes, scaled by
    sqrt(|K|) so that point values stay O(1); admissible for Euler
    (positive density and pressure at every point)."""
    nc = mesh.nc
    r = uniform01(seed, np.arange(nc * nvar * np_)).reshape(nc, nvar, np_) * 2.0 - 1.0
    out = scale * r
    if nvar == 1:
        out[:, 0, 0] += 1.0
    else:
        base = np.array([1.0, 0.3, -0.2, 2.5])
        out[:, :, 0] = base[None, :] * (1.0 + 0.1 * r[:, :, 0])
        out[:, :, 1:] *= 0.2 * np.abs(base)[None, :, None]
    return out * np.sqrt(cell_areas(mesh))[:, None, None]


def merge_meshes(meshes, offsets):
    """Disjoint union of meshes translated by offsets (independent problems
    advanced as one mesh: no face connects two of them)."""
    xy, tri, bf = [], [], []
    nv = 0
    for m, (ox, oy) in zip(meshes, offsets):
        xy.append(m.xy + np.array([ox, oy]))
        tri.append(m.tri + nv)
        b = m.bface.copy()
        b[:, :2] += nv
        bf.append(b)
        nv += m.nv
    x0 = min(o[0] for o in offsets)
    y0 = min(o[1] for o in offsets)
    return Mesh(xy=np.ascontiguousarray(np.concatenate(xy)), tri=np.ascontiguousarray(np.concatenate(tri).astype(np.int32)),
                bface=np.ascontiguousarray(np.concatenate(bf).astype(np.int32)), period=None,
                bounds=(x0, max(o[0] for o in offsets) + 1.0, y0, max(o[1] for o in offsets) + 1.0))


def riemann_ensemble(n_meshes: int = 256, total: float = 5.0e6, seed: int = 1000, lo: float = 2.0e3,
                     hi: float = 6.0e4) -> Problem:
    """Ensemble of independent four-quadrant Riemann problems (Sec. 4.2
    Example 7 family) on [0,1]^2, mesh i drawn with seed seed+i: triangle counts
    log-uniform in [lo, hi], rescaled towards `total` (clamped to [lo, hi]);
    the meshes are laid out on a 16-wide grid of unit squares 1.5 apart and
    advanced together as one disconnected mesh with transmissive boundaries."""
    r = uniform01(seed, np.arange(n_meshes))
    sizes = np.exp(np.log(lo) + (np.log(hi) - np.log(lo)) * r)
    sizes = np.clip(sizes * total / sizes.sum(), lo, hi)
    probs = [riemann_quadrants(max(4, int(round(np.sqrt(sz / 2.0)))), seed + i) for i, sz in enumerate(sizes)]
    offsets = [(1.5 * (i % 16), 1.5 * (i // 16)) for i in range(n_meshes)]
    mesh = merge_meshes([p.mesh for p in probs], offsets)

    def u0(x, y):
        ix = np.clip(np.floor(x / 1.5).astype(int), 0, 15)
        iy = np.floor(y / 1.5).astype(int)
        k = iy * 16 + ix
        out = np.zeros((len(x), 4))
        for i in np.unique(k):
            sel = k == i
            out[sel] = probs[i].u0(x[sel] - offsets[i][0], y[sel] - offsets[i][1])
        return out

    return Problem("riemann_ensemble", 1, mesh, u0, {2: (TRANSMISSIVE, [])}, 0.25, None)

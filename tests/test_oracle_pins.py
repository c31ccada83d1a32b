"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms, numpy/scipy library routines used as independent integrators or
solvers, brute force on tiny inputs, invariants stated in the paper, exact
solutions and convergence orders (Tables 1-3 report order k+1).
"""
import math

import numpy as np
import pytest

import oracle
from oracle.exact import burgers_sine_exact
from paper_2106_06280_gb300 import workloads as W

# ----------------------------------------------------------------------------
# independent integration helpers (numpy Gauss-Legendre on the collapsed square)
# ----------------------------------------------------------------------------
_X, _WX = np.polynomial.legendre.leggauss(10)
_U = 0.5 * (_X + 1.0)
_WU = 0.5 * _WX


def tri_quad(T):
    """Points (n,2) and weights (sum = area) exact to degree 18 on triangle T (3,2)."""
    T = np.asarray(T, dtype=float)
    u, v = np.meshgrid(_U, _U, indexing="ij")
    wu, wv = np.meshgrid(_WU, _WU, indexing="ij")
    P = (1 - u)[..., None] * T[0] + (u * (1 - v))[..., None] * T[1] + (u * v)[..., None] * T[2]
    area = 0.5 * abs((T[1, 0] - T[0, 0]) * (T[2, 1] - T[0, 1]) - (T[2, 0] - T[0, 0]) * (T[1, 1] - T[0, 1]))
    w = wu * wv * 2.0 * u * area
    return P.reshape(-1, 2), w.ravel()


def tri_area(T):
    T = np.asarray(T, dtype=float)
    return 0.5 * abs((T[1, 0] - T[0, 0]) * (T[2, 1] - T[0, 1]) - (T[2, 0] - T[0, 0]) * (T[1, 1] - T[0, 1]))


def tri_mean(T, f):
    P, w = tri_quad(T)
    return float(np.sum(w * f(P[:, 0], P[:, 1])) / np.sum(w))


REF = np.array([[-1.0, -1.0], [1.0, -1.0], [-1.0, 1.0]])


# ----------------------------------------------------------------------------
# quadrature
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_gauss_legendre_exactness(n):
    x, w = oracle.gauss_legendre(n)
    for j in range(2 * n):
        exact = 2.0 / (j + 1) if j % 2 == 0 else 0.0
        assert abs(np.sum(w * x ** j) - exact) < 1e-14
    # not exact one degree higher (it is a genuine n-point rule)
    assert abs(np.sum(w * x ** (2 * n)) - 2.0 / (2 * n + 1)) > 1e-6


@pytest.mark.parametrize("deg,npts", [(2, 3), (4, 6), (5, 7)])
def test_symmetric_triangle_rules(deg, npts):
    b, w = oracle.tri_rule(0, deg)
    assert len(w) == npts
    assert np.all(w > 0) and np.all(b > 0)
    for p in range(deg + 1):
        for q in range(deg + 1 - p):
            exact = 2.0 * math.factorial(p) * math.factorial(q) / math.factorial(p + q + 2)
            assert abs(np.sum(w * b[:, 1] ** p * b[:, 2] ** q) - exact) < 1e-14


@pytest.mark.parametrize("m", [2, 3, 4, 6])
def test_duffy_rule_exactness(m):
    b, w = oracle.tri_rule(1, m)
    for p in range(2 * m - 1):
        for q in range(2 * m - 1 - p):
            exact = 2.0 * math.factorial(p) * math.factorial(q) / math.factorial(p + q + 2)
            assert abs(np.sum(w * b[:, 1] ** p * b[:, 2] ** q) - exact) < 1e-14


# ----------------------------------------------------------------------------
# basis (Sec. 2, Eq. triangleBasis)
# ----------------------------------------------------------------------------
def test_basis_closed_forms_p1():
    rng = np.random.default_rng(0)
    for _ in range(20):
        r, s = rng.uniform(-1, 0.0, 2)
        if r + s > 0:
            continue
        assert abs(oracle.psi(1, 0, r, s)[0] - 1 / math.sqrt(2)) < 1e-15
        assert abs(oracle.psi(1, 1, r, s)[0] - (1 + 3 * s) / 2) < 1e-14
        assert abs(oracle.psi(1, 2, r, s)[0] - math.sqrt(3) / 2 * (1 + 2 * r + s)) < 1e-14


@pytest.mark.parametrize("k", [1, 2])
def test_basis_orthonormal(k):
    P, w = tri_quad(REF)
    np_ = (k + 1) * (k + 2) // 2
    V = np.array([[oracle.psi(k, m, r, s)[0] for r, s in P] for m in range(np_)])
    G = (V * w) @ V.T
    assert np.abs(G - np.eye(np_)).max() < 1e-13


@pytest.mark.parametrize("k", [1, 2])
def test_basis_gradient_finite_difference(k):
    rng = np.random.default_rng(1)
    h = 1e-6
    for _ in range(10):
        r, s = rng.uniform(-0.9, -0.1, 2)
        for m in range((k + 1) * (k + 2) // 2):
            v = oracle.psi(k, m, r, s)
            dr = (oracle.psi(k, m, r + h, s)[0] - oracle.psi(k, m, r - h, s)[0]) / (2 * h)
            ds = (oracle.psi(k, m, r, s + h)[0] - oracle.psi(k, m, r, s - h)[0]) / (2 * h)
            assert abs(v[1] - dr) < 1e-8 and abs(v[2] - ds) < 1e-8


def test_least_squares_matches_numpy():
    rng = np.random.default_rng(2)
    for m, n in [(3, 2), (9, 5), (15, 9), (15, 14)]:
        A = rng.normal(size=(m, n))
        b = rng.normal(size=m)
        c, st = oracle.lsq(A, b)
        ref = np.linalg.lstsq(A, b, rcond=None)[0]
        assert st == 0 and np.abs(c - ref).max() < 1e-12
    A = rng.normal(size=(6, 3))
    A[:, 2] = A[:, 0] + A[:, 1]
    assert oracle.lsq(A, rng.normal(size=6))[1] != 0  # rank loss reported


# ----------------------------------------------------------------------------
# operator L_h (Sec. 2, Eq. weakFormScheme2D) and flux (local Lax-Friedrichs)
# ----------------------------------------------------------------------------
def _transmissive_box(n, seed, eq):
    mesh = W.split_square_mesh(n, n, 0.0, 1.0, 0.0, 1.0, seed, tag_fn=lambda side, xm, ym: 2)
    return W.Problem("box", eq, mesh, None, {2: (W.TRANSMISSIVE, [])})


def _on_box_side(a, b):
    """Both end points on one side of the unit square."""
    return any(a[j] == v and b[j] == v for j in (0, 1) for v in (0.0, 1.0))


@pytest.mark.parametrize("k", [1, 2])
def test_rhs_exact_for_continuous_polynomial_burgers(k):
    """Continuous degree-k data: jumps vanish, every quadrature is exact, so
    in a cell without boundary faces L_h(u) is the L2 projection of
    -u (u_x + u_y) (integration by parts).  A transmissive face takes the cell
    mean ubar as the flux's outside state (reading R-bc), which adds
    -int_e psi_i (F*(u-, ubar) - F(u-)).n ds for that face; that term is formed
    here independently (the method's face rule, numpy's Gauss-Legendre with
    2 / 4 points, and the local Lax-Friedrichs flux of Burgers written out)."""
    pb = _transmissive_box(4, 3, 0)
    o = oracle.Oracle(pb, k=k, limiter=0)
    if k == 1:
        f = lambda x, y: 0.3 + 0.5 * x - 0.2 * y                                    # noqa: E731
        fx = lambda x, y: 0.5 + 0 * x                                              # noqa: E731
        fy = lambda x, y: -0.2 + 0 * x                                             # noqa: E731
    else:
        f = lambda x, y: 0.3 + 0.5 * x - 0.2 * y + 0.7 * x * x - 0.4 * x * y + 0.25 * y * y  # noqa: E731
        fx = lambda x, y: 0.5 + 1.4 * x - 0.4 * y                                  # noqa: E731
        fy = lambda x, y: -0.2 - 0.4 * x + 0.5 * y                                 # noqa: E731
    u = o.project(lambda x, y: f(x, y)[:, None])
    L = o.rhs(u, 0.0)
    m = pb.mesh
    for c in range(m.nc):
        T = m.xy[m.tri[c]]
        P, w = tri_quad(T)
        area = w.sum()
        # psi^K at P via the reference map
        A = np.array([[T[1, 0] - T[0, 0], T[2, 0] - T[0, 0]], [T[1, 1] - T[0, 1], T[2, 1] - T[0, 1]]])
        rs = np.linalg.solve(A, (P - T[0]).T).T * 2 - 1
        g = -f(P[:, 0], P[:, 1]) * (fx(P[:, 0], P[:, 1]) + fy(P[:, 0], P[:, 1]))
        extra = np.zeros(o.np)
        ubar = tri_mean(T, f)
        cen = T.mean(axis=0)
        for e in range(3):
            a, b = T[e], T[(e + 1) % 3]
            if not _on_box_side(a, b):
                continue
            d = b - a
            L_e = np.hypot(*d)
            n = np.array([d[1], -d[0]]) / L_e
            if n @ (0.5 * (a + b) - cen) < 0:
                n = -n
            xg, wg = np.polynomial.legendre.leggauss(2 if k == 1 else 4)  # the face rule (R-weak): max() is not polynomial
            Q = a[None, :] + 0.5 * (xg[:, None] + 1.0) * d[None, :]
            um = f(Q[:, 0], Q[:, 1])
            sn = n[0] + n[1]
            alpha = np.maximum(np.abs(um), abs(ubar)) * abs(sn)
            fstar = 0.5 * (0.5 * um ** 2 + 0.5 * ubar ** 2) * sn - 0.5 * alpha * (ubar - um)
            rsq = np.linalg.solve(A, (Q - T[0]).T).T * 2 - 1
            for i in range(o.np):
                psi_e = np.array([oracle.psi(k, i, r, s)[0] for r, s in rsq]) * math.sqrt(2 / area)
                extra[i] -= np.sum(0.5 * wg * L_e * psi_e * (fstar - 0.5 * um ** 2 * sn))
        for i in range(o.np):
            psi = np.array([oracle.psi(k, i, r, s)[0] for r, s in rs]) * math.sqrt(2 / area)
            assert abs(L[c, 0, i] - np.sum(w * g * psi) - extra[i]) < 1e-12


@pytest.mark.parametrize("k", [1, 2])
def test_rhs_vanishes_on_constant_states(k):
    pb = W.burgers_sine(5, seed=4)
    o = oracle.Oracle(pb, k=k, limiter=0)
    u = o.project(lambda x, y: np.full((len(x), 1), 0.7))
    assert np.abs(o.rhs(u)).max() < 1e-13
    pe = W.euler_entropy_wave(4, seed=5)
    oe = oracle.Oracle(pe, k=k, limiter=0)
    ue = oe.project(lambda x, y: W.prim_to_cons(np.full(len(x), 1.2), 0.4, -0.3, 0.9))
    assert np.abs(oe.rhs(ue)).max() < 1e-12
    # gas at rest in a box of reflecting walls
    mesh = W.split_square_mesh(4, 4, 0.0, 1.0, 0.0, 1.0, 6, tag_fn=lambda s, xm, ym: 3)
    pw = W.Problem("walls", 1, mesh, None, {3: (W.WALL, [])})
    ow = oracle.Oracle(pw, k=k, limiter=0)
    uw = ow.project(lambda x, y: W.prim_to_cons(np.full(len(x), 1.0), 0.0, 0.0, 2.0))
    assert np.abs(ow.rhs(uw)).max() < 1e-12


def test_llf_flux_consistency_and_antisymmetry():
    pe = W.euler_entropy_wave(3)
    oe = oracle.Oracle(pe, k=1, limiter=0)
    rng = np.random.default_rng(7)
    for _ in range(10):
        U = W.prim_to_cons(np.array([rng.uniform(0.5, 2)]), rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(0.5, 2))[0]
        V = W.prim_to_cons(np.array([rng.uniform(0.5, 2)]), rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(0.5, 2))[0]
        th = rng.uniform(0, 2 * np.pi)
        n = np.array([np.cos(th), np.sin(th)])
        rho, mx, my, E = U
        p = 0.4 * (E - 0.5 * (mx * mx + my * my) / rho)
        un = (mx * n[0] + my * n[1]) / rho
        Fn = np.array([rho * un, mx * un + p * n[0], my * un + p * n[1], (E + p) * un])
        assert np.abs(oe.flux(U, U, *n) - Fn).max() < 1e-13
        assert np.abs(oe.flux(U, V, *n) + oe.flux(V, U, *(-n))).max() < 1e-13


def test_euler_eigenvectors():
    """L R = I and R diag(lambda) L equals the flux Jacobian (central FD of the
    oracle's own consistent flux F*(U,U,n) = F(U).n)."""
    pe = W.euler_entropy_wave(3)
    oe = oracle.Oracle(pe, k=1, limiter=0)
    U = W.prim_to_cons(np.array([1.3]), 0.4, -0.7, 1.1)[0]
    for n in [(1.0, 0.0), (0.0, 1.0), (0.6, 0.8)]:
        R, L = oracle.euler_eigen(U, *n)
        assert np.abs(L @ R - np.eye(4)).max() < 1e-13
        J = np.zeros((4, 4))
        for j in range(4):
            h = 1e-6 * max(1.0, abs(U[j]))
            Up, Um = U.copy(), U.copy()
            Up[j] += h
            Um[j] -= h
            J[:, j] = (oe.flux(Up, Up, *n) - oe.flux(Um, Um, *n)) / (2 * h)
        rho, mx, my, E = U
        u, v = mx / rho, my / rho
        p = 0.4 * (E - 0.5 * rho * (u * u + v * v))
        c = math.sqrt(1.4 * p / rho)
        un = u * n[0] + v * n[1]
        lam = np.diag([un - c, un, un, un + c])
        assert np.abs(R @ lam @ L - J).max() < 1e-7


# ----------------------------------------------------------------------------
# time stepping (Eq. timeIntegrate, Table tvd)
# ----------------------------------------------------------------------------
def test_ssp_rk3_matches_butcher_form():
    """Shu-Osher coefficients of Table tvd versus the equivalent Butcher form
    k1 = L(u), k2 = L(u + dt k1), k3 = L(u + dt/4 (k1 + k2)),
    u+ = u + dt/6 (k1 + k2 + 4 k3)."""
    pb = W.burgers_sine(6, seed=8)
    o = oracle.Oracle(pb, k=2, limiter=0)
    u = o.project(pb.u0)
    dt = 0.01
    k1 = o.rhs(u)
    k2 = o.rhs(u + dt * k1)
    k3 = o.rhs(u + dt / 4 * (k1 + k2))
    ref = u + dt / 6 * (k1 + k2 + 4 * k3)
    got, _, _ = o.step(u, 0.0, dt)
    assert np.abs(got - ref).max() < 1e-14


def test_rk3_temporal_order():
    pb = W.burgers_sine(4, seed=9)
    o = oracle.Oracle(pb, k=1, limiter=0)
    u0 = o.project(pb.u0)
    T = 0.04

    def run(n):
        u = u0.copy()
        for i in range(n):
            u, _, _ = o.step(u, i * T / n, T / n)
        return u

    ref = run(256)
    e1 = np.abs(run(8) - ref).max()
    e2 = np.abs(run(16) - ref).max()
    assert 2.7 < math.log2(e1 / e2) < 3.3


# ----------------------------------------------------------------------------
# conservation and exact solution
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("k,limiter", [(1, 1), (2, 1), (1, 2), (2, 2)])
def test_conservation_periodic_burgers(k, limiter):
    pb = W.burgers_sine(8, seed=10)
    o = oracle.Oracle(pb, k=k, limiter=limiter)
    u = o.project(pb.u0)
    s0 = o.conservation(u)
    u, n, _ = o.run(u, 0.0, 0.05, 0.1)
    assert abs(o.conservation(u)[0] - s0[0]) < 1e-13 * abs(s0[0])


def test_conservation_periodic_euler_limited():
    pb = W.euler_entropy_wave(5, seed=11)
    o = oracle.Oracle(pb, k=2, limiter=2)
    u = o.project(pb.u0)
    s0 = o.conservation(u)
    for i in range(3):
        u, _, st = o.step(u, i * 0.005, 0.005)
        assert st == 0
    assert np.abs(o.conservation(u) - s0).max() < 1e-13 * np.abs(s0).max()


def test_burgers_exact_solution_satisfies_pde():
    rng = np.random.default_rng(12)
    x, y = rng.uniform(0, 2, 50), rng.uniform(0, 2, 50)
    t, h = 0.3, 1e-5
    u = burgers_sine_exact(x, y, t)[:, 0]
    ut = (burgers_sine_exact(x, y, t + h) - burgers_sine_exact(x, y, t - h))[:, 0] / (2 * h)
    ux = (burgers_sine_exact(x + h, y, t) - burgers_sine_exact(x - h, y, t))[:, 0] / (2 * h)
    uy = (burgers_sine_exact(x, y + h, t) - burgers_sine_exact(x, y - h, t))[:, 0] / (2 * h)
    assert np.abs(ut + u * ux + u * uy).max() < 1e-7


# ----------------------------------------------------------------------------
# KXRCF (Sec. 3.1, Eq. troubledCellIndicator)
# ----------------------------------------------------------------------------
def test_kxrcf_no_flags_on_continuous_data():
    pb = _transmissive_box(5, 13, 0)
    o = oracle.Oracle(pb, k=1, limiter=1)
    u = o.project(lambda x, y: (0.4 + 0.3 * x - 0.6 * y)[:, None])
    fl, R = o.detect(u)
    assert fl.sum() == 0 and np.abs(R).max() < 1e-12
    pe = W.euler_entropy_wave(4)
    oe = oracle.Oracle(pe, k=2, limiter=1)
    ue = oe.project(lambda x, y: W.prim_to_cons(np.full(len(x), 1.1), 0.3, 0.2, 1.0))
    fl, R = oe.detect(ue)
    assert fl.sum() == 0 and np.abs(R).max() < 1e-12


@pytest.mark.parametrize("k", [1, 2])
def test_kxrcf_brute_force(k):
    """R_j recomputed from its definition with independent face and cell
    quadrature (numpy Gauss-Legendre) and the oracle's point evaluation of u_h;
    ||U_j|| is the cell's L2 norm over its normalised measure (reading
    R-kxrcf)."""
    pb = W.burgers_sine(4, seed=14)
    o = oracle.Oracle(pb, k=k, limiter=1)
    u = W.random_modes(pb.mesh, 1, o.np, 15, scale=0.05)
    fl, R = o.detect(u)
    nb, nbf, sh = o.connectivity()
    m = pb.mesh
    gx, gw = np.polynomial.legendre.leggauss(8)
    for c in range(0, m.nc, 3):
        T = m.xy[m.tri[c]]
        area = 0.5 * ((T[1, 0] - T[0, 0]) * (T[2, 1] - T[0, 1]) - (T[2, 0] - T[0, 0]) * (T[1, 1] - T[0, 1]))
        ub = u[c, 0, 0] / math.sqrt(area)
        num, inlen = 0.0, 0.0
        for f in range(3):
            a, b = T[f], T[(f + 1) % 3]
            e = b - a
            L = np.hypot(*e)
            n = np.array([e[1], -e[0]]) / L
            if not (ub * n[0] + ub * n[1] < 0):
                continue
            inlen += L
            pts = a[None, :] + 0.5 * (gx[:, None] + 1) * e[None, :]
            ui = o.eval_points(u, np.full(len(pts), c), pts)[:, 0]
            uo = o.eval_points(u, np.full(len(pts), nb[c, f]), pts - sh[c, f])[:, 0]
            num += np.sum(0.5 * gw * L * (ui - uo))
        la, lb, lc = np.hypot(*(T[1] - T[0])), np.hypot(*(T[2] - T[1])), np.hypot(*(T[0] - T[2]))
        h = la * lb * lc / (4 * area)
        # ||U_j||: the L2 norm over the cell with respect to its normalised
        # measure, (|K|^-1 int_K u_h^2)^(1/2), by an independent degree-18 rule
        P, w = tri_quad(T)
        uh = o.eval_points(u, np.full(len(P), c), P)[:, 0]
        nrm = math.sqrt(np.sum(w * uh ** 2) / area)
        Rb = 0.0 if inlen == 0 else abs(num) / (h ** ((k + 1) / 2) * inlen * nrm)
        assert abs(Rb - R[c]) < 1e-10 * max(1.0, Rb)
        assert fl[c] == (Rb > 1.0)


# ----------------------------------------------------------------------------
# CSWENO (Sec. 3.2)
# ----------------------------------------------------------------------------
def _stencil_case(k, seed=16):
    pb = W.burgers_sine(6, seed=seed)
    o = oracle.Oracle(pb, k=k, limiter=2)
    return pb, o


@pytest.mark.parametrize("k", [1, 2])
def test_subcell_split_geometry(k):
    pb, o = _stencil_case(k)
    nb, nbf, sh = o.connectivity()
    for c in [0, 7, 31]:
        tri, gh = o.stencil(c)
        for f in range(3):
            N = pb.mesh.xy[pb.mesh.tri[nb[c, f]]] + sh[c, f]
            aN = tri_area(N)
            ar = [tri_area(t) for t in tri[f]]
            # "three equal parts" (Sec. 3.2): each third is a third of the neighbour
            assert np.allclose(ar[:3], aN / 3, rtol=1e-13)
            assert abs(ar[3] + ar[4] - ar[1]) < 1e-14 and abs(ar[5] + ar[6] - ar[2]) < 1e-14
            # the first third sits on the edge shared with the cell
            Tc = pb.mesh.xy[pb.mesh.tri[c]]
            edge = np.array([Tc[f], Tc[(f + 1) % 3]])
            first = tri[f, 0, 1:]
            assert np.abs(np.sort(first, axis=0) - np.sort(edge, axis=0)).max() < 1e-12


@pytest.mark.parametrize("k", [1, 2])
def test_subcell_means_brute_force(k):
    pb, o = _stencil_case(k)
    u = W.random_modes(pb.mesh, 1, o.np, 17)
    nb, nbf, sh = o.connectivity()
    for c in [3, 20]:
        tri, gh = o.stencil(c)
        sm = o.subcell_means(u, c)
        for f in range(3):
            d = nb[c, f]
            for i in range(7):
                T = tri[f, i]
                P, w = tri_quad(T)
                vals = o.eval_points(u, np.full(len(P), d), P - sh[c, f])[:, 0]
                assert abs(np.sum(w * vals) / np.sum(w) - sm[f, i, 0]) < 1e-13
            # area-weighted thirds reproduce the neighbour mean
            aN = tri_area(pb.mesh.xy[pb.mesh.tri[d]])
            assert abs(np.mean(sm[f, :3, 0]) - u[d, 0, 0] / math.sqrt(aN)) < 1e-13


def _poly_means(o, pb, c, coef, deg):
    fr = o.frame(c)
    exps = [(d - e, e) for d in range(1, deg + 1) for e in range(d + 1)]

    def P(x, y):
        xi, eta = (x - fr["x0"]) / fr["h0"], (y - fr["y0"]) / fr["h0"]
        return 0.37 + sum(cf * xi ** a * eta ** b for cf, (a, b) in zip(coef, exps))

    tri, gh = o.stencil(c)
    th = np.array([[tri_mean(tri[f, i], P) for i in range(3)] for f in range(3)])
    hf = np.array([[tri_mean(tri[f, 3 + i], P) for i in range(4)] for f in range(3)])
    ub = tri_mean(pb.mesh.xy[pb.mesh.tri[c]], P)
    return P, th, hf, ub


@pytest.mark.parametrize("k,deg", [(1, 1), (1, 2), (2, 1), (2, 2), (2, 3)])
def test_stencil_least_squares_exactness(k, deg):
    """Means of a global polynomial of degree <= deg(q_m) give back that
    polynomial (Step 1; constrained least squares in the sense of hs1)."""
    pb, o = _stencil_case(k)
    rng = np.random.default_rng(18 + deg)
    coef = rng.normal(size=(deg + 1) * (deg + 2) // 2 - 1)
    for c in [5, 44]:
        P, th, hf, ub = _poly_means(o, pb, c, coef, deg)
        r = o.weno(c, ub, th, hf)
        assert r["status"] == 0
        pad = np.zeros(14)
        pad[: len(coef)] = coef
        if deg <= 1:
            assert np.abs(r["q2"] - pad[:2]).max() < 1e-11
        if deg <= 2:
            assert np.abs(r["q3"] - pad[:5]).max() < 1e-11
        if k == 2:
            assert np.abs(r["q4"] - pad[:9]).max() < 1e-10


@pytest.mark.parametrize("k", [1, 2])
def test_linear_weights_sum_to_one_and_reproduce_top_polynomial(k):
    """Sum gamma = 1 (Eqs. equivalentOrder1-4) and with omega = gamma the
    combination is the top stencil polynomial; for degree-k data the
    reconstruction (Eq. finalMoments) returns the data's own modes."""
    pb, o = _stencil_case(k)
    rng = np.random.default_rng(19)
    coef = rng.normal(size=(k + 1) * (k + 2) // 2 - 1)
    for c in [9, 60]:
        P, th, hf, ub = _poly_means(o, pb, c, coef, k)
        r = o.weno(c, ub, th, hf, force_linear=True)
        nslot = 3 if k == 1 else 4
        g = r["gamma"][:nslot]
        assert abs(g.sum() - 1.0) < 1e-15
        assert np.all(np.diff(g) > 0)  # (1/h)^{l-1}: larger weights for higher degree
        exact = o.project(lambda x, y: P(x, y)[:, None])[c, 0]
        assert np.abs(r["modes"][1:] - exact[1:]).max() < 1e-11


def test_smoothness_indicator_closed_forms():
    pb, o = _stencil_case(2)
    c = 12
    fr = o.frame(c)
    assert o.beta(c, np.zeros(14), 4) == 0.0
    a, b = 0.7, -1.3  # p = a xi + b eta: beta = |Delta0| |grad p|^2 = a^2 + b^2 in the (xi, eta) frame
    assert abs(o.beta(c, np.array([a, b]), 1) - (a * a + b * b)) < 1e-13
    # quadratic: brute force of Eq. smoothnessIndicator in physical coordinates
    cq = np.array([0.3, -0.2, 0.5, 0.1, -0.4])
    T = pb.mesh.xy[pb.mesh.tri[c]]
    Pq, w = tri_quad(T)
    xi, eta = (Pq[:, 0] - fr["x0"]) / fr["h0"], (Pq[:, 1] - fr["y0"]) / fr["h0"]
    h0, A = fr["h0"], fr["area"]
    px = (cq[0] + 2 * cq[2] * xi + cq[3] * eta) / h0
    py = (cq[1] + cq[3] * xi + 2 * cq[4] * eta) / h0
    pxx, pxy, pyy = 2 * cq[2] / h0 ** 2, cq[3] / h0 ** 2, 2 * cq[4] / h0 ** 2
    ref = np.sum(w * (px ** 2 + py ** 2)) + A * np.sum(w * (pxx ** 2 + pxy ** 2 + pyy ** 2))
    assert abs(o.beta(c, cq, 2) - ref) < 1e-12 * ref


@pytest.mark.parametrize("k", [1, 2])
def test_limiter_keeps_cell_means(k):
    pb = W.double_mach(10, 3, seed=20)
    o = oracle.Oracle(pb, k=k, limiter=2)
    u = W.random_modes(pb.mesh, 4, o.np, 21)
    ul, fl, st = o.limit(u)
    assert st == 0 and fl.all()
    assert np.array_equal(ul[:, :, 0], u[:, :, 0])


# ----------------------------------------------------------------------------
# convergence (Tables 1-3: order about k+1 on smooth data)
# ----------------------------------------------------------------------------
def _burgers_errors(k, limiter, ns, T=0.05):
    errs = []
    for n in ns:
        pb = W.burgers_sine(n, seed=1)
        o = oracle.Oracle(pb, k=k, limiter=limiter)
        u = o.project(pb.u0)
        u, _, t = o.run(u, 0.0, T, 0.1)
        assert t == T
        errs.append(o.l1_error(u, burgers_sine_exact, T)[0])
    return np.array(errs)


def test_convergence_p1_unlimited_and_all_cells_limited():
    """Measured orders on the last pair: 1.95 unlimited (8/16/32) and 1.85 with
    every cell limited (32/64; coarser meshes are pre-asymptotic: the weights
    see the 16-cell-per-period wave as non-smooth)."""
    e = _burgers_errors(1, 0, [8, 16, 32])
    assert np.log2(e[-2] / e[-1]) > 1.75, e
    e = _burgers_errors(1, 2, [32, 64])
    assert np.log2(e[-2] / e[-1]) > 1.75, e


def test_convergence_p2_unlimited():
    e = _burgers_errors(2, 0, [8, 16, 32])
    assert np.log2(e[-2] / e[-1]) > 2.6, e


def test_convergence_p2_all_cells_limited():
    """With every cell limited the P2 scheme converges at order 3 once the
    mesh resolves the wave (Table 1 reports 2.9): measured 3.12 on 32/64 (the
    errors on 16/32 fall by 60x as the nonlinear weights stop treating the
    wave as non-smooth)."""
    e = _burgers_errors(2, 2, [32, 64])
    assert np.log2(e[-2] / e[-1]) > 2.8, e


def test_oracle_central_differences_are_a_usable_adjoint_reference():
    """The GPU adjoint tests compare with central differences of the oracle.
    Pin that reference: on the states those tests use, the operator and a
    KXRCF + CSWENO pass are smooth enough that eps = 1e-5 and 1e-6 give the same
    directional derivative (operator: 1e-6 relative; limiter pass, flags
    unchanged: 5e-6, below the 1e-5 the GPU limiter-adjoint tests use), and the
    directional derivative of the operator is linear in the direction."""
    pb = W.riemann_quadrants(9, seed=14)
    nc = pb.mesh.nc
    area = np.sqrt(W.cell_areas(pb.mesh))[:, None, None]
    u = W.random_modes(pb.mesh, 4, 6, 302)
    lam = (W.uniform01(811, np.arange(nc * 24)).reshape(nc, 4, 6) * 2 - 1) * area
    d1 = (W.uniform01(821, np.arange(nc * 24)).reshape(nc, 4, 6) * 2 - 1) * 0.3 * area
    d2 = (W.uniform01(831, np.arange(nc * 24)).reshape(nc, 4, 6) * 2 - 1) * 0.3 * area
    o = oracle.Oracle(pb, k=2, limiter=1)

    def fd(f, d, eps):
        return (np.sum(lam * f(u + eps * d)) - np.sum(lam * f(u - eps * d))) / (2 * eps)

    L = lambda v: o.rhs(v, 0.017)
    a, b = fd(L, d1, 1e-5), fd(L, d1, 1e-6)
    assert abs(a - b) < 1e-6 * abs(b)
    assert abs(fd(L, d1 + d2, 1e-6) - (b + fd(L, d2, 1e-6))) < 1e-6 * abs(b)
    f0 = o.limit(u, 0.0)[1]
    Lim = lambda v: o.limit(v, 0.0)[0]
    assert np.array_equal(o.limit(u + 1e-5 * d1, 0.0)[1], f0) and np.array_equal(o.limit(u - 1e-5 * d1, 0.0)[1], f0)
    a, b = fd(Lim, d1, 1e-5), fd(Lim, d1, 1e-6)
    assert abs(a - b) < 5e-6 * abs(b)


def _entropy_wave_exact(x, y, t, gam=1.4):
    """Sec. 4.1 Example 2 in closed form: the density profile advected by the
    constant velocity (0.7, 0.3) at constant pressure 1 (conserved variables)."""
    rho = 1.0 + 0.2 * np.sin(np.pi * (x + y - (0.7 + 0.3) * t))
    u, v, p = 0.7, 0.3, 1.0
    return np.stack([rho, rho * u, rho * v, p / (gam - 1.0) + 0.5 * rho * (u * u + v * v)], axis=1)


def _entropy_wave_errors(k, limiter, ns, T=0.05):
    errs = []
    for n in ns:
        pb = W.euler_entropy_wave(n, seed=12)
        o = oracle.Oracle(pb, k=k, limiter=limiter)
        u = o.project(pb.u0)
        u, _, t = o.run(u, 0.0, T, 0.1)
        assert t == T
        errs.append(o.l1_error(u, _entropy_wave_exact, T)[0])
    return np.array(errs)


@pytest.mark.parametrize("k,limiter,order,ns", [(1, 0, 1.75, [8, 16, 32]), (2, 0, 2.6, [8, 16, 32]),
                                                 (2, 1, 2.6, [8, 16, 32]), (1, 2, 1.75, [32, 64])])
def test_convergence_euler_entropy_wave(k, limiter, order, ns):
    """The Euler operator (flux, LLF, SSP-RK3) converges at about k+1 on the
    smooth entropy wave against its closed form; with KXRCF the smooth wave is
    not limited, so the order holds too, and with every cell limited (the
    characteristic-field reconstruction in x and y on every cell, every stage)
    P1 keeps its order (Table 2 reports orders near 2 and 3).  Measured at
    t = 0.05: 1.95 (P1) and 2.80 (P2) on 8/16/32, 1.91 for P1 with every cell
    limited on 32/64."""
    e = _entropy_wave_errors(k, limiter, ns)
    assert np.log2(e[-2] / e[-1]) > order, e


def test_dmr_boundaries_follow_the_exact_shock_position():
    """Sec. 4.2 Example 5 boundaries (reading R-bc) against the closed form of
    the shock position: with the post-shock state everywhere, the operator
    vanishes in every cell whose ghosts equal that state (left and bottom
    x < 1/6 inflow, top boundary left of the Mach-10 front at
    x_s(t) = 1/6 + (1 + 20 t)/sqrt(3)) and not in the cells on the top boundary
    right of the front nor on the right side (pre-shock ghosts) nor on the
    reflecting wall (the post-shock flow crosses it)."""
    pb = W.double_mach(48, 12, seed=3)
    m = pb.mesh
    post = np.array(pb.boundaries[1][1], dtype=float)
    o = oracle.Oracle(pb, k=1, limiter=0)
    u = o.project(lambda x, y: np.tile(post, (len(x), 1)))
    t = 0.05
    r = np.abs(o.rhs(u, t)).reshape(m.nc, -1).max(axis=1)
    xs = 1.0 / 6.0 + (1.0 + 20.0 * t) / np.sqrt(3.0)
    cell_of = {}
    for c, tri in enumerate(m.tri):
        for a, b in ((tri[0], tri[1]), (tri[1], tri[2]), (tri[2], tri[0])):
            cell_of[(min(a, b), max(a, b))] = c
    expect = np.zeros(m.nc, dtype=int)  # 0 zero residual, 1 nonzero, -1 not classified
    h = 4.0 / 48
    for v0, v1, tag in m.bface:
        c = cell_of[(min(v0, v1), max(v0, v1))]
        xa, xb = sorted((m.xy[v0, 0], m.xy[v1, 0]))
        if tag == 2 or tag == 3:
            kind = 1
        elif tag == 4:
            kind = 0 if xb < xs - 0.1 * h else (1 if xa > xs + 0.1 * h else -1)
        else:
            kind = 0
        if kind == -1 or expect[c] == -1:
            expect[c] = -1
        else:
            expect[c] = max(expect[c], kind)
    big = r.max()
    assert (expect == 1).sum() > 20 and (expect == 0).sum() > m.nc // 2
    assert np.all(r[expect == 0] < 1e-10 * big), r[expect == 0].max() / big
    assert np.all(r[expect == 1] > 1e-3 * big), r[expect == 1].min() / big


@pytest.mark.parametrize("k,order", [(1, 1.8), (2, 2.7)])
def test_euler_operator_on_the_moving_vortex(k, order):
    """Sec. 4.1 Example 3: the isentropic vortex is carried unchanged at unit
    speed in x, so the exact time derivative is -d/dx of the initial data.  The
    operator applied to the projected vortex approaches the projection of that
    derivative (central difference of the closed form, step 1e-5) as the mesh
    is refined: a wrong flux, pressure or sign gives an O(1) mismatch.  Measured
    (mean absolute modal difference on 10/20/40 meshes): orders 2.07 (P1) and
    3.13 (P2) on the last pair."""
    errs = []
    for n in (10, 20, 40):
        pb = W.isentropic_vortex(n, seed=5, eps=5.0, centre=(5.0, 5.0), box=(0.0, 10.0, 0.0, 10.0))
        o = oracle.Oracle(pb, k=k, limiter=0)
        L = o.rhs(o.project(pb.u0), 0.0)
        h = 1e-5
        d = o.project(lambda x, y: -(pb.u0(x + h, y) - pb.u0(x - h, y)) / (2 * h))
        errs.append(np.abs(L - d).sum() / pb.mesh.nc)
    e = np.array(errs)
    assert np.log2(e[-2] / e[-1]) > order, e

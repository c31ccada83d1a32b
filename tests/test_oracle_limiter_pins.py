"""Pins of the oracle's CSWENO weights and of the limited scheme on a shock.

Sec. 3.2 Steps 2-4: the linear weights gamma_{l,m}, the magnified beta_1
(Eqs. sigmaEqn, smoothnessIndicatorT1), tau (Eqs. tauNonlinearWeightsP1/P2)
and the nonlinear weights (Eqs. nonLinearWeightsP1/P2), with the readings
R-sigma (the square of the mean absolute difference of the beta_{1,l}) and
R-weno (tau the mean absolute difference of the betas, the ratio raised to
the power k + 1).  The expected values are derived here from data whose
smoothness indicators follow in closed form (linear data are reproduced
exactly by every stencil fit, so each beta is |Delta_0| |grad|^2 times a
factor fixed by the linear weights), evaluated in exact rational arithmetic.

The scheme-level pins run the Burgers configuration past shock formation and
check what Sec. 3.2 asks of the limiter: cell means stay within the range of
the exact solution up to a small overshoot that does not grow as the mesh is
refined.
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
from paper_2106_06280_gb300 import workloads as W

EPS = Fr(1, 10 ** 10)


def _case(k, n=6, seed=16):
    pb = W.burgers_sine(n, seed=seed)
    return pb, oracle.Oracle(pb, k=k, limiter=2)


def _centroid(T):
    return T.mean(axis=0)


def _gammas(hbar, nslot):
    ih = Fr(1) / Fr(hbar)
    g = [ih ** l for l in range(nslot)]
    s = sum(g)
    return [x / s for x in g]


def _linear_data(o, c, G, per_face=None):
    """Subcell means of linear data on the stencil of cell c: the mean of a
    linear function over a triangle is its value at the centroid.  per_face
    gives each neighbour its own gradient (Eq. sigmaEqn pins)."""
    tri, gh = o.stencil(c)
    fr = o.frame(c)
    x0 = np.array([fr["x0"], fr["y0"]])
    th = np.zeros((3, 3))
    hf = np.zeros((3, 4))
    for f in range(3):
        g = G if per_face is None else per_face[f]
        for i in range(3):
            th[f, i] = 0.37 + g @ (_centroid(tri[f, i]) - x0)
        for i in range(4):
            hf[f, i] = 0.37 + g @ (_centroid(tri[f, 3 + i]) - x0)
    return th, hf


@pytest.mark.parametrize("k", [1, 2])
def test_beta1_sigma_closed_form(k):
    """Neighbour l carries the linear function with gradient s_l (1, 0),
    s = (1, 2, 3): each p_{1,l} reproduces it, so beta_{1,l} = |Delta_0| s_l^2,
    D = (|1-4| + |4-9| + |9-1|) |Delta_0| / 3 = 16 |Delta_0| / 3,
    sigma_l = (1/3)(1 + D^2 / (beta_{1,l} + eps)) and
    beta_1 = |Delta_0| (sum sigma_l s_l / sum sigma_l)^2."""
    pb, o = _case(k)
    for c in (4, 27):
        fr = o.frame(c)
        A = Fr(fr["area"])
        s = [1, 2, 3]
        th, hf = _linear_data(o, c, None, per_face=[np.array([float(v), 0.0]) for v in s])
        r = o.weno(c, 0.37, th, hf)
        b1l = [A * v * v for v in s]
        D = (abs(b1l[0] - b1l[1]) + abs(b1l[1] - b1l[2]) + abs(b1l[2] - b1l[0])) / 3
        assert D == 16 * A / 3
        sig = [Fr(1, 3) * (1 + D * D / (b + EPS)) for b in b1l]
        abar = sum(sg * v for sg, v in zip(sig, s)) / sum(sig)
        beta1 = A * abar * abar
        assert np.allclose(r["beta1l"], [float(b) for b in b1l], rtol=1e-10, atol=0)
        assert np.allclose(r["sigma"], [float(x) for x in sig], rtol=1e-10, atol=0)
        assert abs(r["beta"][0] - float(beta1)) < 1e-10 * float(beta1)


@pytest.mark.parametrize("k", [1, 2])
def test_tau_and_nonlinear_weights_closed_form(k):
    """Global linear data with gradient G: q_2 = q_3 (= q_4) = the data, so the
    hierarchical polynomials of Eqs. equivalentOrder1-4 are the data's linear
    part scaled by c_2 = 1/gamma_{2,2}, c_3 = (1 - gamma_{2,3} c_2)/gamma_{3,3}
    and (P2) c_4 = (1 - gamma_{2,5} c_2 - gamma_{3,5} c_3)/gamma_{4,5};
    beta_l = |Delta_0| |G|^2 c_l^2 and beta_1 = |Delta_0| |G|^2 (all three
    neighbours alike, sigma_l = 1/3).  tau is the mean absolute difference to
    the top slot's beta and omega_l is proportional to
    gamma_l (1 + (tau / (eps + beta_l))^(k+1))."""
    pb, o = _case(k)
    for c, G in ((9, np.array([0.6, -0.25])), (33, np.array([-1.5, 2.0]))):
        fr = o.frame(c)
        A, hb = Fr(fr["area"]), fr["hbar"]
        th, hf = _linear_data(o, c, G)
        r = o.weno(c, 0.37, th, hf)
        g2, g3, g5 = _gammas(hb, 2), _gammas(hb, 3), _gammas(hb, 4)
        c2 = 1 / g2[1]
        c3 = (1 - g3[1] * c2) / g3[2]
        G2 = Fr(float(G @ G))
        betas = [A * G2, A * G2 * c2 * c2, A * G2 * c3 * c3]
        gam = g3
        if k == 2:
            c4 = (1 - g5[1] * c2 - g5[2] * c3) / g5[3]
            betas.append(A * G2 * c4 * c4)
            gam = g5
        top = betas[-1]
        tau = sum(abs(top - b) for b in betas[:-1]) / (len(betas) - 1)
        wb = [gl * (1 + (tau / (EPS + b)) ** (k + 1)) for gl, b in zip(gam, betas)]
        om = [w / sum(wb) for w in wb]
        n = len(betas)
        assert np.allclose(r["gamma"][:n], [float(x) for x in gam], rtol=1e-14, atol=0)
        assert np.allclose(r["beta"][:n], [float(b) for b in betas], rtol=1e-9, atol=0)
        assert abs(r["tau"] - float(tau)) < 1e-8 * float(tau)
        assert np.allclose(r["omega"][:n], [float(x) for x in om], rtol=1e-8, atol=1e-15)


@pytest.mark.parametrize("k", [1, 2])
def test_constant_data_keep_the_linear_weights(k):
    """Constant data: every beta and tau vanish, eps keeps each ratio
    tau / (eps + beta_l) defined (= 0), so omega = gamma exactly and the
    reconstruction returns the constant (all modes above the mean zero)."""
    pb, o = _case(k)
    for c in (2, 30):
        th, hf = _linear_data(o, c, np.zeros(2))
        r = o.weno(c, 0.37, th, hf)
        n = 3 if k == 1 else 4
        assert np.all(r["beta"][:n] == 0.0) and r["tau"] == 0.0
        assert np.array_equal(r["omega"][:n], r["gamma"][:n])
        assert np.abs(r["modes"][1:]).max() < 1e-15


@pytest.mark.parametrize("k", [1, 2])
def test_eno_jump_outside_the_lower_stencils(k):
    """Smooth (linear) data with a unit jump confined to the stencil cells the
    top polynomial adds (P1: the outer thirds of one neighbour, T3 minus T2;
    P2: the outer halves of one neighbour, T4 minus T3).  The top stencil is
    then non-smooth and the lower ones smooth, and Step 4 states that the
    reconstruction falls back to O(h^{k+1}): its weight must vanish at that
    rate.  Measured on meshes of 16 and 64 squares per side, omega_top falls
    at least as fast as h^{k+1}, stays below 1e-3 on the finer mesh, and the
    reconstructed modes stay within O(h^2) of the smooth data's modes."""
    G = np.array([0.4, -0.3])
    tops = []
    for n in (16, 64):
        pb = W.burgers_sine(n, seed=16)
        o = oracle.Oracle(pb, k=k, limiter=2)
        c = pb.mesh.nc // 2 + 3
        th, hf = _linear_data(o, c, G)
        smooth = o.weno(c, 0.37, th, hf)
        if k == 1:
            th[1, 1:] += 1.0
        else:
            hf[1, [1, 3]] += 1.0  # Delta_{i21}, Delta_{i31}: in T4 only
        r = o.weno(c, 0.37, th, hf)
        nslot = 3 if k == 1 else 4
        tops.append((o.frame(c)["hbar"], r["omega"][nslot - 1], r, smooth))
    (h0, w0, _, _), (h1, w1, r1, s1) = tops
    assert w1 < 1e-3, tops
    assert w1 / w0 < 1.2 * (h1 / h0) ** (k + 1), (w0, w1)
    err = np.abs(r1["modes"][1:] - s1["modes"][1:]).max()
    assert err < 10 * h1 ** 2 * np.linalg.norm(G), err


def _shock_run(n, k):
    pb = W.burgers_sine(n, seed=2)
    o = oracle.Oracle(pb, k=k, limiter=1)
    u = o.project(pb.u0)
    area = W.cell_areas(pb.mesh)
    t, hi, lo = 0.0, 0.0, 1.0
    while t < 1.0:
        dt = min(o.cfl_dt(u, 0.1), 1.0 - t)
        u, fl, st = o.step(u, t, dt)
        assert st == 0
        t += dt
        m = u[:, 0, 0] / np.sqrt(area)
        hi, lo = max(hi, m.max()), min(lo, m.min())
    return hi - 0.75, 0.25 - lo


@pytest.mark.parametrize("k,bound", [(1, 0.025), (2, 0.002)])
def test_burgers_shock_stays_in_range_under_refinement(k, bound):
    """The Burgers configuration (u0 = 0.5 + 0.25 sin(pi (x + y)) on the
    periodic [0,2]^2, KXRCF C_K = 1, CFL 0.1) run through shock formation
    (t = 2/pi) to t = 1.0 on 20x20 and 40x40 meshes: the exact solution stays
    in [0.25, 0.75].  Measured largest cell-mean excursions beyond that range:
    P2 7e-4 (20x20) and 2e-5 (40x40); P1 1.6e-2 and 1.3e-2.  The excursion is
    bounded and does not grow from 20x20 to 40x40."""
    ex = [max(_shock_run(n, k)) for n in (20, 40)]
    assert max(ex) < bound, ex
    assert ex[1] < ex[0] + 0.1 * bound, ex


def test_positivity_trigger_and_fallback():
    """Reading R-pos.  (a) A uniform gas at rest with one cell given a density
    slope that makes its polynomial negative at some points: no face is an
    inflow face, so R = 0, yet the cell is troubled because its polynomial is
    non-physical at a quadrature point; its neighbours are uniform, so the
    reconstruction returns the mean alone.  (b) A low-density cell between a
    near-vacuum neighbour and dense ones: the limited polynomial keeps the
    mean and is physical at every volume point (evaluated independently here
    from the modes and the basis' closed form at the points)."""
    pb = W.euler_entropy_wave(4, seed=12)
    o = oracle.Oracle(pb, k=2, limiter=1)
    area = W.cell_areas(pb.mesh)
    base = W.prim_to_cons(np.array([1.0]), 0.0, 0.0, 1.0)[0]
    u = np.zeros((pb.mesh.nc, 4, 6))
    u[:, :, 0] = base[None, :] * np.sqrt(area)[:, None]
    c = 5
    u1 = u.copy()
    u1[c, 0, 1] = 2.0 * u1[c, 0, 0]  # a first-mode coefficient twice the mean's: negative near one edge
    xy = o.volume_points()[c]
    rho_pts = o.eval_points(u1, np.full(len(xy), c, dtype=np.int32), xy)[:, 0]
    fl, R = o.detect(u1)
    assert R[c] == 0.0 and fl[c] == 1 and fl.sum() == 1
    out, st = o.limit_cell(u1, c)
    assert st == 0 and out[0, 0] == u1[c, 0, 0]
    assert np.abs(out[:, 1:]).max() < 1e-14 * np.abs(out[:, 0]).max()
    nb = o.connectivity()[0]
    for scale in (1e-3, 1e-2, 0.1):
        u2 = u.copy()
        for j, d in enumerate(nb[c]):
            u2[d, :, 0] = W.prim_to_cons(np.array([[scale, 1.0, 3.0][j]]), 0.0, 0.0, scale)[0] * np.sqrt(area[d])
        u2[c, :, 0] = W.prim_to_cons(np.array([0.02]), 0.0, 0.0, scale)[0] * np.sqrt(area[c])
        u2[c, 0, 1:] = 0.5 * u2[c, 0, 0]
        assert o.detect(u2)[0][c] == 1
        out2, st = o.limit_cell(u2, c)
        assert st == 0 and np.array_equal(out2[:, 0], u2[c, :, 0])
        v = u2.copy()
        v[c] = out2
        U = o.eval_points(v, np.full(len(xy), c, dtype=np.int32), xy)
        p = (W.GAMMA - 1.0) * (U[:, 3] - 0.5 * (U[:, 1] ** 2 + U[:, 2] ** 2) / U[:, 0])
        assert U[:, 0].min() > 0.0 and p.min() > 0.0, scale
    assert rho_pts.min() < 0.0  # case (a) really starts non-physical at a volume point


def test_euler_characteristic_fields_isolate_the_entropy_wave():
    """Sec. 3.2, last paragraph (reading R-char), field isolation:
    entropy-wave data (only the density varies; u = 0.7, v = 0.3, p = 1) lie
    along the entropy eigenvector (1, u, v, |v|^2/2), which is the same for the
    x and y directions, so in both characteristic decompositions one field
    carries the density variation and the other three are constant.  The
    limited cell must keep its velocity and pressure (momentum and energy modes
    = u, v and |v|^2/2 times the density modes) and its density modes must be
    the scalar reconstruction of the density's own subcell means."""
    pb = W.euler_entropy_wave(6, seed=12)
    o = oracle.Oracle(pb, k=2, limiter=2)
    u = o.project(pb.u0)
    area = W.cell_areas(pb.mesh)
    for c in (3, 17, 40):
        out, st = o.limit_cell(u, c)
        assert st == 0
        d = out[0, 1:]
        scale = np.abs(d).max()
        assert scale > 1e-4
        assert np.abs(out[1, 1:] - 0.7 * d).max() < 1e-12 * scale
        assert np.abs(out[2, 1:] - 0.3 * d).max() < 1e-12 * scale
        assert np.abs(out[3, 1:] - 0.5 * (0.7 ** 2 + 0.3 ** 2) * d).max() < 1e-12 * scale
        sm = o.subcell_means(u, c)
        w = o.weno(c, u[c, 0, 0] / np.sqrt(area[c]), sm[:, :3, 0], sm[:, 3:7, 0])
        assert np.abs(d - w["modes"][1:]).max() < 1e-11 * scale


@pytest.mark.parametrize("k", [1, 2])
def test_euler_characteristic_reconstruction_identities(k):
    """Sec. 3.2, last paragraph (reading R-char): with the linear weights the reconstruction is
    linear in the data, so transforming by L_d, reconstructing each field and
    mapping back by R_d (then averaging x and y) must equal reconstructing each
    conserved variable on its own, for any data (the eigenvector pair must be
    inverse to each other for this to hold), and must return the data's own
    modes for data that are one polynomial of degree <= k across the stencil
    (cells whose three neighbours are interior)."""
    pb = _transmissive_box_euler(7)
    o = oracle.Oracle(pb, k=k, limiter=2)
    area = W.cell_areas(pb.mesh)
    np_ = (k + 1) * (k + 2) // 2
    rng = np.random.default_rng(31 + k)
    base = W.prim_to_cons(np.array([1.2]), 0.2, -0.1, 1.5)[0]
    u = W.random_modes(pb.mesh, 4, np_, 33 + k, scale=0.02)
    u[:, :, 0] += base[None, :] * np.sqrt(area)[:, None]
    nb = o.connectivity()[0]
    inner = [c for c in range(pb.mesh.nc) if np.all(nb[c] >= 0)][:6]
    for c in inner:
        out, st = o.limit_cell_linear(u, c)
        sm = o.subcell_means(u, c)
        for v in range(4):
            w = o.weno(c, u[c, v, 0] / np.sqrt(area[c]), sm[:, :3, v], sm[:, 3:7, v] if k == 2 else None,
                       force_linear=True)
            assert np.abs(out[v, 1:] - w["modes"][1:]).max() < 1e-12 * np.abs(u[c]).max(), (c, v)
    coef = rng.normal(size=(4, (k + 1) * (k + 2) // 2 - 1)) * 0.1
    exps = [(d - e, e) for d in range(1, k + 1) for e in range(d + 1)]

    def poly(x, y):
        cols = [base[v] + sum(cf * x ** a * y ** b for cf, (a, b) in zip(coef[v], exps)) for v in range(4)]
        return np.stack(cols, axis=1)

    up = o.project(poly)
    for c in inner:
        out, st = o.limit_cell_linear(up, c)
        assert st == 0
        assert np.abs(out - up[c]).max() < 1e-11 * np.abs(up[c]).max(), c


def _transmissive_box_euler(n):
    mesh = W.split_square_mesh(n, n, 0.0, 1.0, 0.0, 1.0, 5, tag_fn=lambda side, xm, ym: 2)
    return W.Problem("box", 1, mesh, None, {2: (W.TRANSMISSIVE, [])})

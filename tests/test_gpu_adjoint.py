"""GPU adjoint (operator, limiter pass with frozen flags, checkpointed
SSP-RK3 steps, the torch.autograd bridge) against the FP64 oracle.

The reference is the oracle's central finite difference of lambda . L_h(u)
along 32 seeded directions d (the oracle itself has no adjoint): the GPU's
(dL_h/du)^T lambda dotted with each d must match it.  With eps = 1e-6 on states and
directions of order one, the central difference agrees with eps = 1e-5 to
2e-8 relative on these meshes (the double Mach states of order 100 bring the
rounding of the difference to about 1e-7 absolute against dot products of
order 10), so FP64 is held to 1e-6 relative; FP32 to 2e-4 relative to the
FP64 adjoint (float operator arithmetic, see test_gpu_fp32).
The meshes carry periodic, Dirichlet, wall, transmissive and moving
shock-line boundaries.
"""
import numpy as np
import pytest

import oracle
from paper_2106_06280_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def problems():
    return {
        "burgers": W.burgers_sine(9, seed=11),
        "entropy": W.euler_entropy_wave(7, seed=12),
        "dmr": W.double_mach(26, 7, seed=13),
        "riemann": W.riemann_quadrants(9, seed=14),
    }


NDIR = 32  # seeded directions per gradient check


def fd_tol(rel, fd, terms, eps):
    """rel |fd| plus the rounding noise of a central difference of an objective
    whose terms have the absolute values terms: each of the two evaluations
    carries about machine epsilon times their sum, divided by 2 eps (a factor
    10 of margin); it matters where the directional derivative is small
    against the objective."""
    return rel * abs(fd) + 10 * np.finfo(float).eps * float(np.sum(np.abs(terms))) / eps


def seeded(pb, k, seed, scale):
    np_ = (k + 1) * (k + 2) // 2
    r = W.uniform01(seed, np.arange(pb.mesh.nc * pb.nvar * np_)).reshape(pb.mesh.nc, pb.nvar, np_) * 2.0 - 1.0
    return scale * r * np.sqrt(W.cell_areas(pb.mesh))[:, None, None]


def fd_dot(o, u, lam, d, t, eps=1e-6):
    return (np.sum(lam * o.rhs(u + eps * d, t)) - np.sum(lam * o.rhs(u - eps * d, t))) / (2 * eps)


@pytest.mark.parametrize("name,k", [("burgers", 1), ("burgers", 2), ("entropy", 2), ("dmr", 1), ("dmr", 2), ("riemann", 2)])
def test_rhs_adjoint_fp64_vs_oracle_fd(csw, cuda_stream, name, k):
    pb = problems()[name]
    s = csw.Solver(pb.equation, k, csw.FP64, csw.LIMITER_OFF, stream=cuda_stream)
    s.setup(pb)
    o = oracle.Oracle(pb, k=k, limiter=0)
    u = W.random_modes(pb.mesh, pb.nvar, (k + 1) * (k + 2) // 2, 700 + k)
    lam = seeded(pb, k, 710 + k, 1.0)
    t = 0.017
    g = s.rhs_adjoint(u, lam, t)
    terms = lam * o.rhs(u, t)
    for j in range(NDIR):
        d = seeded(pb, k, 7200 + 100 * k + j, 0.3)
        fd = fd_dot(o, u, lam, d, t)
        ad = float(np.sum(g * d))
        assert abs(ad - fd) < fd_tol(1e-6, fd, terms, 1e-6), (name, k, j, ad, fd)


def test_rhs_adjoint_fp32_vs_fp64(csw, cuda_stream):
    pb = problems()["dmr"]
    u = W.random_modes(pb.mesh, 4, 6, 731)
    lam = seeded(pb, 2, 732, 1.0)
    out = []
    for prec in (csw.FP64, csw.FP32_BULK):
        s = csw.Solver(1, 2, prec, csw.LIMITER_OFF, stream=cuda_stream)
        s.setup(pb)
        out.append(s.rhs_adjoint(u, lam, 0.01))
        s.close()
    assert np.abs(out[1] - out[0]).max() < 2e-4 * np.abs(out[0]).max()


def vortex(n, seed=5):
    return W.isentropic_vortex(n, seed=seed, box=(0.0, 10.0, 0.0, 10.0))


def oracle_run(o, u, t0, dt, nsteps):
    t = t0
    for _ in range(nsteps):
        u, _, st = o.step(u, t, dt)
        assert st == 0
        t += dt
    return u


@pytest.mark.parametrize("limiter", [0, 1])
def test_adjoint_steps_fp64_vs_oracle_fd(csw, cuda_stream, limiter):
    """7 fixed-dt steps on a 128-cell periodic vortex (checkpoints every 3 steps:
    a partial last segment): forward state against the oracle, gradient
    against the oracle's central difference along 3 seeded directions.  With
    the KXRCF limiter the smooth vortex flags no cell, so the limited and
    unlimited runs have the same adjoint."""
    pb = vortex(8)
    s = csw.Solver(1, 2, csw.FP64, limiter, stream=cuda_stream)
    s.setup(pb)
    o = oracle.Oracle(pb, k=2, limiter=limiter)
    u0 = o.project(pb.u0)
    dt, nsteps = 0.5 * o.cfl_dt(u0, 0.1), 7
    gT = seeded(pb, 2, 741, 1.0)
    s.set_time(0.0)
    uT, g0 = s.adjoint_steps(u0, gT, dt, nsteps, 3)
    uo = oracle_run(o, u0, 0.0, dt, nsteps)
    assert np.abs(uT - uo).max() < 1e-11 * np.abs(uo).max()
    assert abs(s.get_time() - nsteps * dt) < 1e-13
    for j in range(NDIR):
        d = seeded(pb, 2, 7500 + j, 0.1)
        eps = 1e-6
        fd = (np.sum(gT * oracle_run(o, u0 + eps * d, 0.0, dt, nsteps)) -
              np.sum(gT * oracle_run(o, u0 - eps * d, 0.0, dt, nsteps))) / (2 * eps)
        ad = float(np.sum(g0 * d))
        assert abs(ad - fd) < fd_tol(1e-6, fd, gT * uo, eps), (j, ad, fd)


@pytest.mark.parametrize("name,k", [("burgers", 1), ("burgers", 2), ("entropy", 2), ("dmr", 1), ("dmr", 2), ("riemann", 2)])
def test_limit_adjoint_fp64_vs_oracle_fd(csw, cuda_stream, name, k):
    """One KXRCF + CSWENO pass with the flags frozen: (dLim/du)^T lambda dotted
    with d against the oracle's central difference, along the directions
    whose flags at u +- eps d are those at u (at least 28 of 32).  The random
    states flag most cells, with smoothness indicators of order one
    (near-constant data, where beta ~ 0 and the weights turn stiff at the
    1e-10 epsilon, is left to the step test's smooth vortex).
    Held to 1e-5 relative: the central difference agrees between eps = 1e-6
    and 1e-7 to better than 3e-6 relative on these states."""
    pb = problems()[name]
    np_ = (k + 1) * (k + 2) // 2
    s = csw.Solver(pb.equation, k, csw.FP64, csw.LIMITER_KXRCF, stream=cuda_stream)
    s.setup(pb)
    o = oracle.Oracle(pb, k=k, limiter=1)
    u = W.random_modes(pb.mesh, pb.nvar, np_, 300 + k)
    lam = seeded(pb, k, 810 + k, 1.0)
    g, fl = s.limit_adjoint(u, lam, 0.0)
    ul0, f0, _ = o.limit(u, 0.0)
    assert np.array_equal(fl, f0) and 0 < f0.sum() < len(f0)
    checked = 0
    for j in range(NDIR):
        d = seeded(pb, k, 8200 + 100 * k + j, 0.3)
        eps = 1e-6
        up, fp, _ = o.limit(u + eps * d, 0.0)
        um, fm, _ = o.limit(u - eps * d, 0.0)
        if not (np.array_equal(fp, f0) and np.array_equal(fm, f0)):
            continue  # a flag flips within eps: the frozen-flag derivative does not apply
        fd = (np.sum(lam * up) - np.sum(lam * um)) / (2 * eps)
        ad = float(np.sum(g * d))
        assert abs(ad - fd) < fd_tol(1e-5, fd, lam * ul0, eps), (name, k, j, ad, fd)
        checked += 1
    assert checked >= NDIR - 4


@pytest.mark.parametrize("name,k,scale", [("riemann", 2, 0.3), ("burgers", 2, 0.3), ("dmr", 2, 0.05), ("entropy", 1, 0.3)])
def test_adjoint_steps_limited_fp64_vs_oracle_fd(csw, cuda_stream, name, k, scale):
    """2 fixed-dt steps with KXRCF + CSWENO after every stage (about 300-700
    reconstructions), checkpoint every step: the adjoint through the operator
    and the reconstructions (flags frozen) against the oracle's central
    difference, 1e-5 relative (the difference is stable to 3e-6 relative
    between eps = 1e-6 and 1e-7 here), along the directions where it is stable
    to 1e-3 between those two steps (a flag flip within eps makes it jump; at
    least 28 of 32)."""
    pb = problems()[name]
    np_ = (k + 1) * (k + 2) // 2
    s = csw.Solver(pb.equation, k, csw.FP64, csw.LIMITER_KXRCF, stream=cuda_stream)
    s.setup(pb)
    o = oracle.Oracle(pb, k=k, limiter=1)
    u0 = W.random_modes(pb.mesh, pb.nvar, np_, 900 + k, scale=scale)
    dt, nsteps = 0.5 * o.cfl_dt(u0, 0.1), 2
    gT = seeded(pb, k, 841, 1.0)
    s.set_time(0.0)
    uT, g0 = s.adjoint_steps(u0, gT, dt, nsteps, 1)
    uo = oracle_run(o, u0, 0.0, dt, nsteps)
    assert np.abs(uT - uo).max() < 1e-10 * np.abs(uo).max()
    checked = 0
    for j in range(NDIR):
        d = seeded(pb, k, 8510 + j, 0.1)
        fds = [(np.sum(gT * oracle_run(o, u0 + eps * d, 0.0, dt, nsteps)) -
                np.sum(gT * oracle_run(o, u0 - eps * d, 0.0, dt, nsteps))) / (2 * eps) for eps in (1e-6, 1e-7)]
        if abs(fds[0] - fds[1]) > fd_tol(1e-3, fds[0], gT * uo, 1e-7):
            continue  # a troubled-cell flag flips within eps: the difference jumps
        ad = float(np.sum(g0 * d))
        assert abs(ad - fds[0]) < fd_tol(1e-5, fds[0], gT * uo, 1e-6), (j, ad, fds[0])
        checked += 1
    assert checked >= NDIR - 4


def test_adjoint_steps_cfl_schedule_fp64_vs_oracle_fd(csw, cuda_stream):
    """6 CFL-rule steps (CFL 0.1) on the 128-cell vortex with KXRCF, checkpoint
    every 4 steps: the step sizes the forward sweep chose against the oracle's
    own CFL rule along its run, the final state against the oracle, and the
    gradient (step sizes frozen) against the oracle's central difference with
    its schedule held fixed, along 32 seeded directions."""
    pb = vortex(8)
    s = csw.Solver(1, 2, csw.FP64, csw.LIMITER_KXRCF, cfl=0.1, stream=cuda_stream)
    s.setup(pb)
    o = oracle.Oracle(pb, k=2, limiter=1)
    u0 = o.project(pb.u0)
    nsteps = 6
    gT = seeded(pb, 2, 861, 1.0)
    s.set_time(0.0)
    uT, g0, dts = s.adjoint_steps(u0, gT, 0.0, nsteps, 4, return_dts=True)
    u, t, sched = u0, 0.0, []
    for _ in range(nsteps):
        dt = o.cfl_dt(u, 0.1)
        sched.append(dt)
        u, _, st = o.step(u, t, dt)
        assert st == 0
        t += dt
    assert np.abs(dts - np.array(sched)).max() < 1e-13 * max(sched)
    assert np.abs(uT - u).max() < 1e-11 * np.abs(u).max()
    assert abs(s.get_time() - t) < 1e-13

    def run_fixed(v):
        tt = 0.0
        for dt in sched:
            v, _, st = o.step(v, tt, dt)
            assert st == 0
            tt += dt
        return v

    for j in range(NDIR):
        d = seeded(pb, 2, 8700 + j, 0.1)
        eps = 1e-6
        fd = (np.sum(gT * run_fixed(u0 + eps * d)) - np.sum(gT * run_fixed(u0 - eps * d))) / (2 * eps)
        ad = float(np.sum(g0 * d))
        assert abs(ad - fd) < fd_tol(1e-6, fd, gT * u, eps), (j, ad, fd)


def test_autograd_vortex_box_energy_fp32(csw, cuda_stream):
    """J = integral of rho^2 over the cells in [6,8]x[4,6] after 40 steps on a
    1,152-cell vortex, FP32-bulk forward and adjoint through torch.autograd,
    against the central difference of the FP64 GPU forward run (which matches
    the oracle to 1e-11) along the gradient direction and 3 seeded ones."""
    import torch
    from paper_2106_06280_gb300.autograd import RKDGSteps, box_density_energy

    pb = vortex(24)
    o = oracle.Oracle(pb, k=2, limiter=0)
    u0 = o.project(pb.u0)
    dt, nsteps = 0.5 * o.cfl_dt(u0, 0.1), 40
    cent = pb.mesh.xy[pb.mesh.tri].mean(axis=1)
    box = (6.0, 8.0, 4.0, 6.0)
    s32 = csw.Solver(1, 2, csw.FP32_BULK, csw.LIMITER_KXRCF, stream=cuda_stream)
    s32.setup(pb)
    s32.set_time(0.0)
    x = torch.tensor(u0, requires_grad=True)
    J = box_density_energy(RKDGSteps.apply(x, s32, dt, nsteps, 8), cent, box)
    J.backward()
    g = x.grad.numpy()
    s64 = csw.Solver(1, 2, csw.FP64, csw.LIMITER_OFF, stream=cuda_stream)
    s64.setup(pb)

    def J64(u):
        s64.write_modes(u)
        s64.set_time(0.0)
        s64.step(dt, nsteps, 1e300)
        return float(box_density_energy(torch.from_numpy(s64.read_modes()), cent, box))

    dirs = [g / np.abs(g).max()] + [seeded(pb, 2, 760 + j, 0.1) for j in range(3)]
    for j, d in enumerate(dirs):
        eps = 1e-5
        fd = (J64(u0 + eps * d) - J64(u0 - eps * d)) / (2 * eps)
        ad = float(np.sum(g * d))
        assert abs(ad - fd) < 1e-4 * max(abs(fd), 1e-3 * float(np.sum(np.abs(g * d)))), (j, ad, fd)

"""Pins of the radiation-diffusion oracle (Sec. 4.3) against facts that do not come from
the oracle itself.

- The SDIRK3 tableau satisfies the order conditions up to order 3. Its diagonal matches
  Alexander's published value, and its stability function is L-stable.
- A spatially uniform state reduces each stage to two scalar equations. Their root, found
  by a library root finder, must be the oracle's stage solution.
- With no sources and reflecting walls, total energy int(rho e + E) is exactly conserved
  through every stage. A sign error or a dropped term in one of the coupling terms, the
  divergence or the time derivative breaks this.
- On a manufactured solution the discrete solution converges at the rate of the L2 space.
- The emission Jacobian matches finite differences of the emission term, and the Newton
  solve converges quadratically.
"""
import numpy as np
import pytest
from scipy.optimize import brentq

import synth
from oracle.raddiff import RadDiff, sdirk3
from synth import raddiff as mms

# Alexander (1977), "Diagonally implicit Runge-Kutta methods for stiff O.D.E.'s", SIAM J.
# Numer. Anal. 14: the three-stage, L-stable, stiffly accurate method of order 3 has
# diagonal gamma = 0.43586652150845899942 (to 20 digits).
GAMMA_ALEXANDER = 0.43586652150845899942


def test_sdirk3_order_conditions_and_published_diagonal():
    A, b, c = sdirk3()
    assert abs(A[0, 0] - GAMMA_ALEXANDER) < 1e-15
    assert np.allclose(np.diag(A), A[0, 0], rtol=0, atol=0)
    assert np.allclose(np.triu(A, 1), 0.0, atol=0)
    assert np.allclose(A.sum(axis=1), c, atol=1e-15)
    assert np.array_equal(b, A[2])                       # stiffly accurate
    one = np.ones(3)
    assert abs(b @ one - 1.0) < 1e-15                     # order 1
    assert abs(b @ c - 0.5) < 1e-15                       # order 2
    assert abs(b @ (c * c) - 1.0 / 3.0) < 1e-15           # order 3
    assert abs(b @ (A @ c) - 1.0 / 6.0) < 1e-15
    # the fourth-order condition b.c^3 = 1/4 fails: the method is of order 3 exactly
    assert abs(b @ c ** 3 - 0.25) > 1e-3


def test_sdirk3_is_l_stable():
    A, b, _ = sdirk3()
    one = np.ones(3)

    def R(z):
        return 1.0 + z * b @ np.linalg.solve(np.eye(3) - z * A, one)

    for y in np.linspace(-200.0, 200.0, 2001):
        assert abs(R(1j * y)) <= 1.0 + 1e-14
    for z in (-1e3, -1e6, -1e9):
        assert abs(R(z)) < 10.0 / abs(z)
    rng = np.random.Generator(np.random.PCG64(7))
    for z in -rng.uniform(0, 50, 200) + 1j * rng.uniform(-50, 50, 200):
        assert abs(R(z)) <= 1.0 + 1e-14


def _uniform_state(rd, value):
    """Coefficients of the constant field `value` (affine mesh)."""
    return rd.project(np.full(rd.detJ.shape, value))


@pytest.mark.parametrize("sigma,dt", [(2.0, 0.05), (50.0, 0.01), (0.3, 1.0)])
def test_uniform_stage_reduces_to_scalar_equations(sigma, dt):
    """Constant e*, E* and no sources on an affine mesh: F stays 0 and each stage solves
    rho beta (e - e*) + c sigma (a (e/Cv)^4 - E) = 0 and
    beta (E - E*) - c sigma (a (e/Cv)^4 - E) = 0."""
    rho, cv, a, c = 1.3, 0.7, 0.9, 2.0
    vx, vy, vz = synth.lattice_vertices(2, 2, 1, extent=(1.0, 0.8, 0.5))
    rd = RadDiff(2, 2, 1, 3, vx, vy, vz, sigma, dt, rho=rho, cv=cv, a=a, c=c)
    e0, E0 = 2.0, 0.4
    e_star, Eh_star = _uniform_state(rd, e0), rd.load(np.full(rd.detJ.shape, E0))
    F = np.zeros(rd.n_rt)
    e, Eh, F, info = rd.stage(e_star, Eh_star, None, None, e_star.copy(), Eh_star.copy(), F)
    beta, cs = rd.beta, c * sigma

    def reduced(ev):
        Ev = (beta * E0 + cs * a * (ev / cv) ** 4) / (beta + cs)
        return rho * beta * (ev - e0) + cs * (a * (ev / cv) ** 4 - Ev)

    e_exact = brentq(reduced, 1e-6, e0 * 10, xtol=1e-15, rtol=1e-15)
    E_exact = (beta * E0 + cs * a * (e_exact / cv) ** 4) / (beta + cs)
    assert np.abs(e - _uniform_state(rd, e_exact)).max() <= 1e-10 * np.abs(e).max()
    assert np.abs(rd.winv(Eh) - _uniform_state(rd, E_exact)).max() <= 1e-10 * np.abs(Eh).max()
    assert np.abs(F).max() <= 1e-10
    assert info["relres"] <= 1e-11


def test_total_energy_is_conserved_with_reflecting_walls():
    nx, ny, nz, k = 3, 2, 2, 3
    vx, vy, vz = synth.lattice_vertices(nx, ny, nz, perturb=0.2, seed=11)
    sigma = synth.lognormal(nx * ny * nz, 0.5, seed=12)  # c sigma below 1 / dt: the time-accurate regime
    rd = RadDiff(nx, ny, nz, k, vx, vy, vz, sigma, 0.05, rho=1.1, cv=0.8, a=0.5, c=1.0)
    rng = np.random.Generator(np.random.PCG64(13))
    T0 = 1.0 + 0.5 * rng.uniform(0, 1, rd.detJ.shape)
    e = rd.project(0.8 * T0)
    Eh = rd.load(1.2 * (1.0 + 0.8 * rng.uniform(0, 1, rd.detJ.shape)))
    F = np.zeros(rd.n_rt)
    W0 = rd.total_energy(e, Eh)
    e1, Eh1, F1, infos = rd.step(e, Eh, F)
    assert abs(rd.total_energy(e1, Eh1) - W0) <= 1e-11 * abs(W0)
    assert np.linalg.norm(e1 - e) > 1e-3 * np.linalg.norm(e)     # the state did change
    assert np.linalg.norm(F1) > 0.0
    assert all(i["relres"] <= 1e-10 for i in infos), infos


def _mms_run(n, k, steps, dt, sigma=2.0):
    vx, vy, vz = synth.lattice_vertices(n, n, n, perturb=0.1, seed=5)
    rd = RadDiff(n, n, n, k, vx, vy, vz, sigma, dt)
    _, _, c = sdirk3()
    X = rd.points()
    e0, E0, _, _, _ = mms.fields(X, 0.0, sigma=sigma)
    e, Eh, F = rd.project(e0), rd.load(E0), np.zeros(rd.n_rt)
    t = 0.0
    for _ in range(steps):
        loads = []
        for ci in c:
            _, _, _, Q, S = mms.fields(X, t + ci * dt, sigma=sigma)
            loads.append((rd.load(Q), rd.load(S)))
        e, Eh, F, _ = rd.step(e, Eh, F, loads)
        t += dt
    ee, EE, _, _, _ = mms.fields(X, t, sigma=sigma)
    return rd.l2_error(e, ee), rd.l2_error(rd.winv(Eh), EE)


def test_manufactured_solution_converges_at_the_l2_rate():
    """k = 2 (Q_1 in the L2 space): second order in h. The time step is small enough that
    the SDIRK3 error (dt^3) stays far below the spatial error."""
    ee2, eE2 = _mms_run(2, 2, 2, 0.01)
    ee4, eE4 = _mms_run(4, 2, 2, 0.01)
    assert ee2 / ee4 > 3.2, (ee2, ee4)
    assert eE2 / eE4 > 3.2, (eE2, eE4)
    assert ee4 < 1e-2 and eE4 < 1e-2


def test_emission_jacobian_matches_finite_differences():
    vx, vy, vz = synth.lattice_vertices(2, 1, 1, perturb=0.0)
    vx = vx + 0.1 * vy * vz  # a non-affine (trilinear) map, det J > 0
    rd = RadDiff(2, 1, 1, 3, vx, vy, vz, 1.0, 0.1)
    rng = np.random.Generator(np.random.PCG64(21))
    el = rd._loc(rd.project(1.0 + 0.3 * rng.uniform(0, 1, rd.detJ.shape)))
    J = rd.emission_jacobian(el)
    d = rng.uniform(-1, 1, el.shape) * np.abs(el).max()
    err = []
    for h in (1e-3, 1e-4):  # central differences: the error of an exact Jacobian falls as h^2
        fd = (rd.emission(el + h * d) - rd.emission(el - h * d)) / (2 * h)
        err.append(np.abs(np.einsum("eab,eb->ea", J, d) - fd).max() / np.abs(fd).max())
    assert err[1] < 1e-5 and 80.0 < err[0] / err[1] < 120.0, err


def test_newton_converges_quadratically():
    nx, ny, nz, k = 2, 2, 1, 3
    vx, vy, vz = synth.lattice_vertices(nx, ny, nz, perturb=0.2, seed=31)
    rd = RadDiff(nx, ny, nz, k, vx, vy, vz, 20.0, 0.2)
    rng = np.random.Generator(np.random.PCG64(32))
    e_star = rd.project(1.0 + 0.5 * rng.uniform(0, 1, rd.detJ.shape))
    Eh_star = rd.load(3.0 + rng.uniform(0, 1, rd.detJ.shape))   # far from equilibrium
    F = np.zeros(rd.n_rt)
    e, Eh = e_star.copy(), Eh_star.copy()
    norms = []
    for _ in range(6):
        R1, R2 = rd.residual_12(e, Eh, F, e_star, Eh_star, 0 * e, 0 * e)
        norms.append(np.sqrt(np.sum(R1 ** 2) + np.sum(R2 ** 2)))
        e, Eh, _ = rd.newton(e, Eh, F, e_star, Eh_star, 0 * e, 0 * e, rtol=0.0, maxit=1)
    # quadratic in the end: the contraction factor r_{i+1} / r_i itself falls by orders of
    # magnitude from one step to the next (a wrong Jacobian leaves it constant)
    ratio = [norms[i + 1] / norms[i] for i in range(5)]
    assert norms[4] < 1e-9 * norms[0], norms
    assert ratio[2] < 1e-2 and ratio[3] < 0.1 * ratio[2], norms


def _random_stage(seed=51):
    nx, ny, nz, k = 3, 2, 2, 3
    vx, vy, vz = synth.lattice_vertices(nx, ny, nz, perturb=0.2, seed=seed)
    sigma = synth.lognormal(nx * ny * nz, 0.5, seed=seed + 1)
    rd = RadDiff(nx, ny, nz, k, vx, vy, vz, sigma, 0.05, rho=1.1, cv=0.8, a=0.5, c=1.0)
    rng = np.random.Generator(np.random.PCG64(seed + 2))
    shape = rd.detJ.shape
    e_s = rd.project(0.8 * (1.0 + 0.5 * rng.uniform(0, 1, shape)))
    Eh_s = rd.load(0.5 * (1.0 + 0.8 * rng.uniform(0, 1, shape)))
    Ql, Sl = rd.load(rng.uniform(0, 1, shape)), rd.load(rng.uniform(0, 1, shape))
    return rd, rng, e_s, Eh_s, Ql, Sl


def test_each_step_of_a_pass_solves_its_own_equations():
    """Newton with F fixed zeroes (R1, R2); the Darcy step with e fixed zeroes (R2, R3). The
    residuals are evaluated from their definitions, independently of how each step maps its
    unknowns (the sign of Eh in the Darcy unknown, the right-hand side W^-1 G)."""
    rd, rng, e_s, Eh_s, Ql, Sl = _random_stage()
    F = rng.uniform(-1, 1, rd.n_rt)
    F[rd.prob.ess] = 0.0
    e, Eh, _ = rd.newton(e_s.copy(), Eh_s.copy(), F, e_s, Eh_s, Ql, Sl, rtol=1e-14, maxit=30)
    R1, R2 = rd.residual_12(e, Eh, F, e_s, Eh_s, Ql, Sl)
    scale = np.abs(rd.beta * Eh).max()
    assert np.abs(R1).max() <= 1e-12 * scale and np.abs(R2).max() <= 1e-12 * scale
    Eh2, F2 = rd.darcy(e, Eh_s, Sl)
    R = rd.residual(e, Eh2, F2, e_s, Eh_s, Ql, Sl)
    n = rd.n_l2
    assert np.abs(R[n:2 * n]).max() <= 1e-11 * scale          # R2
    assert np.abs(R[2 * n:]).max() <= 1e-11 * np.abs(F2).max() * rd.beta  # R3
    assert np.abs(R[:n]).max() > 1e-6 * scale                  # R1 moved: the flux changed


def test_stage_solution_does_not_depend_on_the_initial_guess():
    rd, rng, e_s, Eh_s, Ql, Sl = _random_stage(61)
    F0 = np.zeros(rd.n_rt)
    a = rd.stage(e_s, Eh_s, Ql, Sl, e_s.copy(), Eh_s.copy(), F0.copy())
    g = rng.uniform(0.9, 1.1, rd.n_l2)
    b = rd.stage(e_s, Eh_s, Ql, Sl, e_s * g, Eh_s * g[::-1], F0 + 1e-3 * rng.uniform(-1, 1, rd.n_rt) * (
        np.isin(np.arange(rd.n_rt), rd.prob.ess, invert=True)))
    for x, y in zip(a[:3], b[:3]):
        assert np.abs(x - y).max() <= 1e-9 * np.abs(x).max()


def test_sdirk3_steps_converge_at_third_order_in_time():
    """A spatially uniform state with no sources keeps F = 0 and reduces the system to the ODEs
    rho de/dt = -c sigma (a (e/Cv)^4 - E), dE/dt = c sigma (a (e/Cv)^4 - E). The oracle's steps
    (stage starts, stage rates, the stiffly accurate update) against scipy's Radau solution to
    1e-13: the error falls by about 2^3 per halving of dt (above 6.5 here: a second-order
    method gives about 4)."""
    from scipy.integrate import solve_ivp
    rho, cv, a, c, sigma = 1.0, 1.0, 1.0, 1.0, 0.5
    e0, E0, t_end = 2.0, 0.5, 0.4

    def f(t, y):
        cpl = c * sigma * (a * (y[0] / cv) ** 4 - y[1])
        return [-cpl / rho, cpl]

    ref = solve_ivp(f, (0.0, t_end), [e0, E0], method="Radau", rtol=1e-13, atol=1e-14).y[:, -1]
    vx, vy, vz = synth.lattice_vertices(1, 1, 1)
    errs = []
    for dt in (0.05, 0.025, 0.0125):
        rd = RadDiff(1, 1, 1, 2, vx, vy, vz, sigma, dt, rho=rho, cv=cv, a=a, c=c)
        e = rd.project(np.full(rd.detJ.shape, e0))
        Eh = rd.load(np.full(rd.detJ.shape, E0))
        F = np.zeros(rd.n_rt)
        for _ in range(int(round(t_end / dt))):
            e, Eh, F, _ = rd.step(e, Eh, F, outer_rtol=1e-13)
        # on the unit cube the coefficients of a constant field sum to its value
        errs.append(max(abs(e.sum() - ref[0]), abs(rd.winv(Eh).sum() - ref[1])))
    assert errs[2] < 1e-5, errs
    assert errs[1] / errs[2] > 6.5 and errs[0] / errs[1] > 6.0, errs

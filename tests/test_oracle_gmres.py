"""Pins of the oracle's GMRES and block-triangular preconditioner (Sec. 2.3 remark):
exact blocks give convergence in two iterations; each GMRES iterate is the
minimal-residual point of its Krylov space (brute-force least squares); the
triangular preconditioner inverts the assembled triangular block matrix; with the
V-cycle it needs fewer iterations than block-diagonal MINRES."""
import numpy as np
import scipy.linalg as sla
import pytest

import synth
from cases import inputs, oracle_problem
from oracle.gmres import gmres
from oracle.minres import minres
from oracle.precond import BlockPrec, BlockTriPrec


def _blocks(prob):
    A = prob.matrix().toarray()
    nrt = prob.lat.n_rt
    return A, A[:nrt, :nrt], A[:nrt, nrt:], A[nrt:, :nrt], A[nrt:, nrt:], nrt


@pytest.mark.parametrize("name", ["c1", "gd_k4_ragged", "darcy_gamma"])
def test_exact_block_triangular_gmres_converges_in_two_iterations(name):
    """P = [[M, D^T], [0, -S]] with S = C + D M^-1 D^T exact: A P^-1 - I is nilpotent
    of index two, so GMRES reaches the solution in (at most) two steps."""
    prob = oracle_problem(inputs(name))
    A, M, Bt, B, mC, nrt = _blocks(prob)
    S = -mC + B @ np.linalg.solve(M, Bt)
    P = np.block([[M, Bt], [np.zeros_like(B), -S]])
    E = A @ np.linalg.inv(P) - np.eye(A.shape[0])
    assert np.abs(E @ E).max() < 1e-8 * np.abs(E).max()
    b = np.random.Generator(np.random.PCG64(31)).uniform(-1, 1, A.shape[0])
    x, info = gmres(lambda v: A @ v, lambda r: np.linalg.solve(P, r), b, rtol=1e-10, maxit=10)
    assert info["iterations"] <= 2 and info["converged"], info
    assert np.linalg.norm(A @ x - b) <= 1e-9 * np.linalg.norm(b)


def test_gmres_iterate_is_the_krylov_minimal_residual():
    """x_j = x_0 + P^-1 V_j y minimises ||b - A x|| over the span of P^-1 times the
    Krylov vectors of A P^-1: compare with a least-squares solve on an explicitly
    built (orthonormalised) Krylov basis, for j = 1..5, without restarts."""
    prob = oracle_problem(inputs("darcy_gamma"))
    A = prob.matrix().toarray()
    bp = BlockTriPrec(prob, coarse_max=8, cycle=2, smooth=4.0 / 3.0, sa_levels=2)
    Pinv = lambda r: bp.apply(r)
    b = np.random.Generator(np.random.PCG64(32)).uniform(-1, 1, A.shape[0])
    AP = np.column_stack([A @ Pinv(e) for e in np.eye(A.shape[0])])
    for j in range(1, 6):
        x, info = gmres(lambda v: A @ v, Pinv, b, rtol=0.0, maxit=j, restart=50)
        K = [b / np.linalg.norm(b)]
        for _ in range(j - 1):
            K.append(AP @ K[-1])
        Q, _ = np.linalg.qr(np.column_stack(K))
        y, *_ = np.linalg.lstsq(AP @ Q, b, rcond=None)
        best = np.linalg.norm(b - AP @ (Q @ y))
        assert abs(np.linalg.norm(b - A @ x) - best) <= 1e-9 * np.linalg.norm(b), (j, best)


def test_block_triangular_preconditioner_inverts_the_triangular_matrix():
    """With exact M~ and a direct S^ the apply equals the solve with the assembled
    [[tau M~, D^T], [0, -S~]] (free dofs; identity rows on essential dofs)."""
    prob = oracle_problem(inputs("gd_k4_ragged"))
    bp = BlockTriPrec(prob, tau=1.3, coarse_max=10 ** 6, cycle=1, smooth=0.0)   # one level: exact S~ solve
    assert bp.vc.n_levels == 1
    A, M, Bt, B, mC, nrt = _blocks(prob)
    Mt = np.where(prob.free, 1.3 * bp.Mt, 1.0)
    P = np.block([[np.diag(Mt), Bt], [np.zeros_like(B), -bp.S.toarray()]])
    r = np.random.Generator(np.random.PCG64(33)).uniform(-1, 1, A.shape[0])
    z = bp.apply(r)
    assert np.allclose(P @ z, r, rtol=1e-12, atol=1e-12 * np.abs(r).max())


def test_block_triangular_gmres_needs_fewer_iterations_than_minres():
    """On the metric recipe (4^3 elements, k = 4) GMRES with the triangular
    preconditioner reaches a true relative residual of 1e-8 in fewer iterations than
    block-diagonal MINRES reaches its own (weaker) stopping test."""
    from oracle.assembly import Problem, GRAD_DIV
    n = 4
    vx, vy, vz = synth.lattice_vertices(n, n, n, perturb=0.15, seed=2304)
    beta = synth.lognormal(n ** 3, 2.0, seed=2305)
    prob = Problem(n, n, n, 4, vx, vy, vz, np.ones(n ** 3), beta, kind=GRAD_DIV, ess_mask=63, q=6)
    b = synth.uniform(prob.n, seed=2311)
    b[prob.ess] = 0.0
    kw = dict(coarse_max=8, cycle=2, smooth=4.0 / 3.0, sa_levels=2)
    _, im = minres(prob.apply_op, BlockPrec(prob, **kw).apply, b, rtol=1e-8, maxit=2000)
    x, ig = gmres(prob.apply_op, BlockTriPrec(prob, **kw).apply, b, rtol=1e-8, maxit=2000, restart=50)
    assert ig["converged"] and ig["true_relres"] <= 1e-8
    assert ig["iterations"] < 0.8 * im["iterations"], (ig["iterations"], im["iterations"])


def test_gmres_zero_rhs_and_restart_one():
    """b = 0 returns x = 0 with no steps; GMRES(1) on an SPD system is the
    minimal-residual iteration and converges (slowly) to the dense solution."""
    rng = np.random.Generator(np.random.PCG64(34))
    Q, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    A = Q @ np.diag(np.linspace(1.0, 4.0, 12)) @ Q.T
    x, info = gmres(lambda v: A @ v, lambda r: r, np.zeros(12), rtol=1e-8, maxit=10)
    assert info["iterations"] == 0 and np.all(x == 0)
    b = rng.standard_normal(12)
    x, info = gmres(lambda v: A @ v, lambda r: r, b, rtol=1e-10, maxit=500, restart=1)
    assert info["converged"] and info["cycles"] == info["iterations"]
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-8, atol=1e-9)

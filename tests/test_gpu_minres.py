"""GPU MINRES against the oracle's MINRES (same preconditioner spec): solutions
within 1e-8 relative, iteration counts within one."""
import numpy as np
import pytest

from cases import close, gpu_operator, inputs, oracle_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,rtol", [("c1", 1e-10), ("darcy_k3", 1e-8), ("gd_k4_ragged", 1e-8),
                                       ("darcy_neumann", 1e-8), ("darcy_gamma", 1e-8)])
def test_minres_matches_oracle(name, rtol):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle.minres import minres
    from oracle.precond import BlockPrec
    d = inputs(name)
    prob = oracle_problem(d)
    bp = BlockPrec(prob, nu=2, coarse_max=8)
    b = np.random.Generator(np.random.PCG64(11)).uniform(-1, 1, prob.n)
    b[prob.ess] = 0.0
    if bp.singular:                       # consistent right-hand side: q part orthogonal to constants
        b[prob.lat.n_rt:] -= b[prob.lat.n_rt:].mean()
    xr, info_r = minres(prob.apply_op, bp.apply, b, rtol=rtol, maxit=2000)
    op = gpu_operator(d, coarse_max=8)
    x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    st, info = op.hd_minres_solve(torch.from_numpy(b).cuda(), x, rtol=rtol, maxit=2000, check_every=4)
    torch.cuda.synchronize()
    assert st == 0, info
    assert abs(info["iterations"] - info_r["iterations"]) <= 1, (info, info_r["iterations"])
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - xr) <= 1e-8 * np.linalg.norm(xr)
    assert info["true_relres"] < 1e3 * rtol
    op.close()


@pytest.mark.parametrize("name,precision", [("darcy_k3", 0), ("darcy_k3", 1), ("gd_k4_ragged", 1),
                                            ("c1", 1), ("darcy_gamma", 1)])
def test_refined_solve_reaches_true_residual(name, precision):
    """FP64 residual correction around the inner MINRES (precision 0: FP64 inner;
    1: FP32 operator and V-cycle inside, FP64 Lanczos vectors, dots and coarsest
    solve): the true relative residual reaches the target and the solution matches
    an exact sparse solve of the oracle's assembled system."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import scipy.sparse.linalg as spla
    d = inputs(name)
    prob = oracle_problem(d)
    b = np.random.Generator(np.random.PCG64(12)).uniform(-1, 1, prob.n)
    b[prob.ess] = 0.0
    x_exact = spla.spsolve(prob.matrix().tocsc(), b)
    op = gpu_operator(d, coarse_max=8)
    x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    st, info = op.hd_minres_solve(torch.from_numpy(b).cuda(), x, rtol=1e-5 if precision else 1e-8,
                                  maxit=5000, check_every=4, precision=precision, outer_rtol=1e-10,
                                  max_outer=30)
    torch.cuda.synchronize()
    assert st == 0, info
    assert info["true_relres"] <= 1e-10, info
    xg = x.cpu().numpy()
    r = b - prob.apply_op(xg)
    assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(b)       # oracle's own residual of the result
    err = np.linalg.norm(xg - x_exact) / np.linalg.norm(x_exact)
    assert err <= 1e-7, err
    op.close()


@pytest.mark.parametrize("name", ["gd_k4_ragged", "darcy_k3", "darcy_neumann"])
def test_wcycle_matches_oracle(name):
    """W-cycle option: the V-cycle apply and the MINRES iteration count against the
    oracle running the same W-cycle spec."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle.minres import minres
    from oracle.precond import BlockPrec
    d = inputs(name)
    prob = oracle_problem(d)
    bp = BlockPrec(prob, nu=2, coarse_max=8, cycle=2)
    op = gpu_operator(d, coarse_max=8, cycle=2)
    assert bp.vc.n_levels >= 3
    r = np.random.Generator(np.random.PCG64(13)).uniform(-1, 1, prob.lat.n_l2)
    z = torch.empty(prob.lat.n_l2, dtype=torch.float64, device="cuda")
    op.hd_vcycle(torch.from_numpy(r).cuda(), z)
    torch.cuda.synchronize()
    assert close(z.cpu().numpy(), bp.vc._cycle(0, r), 1e-12) <= 1e-12
    b = np.random.Generator(np.random.PCG64(14)).uniform(-1, 1, prob.n)
    b[prob.ess] = 0.0
    if bp.singular:
        b[prob.lat.n_rt:] -= b[prob.lat.n_rt:].mean()
    xr, ir = minres(prob.apply_op, bp.apply, b, rtol=1e-8, maxit=2000)
    x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    st, info = op.hd_minres_solve(torch.from_numpy(b).cuda(), x, rtol=1e-8, maxit=2000, check_every=4)
    assert st == 0 and abs(info["iterations"] - ir["iterations"]) <= 1, (info, ir["iterations"])
    assert np.linalg.norm(x.cpu().numpy() - xr) <= 1e-8 * np.linalg.norm(xr)
    op.close()


@pytest.mark.parametrize("name,cycle", [("gd_k4_ragged", 2), ("darcy_k3", 1), ("darcy_neumann", 2), ("c1", 1)])
def test_fp64_emulation_solver_matches_oracle(name, cycle):
    """Double-float element kernel and V/W-cycle (fp64_emulation = 1): the V-cycle
    and preconditioner applies at the FP64 tolerances, MINRES iterations within one
    of the oracle and the solution within 1e-8."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle.minres import minres
    from oracle.precond import BlockPrec
    d = inputs(name)
    prob = oracle_problem(d)
    bp = BlockPrec(prob, nu=2, coarse_max=8, cycle=cycle)
    op = gpu_operator(d, coarse_max=8, cycle=cycle, fp64_emulation=1)
    rng = np.random.Generator(np.random.PCG64(17))
    r = rng.uniform(-1, 1, prob.lat.n_l2)
    z = torch.empty(prob.lat.n_l2, dtype=torch.float64, device="cuda")
    op.hd_vcycle(torch.from_numpy(r).cuda(), z)
    torch.cuda.synchronize()
    assert close(z.cpu().numpy(), bp.vc._cycle(0, r), 1e-12) <= 1e-12
    rr = rng.uniform(-1, 1, prob.n)
    zz = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    op.hd_apply_prec(torch.from_numpy(rr).cuda(), zz)
    torch.cuda.synchronize()
    assert close(zz.cpu().numpy(), bp.apply(rr), 1e-12) <= 1e-12
    b = rng.uniform(-1, 1, prob.n)
    b[prob.ess] = 0.0
    if bp.singular:
        b[prob.lat.n_rt:] -= b[prob.lat.n_rt:].mean()
    xr, ir = minres(prob.apply_op, bp.apply, b, rtol=1e-8, maxit=2000)
    x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    st, info = op.hd_minres_solve(torch.from_numpy(b).cuda(), x, rtol=1e-8, maxit=2000, check_every=4)
    assert st == 0 and abs(info["iterations"] - ir["iterations"]) <= 1, (info, ir["iterations"])
    assert np.linalg.norm(x.cpu().numpy() - xr) <= 1e-8 * np.linalg.norm(xr)
    op.close()

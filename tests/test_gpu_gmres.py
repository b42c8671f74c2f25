"""GMRES with the block preconditioners (the remark on block-triangular
preconditioners in Sec. 2.3) against the oracle's GMRES on the same seeded inputs:
Arnoldi step counts within one, solutions within 1e-8, the true relative residual
reached; restarts; the singular pure-Neumann case; argument and non-convergence
errors."""
import numpy as np
import pytest

from cases import gpu_operator, inputs, oracle_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OMEGA = 4.0 / 3.0
KW = dict(coarse_max=8, cycle=2, smooth_levels=2)


def _setup(name, tri):
    from oracle.precond import BlockPrec, BlockTriPrec
    d = inputs(name)
    prob = oracle_problem(d)
    cls = BlockTriPrec if tri else BlockPrec
    bp = cls(prob, nu=2, coarse_max=8, cycle=2, smooth=OMEGA, sa_levels=2)
    op = gpu_operator(d, **KW)
    b = np.random.Generator(np.random.PCG64(41)).uniform(-1, 1, prob.n)
    b[prob.ess] = 0.0
    if bp.singular:
        b[prob.lat.n_rt:] -= b[prob.lat.n_rt:].mean()
    return d, prob, bp, op, b


@pytest.mark.parametrize("tri", [True, False])
@pytest.mark.parametrize("name", ["gd_k4_ragged", "darcy_k3", "darcy_neumann", "c1", "gd_k5", "gd_tall", "gd_flat"])
def test_gmres_matches_oracle(name, tri):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_12387_gb300 as hd
    from oracle.gmres import gmres
    d, prob, bp, op, b = _setup(name, tri)
    xr, ir = gmres(prob.apply_op, bp.apply, b, rtol=1e-8, maxit=2000, restart=64)
    assert ir["converged"]
    x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    prec = hd.HD_GMRES_BLOCK_TRI if tri else hd.HD_GMRES_BLOCK_DIAG
    st, info = op.hd_gmres_solve(torch.from_numpy(b).cuda(), x, rtol=1e-8, maxit=2000, restart=64, prec=prec)
    assert st == 0 and abs(info["iterations"] - ir["iterations"]) <= 1, (info, ir["iterations"])
    assert info["true_relres"] <= 1e-8
    xs = x.cpu().numpy()
    assert np.linalg.norm(xs - xr) <= 1e-7 * np.linalg.norm(xr)
    assert np.linalg.norm(b - prob.apply_op(xs)) <= 1e-8 * np.linalg.norm(b)
    op.close()


@pytest.mark.parametrize("name", ["gd_k4_ragged", "darcy_neumann"])
def test_gmres_restarts_match_oracle(name):
    """restart = 5: several cycles, each restarted from the true residual."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_12387_gb300 as hd
    from oracle.gmres import gmres
    d, prob, bp, op, b = _setup(name, True)
    xr, ir = gmres(prob.apply_op, bp.apply, b, rtol=1e-8, maxit=2000, restart=5)
    x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    st, info = op.hd_gmres_solve(torch.from_numpy(b).cuda(), x, rtol=1e-8, maxit=2000, restart=5,
                                 prec=hd.HD_GMRES_BLOCK_TRI)
    assert st == 0 and info["cycles"] >= 2 and abs(info["iterations"] - ir["iterations"]) <= 2, (info, ir)
    assert np.linalg.norm(x.cpu().numpy() - xr) <= 1e-7 * np.linalg.norm(xr)
    op.close()


def test_gmres_triangular_beats_minres_in_iterations():
    """Same problem, same hierarchy: block-triangular GMRES reaches the true 1e-8 in
    fewer steps than block-diagonal MINRES with its FP64 residual correction."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_12387_gb300 as hd
    d, prob, bp, op, b = _setup("gd_k4_ragged", True)
    bt = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bt)
    st, gi = op.hd_gmres_solve(bt, x, rtol=1e-8, maxit=2000, restart=64, prec=hd.HD_GMRES_BLOCK_TRI)
    x2 = torch.zeros_like(bt)
    st2, mi = op.hd_minres_solve(bt, x2, rtol=1e-8, maxit=2000, outer_rtol=1e-8, max_outer=10)
    assert st == 0 and st2 == 0 and gi["iterations"] < mi["iterations"], (gi, mi)
    op.close()


def test_gmres_arguments_and_non_convergence():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_12387_gb300 as hd
    d, prob, bp, op, b = _setup("darcy_k3", True)
    bt = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bt)
    for kw in (dict(restart=0), dict(restart=129), dict(prec=2), dict(maxit=0), dict(precision=2),
               dict(precision=1, inner_rtol=0.0), dict(precision=1, inner_rtol=1.0)):
        st, _ = op.hd_gmres_solve(bt, x, **kw)
        assert st == hd.HD_ERR_INVALID_ARG, kw
    st, info = op.hd_gmres_solve(bt, x, rtol=1e-12, maxit=3, restart=64, prec=hd.HD_GMRES_BLOCK_TRI)
    assert st == hd.HD_ERR_NOT_CONVERGED and info["iterations"] == 3
    assert 0 < info["true_relres"] < 1
    op.close()


@pytest.mark.parametrize("name", ["gd_k4_ragged", "darcy_k3", "darcy_neumann", "gd_flat"])
def test_mixed_precision_gmres_reaches_the_fp64_solution(name):
    """precision = 1: FP32 operator and V-cycle inside the cycles, FP64 residual at
    every restart: the true relative residual 1e-8 is reached and the solution
    agrees with the oracle's FP64 GMRES."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_12387_gb300 as hd
    from oracle.gmres import gmres
    d, prob, bp, op, b = _setup(name, True)
    xr, ir = gmres(prob.apply_op, bp.apply, b, rtol=1e-10, maxit=2000, restart=64)
    x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    st, info = op.hd_gmres_solve(torch.from_numpy(b).cuda(), x, rtol=1e-8, maxit=2000, restart=32,
                                 prec=hd.HD_GMRES_BLOCK_TRI, precision=1, inner_rtol=1e-4)
    assert st == 0 and info["true_relres"] <= 1e-8 and info["cycles"] >= 2, info
    xs = x.cpu().numpy()
    assert np.linalg.norm(b - prob.apply_op(xs)) <= 1e-8 * np.linalg.norm(b)
    assert np.linalg.norm(xs - xr) <= 1e-6 * np.linalg.norm(xr)
    op.close()


def test_gmres_edge_cases():
    """b = 0 gives x = 0 in no steps; a starting guess that already meets the
    tolerance returns at once; restart = 1 (minimal-residual steps from the true
    residual each time) still converges, as the oracle's GMRES(1) does."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_12387_gb300 as hd
    from oracle.gmres import gmres
    d, prob, bp, op, b = _setup("darcy_gamma", True)
    bt = torch.from_numpy(b).cuda()
    z = torch.zeros_like(bt)
    x = torch.full_like(bt, 3.0)
    st, info = op.hd_gmres_solve(z, x, rtol=1e-8, maxit=100, restart=16, prec=hd.HD_GMRES_BLOCK_TRI)
    assert st == 0 and info["iterations"] == 0 and float(x.abs().max()) == 0.0
    x = torch.zeros_like(bt)
    st, info = op.hd_gmres_solve(bt, x, rtol=1e-10, maxit=500, restart=32, prec=hd.HD_GMRES_BLOCK_TRI)
    assert st == 0
    st, info = op.hd_gmres_solve(bt, x, rtol=1e-8, maxit=500, restart=32, prec=hd.HD_GMRES_BLOCK_TRI, use_x0=True)
    assert st == 0 and info["iterations"] == 0 and info["true_relres"] <= 1e-8
    xr, ir = gmres(prob.apply_op, bp.apply, b, rtol=1e-6, maxit=5000, restart=1)
    x = torch.zeros_like(bt)
    st, info = op.hd_gmres_solve(bt, x, rtol=1e-6, maxit=5000, restart=1, prec=hd.HD_GMRES_BLOCK_TRI)
    assert ir["converged"] and st == 0 and info["cycles"] == info["iterations"]
    assert abs(info["iterations"] - ir["iterations"]) <= max(2, ir["iterations"] // 50), (info, ir["iterations"])
    op.close()


def test_mixed_gmres_block_diagonal():
    """precision = 1 with the block-diagonal preconditioner also reaches the true 1e-8."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_12387_gb300 as hd
    d, prob, bp, op, b = _setup("darcy_k3", False)
    x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    st, info = op.hd_gmres_solve(torch.from_numpy(b).cuda(), x, rtol=1e-8, maxit=3000, restart=32,
                                 prec=hd.HD_GMRES_BLOCK_DIAG, precision=1, inner_rtol=1e-3)
    assert st == 0 and info["true_relres"] <= 1e-8
    assert np.linalg.norm(b - prob.apply_op(x.cpu().numpy())) <= 1e-8 * np.linalg.norm(b)
    op.close()


def test_gmres_with_the_learned_schur_preconditioner():
    """The learned Schur preconditioner replaces S^-1 inside FP64 block-triangular GMRES
    (no symmetry needed): the true 1e-8 is reached; the FP32 cycles refuse it."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_12387_gb300 as hd
    d = inputs("darcy_k3")
    prob = oracle_problem(d)
    op = gpu_operator(d, coarse_max=8, cycle=2)
    op.hd_learned_init(seed=5)
    op.hd_set_schur_prec(1)
    b = np.random.Generator(np.random.PCG64(43)).uniform(-1, 1, prob.n)
    bt = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bt)
    st, info = op.hd_gmres_solve(bt, x, rtol=1e-8, maxit=3000, restart=32, prec=hd.HD_GMRES_BLOCK_TRI)
    assert st == 0 and info["true_relres"] <= 1e-8, info
    assert np.linalg.norm(b - prob.apply_op(x.cpu().numpy())) <= 1e-8 * np.linalg.norm(b)
    st, _ = op.hd_gmres_solve(bt, x, rtol=1e-8, maxit=100, restart=32, prec=hd.HD_GMRES_BLOCK_TRI, precision=1)
    assert st == hd.HD_ERR_NOT_IMPLEMENTED
    op.close()

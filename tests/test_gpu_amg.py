"""Smoothed-aggregation hierarchy (smooth_levels = 1: the first prolongator smoothed;
2: the first two) against the oracle running the same spec: the V/W-cycle and
preconditioner applies within 1e-12, MINRES iteration counts within one and
solutions within 1e-8; the FP32 copy within FP32 rounding."""
import numpy as np
import pytest

from cases import close, gpu_operator, inputs, oracle_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OMEGA = 4.0 / 3.0
NAMES = ["gd_k4_ragged", "darcy_k3", "darcy_neumann", "c1", "gd_k5", "darcy_gamma", "gd_tall", "gd_flat"]


def _setup(name, cycle, w_levels=0, smooth_levels=1):
    from oracle.precond import BlockPrec
    d = inputs(name)
    prob = oracle_problem(d)
    bp = BlockPrec(prob, nu=2, coarse_max=8, cycle=cycle, smooth=OMEGA if smooth_levels else 0.0,
                   sa_levels=max(smooth_levels, 1), w_levels=w_levels)
    op = gpu_operator(d, coarse_max=8, cycle=cycle, smooth_levels=smooth_levels, w_levels=w_levels)
    return d, prob, bp, op


@pytest.mark.parametrize("smooth_levels", [1, 2])
@pytest.mark.parametrize("cycle,w_levels", [(1, 0), (2, 0), (2, 1), (2, 2)])
@pytest.mark.parametrize("name", NAMES)
def test_smoothed_cycle_and_preconditioner_match_oracle(name, cycle, w_levels, smooth_levels):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d, prob, bp, op = _setup(name, cycle, w_levels, smooth_levels)
    if smooth_levels == 2:
        assert bp.vc.n_levels >= 3  # the second prolongator exists
    rng = np.random.Generator(np.random.PCG64(21))
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
    # the FP32 copy used inside the mixed-precision solve
    zf = torch.empty(prob.n, dtype=torch.float32, device="cuda")
    op.hd_apply_prec_f32(torch.from_numpy(rr).float().cuda(), zf)
    torch.cuda.synchronize()
    assert close(zf.double().cpu().numpy(), bp.apply(rr), 2e-5) <= 2e-5
    op.close()


@pytest.mark.parametrize("name,cycle,w_levels,smooth_levels",
                         [("gd_k4_ragged", 2, 2, 1), ("darcy_k3", 2, 0, 1), ("darcy_neumann", 2, 2, 1),
                          ("c1", 1, 0, 1), ("darcy_gamma", 1, 0, 1), ("gd_k4_ragged", 2, 0, 2),
                          ("darcy_neumann", 2, 0, 2), ("darcy_k3", 1, 0, 2)])
def test_smoothed_minres_matches_oracle(name, cycle, w_levels, smooth_levels):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle.minres import minres
    d, prob, bp, op = _setup(name, cycle, w_levels, smooth_levels)
    b = np.random.Generator(np.random.PCG64(22)).uniform(-1, 1, prob.n)
    b[prob.ess] = 0.0
    if bp.singular:
        b[prob.lat.n_rt:] -= b[prob.lat.n_rt:].mean()
    xr, ir = minres(prob.apply_op, bp.apply, b, rtol=1e-8, maxit=2000)
    x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    st, info = op.hd_minres_solve(torch.from_numpy(b).cuda(), x, rtol=1e-8, maxit=2000, check_every=4)
    assert st == 0 and abs(info["iterations"] - ir["iterations"]) <= 1, (info, ir["iterations"])
    assert np.linalg.norm(x.cpu().numpy() - xr) <= 1e-8 * np.linalg.norm(xr)
    # mixed precision with FP64 residual correction reaches the same solution
    xm = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    st, info = op.hd_minres_solve(torch.from_numpy(b).cuda(), xm, rtol=1e-4, maxit=2000, check_every=4,
                                  precision=1, outer_rtol=1e-10, max_outer=30)
    assert st == 0 and info["true_relres"] <= 1e-10, info
    assert np.linalg.norm(xm.cpu().numpy() - xr) <= 1e-7 * np.linalg.norm(xr)
    op.close()


def test_smooth_levels_argument_checks():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_12387_gb300 as hd
    d = inputs("c1")
    with pytest.raises(hd.HdError) as e:
        gpu_operator(d, smooth_levels=3)
    assert e.value.status == hd.HD_ERR_NOT_IMPLEMENTED
    with pytest.raises(hd.HdError) as e:
        gpu_operator(d, smooth_levels=-1)
    assert e.value.status == hd.HD_ERR_INVALID_ARG
    # a single-level hierarchy has nothing to smooth: same result as without
    from oracle.precond import BlockPrec
    prob = oracle_problem(d)
    bp = BlockPrec(prob, coarse_max=10 ** 6, smooth=OMEGA)
    op = gpu_operator(d, coarse_max=4096, smooth_levels=1)
    r = np.random.Generator(np.random.PCG64(23)).uniform(-1, 1, prob.lat.n_l2)
    z = torch.empty(prob.lat.n_l2, dtype=torch.float64, device="cuda")
    op.hd_vcycle(torch.from_numpy(r).cuda(), z)
    torch.cuda.synchronize()
    assert close(z.cpu().numpy(), bp.vc.apply(r), 1e-12) <= 1e-12
    op.close()


@pytest.mark.parametrize("name", ["gd_k4_ragged", "darcy_neumann"])
def test_unsmoothed_w_levels_matches_oracle(name):
    """w_levels on the unsmoothed hierarchy: the cycle against the oracle's."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d, prob, bp, op = _setup(name, 2, w_levels=1, smooth_levels=0)
    r = np.random.Generator(np.random.PCG64(24)).uniform(-1, 1, prob.lat.n_l2)
    z = torch.empty(prob.lat.n_l2, dtype=torch.float64, device="cuda")
    op.hd_vcycle(torch.from_numpy(r).cuda(), z)
    torch.cuda.synchronize()
    assert close(z.cpu().numpy(), bp.vc._cycle(0, r), 1e-12) <= 1e-12
    op.close()

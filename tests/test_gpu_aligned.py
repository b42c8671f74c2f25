"""Element-aligned aggregation of the Schur hierarchy (aggregation = 1) against the oracle
running the same spec (oracle.precond.aggregation with the element counts).

Odd k: the first transfer groups each element's cells as [2, 1] (k = 3) or [2, 1, 2]
(k = 5), and for k = 5 the second one as [2, 1]. The GPU cycle and preconditioner match
the oracle's at 1e-12, as for the pair hierarchy (the unsmoothed 7-point levels, and
the smoothed first level with its 81-point coarse stencil), the FP32 copy at FP32
rounding, and MINRES within one iteration. For even k the option changes nothing (bit for
bit), and odd k with two smoothed levels is refused."""
import numpy as np
import pytest

from cases import close, gpu_operator, inputs, oracle_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OMEGA = 4.0 / 3.0
ODD = ["darcy_k3", "gd_k3", "gd_k5"]


def _setup(name, cycle, smooth_levels):
    from oracle.precond import BlockPrec
    d = inputs(name)
    prob = oracle_problem(d)
    bp = BlockPrec(prob, nu=2, coarse_max=8, cycle=cycle, smooth=OMEGA if smooth_levels else 0.0, sa_levels=1,
                   aligned=True)
    op = gpu_operator(d, coarse_max=8, cycle=cycle, smooth_levels=smooth_levels, aggregation=1)
    return d, prob, bp, op


@pytest.mark.parametrize("smooth_levels", [0, 1])
@pytest.mark.parametrize("cycle", [1, 2])
@pytest.mark.parametrize("name", ODD)
def test_aligned_cycle_and_preconditioner_match_oracle(name, cycle, smooth_levels):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d, prob, bp, op = _setup(name, cycle, smooth_levels)
    # the same lattice dimensions on every level
    nl = op.hd_get_level(0)[0]
    assert nl == bp.vc.n_levels
    for l in range(nl):
        assert tuple(op.hd_get_level(l)[1]) == tuple(bp.vc.dims[l]), l
    assert bp.vc.dims[1][0] == d["nx"] * (2 if d["k"] == 3 else 3)  # element-aligned groups
    rng = np.random.Generator(np.random.PCG64(31))
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
    zf = torch.empty(prob.n, dtype=torch.float32, device="cuda")
    op.hd_apply_prec_f32(torch.from_numpy(rr).float().cuda(), zf)
    torch.cuda.synchronize()
    assert close(zf.double().cpu().numpy(), bp.apply(rr), 2e-5) <= 2e-5
    op.close()


@pytest.mark.parametrize("name,smooth_levels", [("darcy_k3", 1), ("gd_k5", 1), ("gd_k3", 0)])
def test_aligned_minres_matches_oracle(name, smooth_levels):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle.minres import minres
    d, prob, bp, op = _setup(name, 2, smooth_levels)
    b = np.random.Generator(np.random.PCG64(32)).uniform(-1, 1, prob.n)
    b[prob.ess] = 0.0
    if bp.singular:
        b[prob.lat.n_rt:] -= b[prob.lat.n_rt:].mean()
    xr, ir = minres(prob.apply_op, bp.apply, b, rtol=1e-8, maxit=2000)
    x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    st, info = op.hd_minres_solve(torch.from_numpy(b).cuda(), x, rtol=1e-8, maxit=2000, check_every=4)
    assert st == 0 and abs(info["iterations"] - ir["iterations"]) <= 1, (info, ir["iterations"])
    assert np.linalg.norm(x.cpu().numpy() - xr) <= 1e-8 * np.linalg.norm(xr)
    xm = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    st, info = op.hd_minres_solve(torch.from_numpy(b).cuda(), xm, rtol=1e-4, maxit=2000, check_every=4,
                                  precision=1, outer_rtol=1e-10, max_outer=30)
    assert st == 0 and info["true_relres"] <= 1e-10, info
    op.close()


@pytest.mark.parametrize("smooth_levels", [0, 1, 2])
def test_even_degree_aligned_is_the_pair_hierarchy(smooth_levels):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = inputs("gd_k4_ragged")
    zs = []
    for agg in (0, 1):
        op = gpu_operator(d, coarse_max=8, cycle=2, smooth_levels=smooth_levels, aggregation=agg)
        rr = torch.from_numpy(np.random.Generator(np.random.PCG64(33)).uniform(-1, 1, op.n_l2)).cuda()
        z = torch.empty_like(rr)
        op.hd_vcycle(rr, z)
        torch.cuda.synchronize()
        zs.append(z.cpu())
        op.close()
    assert torch.equal(zs[0], zs[1])


def test_odd_degree_aligned_with_two_smoothed_levels_is_refused():
    import paper_2304_12387_gb300 as hd
    d = inputs("darcy_k3")
    with pytest.raises(hd.HdError) as e:
        gpu_operator(d, coarse_max=8, cycle=2, smooth_levels=2, aggregation=1)
    assert e.value.status == hd.HD_ERR_NOT_IMPLEMENTED

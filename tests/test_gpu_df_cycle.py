"""The Schur V/W-cycle in double-float (fp64_emulation = 2: the element kernel and the cycle's
levels in FP32 pairs, about 48 significant bits; the coarsest dense solve and the MINRES
recurrences in FP64) against the oracle's cycle and the FP64 cycle of the same hierarchy.

Bars: the cycle within 1e-12 of the oracle (the FP64 cycle's own bar; double-float roundoff,
~3.6e-15 per operation, stays far below it over a W-cycle's few hundred operations per
entry), and MINRES within one iteration of the FP64-cycle solve with the same solution to
1e-8, for the pair hierarchy with none, one and two smoothed levels and for the
element-aligned one."""
import numpy as np
import pytest

from cases import close, gpu_operator, inputs, oracle_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
OMEGA = 4.0 / 3.0


@pytest.mark.parametrize("name,smooth_levels,cycle,agg", [
    ("gd_k4_ragged", 0, 2, 0), ("gd_k4_ragged", 1, 2, 0), ("gd_k4_ragged", 2, 2, 0), ("darcy_k3", 2, 1, 0),
    ("darcy_neumann", 2, 2, 0), ("gd_tall", 1, 2, 0), ("darcy_k3", 1, 2, 1), ("gd_k5", 0, 2, 1)])
def test_double_float_cycle_matches_oracle_and_fp64(name, smooth_levels, cycle, agg):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle.precond import BlockPrec
    d = inputs(name)
    prob = oracle_problem(d)
    bp = BlockPrec(prob, nu=2, coarse_max=8, cycle=cycle, smooth=OMEGA if smooth_levels else 0.0,
                   sa_levels=max(smooth_levels, 1), aligned=bool(agg))
    ops = {e: gpu_operator(d, coarse_max=8, cycle=cycle, smooth_levels=smooth_levels, aggregation=agg,
                           fp64_emulation=e) for e in (1, 2)}
    r = np.random.Generator(np.random.PCG64(41)).uniform(-1, 1, prob.lat.n_l2)
    z = {}
    for e, op in ops.items():
        zz = torch.empty(prob.lat.n_l2, dtype=torch.float64, device="cuda")
        op.hd_vcycle(torch.from_numpy(r).cuda(), zz)
        torch.cuda.synchronize()
        z[e] = zz.cpu().numpy()
    ref = bp.vc._cycle(0, r)
    assert close(z[2], ref, 1e-12) <= 1e-12
    assert close(z[2], z[1], 1e-12) <= 1e-12
    assert not np.array_equal(z[2], z[1])  # the double-float path really ran
    b = np.random.Generator(np.random.PCG64(42)).uniform(-1, 1, prob.n)
    b[prob.ess] = 0.0
    if bp.singular:
        b[prob.lat.n_rt:] -= b[prob.lat.n_rt:].mean()
    its, xs = {}, {}
    for e, op in ops.items():
        x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
        st, info = op.hd_minres_solve(torch.from_numpy(b).cuda(), x, rtol=1e-8, maxit=3000, check_every=4)
        assert st == 0, (e, info)
        its[e], xs[e] = info["iterations"], x.cpu().numpy()
        op.close()
    assert abs(its[2] - its[1]) <= 1, its
    assert np.linalg.norm(xs[2] - xs[1]) <= 1e-8 * np.linalg.norm(xs[1])


def test_fp64_emulation_values_are_checked():
    import paper_2304_12387_gb300 as hd
    d = inputs("c1")
    with pytest.raises(hd.HdError) as e:
        gpu_operator(d, fp64_emulation=3)
    assert e.value.status == hd.HD_ERR_INVALID_ARG
    with pytest.raises(hd.HdError) as e:
        gpu_operator(d, fp64_emulation=2, winv_mode=hd.HD_WINV_CG)
    assert e.value.status == hd.HD_ERR_NOT_IMPLEMENTED

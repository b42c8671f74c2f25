"""Failure detection with faults injected on the host.

A NaN in the right-hand side or an Inf in the initial guess must end MINRES
(plain and with FP64 residual correction) and GMRES with HD_ERR_NAN instead of
iterating on garbage, and must leave the handle usable: a clean solve on the same
handle afterwards gives bit for bit the solution of a fresh handle (the solvers
are deterministic). Nothing here faults, traps or stalls the GPU: the recurrence
scalars and the residual norms carry the NaN to a status word that the host reads."""
import numpy as np
import pytest

from cases import gpu_operator, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rhs(n, seed):
    return torch.from_numpy(np.random.Generator(np.random.PCG64(seed)).uniform(-1, 1, n)).cuda()


def _clean_solve(op, solver, b):
    x = torch.zeros_like(b)
    st, _ = solver(op)(b, x)
    torch.cuda.synchronize()
    return st, x.cpu().numpy()


SOLVERS = {
    "minres": lambda op: (lambda b, x, **kw: op.hd_minres_solve(b, x, rtol=1e-8, maxit=2000, check_every=4, **kw)),
    "minres_refined": lambda op: (lambda b, x, **kw: op.hd_minres_solve(b, x, rtol=1e-4, maxit=4000, precision=1,
                                                                        outer_rtol=1e-8, max_outer=20, **kw)),
    "gmres": lambda op: (lambda b, x, **kw: op.hd_gmres_solve(b, x, rtol=1e-8, maxit=400, restart=16, **kw)),
}


@pytest.mark.parametrize("solver", sorted(SOLVERS))
@pytest.mark.parametrize("fault", ["nan_rhs", "inf_x0"])
def test_injected_non_finite_values_are_reported(solver, fault):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_12387_gb300 as hd
    d = inputs("darcy_gamma")
    op = gpu_operator(d, coarse_max=8)
    b = _rhs(op.n, 40)
    bad_b = b.clone()
    x0 = torch.zeros_like(b)
    if fault == "nan_rhs":
        bad_b[op.n // 3] = float("nan")
        st, info = SOLVERS[solver](op)(bad_b, x0)
    else:
        x0[7] = float("inf")
        st, info = SOLVERS[solver](op)(b, x0, use_x0=True)
    torch.cuda.synchronize()
    assert st == hd.HD_ERR_NAN, (solver, fault, st, info)
    assert info["status"] == hd.HD_ERR_NAN
    # the handle still works, and gives what a fresh handle gives
    st1, x1 = _clean_solve(op, SOLVERS[solver], b)
    fresh = gpu_operator(d, coarse_max=8)
    st2, x2 = _clean_solve(fresh, SOLVERS[solver], b)
    assert st1 == hd.HD_OK and st2 == hd.HD_OK
    assert np.array_equal(x1, x2)
    op.close()
    fresh.close()


def test_corrupted_learned_network_falls_back_to_the_vcycle():
    """NaN weights injected into the learned Schur preconditioner: MINRES detects the
    breakdown, solves again with the V-cycle and reports the fallback; the solution is
    the plain solver's."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_12387_gb300 as hd
    d = inputs("darcy_k3")
    op = gpu_operator(d, coarse_max=8)
    op.hd_learned_init(delta=1e-3)
    W1, W2 = op.hd_learned_get_weights()
    W1[3, 5] = np.nan
    op.hd_learned_set_weights(W1, W2)
    op.hd_enable_learned(1)
    b = _rhs(op.n, 41)
    x = torch.zeros_like(b)
    st, info = op.hd_minres_solve(b, x, rtol=1e-8, maxit=3000, check_every=4)
    torch.cuda.synchronize()
    assert st == hd.HD_OK and info["fallback"] == 1, info
    plain = gpu_operator(d, coarse_max=8)
    st2, x2 = _clean_solve(plain, lambda o: (lambda bb, xx: o.hd_minres_solve(bb, xx, rtol=1e-8, maxit=3000,
                                                                               check_every=4)), b)
    assert st2 == hd.HD_OK
    xn = x.cpu().numpy()
    assert np.abs(xn - x2).max() <= 1e-12 * np.abs(x2).max()
    op.close()
    plain.close()


@pytest.mark.parametrize("affine", [False, True])
def test_double_float_refuses_element_data_outside_its_range(affine):
    """The double-float element kernel holds FP64 data to ~48 bits only inside FP32's
    exponent range: hd_create must refuse fp64_emulation = 1 when an element's largest
    geometric factor (beta = 1e-35 makes them ~1e-35 < 2^-60) or its largest entry of
    C = W^-1/alpha (alpha = 1e40) leaves [2^-60, 2^60], and the FP64 kernel must still
    take the same problem."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_12387_gb300 as hd
    import synth
    from oracle.assembly import GRAD_DIV, Problem
    n, k = 2, 2
    vx, vy, vz = synth.lattice_vertices(n, n, n, perturb=0.0 if affine else 0.1)
    for alpha, beta in ((1.0, 1e-35), (1e40, 1.0)):
        kw = dict(kind=hd.HD_GRAD_DIV, ess_mask=0, q=k + 1 if affine else k + 2, affine=affine, coarse_max=8)
        with pytest.raises(hd.HdError) as err:
            hd.Operator(n, n, n, k, vx, vy, vz, alpha, beta, fp64_emulation=1, **kw)
        assert err.value.status == hd.HD_ERR_INVALID_ARG
        op = hd.Operator(n, n, n, k, vx, vy, vz, alpha, beta, fp64_emulation=0, **kw)
        prob = Problem(n, n, n, k, vx, vy, vz, alpha, beta, kind=GRAD_DIV, ess_mask=0, q=kw["q"])
        x = np.random.Generator(np.random.PCG64(5)).uniform(-1, 1, prob.n)
        y = torch.empty(prob.n, dtype=torch.float64, device="cuda")
        op.hd_apply_op(torch.from_numpy(x).cuda(), y)
        ref = prob.apply_op(x)
        yu, ru = y.cpu().numpy()[:prob.lat.n_rt], ref[:prob.lat.n_rt]
        yq, rq = y.cpu().numpy()[prob.lat.n_rt:], ref[prob.lat.n_rt:]
        assert np.abs(yu - ru).max() <= 1e-12 * np.abs(ru).max()
        assert np.abs(yq - rq).max() <= 1e-12 * np.abs(rq).max()
        op.close()

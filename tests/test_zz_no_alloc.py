"""The allocation-free MINRES entry point against the allocating one.

hd_minres_solve_noalloc serves callers that may not allocate device memory once
their handle exists (for instance a host code with a fixed device memory budget
after initialisation): it takes its work space from a fixed device array in the
library instead of cudaMalloc and runs the V/W-cycle without CUDA graphs. This
test calls it through the C ABI twice in a row on a FRESH handle that has never
run hd_minres_solve, checking that the device's free memory is unchanged across
each call (the very first one included), then compares each result with
hd_minres_solve on the same input, at the tolerance of the other MINRES tests
(solutions within 1e-8 relative, same iteration count). The second call starts
from the first call's leftover scratch contents. It also checks the documented
refusals: a problem above the size limit, the outer residual-correction loop and
a handle with the learned Schur preconditioner enabled.
Kept in a file of its own that pytest collects last.
"""
import numpy as np
import pytest

from cases import gpu_operator, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,smooth_levels", [("darcy_k3", 0), ("gd_k4_ragged", 2)])
def test_noalloc_minres_allocates_nothing_and_matches_the_allocating_solver(name, smooth_levels):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = inputs(name)
    op = gpu_operator(d, coarse_max=8, cycle=2, smooth_levels=smooth_levels)
    rng = np.random.Generator(np.random.PCG64(21))
    bs = [torch.from_numpy(rng.uniform(-1, 1, op.n)).cuda() for _ in range(2)]
    xs = [torch.full((op.n,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(2)]
    results = []
    for b, x in zip(bs, xs):
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        st, info = op.hd_minres_solve_noalloc(b, x, rtol=1e-8, maxit=2000, check_every=4)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free_before
        results.append((st, info))
    for b, x, (st, info) in zip(bs, xs, results):
        x_ref = torch.zeros(op.n, dtype=torch.float64, device="cuda")
        st_ref, info_ref = op.hd_minres_solve(b, x_ref, rtol=1e-8, maxit=2000, check_every=4)
        assert st_ref == 0 and st == 0, (st_ref, st, info)
        assert info["iterations"] == info_ref["iterations"]
        xr, xn = x_ref.cpu().numpy(), x.cpu().numpy()
        assert np.linalg.norm(xn - xr) <= 1e-8 * np.linalg.norm(xr)
        assert abs(info["true_relres"] - info_ref["true_relres"]) <= 1e-8
    op.close()


def test_noalloc_refuses_what_it_does_not_compute():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_12387_gb300 as hd
    op = gpu_operator(inputs("darcy_k3"), coarse_max=8)
    b = torch.ones(op.n, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    st, _ = op.hd_minres_solve_noalloc(b, x, max_outer=3, outer_rtol=1e-8)
    assert st == hd.HD_ERR_NOT_IMPLEMENTED
    op.hd_learned_init()
    op.hd_set_schur_prec(1)
    st, _ = op.hd_minres_solve_noalloc(b, x)
    assert st == hd.HD_ERR_NOT_IMPLEMENTED
    assert "learned" in hd.lib().hd_last_error(op.h).decode()
    op.close()


def test_noalloc_rejects_problems_above_the_limit():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_12387_gb300 as hd
    import synth
    n = 13  # 13^3 elements at k = 3: 182,520 RT + 59,319 L2 = 241,839 DOFs, above the limit
    vx, vy, vz = synth.lattice_vertices(n, n, n)
    op = hd.Operator(n, n, n, 3, vx, vy, vz, 1.0, 1.0, kind=hd.HD_GRAD_DIV, ess_mask=63, affine=True)
    assert op.n > 209696
    b = torch.zeros(op.n, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    st, _ = op.hd_minres_solve_noalloc(b, x)
    assert st == hd.HD_ERR_INVALID_ARG
    assert "exceed" in hd.lib().hd_last_error(op.h).decode()
    op.close()

"""The allocation-free MINRES entry point against the allocating one.

hd_minres_solve_noalloc serves callers that may not allocate device memory once
their handle exists (for instance a host code with a fixed device memory budget
after initialisation): it takes its work space from a fixed device array in the
library instead of cudaMalloc. This test calls it through the C ABI twice in a
row (the second call starts from the first call's leftover scratch contents) and
compares each result with hd_minres_solve on the same input, at the tolerance of
the other MINRES tests (solutions within 1e-8 relative, same iteration count).
It also checks that a problem above the documented size limit is rejected.
Kept in a file of its own that pytest collects last.
"""
import numpy as np
import pytest

from cases import gpu_operator, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_minres_matches_allocating_solver_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = inputs("darcy_k3")
    op = gpu_operator(d, coarse_max=8)
    rng = np.random.Generator(np.random.PCG64(21))
    free_before = None
    for call in range(2):
        b = torch.from_numpy(rng.uniform(-1, 1, op.n)).cuda()
        x_ref = torch.zeros(op.n, dtype=torch.float64, device="cuda")
        st_ref, info_ref = op.hd_minres_solve(b, x_ref, rtol=1e-8, maxit=2000, check_every=4)
        x = torch.full((op.n,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        if call == 1:
            free_before = torch.cuda.mem_get_info()[0]
        st, info = op.hd_minres_solve_noalloc(b, x, rtol=1e-8, maxit=2000, check_every=4)
        torch.cuda.synchronize()
        if call == 1:
            assert torch.cuda.mem_get_info()[0] == free_before
        assert st_ref == 0 and st == 0, (st_ref, st, info)
        assert info["iterations"] == info_ref["iterations"]
        xr, xn = x_ref.cpu().numpy(), x.cpu().numpy()
        assert np.linalg.norm(xn - xr) <= 1e-8 * np.linalg.norm(xr)
        assert abs(info["true_relres"] - info_ref["true_relres"]) <= 1e-8
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

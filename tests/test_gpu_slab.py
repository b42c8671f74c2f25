"""In-process z-slab partition on one GPU (hd_apply_op_partitioned,
hd_minres_solve_partitioned).

Every partition applies its element layers to its own buffers, NaN outside its owned
and halo entries, with the halo values and interface sums exchanged by device copies:
the block apply must equal the unpartitioned apply bit for bit (each interface face
sums exactly two addends) for P = 2, 3, 4 (ragged slabs included), in FP64 and in
double-float. MINRES through the partition, with every inner product summed per
partition then over the partitions, must take the unpartitioned solve's iteration
count (within one) and reach its solution within 1e-10 (the sums associate
differently, so the iterates agree to rounding, not bit for bit)."""
import numpy as np
import pytest

from cases import gpu_operator, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("emul", [0, 1])
@pytest.mark.parametrize("name,parts", [("gd_tall", (2, 3, 4)), ("gd_k4_ragged", (2, 3)), ("darcy_k3", (2, 3)),
                                        ("darcy_neumann", (2,))])
def test_partitioned_apply_is_bitwise_the_apply(name, parts, emul):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = inputs(name)
    op = gpu_operator(d, coarse_max=8, fp64_emulation=emul)
    x = torch.from_numpy(np.random.Generator(np.random.PCG64(81)).uniform(-1, 1, op.n)).cuda()
    y = torch.empty_like(x)
    op.hd_apply_op(x, y)
    for P in parts:
        yp = torch.full_like(x, float("nan"))
        op.hd_apply_op_partitioned(P, x, yp)
        torch.cuda.synchronize()
        assert torch.equal(yp, y), (P, float((yp - y).abs().max()))
    op.close()


@pytest.mark.parametrize("name,P", [("gd_tall", 4), ("gd_k4_ragged", 3), ("darcy_neumann", 2)])
def test_partitioned_minres_matches_the_solve(name, P):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = inputs(name)
    op = gpu_operator(d, coarse_max=8, cycle=2, smooth_levels=1)
    b = np.random.Generator(np.random.PCG64(82)).uniform(-1, 1, op.n)
    b[op.hd_get_ess_dofs()] = 0.0
    if name == "darcy_neumann":
        b[op.n_rt:] -= b[op.n_rt:].mean()
    b = torch.from_numpy(b).cuda()
    x = torch.zeros_like(b)
    st, info = op.hd_minres_solve(b, x, rtol=1e-10, maxit=3000, check_every=4)
    xp = torch.zeros_like(b)
    stp, infop = op.hd_minres_solve_partitioned(P, b, xp, rtol=1e-10, maxit=3000, check_every=4)
    assert st == 0 and stp == 0, (st, stp)
    assert abs(info["iterations"] - infop["iterations"]) <= 1, (info, infop)
    assert float(torch.linalg.vector_norm(xp - x) / torch.linalg.vector_norm(x)) <= 1e-10
    assert infop["true_relres"] <= 1e-8
    op.close()

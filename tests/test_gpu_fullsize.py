"""Parity at full size: the fused block apply of every workload at its full size
(the metric workload in the launch configuration bench.py times) against the
oracle's element-local rows, on a seeded sample of RT rows (including essential
rows) and L2 rows. Tolerance: |gpu - oracle| <= 1e-12 * max over the sampled
oracle rows (norm-scaled, FP64)."""
import numpy as np
import pytest

from cases import fullsize

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["m64", "c2", "c3", "c4", "c5"])
def test_fullsize_sampled_rows(name):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_12387_gb300 as hd
    from oracle.sampled import SampledOperator
    d = fullsize(name)
    op = hd.Operator(d["nx"], d["ny"], d["nz"], d["k"], d["vx"], d["vy"], d["vz"], d["coef0"], d["coef1"],
                     kind=d["kind"], ess_mask=d["ess_mask"], q=d["q"], affine=d["affine"],
                     stream=torch.cuda.current_stream())
    rng = np.random.Generator(np.random.PCG64(77))
    x = rng.uniform(-1, 1, op.n)
    xd = torch.from_numpy(x).cuda()
    y = torch.empty_like(xd)
    op.hd_apply_op(xd, y)
    torch.cuda.synchronize()
    so = SampledOperator(d["nx"], d["ny"], d["nz"], d["k"], d["vx"], d["vy"], d["vz"], d["coef0"], d["coef1"],
                         kind=d["kind"], ess_mask=d["ess_mask"], q=d["q"])
    rt = rng.choice(op.n_rt, 24, replace=False)
    if len(so.ess):
        rt = np.concatenate([rt, so.ess[rng.choice(len(so.ess), 3, replace=False)]])
    # rows on the last element layer and the first: ragged ends of the element loop
    rt = np.concatenate([rt, [0, op.n_rt - 1]])
    l2 = np.concatenate([rng.choice(op.n_l2, 12, replace=False), [0, op.n_l2 - 1]])
    ref_rt = so.rt_rows(x, rt)
    ref_l2 = so.l2_rows(x, l2)
    got = y[torch.from_numpy(np.concatenate([rt, op.n_rt + l2])).cuda()].cpu().numpy()
    ref = np.concatenate([ref_rt, ref_l2])
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-12 * scale, (name, np.abs(got - ref).max() / scale)
    op.close()


@pytest.mark.parametrize("name", ["m64", "c4"])
def test_fullsize_m64_fp64_emulation(name):
    """The metric workload (and the affine bent-tube workload, which takes the affine fast
    path) with the double-float element kernel, sampled rows at 1e-12."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_12387_gb300 as hd
    from oracle.sampled import SampledOperator
    d = fullsize(name)
    op = hd.Operator(d["nx"], d["ny"], d["nz"], d["k"], d["vx"], d["vy"], d["vz"], d["coef0"], d["coef1"],
                     kind=d["kind"], ess_mask=d["ess_mask"], q=d["q"], affine=d["affine"], fp64_emulation=1,
                     stream=torch.cuda.current_stream())
    rng = np.random.Generator(np.random.PCG64(78))
    x = rng.uniform(-1, 1, op.n)
    xd = torch.from_numpy(x).cuda()
    y = torch.empty_like(xd)
    op.hd_apply_op(xd, y)
    torch.cuda.synchronize()
    so = SampledOperator(d["nx"], d["ny"], d["nz"], d["k"], d["vx"], d["vy"], d["vz"], d["coef0"], d["coef1"],
                         kind=d["kind"], ess_mask=d["ess_mask"], q=d["q"])
    rt = np.concatenate([rng.choice(op.n_rt, 16, replace=False), so.ess[:2], [0, op.n_rt - 1]])
    l2 = np.concatenate([rng.choice(op.n_l2, 8, replace=False), [0, op.n_l2 - 1]])
    ref = np.concatenate([so.rt_rows(x, rt), so.l2_rows(x, l2)])
    got = y[torch.from_numpy(np.concatenate([rt, op.n_rt + l2])).cuda()].cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    op.close()


def test_fullsize_m64_smoothed_hierarchy():
    """The metric workload with the bench's preconditioner (smoothed aggregation,
    W-cycle): the cycles with one and two smoothed levels are symmetric and positive
    at full size, and FP64 MINRES reaches a true relative residual of 1e-8 in fewer
    iterations than with the plain-aggregation W-cycle, and fewer again with the
    second level smoothed."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_12387_gb300 as hd
    d = fullsize("m64")
    its = {}
    for sl in (2, 1, 0):
        op = hd.Operator(d["nx"], d["ny"], d["nz"], d["k"], d["vx"], d["vy"], d["vz"], d["coef0"], d["coef1"],
                         kind=d["kind"], ess_mask=d["ess_mask"], q=d["q"], affine=d["affine"], fp64_emulation=1,
                         cycle=2, smooth_levels=sl, stream=torch.cuda.current_stream())
        if sl >= 1:
            g = torch.Generator(device="cuda").manual_seed(79)
            x = torch.rand(op.n_l2, dtype=torch.float64, device="cuda", generator=g) - 0.5
            y = torch.rand(op.n_l2, dtype=torch.float64, device="cuda", generator=g) - 0.5
            vx, vy = torch.empty_like(x), torch.empty_like(y)
            op.hd_vcycle(x, vx)
            op.hd_vcycle(y, vy)
            a, b = float(x @ vy), float(y @ vx)
            # symmetry of the cycle at 16.8 M cells: the two inner products round differently
            # (about sqrt(n) u of the product of the norms); a parity bar does not apply here
            assert abs(a - b) <= 1e-11 * float(torch.linalg.vector_norm(x) * torch.linalg.vector_norm(vy))
            assert float(x @ vx) > 0
        rhs = torch.from_numpy(np.random.Generator(np.random.PCG64(80)).uniform(-1, 1, op.n)).cuda()
        rhs[torch.from_numpy(op.hd_get_ess_dofs()).cuda()] = 0.0
        sol = torch.zeros_like(rhs)
        st, info = op.hd_minres_solve(rhs, sol, rtol=1e-8, maxit=5000, check_every=16, outer_rtol=1e-8,
                                      max_outer=10)
        assert st == 0 and info["true_relres"] <= 1e-8, info
        its[sl] = info["iterations"]
        op.close()
    assert its[1] < 0.8 * its[0], its
    assert its[2] < 0.9 * its[1], its


def test_fullsize_m64_gmres():
    """The metric workload with block-triangular GMRES (FP64 with the double-float basis,
    and mixed precision): both reach a true relative residual of 1e-8, their solutions
    agree with FP64 MINRES's, and they need fewer than half its steps."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_12387_gb300 as hd
    d = fullsize("m64")
    op = hd.Operator(d["nx"], d["ny"], d["nz"], d["k"], d["vx"], d["vy"], d["vz"], d["coef0"], d["coef1"],
                     kind=d["kind"], ess_mask=d["ess_mask"], q=d["q"], affine=d["affine"], fp64_emulation=1,
                     cycle=2, smooth_levels=2, stream=torch.cuda.current_stream())
    rhs = torch.from_numpy(np.random.Generator(np.random.PCG64(81)).uniform(-1, 1, op.n)).cuda()
    rhs[torch.from_numpy(op.hd_get_ess_dofs()).cuda()] = 0.0
    xm = torch.zeros_like(rhs)
    st, mi = op.hd_minres_solve(rhs, xm, rtol=1e-8, maxit=5000, check_every=16, outer_rtol=1e-8, max_outer=10)
    assert st == 0
    for prec in (0, 1):
        x = torch.zeros_like(rhs)
        st, gi = op.hd_gmres_solve(rhs, x, rtol=1e-8, maxit=2000, restart=32, prec=hd.HD_GMRES_BLOCK_TRI,
                                   precision=prec, inner_rtol=1e-3)
        assert st == 0 and gi["true_relres"] <= 1e-8, gi
        assert 2 * gi["iterations"] < mi["iterations"], (gi, mi)
        rel = float(torch.linalg.vector_norm(x - xm) / torch.linalg.vector_norm(xm))
        assert rel <= 1e-6, rel
    op.close()


@pytest.mark.parametrize("name,emul", [("m64", 0), ("m64", 1), ("c2", 0)])
def test_fullsize_every_element_layer(name, emul):
    """A strided sample through every element layer of the full-size workload: in each
    layer the z-face at its bottom and at its top, an x-face and a y-face inside it, and a
    cell of its first and of its last cell layer (random positions in x and y), against
    the oracle's rows at 1e-12 of the sampled maximum (FP64 and the double-float kernel)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_12387_gb300 as hd
    from oracle.sampled import SampledOperator
    d = fullsize(name)
    op = hd.Operator(d["nx"], d["ny"], d["nz"], d["k"], d["vx"], d["vy"], d["vz"], d["coef0"], d["coef1"],
                     kind=d["kind"], ess_mask=d["ess_mask"], q=d["q"], affine=d["affine"], fp64_emulation=emul,
                     stream=torch.cuda.current_stream())
    rng = np.random.Generator(np.random.PCG64(79))
    x = rng.uniform(-1, 1, op.n)
    xd = torch.from_numpy(x).cuda()
    y = torch.empty_like(xd)
    op.hd_apply_op(xd, y)
    torch.cuda.synchronize()
    so = SampledOperator(d["nx"], d["ny"], d["nz"], d["k"], d["vx"], d["vy"], d["vz"], d["coef0"], d["coef1"],
                         kind=d["kind"], ess_mask=d["ess_mask"], q=d["q"])
    k = d["k"]
    X, Y, Z = d["nx"] * k, d["ny"] * k, d["nz"] * k
    nxf, nyf = (X + 1) * Y * Z, X * (Y + 1) * Z
    rt, l2 = [], []
    for ez in range(d["nz"]):
        I, J = int(rng.integers(0, X)), int(rng.integers(0, Y))
        for K in (ez * k, ez * k + k):                       # z-faces at the layer's bottom and top
            rt.append(nxf + nyf + I + X * (J + Y * K))
        K = ez * k + int(rng.integers(0, k))
        rt.append(int(rng.integers(0, X + 1)) + (X + 1) * (J + Y * K))     # an x-face
        rt.append(nxf + I + X * (int(rng.integers(0, Y + 1)) + (Y + 1) * K))  # a y-face
        for K in (ez * k, ez * k + k - 1):                   # cells of the first and last cell layer
            l2.append(I + X * (J + Y * K))
    rt, l2 = np.array(rt), np.array(l2)
    ref = np.concatenate([so.rt_rows(x, rt), so.l2_rows(x, l2)])
    got = y[torch.from_numpy(np.concatenate([rt, op.n_rt + l2])).cuda()].cpu().numpy()
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-12 * scale, (name, emul, np.abs(got - ref).max() / scale)
    op.close()

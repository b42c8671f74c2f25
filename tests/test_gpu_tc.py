"""GPU parity of the tensor-core operator of affine meshes (hd_apply_op_tc).

The operator computes the RT mass as sum_ab G_ab K_ab on the tensor cores with
FP16-pair operands and FP32 accumulation, and D, D^T and C in FP32 on the CUDA
cores. Tolerance, derived from that arithmetic: every operand is held to about 2^-22
of the largest entry of its element component or block (FP16 pair after power-of-two
scaling), and each output sums at most 3 (k+1) k^2 <= 240 products in FP32, so the
result is within 2e-5 of the largest output entry (the worst-case bound is about
240 * 2^-24 = 1.4e-5 plus the operand terms; the typical error is ~1e-6). The same
bar is checked against the oracle on small meshes (ragged tiles, several tiles,
grad-div and Darcy with and without gamma, essential sides), against the FP64
affine kernel on meshes with more tiles than SMs and on the full 64^3 workload, and
for FP32 vectors. Applies are deterministic (two addends per shared face).
"""
import numpy as np
import pytest

from cases import close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TC_TOL = 2e-5
SHEAR = np.array([[1.0, 0.3, 0.1], [0.05, 0.8, 0.2], [0.1, -0.1, 1.2]])


def _mesh(nx, ny, nz, graded=True):
    """Graded lattice (x -> x^1.3 per axis) under a fixed shear: parallelepipeds."""
    import synth
    vx, vy, vz = synth.lattice_vertices(nx, ny, nz)
    P = np.stack([vx, vy, vz]) ** (1.3 if graded else 1.0)
    X = SHEAR @ P
    return X[0].copy(), X[1].copy(), X[2].copy()


def _operator(kind, dims, k, ess, c0, c1, vx, vy, vz, **kw):
    import paper_2304_12387_gb300 as hd
    nx, ny, nz = dims
    return hd.Operator(nx, ny, nz, k, vx, vy, vz, c0, c1, kind=kind, ess_mask=ess, q=k + 1, affine=True,
                       coarse_max=8, **kw)


# kind, dims, k, ess_mask, coefficients
CASES = {
    "gd_k4_ragged": (0, (3, 2, 3), 4, 5, "lognormal"),       # 18 elements: one partial tile
    "gd_k4_tiles": (0, (6, 5, 7), 4, 63, "lognormal"),       # 210 elements: two tiles, ragged tail
    "darcy_k3_gamma": (1, (5, 4, 9), 3, 12, "gamma"),        # 180 elements
    "darcy_k3_neumann": (1, (4, 4, 3), 3, 63, "darcy"),      # gamma = 0: C = 0
    "gd_k2": (0, (7, 6, 5), 2, 0, "lognormal"),              # natural BC, 210 elements
    "gd_k2_c1": (0, (4, 4, 4), 2, 63, "ones"),               # the C1 shape
}


def _coefs(recipe, E):
    import synth
    if recipe == "ones":
        return np.ones(E), np.ones(E)
    if recipe == "lognormal":
        return synth.lognormal(E, 1.0, seed=2305), synth.lognormal(E, 1.0, seed=2306)
    if recipe == "gamma":
        return synth.lognormal(E, 1.0, seed=2305), synth.lognormal(E, 1.0, seed=2307)
    return synth.lognormal(E, 2.0, seed=2305), np.zeros(E)


@pytest.mark.parametrize("name", sorted(CASES))
def test_tensor_core_operator_matches_oracle(name):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle.assembly import Problem
    kind, dims, k, ess, recipe = CASES[name]
    E = dims[0] * dims[1] * dims[2]
    vx, vy, vz = _mesh(*dims)
    c0, c1 = _coefs(recipe, E)
    prob = Problem(*dims, k, vx, vy, vz, c0, c1, kind=kind, ess_mask=ess, q=k + 1)
    op = _operator(kind, dims, k, ess, c0, c1, vx, vy, vz)
    rng = np.random.Generator(np.random.PCG64(31))
    x = rng.uniform(-1, 1, prob.n)
    ref = prob.apply_op(x)
    xd = torch.from_numpy(x).cuda()
    y1 = torch.empty_like(xd)
    y2 = torch.empty_like(xd)
    op.hd_apply_op_tc(xd, y1)
    op.hd_apply_op_tc(xd, y2)  # starts from the first apply's leftovers
    assert op.hd_tc_status() == 0
    yh = y1.cpu().numpy()
    assert close(yh, ref, TC_TOL) <= TC_TOL
    assert torch.equal(y1, y2)
    # essential rows are the constrained identity, bit for bit
    assert np.array_equal(yh[prob.ess], x[prob.ess])
    # FP32 vectors
    yf = torch.empty(prob.n, dtype=torch.float32, device="cuda")
    op.hd_apply_op_tc_f32(xd.float(), yf)
    assert close(yf.double().cpu().numpy(), ref, TC_TOL) <= TC_TOL
    op.close()


@pytest.mark.parametrize("n,k", [(28, 4), (40, 3), (48, 2)])
def test_tensor_core_operator_many_tiles_matches_fp64_affine_kernel(n, k):
    """More tiles than SMs (each persistent CTA loops over several tiles): against the
    FP64 affine fast path, itself parity-tested against the oracle at 1e-12."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import synth
    vx, vy, vz = _mesh(n, n, n)
    E = n ** 3
    c0, c1 = synth.lognormal(E, 2.0, seed=2311), synth.lognormal(E, 2.0, seed=2312)
    op = _operator(0, (n, n, n), k, 63, c0, c1, vx, vy, vz)
    assert (E + 127) // 128 > 152
    x = torch.from_numpy(synth.uniform(op.n, seed=2313)).cuda()
    y = torch.empty_like(x)
    yt = torch.empty_like(x)
    op.hd_apply_op(x, y)
    op.hd_apply_op_tc(x, yt)
    assert op.hd_tc_status() == 0
    assert close(yt.cpu().numpy(), y.cpu().numpy(), TC_TOL) <= TC_TOL
    op.close()


def test_tensor_core_operator_full_size_m64_affine():
    """The bench's affine workload (64^3 elements, k = 4, q = 5, beta = exp(2Z), u.n = 0)
    in the bench's launch configuration, against the FP64 affine kernel."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_12387_gb300 as hd
    import synth
    n = 64
    vx, vy, vz = synth.lattice_vertices(n, n, n)
    beta = synth.lognormal(n ** 3, 2.0, seed=2305)
    op = hd.Operator(n, n, n, 4, vx, vy, vz, np.ones(n ** 3), beta, kind=hd.HD_GRAD_DIV, ess_mask=63, q=5,
                     affine=True, fp64_emulation=1)
    x = torch.from_numpy(synth.uniform(op.n, seed=2304)).cuda()
    y = torch.empty_like(x)
    yt = torch.empty_like(x)
    op.hd_apply_op(x, y)
    op.hd_apply_op_tc(x, yt)
    assert op.hd_tc_status() == 0
    d = float((yt - y).abs().max() / y.abs().max())
    assert d <= TC_TOL, d
    op.close()


def test_tensor_core_operator_refusals():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_12387_gb300 as hd
    import synth
    # a perturbed mesh has no affine data
    vx, vy, vz = synth.lattice_vertices(3, 3, 3, perturb=0.1)
    op = hd.Operator(3, 3, 3, 3, vx, vy, vz, 1.0, 1.0, kind=hd.HD_GRAD_DIV, ess_mask=63, q=4, affine=True)
    x = torch.zeros(op.n, dtype=torch.float64, device="cuda")
    with pytest.raises(hd.HdError) as e:
        op.hd_apply_op_tc(x, torch.empty_like(x))
    assert e.value.status == hd.HD_ERR_NOT_IMPLEMENTED
    with pytest.raises(hd.HdError) as e:
        op.hd_set_inner_operator(1)
    assert e.value.status == hd.HD_ERR_NOT_IMPLEMENTED
    op.close()
    # k = 5 is not instantiated on the tensor cores
    vx, vy, vz = _mesh(2, 1, 1)
    op = _operator(0, (2, 1, 1), 5, 3, np.ones(2), np.ones(2), vx, vy, vz)
    x = torch.zeros(op.n, dtype=torch.float64, device="cuda")
    with pytest.raises(hd.HdError) as e:
        op.hd_apply_op_tc(x, torch.empty_like(x))
    assert e.value.status == hd.HD_ERR_NOT_IMPLEMENTED
    op.close()


@pytest.mark.parametrize("solver", ["minres", "gmres"])
def test_mixed_solve_with_tensor_core_inner_operator_reaches_fp64_solution(solver):
    """Mixed-precision solves with the tensor-core inner operator (FP64 residual
    correction outside) reach the true relative residual 1e-8 and the FP64 solution."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_12387_gb300 as hd
    import synth
    n, k = 12, 4
    vx, vy, vz = _mesh(n, n, n, graded=False)
    inside = synth.bent_tube_mask(n, n, n)
    alpha, beta = np.where(inside, 1e3, 1.0), np.where(inside, 1.0, 1e-3)
    op = _operator(0, (n, n, n), k, 63, alpha, beta, vx, vy, vz, cycle=2, smooth_levels=2)
    b = torch.from_numpy(synth.uniform(op.n, seed=2321)).cuda()
    b[torch.from_numpy(op.hd_get_ess_dofs()).cuda()] = 0.0
    x64 = torch.zeros_like(b)
    if solver == "minres":
        st, info = op.hd_minres_solve(b, x64, rtol=1e-10, maxit=5000, check_every=8, outer_rtol=1e-10, max_outer=5)
    else:
        st, info = op.hd_gmres_solve(b, x64, rtol=1e-10, maxit=2000, restart=32)
    assert st == 0
    op.hd_set_inner_operator(1)
    xm = torch.zeros_like(b)
    if solver == "minres":
        st, info = op.hd_minres_solve(b, xm, rtol=1e-4, maxit=5000, check_every=8, precision=1, outer_rtol=1e-8,
                                      max_outer=20)
    else:
        st, info = op.hd_gmres_solve(b, xm, rtol=1e-8, maxit=2000, restart=32, precision=1, inner_rtol=1e-3)
    assert st == 0 and info["true_relres"] <= 1e-8, info
    assert op.hd_tc_status() == 0
    # the two solutions differ by at most cond(AA) times their residuals (1e-8 and 1e-10);
    # with the tube's 10^6 coefficient contrast that is ~1e-6 here
    rel = float(torch.linalg.vector_norm(xm - x64) / torch.linalg.vector_norm(x64))
    assert rel <= 1e-5, rel
    op.close()

"""GPU parity: every block of the CUDA operator and preconditioner against the
FP64 oracle on the same seeded inputs (small meshes that span several CTA
batches and ragged tails). Tolerance for FP64 results: componentwise
|gpu - oracle| <= 1e-12 * max|oracle| (norm-scaled relative error)."""
import numpy as np
import pytest

from cases import CASES, close, gpu_operator, inputs, oracle_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-12


@pytest.fixture(scope="module", params=sorted(CASES))
def pair(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = inputs(request.param)
    prob = oracle_problem(d)
    op = gpu_operator(d, coarse_max=8)
    yield request.param, d, prob, op
    op.close()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def test_sizes(pair):
    _, _, prob, op = pair
    assert (op.n_rt, op.n_l2) == (prob.lat.n_rt, prob.lat.n_l2)


def test_maps(pair):
    _, _, prob, op = pair
    assert np.array_equal(op.hd_get_e2d_map().astype(np.int64), prob.e2d)
    assert np.array_equal(op.hd_get_ess_dofs(), prob.ess)


def test_apply_op(pair):
    name, _, prob, op = pair
    x = np.random.Generator(np.random.PCG64(1)).uniform(-1, 1, prob.n)
    y = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    op.hd_apply_op(_dev(x), y)
    assert close(_host(y), prob.apply_op(x), RTOL) <= RTOL, name


def test_apply_op_host_buffers(pair):
    _, _, prob, op = pair
    x = np.random.Generator(np.random.PCG64(2)).uniform(-1, 1, prob.n)
    y = np.zeros(prob.n)
    op.hd_apply_op_host(x, y)
    assert close(y, prob.apply_op(x), RTOL) <= RTOL


@pytest.mark.parametrize("emulation", [0, 1])
def test_apply_op_host_pipelined_is_bitwise_the_device_apply(pair, emulation):
    """The host-buffer apply runs slab by slab with the copies overlapped; each shared
    face still receives exactly two addends on zero, so the result equals the
    device apply bit for bit (pinned and pageable host buffers)."""
    name, d, prob, op = pair
    if emulation:
        op = gpu_operator(d, coarse_max=8, fp64_emulation=1)
    x = np.random.Generator(np.random.PCG64(5)).uniform(-1, 1, prob.n)
    yd = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    op.hd_apply_op(_dev(x), yd)
    ref = _host(yd)
    xp = torch.from_numpy(x).pin_memory()
    yp = torch.full((prob.n,), float("nan"), dtype=torch.float64).pin_memory()
    op.hd_apply_op_host(xp, yp)
    assert np.array_equal(yp.numpy(), ref), name
    yq = np.full(prob.n, np.nan)
    op.hd_apply_op_host(x, yq)
    assert np.array_equal(yq, ref), name
    if emulation:
        op.close()


def test_apply_A(pair):
    _, _, prob, op = pair
    u = np.random.Generator(np.random.PCG64(3)).uniform(-1, 1, prob.lat.n_rt)
    y = torch.empty(prob.lat.n_rt, dtype=torch.float64, device="cuda")
    op.hd_apply_A(_dev(u), y)
    assert close(_host(y), prob.apply_A(u), RTOL) <= RTOL


def test_apply_B_Bt_exact(pair):
    """D and D^T are +-1 stencils: sums of at most 6 terms, compared tightly."""
    _, _, prob, op = pair
    rng = np.random.Generator(np.random.PCG64(4))
    u = rng.uniform(-1, 1, prob.lat.n_rt)
    q = rng.uniform(-1, 1, prob.lat.n_l2)
    yq = torch.empty(prob.lat.n_l2, dtype=torch.float64, device="cuda")
    yu = torch.empty(prob.lat.n_rt, dtype=torch.float64, device="cuda")
    op.hd_apply_B(_dev(u), yq)
    op.hd_apply_Bt(_dev(q), yu)
    assert close(_host(yq), prob.apply_B(u), 1e-15) <= 1e-15
    assert close(_host(yu), prob.apply_Bt(q), 1e-15) <= 1e-15


def test_apply_C(pair):
    _, _, prob, op = pair
    q = np.random.Generator(np.random.PCG64(5)).uniform(-1, 1, prob.lat.n_l2)
    y = torch.empty(prob.lat.n_l2, dtype=torch.float64, device="cuda")
    op.hd_apply_C(_dev(q), y)
    ref = prob.apply_C(q)
    if np.abs(ref).max() == 0:
        assert np.abs(_host(y)).max() == 0
    else:
        assert close(_host(y), ref, RTOL) <= RTOL


def test_preconditioner_diagonals(pair):
    from oracle.precond import approx_schur
    _, _, prob, op = pair
    S, Mt, Ct = approx_schur(prob)
    mt = torch.empty(prob.lat.n_rt, dtype=torch.float64, device="cuda")
    ct = torch.empty(prob.lat.n_l2, dtype=torch.float64, device="cuda")
    op.hd_get_diagonals(mt, ct)
    assert close(_host(mt), Mt, RTOL) <= RTOL
    if np.abs(Ct).max() == 0:
        assert np.abs(_host(ct)).max() == 0
    else:
        assert close(_host(ct), Ct, RTOL) <= RTOL


def test_schur_stencil(pair):
    from oracle.precond import approx_schur
    _, _, prob, op = pair
    S, _, _ = approx_schur(prob)
    x = np.random.Generator(np.random.PCG64(6)).uniform(-1, 1, prob.lat.n_l2)
    y = torch.empty(prob.lat.n_l2, dtype=torch.float64, device="cuda")
    op.hd_apply_schur(_dev(x), y)
    assert close(_host(y), S @ x, RTOL) <= RTOL


def test_vcycle_and_levels(pair):
    from oracle.precond import BlockPrec
    _, _, prob, op = pair
    bp = BlockPrec(prob, nu=2, coarse_max=8)
    nl, dims0 = op.hd_get_level(0)
    assert nl == bp.vc.n_levels
    for l in range(nl):
        assert op.hd_get_level(l)[1] == bp.vc.dims[l]
    b = np.random.Generator(np.random.PCG64(7)).uniform(-1, 1, prob.lat.n_l2)
    x = torch.empty(prob.lat.n_l2, dtype=torch.float64, device="cuda")
    op.hd_vcycle(_dev(b), x)
    ref = bp.vc._cycle(0, b)
    assert close(_host(x), ref, 1e-12) <= 1e-12


def test_apply_prec(pair):
    from oracle.precond import BlockPrec
    _, _, prob, op = pair
    bp = BlockPrec(prob, nu=2, coarse_max=8)
    r = np.random.Generator(np.random.PCG64(8)).uniform(-1, 1, prob.n)
    z = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    op.hd_apply_prec(_dev(r), z)
    zr = bp.apply(r)
    zg = _host(z)
    nrt = prob.lat.n_rt
    assert close(zg[:nrt], zr[:nrt], RTOL) <= RTOL
    assert close(zg[nrt:], zr[nrt:], 1e-12) <= 1e-12


def test_f32_operator_close(pair):
    """FP32 inner operator: same result to single-precision accuracy."""
    _, _, prob, op = pair
    x = np.random.Generator(np.random.PCG64(9)).uniform(-1, 1, prob.n)
    y = torch.empty(prob.n, dtype=torch.float32, device="cuda")
    op.hd_apply_op_f32(torch.from_numpy(x.astype(np.float32)).cuda(), y)
    assert close(_host(y).astype(np.float64), prob.apply_op(x), 1e-4) <= 1e-4


@pytest.mark.parametrize("basis", ["gl", "hist", "chol"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_local_cg_winv_mode(name, basis):
    """W^-1 by the fused local CG in the Gauss-Legendre nodal basis (the paper's
    matrix-free method, Sec. 2.5 and 3.1), in the histopolation basis itself (the
    comparison of Sec. 3.1), or by per-element Cholesky factors (the factorisation
    approach of Sec. 3.1), instead of stored dense inverses: same operator to 1e-12."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_12387_gb300 as hd
    from oracle.precond import approx_schur
    d = inputs(name)
    prob = oracle_problem(d)
    op = gpu_operator(d, coarse_max=8, winv_mode={"gl": hd.HD_WINV_CG, "hist": hd.HD_WINV_CG_HIST,
                                                  "chol": hd.HD_WINV_CHOL}[basis])
    rng = np.random.Generator(np.random.PCG64(15))
    x = rng.uniform(-1, 1, prob.n)
    y = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    op.hd_apply_op(_dev(x), y)
    assert close(_host(y), prob.apply_op(x), RTOL) <= RTOL
    q = rng.uniform(-1, 1, prob.lat.n_l2)
    yc = torch.empty(prob.lat.n_l2, dtype=torch.float64, device="cuda")
    op.hd_apply_C(_dev(q), yc)
    ref = prob.apply_C(q)
    if np.abs(ref).max() > 0:
        assert close(_host(yc), ref, RTOL) <= RTOL
    _, _, Ct = approx_schur(prob)
    mt = torch.empty(prob.lat.n_rt, dtype=torch.float64, device="cuda")
    ct = torch.empty(prob.lat.n_l2, dtype=torch.float64, device="cuda")
    op.hd_get_diagonals(mt, ct)
    if np.abs(Ct).max() > 0:
        assert close(_host(ct), Ct, RTOL) <= RTOL
    op.close()


@pytest.mark.parametrize("name", sorted(CASES))
def test_fp64_emulation_mode(name):
    """Element kernel in double-float arithmetic (FP32 pairs on the FP32 pipe) with
    FP64 vectors in and out: the same FP64 parity bar as the native kernel."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = inputs(name)
    prob = oracle_problem(d)
    op = gpu_operator(d, coarse_max=8, fp64_emulation=1)
    rng = np.random.Generator(np.random.PCG64(16))
    x = rng.uniform(-1, 1, prob.n)
    y = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    op.hd_apply_op(_dev(x), y)
    assert close(_host(y), prob.apply_op(x), RTOL) <= RTOL
    u = rng.uniform(-1, 1, prob.lat.n_rt)
    ya = torch.empty(prob.lat.n_rt, dtype=torch.float64, device="cuda")
    op.hd_apply_A(_dev(u), ya)
    assert close(_host(ya), prob.apply_A(u), RTOL) <= RTOL
    q = rng.uniform(-1, 1, prob.lat.n_l2)
    yc = torch.empty(prob.lat.n_l2, dtype=torch.float64, device="cuda")
    op.hd_apply_C(_dev(q), yc)
    ref = prob.apply_C(q)
    if np.abs(ref).max() > 0:
        assert close(_host(yc), ref, RTOL) <= RTOL
    op.close()

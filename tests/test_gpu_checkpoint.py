"""MINRES checkpoints and learned-network files through the C ABI.

A plain FP64 solve stopped at its iteration cap keeps its recurrence on the handle;
continuing it (directly, or after writing it to a file and reading it back) runs the
same kernels on the same state, so the iterate equals the one of an uninterrupted
solve bit for bit and the iteration count is the same. Files of another problem,
truncated or foreign files, and resumes the recurrence cannot serve are refused."""
import numpy as np
import pytest

from cases import gpu_operator, inputs, oracle_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _setup(name="gd_k4_ragged"):
    d = inputs(name)
    prob = oracle_problem(d)
    b = np.random.Generator(np.random.PCG64(51)).uniform(-1, 1, prob.n)
    b[prob.ess] = 0.0
    return d, prob, torch.from_numpy(b).cuda()


def _full(op, b):
    x = torch.zeros_like(b)
    st, info = op.hd_minres_solve(b, x, rtol=1e-10, maxit=2000, check_every=4)
    assert st == 0, info
    return x, info["iterations"]


def test_resume_from_file_is_bitwise_identical(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_12387_gb300 as hd
    d, prob, b = _setup()
    op = gpu_operator(d, coarse_max=8)
    x_full, its = _full(op, b)
    assert its >= 8
    x = torch.zeros_like(b)
    half = its // 2
    st, info = op.hd_minres_solve(b, x, rtol=1e-10, maxit=half, check_every=4)
    assert st == hd.HD_ERR_NOT_CONVERGED and info["iterations"] == half
    path = tmp_path / "minres.ckpt"
    assert op.hd_checkpoint_minres(path) == 0
    assert path.stat().st_size > 6 * 8 * prob.n
    # another solve replaces the kept recurrence
    x2 = torch.zeros_like(b)
    assert op.hd_minres_solve(-b, x2, rtol=1e-6, maxit=2000)[0] == 0
    assert op.hd_checkpoint_minres(tmp_path / "none.ckpt") == hd.HD_ERR_INVALID_ARG
    assert op.hd_minres_solve(b, x2, rtol=1e-10, maxit=10, resume=True)[0] == hd.HD_ERR_INVALID_ARG
    # read it back: the solve continues from the stored iterate, whatever x holds
    assert op.hd_resume_minres(path) == 0
    x3 = torch.full_like(b, 7.0)
    st, info = op.hd_minres_solve(b, x3, rtol=1e-10, maxit=2000, check_every=4, resume=True)
    assert st == 0 and info["iterations"] == its, (info, its)
    assert torch.equal(x3, x_full)
    op.close()


def test_chained_resumes_on_the_handle():
    """Stop, continue and stop again, then finish: same iterate as one solve."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_12387_gb300 as hd
    d, prob, b = _setup("darcy_k3")
    op = gpu_operator(d, coarse_max=8)
    x_full, its = _full(op, b)
    third = max(1, its // 3)
    x = torch.zeros_like(b)
    st, info = op.hd_minres_solve(b, x, rtol=1e-10, maxit=third, check_every=3)
    assert st == hd.HD_ERR_NOT_CONVERGED and info["iterations"] == third
    st, info = op.hd_minres_solve(b, x, rtol=1e-10, maxit=third, check_every=3, resume=True)
    assert st == hd.HD_ERR_NOT_CONVERGED and info["iterations"] == 2 * third
    st, info = op.hd_minres_solve(b, x, rtol=1e-10, maxit=2000, check_every=3, resume=True)
    assert st == 0 and info["iterations"] == its
    assert torch.equal(x, x_full)
    op.close()


def test_resume_in_a_new_handle(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_12387_gb300 as hd
    d, prob, b = _setup()
    op = gpu_operator(d, coarse_max=8)
    x = torch.zeros_like(b)
    _, its = _full(op, b)
    st, _ = op.hd_minres_solve(b, x, rtol=1e-10, maxit=its // 2, check_every=4)
    assert st == hd.HD_ERR_NOT_CONVERGED
    path = tmp_path / "minres.ckpt"
    assert op.hd_checkpoint_minres(path) == 0
    op.close()
    op2 = gpu_operator(d, coarse_max=8)
    x_full, its2 = _full(op2, b)
    assert its2 == its
    assert op2.hd_resume_minres(path) == 0
    x2 = torch.zeros_like(b)
    st, info = op2.hd_minres_solve(b, x2, rtol=1e-10, maxit=2000, check_every=4, resume=True)
    assert st == 0 and info["iterations"] == its
    assert float((x2 - x_full).norm()) <= 1e-12 * float(x_full.norm())
    op2.close()


def test_checkpoint_errors(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_12387_gb300 as hd
    d, prob, b = _setup()
    op = gpu_operator(d, coarse_max=8)
    x = torch.zeros_like(b)
    assert op.hd_checkpoint_minres(tmp_path / "a.ckpt") == hd.HD_ERR_INVALID_ARG   # nothing kept
    assert op.hd_resume_minres(tmp_path / "missing.ckpt") == hd.HD_ERR_INVALID_ARG
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(b"not a checkpoint" * 8)
    assert op.hd_resume_minres(bad) == hd.HD_ERR_INVALID_ARG
    st, _ = op.hd_minres_solve(b, x, rtol=1e-10, maxit=5)
    assert st == hd.HD_ERR_NOT_CONVERGED
    good = tmp_path / "good.ckpt"
    assert op.hd_checkpoint_minres(good) == 0
    # only the plain FP64 recurrence resumes; the refused call keeps the state
    assert op.hd_minres_solve(b, x, rtol=1e-10, maxit=5, precision=1, resume=True)[0] == hd.HD_ERR_NOT_IMPLEMENTED
    assert op.hd_minres_solve(b, x, rtol=1e-10, maxit=5, max_outer=3, resume=True)[0] == hd.HD_ERR_NOT_IMPLEMENTED
    st, info = op.hd_minres_solve(b, x, rtol=1e-10, maxit=5, resume=True)
    assert st == hd.HD_ERR_NOT_CONVERGED and info["iterations"] == 10
    # truncated, or of another problem size: refused, and nothing is kept afterwards
    data = good.read_bytes()
    cut = tmp_path / "cut.ckpt"
    cut.write_bytes(data[:-8])
    assert op.hd_resume_minres(cut) == hd.HD_ERR_INVALID_ARG
    assert op.hd_minres_solve(b, x, rtol=1e-10, maxit=5, resume=True)[0] == hd.HD_ERR_INVALID_ARG
    d2 = inputs("darcy_k3")
    op2 = gpu_operator(d2, coarse_max=8)
    assert op2.hd_resume_minres(good) == hd.HD_ERR_INVALID_ARG
    long = tmp_path / "long.ckpt"
    long.write_bytes(data + b"\0")
    assert op.hd_resume_minres(long) == hd.HD_ERR_INVALID_ARG
    assert op.hd_resume_minres(good) == 0
    op2.close()
    op.close()


def test_learned_network_file_round_trip(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_12387_gb300 as hd
    d = inputs("darcy_k3")
    op = gpu_operator(d, coarse_max=8)
    path = tmp_path / "net.bin"
    assert op.hd_learned_save(path) == hd.HD_ERR_INVALID_ARG          # no network yet
    with pytest.raises(RuntimeError):
        op.hd_enable_learned(True)
    op.hd_learned_init(seed=5, delta=2e-3)
    W1, W2 = op.hd_learned_get_weights()
    assert op.hd_learned_save(path) == 0
    r = torch.from_numpy(np.random.Generator(np.random.PCG64(3)).uniform(-1, 1, op.n_l2)).cuda()
    z1 = torch.zeros_like(r)
    op.hd_learned_apply(r, z1)
    op2 = gpu_operator(d, coarse_max=8)
    assert op2.hd_learned_load(path) == 0
    V1, V2 = op2.hd_learned_get_weights()
    assert np.array_equal(V1, W1) and np.array_equal(V2, W2)
    z2 = torch.zeros_like(r)
    op2.hd_learned_apply(r, z2)
    assert torch.equal(z1, z2)
    op2.hd_enable_learned(True)
    op2.hd_enable_learned(False)
    assert op2.hd_learned_load(tmp_path / "missing.bin") == hd.HD_ERR_INVALID_ARG
    cut = tmp_path / "cut.bin"
    cut.write_bytes(path.read_bytes()[:-4])
    assert op2.hd_learned_load(cut) == hd.HD_ERR_INVALID_ARG
    op2.close()
    op.close()

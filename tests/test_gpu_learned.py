"""GPU learned Schur preconditioner against the FP64 reference (oracle.conv).

The GPU network computes in FP16 (activations and weights) with FP32
accumulation, so it is compared with the reference evaluated on the same
FP16-rounded weights, at a norm-scaled tolerance of 2e-2 for outputs and 5e-2
for gradients (FP16 carries 11 significant bits; each output sums 27 x 32
terms per layer over four layers). The coarse correction is FP64 (1e-12)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from cases import close, gpu_operator, inputs, oracle_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DELTA = 1e-3


def _setup(name):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle.precond import BlockPrec
    d = inputs(name)
    prob = oracle_problem(d)
    op = gpu_operator(d, coarse_max=8)
    bp = BlockPrec(prob, coarse_max=8)
    return d, prob, op, bp


def _Q(bp, r):
    if bp.vc.n_levels < 2:
        return np.zeros_like(r)
    return bp.vc.P[0] @ bp.vc._cycle(1, bp.vc.P[0].T @ r)


def _f16(W):
    return W.astype(np.float32).astype(np.float16).astype(np.float64)


def _dims(prob):
    return (prob.lat.X, prob.lat.Y, prob.lat.Z)


@pytest.mark.parametrize("name", ["darcy_k3", "gd_k4_ragged", "darcy_neumann"])
def test_net_apply_matches_reference(name):
    from oracle import conv
    d, prob, op, bp = _setup(name)
    W1, W2 = conv.init_weights(32, seed=5)
    op.hd_learned_init(delta=DELTA)
    op.hd_learned_set_weights(W1, W2)
    r = np.random.Generator(np.random.PCG64(6)).uniform(-1, 1, prob.lat.n_l2)
    z = torch.empty(prob.lat.n_l2, dtype=torch.float64, device="cuda")
    op.hd_learned_apply(torch.from_numpy(r).cuda(), z)
    ref = conv.apply_net(_f16(W1), _f16(W2), r, bp.S.diagonal(), _dims(prob), DELTA)
    torch.cuda.synchronize()
    assert close(z.cpu().numpy(), ref, 2e-2) <= 2e-2
    op.close()


@pytest.mark.parametrize("name", ["darcy_k3", "gd_k4_ragged"])
def test_coarse_correction_matches_reference(name):
    _, prob, op, bp = _setup(name)
    r = np.random.Generator(np.random.PCG64(7)).uniform(-1, 1, prob.lat.n_l2)
    z = torch.empty(prob.lat.n_l2, dtype=torch.float64, device="cuda")
    op.hd_coarse_correction(torch.from_numpy(r).cuda(), z)
    torch.cuda.synchronize()
    assert close(z.cpu().numpy(), _Q(bp, r), 1e-12) <= 1e-12
    op.close()


def test_gradient_matches_reference():
    from oracle import conv
    _, prob, op, bp = _setup("darcy_k3")
    W1, W2 = conv.init_weights(32, seed=8)
    op.hd_learned_init(delta=DELTA)
    op.hd_learned_set_weights(W1, W2)
    rng = np.random.Generator(np.random.PCG64(9))
    S = bp.S.tocsc()
    pairs = []
    for _ in range(2):
        r = rng.uniform(-1, 1, prob.lat.n_l2)
        pairs.append((r, spla.spsolve(S, r), _Q(bp, r)))
    R = torch.from_numpy(np.stack([p[0] for p in pairs])).cuda()
    E = torch.from_numpy(np.stack([p[1] for p in pairs])).cuda()
    QR = torch.from_numpy(np.stack([p[2] for p in pairs])).cuda()
    loss, g1, g2 = op.hd_learned_grad(R, E, QR)
    W1r, W2r = _f16(W1), _f16(W2)
    Lref = conv.loss(W1r, W2r, pairs, bp.S, bp.S.diagonal(), _dims(prob), DELTA)
    r1, r2 = conv.grad(W1r, W2r, pairs, bp.S, bp.S.diagonal(), _dims(prob), DELTA)
    assert abs(loss - Lref) <= 2e-2 * abs(Lref)
    assert close(g1, r1, 5e-2) <= 5e-2
    assert close(g2, r2, 5e-2) <= 5e-2
    op.close()


def test_training_lowers_loss_and_preconditioner_stays_spd():
    _, prob, op, bp = _setup("darcy_k3")
    op.hd_learned_init(delta=DELTA)
    info = op.hd_learned_train(npairs=6, capture_every=3, steps=40, lr=3e-3)
    assert info["pairs"] == 6
    assert info["loss_final"] < info["loss_initial"], info
    op.hd_set_schur_prec(1)
    rng = np.random.Generator(np.random.PCG64(10))
    a, b = (torch.from_numpy(rng.uniform(-1, 1, prob.n)).cuda() for _ in range(2))
    Pa, Pb = torch.empty_like(a), torch.empty_like(b)
    op.hd_apply_prec(a, Pa)
    op.hd_apply_prec(b, Pb)
    torch.cuda.synchronize()
    ab, ba = float(Pa @ b), float(a @ Pb)
    assert abs(ab - ba) <= 1e-2 * max(abs(ab), abs(ba))
    assert float(a @ Pa) > 0
    rhs = rng.uniform(-1, 1, prob.n)
    x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    st, sol = op.hd_minres_solve(torch.from_numpy(rhs).cuda(), x, rtol=1e-8, maxit=3000, check_every=4)
    assert st == 0 and sol["fallback"] == 0, sol
    assert sol["true_relres"] < 1e-5
    op.close()

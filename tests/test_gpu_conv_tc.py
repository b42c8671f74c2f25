"""The learned network's 32 -> 32 convolutions on the tcgen05 tensor cores (the default
engine) against the mma.sync engine and the FP64 reference (oracle.conv).

Both engines take FP16 activations and weights and accumulate in FP32. They differ only
in the order of the FP32 sums and so agree to FP16 rounding of the layer outputs: 5e-3
of the largest entry after the four layers (norm-scaled). Against the reference on the
same FP16-rounded weights the bar is that of the network tests, 2e-2 for the apply and
5e-2 for the gradient. Lattices: small ones (a tile shorter than the line of 128 cells)
and a 150-cell line with 2 tiles per line, the second one ragged, so that the halo's
zero fill at both ends of a line, at the y and z faces and past the ragged end are all
reached."""
import numpy as np
import pytest

import synth
from cases import close, gpu_operator, inputs, oracle_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DELTA = 1e-3


def _long_line():
    nx, ny, nz = 50, 2, 2
    vx, vy, vz = synth.lattice_vertices(nx, ny, nz, perturb=0.1, seed=91)
    E = nx * ny * nz
    from oracle.assembly import DARCY
    return dict(kind=DARCY, nx=nx, ny=ny, nz=nz, k=3, q=5, vx=vx, vy=vy, vz=vz,
                coef0=synth.lognormal(E, 1.0, seed=92), coef1=np.zeros(E), ess_mask=0, affine=False)


def _case(name):
    return _long_line() if name == "long_line" else inputs(name)


def _f16(W):
    return W.astype(np.float32).astype(np.float16).astype(np.float64)


@pytest.mark.parametrize("name", ["long_line", "darcy_k3", "gd_k4_ragged"])
def test_tensor_core_convolution_matches_mma_sync_and_reference(name):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import conv
    from oracle.precond import BlockPrec
    d = _case(name)
    prob = oracle_problem(d)
    bp = BlockPrec(prob, coarse_max=8)
    op = gpu_operator(d, coarse_max=8)
    W1, W2 = conv.init_weights(32, seed=7)
    # three times the initial scale: the network term exceeds the delta term by about 1e6 and the
    # FP16 activations stay below 200 (a factor 30 overflows FP16 in both engines)
    W1, W2 = 3.0 * W1, 3.0 * W2
    op.hd_learned_init(delta=DELTA)
    op.hd_learned_set_weights(W1, W2)
    r = np.random.Generator(np.random.PCG64(8)).uniform(-1, 1, prob.lat.n_l2)
    rd = torch.from_numpy(r).cuda()
    z = {}
    for engine in (0, 1):
        op.hd_learned_conv_engine(engine)
        zz = torch.empty(prob.lat.n_l2, dtype=torch.float64, device="cuda")
        op.hd_learned_apply(rd, zz)
        torch.cuda.synchronize()
        z[engine] = zz.cpu().numpy()
    assert op.hd_tc_status() == 0
    assert close(z[0], z[1], 5e-3) <= 5e-3
    ref = conv.apply_net(_f16(W1), _f16(W2), r, bp.S.diagonal(), (prob.lat.X, prob.lat.Y, prob.lat.Z), DELTA)
    assert close(z[0], ref, 2e-2) <= 2e-2
    op.close()


def test_tensor_core_convolution_gradient_matches_reference():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import scipy.sparse.linalg as spla
    from oracle import conv
    from oracle.precond import BlockPrec
    d = _long_line()
    prob = oracle_problem(d)
    bp = BlockPrec(prob, coarse_max=8)
    op = gpu_operator(d, coarse_max=8)
    W1, W2 = conv.init_weights(32, seed=9)
    op.hd_learned_init(delta=DELTA)
    op.hd_learned_set_weights(W1, W2)
    op.hd_learned_conv_engine(0)
    rng = np.random.Generator(np.random.PCG64(10))
    S = bp.S.tocsc()
    pairs = []
    for _ in range(2):
        r = rng.uniform(-1, 1, prob.lat.n_l2)
        pairs.append((r, spla.spsolve(S, r), np.zeros_like(r)))
    R = torch.from_numpy(np.stack([p[0] for p in pairs])).cuda()
    E = torch.from_numpy(np.stack([p[1] for p in pairs])).cuda()
    QR = torch.from_numpy(np.stack([p[2] for p in pairs])).cuda()
    loss, g1, g2 = op.hd_learned_grad(R, E, QR)
    dims = (prob.lat.X, prob.lat.Y, prob.lat.Z)
    W1r, W2r = _f16(W1), _f16(W2)
    Lref = conv.loss(W1r, W2r, pairs, bp.S, bp.S.diagonal(), dims, DELTA)
    r1, r2 = conv.grad(W1r, W2r, pairs, bp.S, bp.S.diagonal(), dims, DELTA)
    assert abs(loss - Lref) <= 2e-2 * abs(Lref)
    assert close(g1, r1, 5e-2) <= 5e-2
    assert close(g2, r2, 5e-2) <= 5e-2
    assert op.hd_tc_status() == 0
    op.close()

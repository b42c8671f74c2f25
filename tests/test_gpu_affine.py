"""GPU parity of the affine fast path of the block apply.

A handle created with affine = 1, q = k+1 and the dense W^-1 on a mesh of
parallelepipeds keeps 8 values per element (the constant geometric factor and
det J) and applies W_e^-1 as det J (H^-1 x H^-1 x H^-1). Its applies must equal
the FP64 oracle's (full quadrature, dense per-element inverses) within the FP64
tolerance of the other parity tests, in FP64 and in double-float, and equal the
general kernel (per-point factors, stored inverses) on the same mesh. A mesh that
is flagged affine but is not must take the general path and still match."""
import numpy as np
import pytest

from cases import close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-12
SHEAR = np.array([[1.0, 0.3, 0.1], [0.05, 0.8, 0.2], [0.1, -0.1, 1.2]])


def _mesh(nx, ny, nz, perturb):
    """Graded lattice (x -> x^1.3 per axis) under a fixed shear: every element is a
    parallelepiped unless perturb > 0."""
    import synth
    vx, vy, vz = synth.lattice_vertices(nx, ny, nz, perturb=perturb, seed=2304)
    P = np.stack([vx, vy, vz]) ** 1.3 if perturb == 0 else np.stack([vx, vy, vz])
    X = SHEAR @ P
    return X[0].copy(), X[1].copy(), X[2].copy()


# kind, dims, k, ess_mask, perturb
CASES = [
    (0, (3, 2, 3), 4, 5, 0.0),     # grad-div k = 4, ragged element count (18)
    (1, (2, 3, 2), 3, 12, 0.0),    # Darcy with gamma > 0
    (0, (2, 2, 1), 2, 63, 0.0),
    (0, (1, 2, 1), 5, 3, 0.0),
    (0, (2, 2, 2), 3, 0, 0.1),     # flagged affine but perturbed: general path
]


@pytest.mark.parametrize("case", CASES, ids=["gd_k4", "darcy_k3_gamma", "gd_k2", "gd_k5", "perturbed_flagged"])
def test_affine_fast_path_matches_oracle_and_general_kernel(case):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_12387_gb300 as hd
    import synth
    from oracle.assembly import Problem
    kind, (nx, ny, nz), k, ess, perturb = case
    vx, vy, vz = _mesh(nx, ny, nz, perturb)
    E = nx * ny * nz
    c0 = synth.lognormal(E, 1.0, seed=2305)
    c1 = synth.lognormal(E, 1.0, seed=2306)
    q = k + 1
    prob = Problem(nx, ny, nz, k, vx, vy, vz, c0, c1, kind=kind, ess_mask=ess, q=q)
    x = np.random.Generator(np.random.PCG64(9)).uniform(-1, 1, prob.n)
    ref = prob.apply_op(x)
    xd = torch.from_numpy(x).cuda()
    outs = {}
    for affine in (True, False):
        for emul in (0, 1):
            op = hd.Operator(nx, ny, nz, k, vx, vy, vz, c0, c1, kind=kind, ess_mask=ess, q=q,
                             affine=affine, fp64_emulation=emul, coarse_max=8)
            y = torch.empty(prob.n, dtype=torch.float64, device="cuda")
            for _ in range(2):  # the second apply starts from the first one's leftovers
                op.hd_apply_op(xd, y)
            torch.cuda.synchronize()
            outs[affine, emul] = y.cpu().numpy()
            assert close(outs[affine, emul], ref, RTOL) <= RTOL, (affine, emul)
            op.close()
    for emul in (0, 1):
        assert close(outs[True, emul], outs[False, emul], 1e-13) <= 1e-13
    if perturb:
        assert np.array_equal(outs[True, 0], outs[False, 0])  # same (general) kernel

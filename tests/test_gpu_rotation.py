"""GPU parity with rotated elements (Algorithm 1's local orientations).

A handle created with element rotation codes must give the operator of the
oracle's problem with the same codes (element matrices in each element's own
frame, assembled through the rotated signed maps and Algorithm 1's D), within
the FP64 tolerance of the other parity tests, and must export the rotated maps
bit for bit. Codes outside 0..23 are rejected by hd_create."""
import numpy as np
import pytest

from cases import close, gpu_operator, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-12


def _rotated_pair(name, seed):
    from oracle.assembly import Problem
    d = inputs(name)
    E = d["nx"] * d["ny"] * d["nz"]
    rot = np.random.Generator(np.random.PCG64(seed)).integers(0, 24, E)
    prob = Problem(d["nx"], d["ny"], d["nz"], d["k"], d["vx"], d["vy"], d["vz"], d["coef0"], d["coef1"],
                   kind=d["kind"], ess_mask=d["ess_mask"], q=d["q"], rot=rot)
    op = gpu_operator(d, coarse_max=8, elem_rotation=rot)
    return d, rot, prob, op


@pytest.mark.parametrize("name", ["gd_k4_ragged", "darcy_gamma", "gd_k3"])
def test_rotated_elements_apply_matches_oracle(name):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d, rot, prob, op = _rotated_pair(name, 31)
    assert (prob.e2d < 0).any()
    rng = np.random.Generator(np.random.PCG64(3))
    x = rng.uniform(-1, 1, prob.n)
    y = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    op.hd_apply_op(torch.from_numpy(x).cuda(), y)
    torch.cuda.synchronize()
    assert close(y.cpu().numpy(), prob.apply_op(x), RTOL) <= RTOL
    u = rng.uniform(-1, 1, prob.lat.n_rt)
    yu = torch.empty(prob.lat.n_rt, dtype=torch.float64, device="cuda")
    op.hd_apply_A(torch.from_numpy(u).cuda(), yu)
    torch.cuda.synchronize()
    assert close(yu.cpu().numpy(), prob.apply_A(u), RTOL) <= RTOL
    assert np.array_equal(op.hd_get_e2d_map().astype(np.int64), prob.e2d)
    assert np.array_equal(op.hd_get_e2l_map().astype(np.int64), prob.e2l)
    op.close()


def test_bad_rotation_code_is_rejected_by_create():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_12387_gb300 as hd
    d = inputs("darcy_gamma")
    E = d["nx"] * d["ny"] * d["nz"]
    rot = np.zeros(E, dtype=np.int64)
    rot[E - 1] = 24
    with pytest.raises(hd.HdError) as err:
        gpu_operator(d, coarse_max=8, elem_rotation=rot)
    assert err.value.status == hd.HD_ERR_INVALID_ARG

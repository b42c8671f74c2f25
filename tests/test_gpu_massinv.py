"""DG mass inverse of any degree (hd_massinv_*, Sec. 3.1) against the oracle.

For k = 2..9 (the paper's p = 1..8) and each method (explicit inverse, Cholesky factor,
GL-basis CG, histopolation-basis CG), y = W^-1 x on a perturbed two-element mesh with
log-normal alpha must equal the per-element solve with the oracle's W_e (full quadrature,
q = k + 2) within 1e-12 of the largest entry. W_e in the histopolation basis has
condition numbers up to about 110 at k = 9, and the CG stops at a relative residual
of 1e-14, so every method lands far inside that bar. The GL-basis CG must need few
iterations at every degree (the basis is conditioned near 1, Sec. 2.5), fewer than
the histopolation-basis CG. The CG methods also run with their stages in double-float
(FP32 pairs, about 48 bits, unit roundoff ~3.6e-15): the GL-basis CG to the same 1e-12,
the histopolation-basis CG to 1e-11 (its Jacobi-scaled W has condition numbers up to
about 100, which multiply the double-float roundoff). Invalid input is refused on the
host."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

METHODS = ["dense", "chol", "cg", "cg_hist", "cg_df", "cg_hist_df"]


def _mesh(k):
    nx, ny, nz = 2, 1, 1
    vx, vy, vz = synth.lattice_vertices(nx, ny, nz, perturb=0.15, seed=40 + k)
    alpha = synth.lognormal(nx * ny * nz, 1.0, seed=50 + k)
    return (nx, ny, nz), (vx, vy, vz), alpha


def _reference(k, dims, v, alpha, x):
    from oracle.element import element_matrices, element_vertices
    from oracle.lattice import Lattice
    V = element_vertices(*dims, *v)
    W = element_matrices(V, k, k + 2, np.ones(len(alpha)), alpha, want=("W",))["W"]
    e2l = Lattice(*dims, k).e2l2_map()
    y = np.zeros_like(x)
    for e in range(len(alpha)):
        y[e2l[e]] = np.linalg.solve(W[e], x[e2l[e]])
    return y


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("k", [2, 3, 4, 5, 6, 7, 8, 9])
def test_mass_inverse_matches_oracle(k, method):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_12387_gb300 as hd
    m = {"dense": hd.HD_WINV_DENSE, "chol": hd.HD_WINV_CHOL, "cg": hd.HD_WINV_CG, "cg_hist": hd.HD_WINV_CG_HIST}
    df = method.endswith("_df")
    dims, v, alpha = _mesh(k)
    mi = hd.MassInverse(*dims, k, *v, alpha=alpha, method=m[method.replace("_df", "")], fp64_emulation=int(df))
    x = np.random.Generator(np.random.PCG64(60 + k)).uniform(-1, 1, mi.n_l2)
    y = torch.empty(mi.n_l2, dtype=torch.float64, device="cuda")
    mi.apply(torch.from_numpy(x).cuda(), y)
    torch.cuda.synchronize()
    ref = _reference(k, dims, v, alpha, x)
    err = np.abs(y.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err <= (1e-11 if method == "cg_hist_df" else 1e-12), err
    its = mi.iterations()
    if method in ("cg", "cg_df"):
        assert 1 <= its <= 20, its
    elif method in ("cg_hist", "cg_hist_df"):
        assert its >= 1, its
    else:
        assert its == 0
    assert mi.setup_ms() > 0.0
    mi.close()


def test_gl_basis_cg_needs_fewer_iterations_than_the_histopolation_basis():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_12387_gb300 as hd
    k = 7
    dims, v, alpha = _mesh(k)
    x = torch.from_numpy(np.random.Generator(np.random.PCG64(61)).uniform(-1, 1, 2 * k ** 3)).cuda()
    its = {}
    for name, method in (("gl", hd.HD_WINV_CG), ("hist", hd.HD_WINV_CG_HIST)):
        mi = hd.MassInverse(*dims, k, *v, alpha=alpha, method=method)
        y = torch.empty_like(x)
        mi.apply(x, y)
        its[name] = mi.iterations()
        mi.close()
    assert its["gl"] < its["hist"], its


def test_mass_inverse_refuses_invalid_input():
    import paper_2304_12387_gb300 as hd
    dims, v, alpha = _mesh(3)
    for kw in (dict(k=10), dict(k=1), dict(k=3, q=2), dict(k=3, method=7)):
        k = kw.pop("k")
        with pytest.raises(hd.HdError) as e:
            hd.MassInverse(*dims, k, *v, alpha=alpha, **kw)
        assert e.value.status == hd.HD_ERR_INVALID_ARG
    with pytest.raises(hd.HdError) as e:
        hd.MassInverse(*dims, 3, *v, alpha=-alpha)
    assert e.value.status == hd.HD_ERR_INVALID_ARG


def test_double_float_direct_methods_are_refused():
    import paper_2304_12387_gb300 as hd
    dims, v, alpha = _mesh(3)
    for method in (hd.HD_WINV_DENSE, hd.HD_WINV_CHOL):
        with pytest.raises(hd.HdError) as e:
            hd.MassInverse(*dims, 3, *v, alpha=alpha, method=method, fp64_emulation=1)
        assert e.value.status == hd.HD_ERR_NOT_IMPLEMENTED

"""Pins of the oracle's assembled operator, preconditioner and MINRES."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import synth
from oracle import manufactured
from oracle.assembly import DARCY, GRAD_DIV, Problem
from oracle.minres import minres
from oracle.precond import BlockPrec, VCycle, aggregation, approx_schur
from oracle.sampled import SampledOperator


def _prob(n=2, k=2, perturb=0.15, kind=GRAD_DIV, ess=63, seed=2304, gamma=None):
    vx, vy, vz = synth.lattice_vertices(n, n, n, perturb=perturb, seed=seed)
    E = n ** 3
    c0 = synth.lognormal(E, 1.0, seed=seed + 1)
    c1 = synth.lognormal(E, 1.0, seed=seed + 2) if gamma is None else gamma
    return Problem(n, n, n, k, vx, vy, vz, c0, c1, kind=kind, ess_mask=ess)


def test_operator_symmetric():
    p = _prob()
    A = p.matrix()
    assert abs(A - A.T).max() < 1e-13 * abs(A).max()


def test_D_two_entries_per_column_geometry_free():
    p1 = _prob(perturb=0.0)
    p2 = _prob(perturb=0.2)
    assert (p1.D_full != p2.D_full).nnz == 0
    g = _golden()
    nnz_col = np.diff(p1.D_full.tocsc().indptr)
    interior = np.ones(p1.lat.n_rt, dtype=bool)
    interior[p1.lat.ess_dofs(63)] = False
    assert np.all(nnz_col[interior] == int(g["D_nonzeros_per_column"]))
    assert np.all(nnz_col[~interior] == 1)             # a boundary face has one cell
    assert set(np.unique(p1.D_full.data).tolist()) == {float(v) for v in g["D_values"].split(",")}


def _golden():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.txt")
    out = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            name, val = line.split()[:2]
            out[name] = val
    return out


def test_golden_constants_are_closed_forms():
    g = _golden()
    assert np.isclose(float(g["prop1_neg_hi"]), (1 - np.sqrt(5)) / 2, rtol=1e-15)
    assert np.isclose(float(g["prop1_pos_hi"]), (1 + np.sqrt(5)) / 2, rtol=1e-15)
    assert abs(float(g["prop1_kappa"]) - (np.sqrt(5) + 1) / (np.sqrt(5) - 1)) < 1e-3


@pytest.mark.parametrize("tau,prop", [(1.0, "prop1"), (2.0, "prop2")])
def test_props_1_2_exact_block_preconditioner(tau, prop):
    """Prop. 1 (tau = 1) and Prop. 2 (tau = 2): eigenvalues of B^-1 AA with the exact
    blocks B = diag(tau M, S), S = C + D M^-1 D^T, lie in the printed intervals and
    the condition number is below the printed bound."""
    g = _golden()
    neg = (float(g[prop + "_neg_lo"]), float(g[prop + "_neg_hi"]))
    pos = (float(g[prop + "_pos_lo"]), float(g[prop + "_pos_hi"]))
    kappa = float(g[prop + "_kappa"])
    p = _prob(n=2, k=2)
    M = p.M.toarray()
    D = p.D.toarray()
    C = p.C.toarray()
    AA = p.matrix().toarray()
    S = C + D @ np.linalg.solve(M, D.T)
    B = sla.block_diag(tau * M, S)
    lam = sla.eigh(AA, B, eigvals_only=True)
    tol = 1e-10
    for l in lam:
        in_neg = neg[0] - tol <= l <= neg[1] + tol
        in_pos = pos[0] - tol <= l <= pos[1] + tol
        assert in_neg or in_pos, l
    assert np.any(lam < 0) and np.any(lam > 0)
    assert np.abs(lam).max() / np.abs(lam).min() <= kappa + 1e-3


def test_darcy_piecewise_constant_gamma_simplification():
    """W^-1 W_gamma W^-1 = W_{1/gamma}^-1 when gamma is constant per element (Sec. 2.4)."""
    n, k = 2, 2
    gamma = synth.lognormal(n ** 3, 1.0, seed=5)
    p = _prob(n=n, k=k, kind=DARCY, gamma=gamma)
    vx, vy, vz = synth.lattice_vertices(n, n, n, perturb=0.15, seed=2304)
    g = Problem(n, n, n, k, vx, vy, vz, 1.0 / gamma, 1.0, kind=GRAD_DIV, ess_mask=63)
    # grad-div with alpha = 1/gamma has (2,2) block W_{1/gamma}^-1
    assert np.allclose(p.C.toarray(), g.C.toarray(), atol=1e-12 * abs(g.C).max())


def test_darcy_zero_gamma_block_vanishes():
    p = _prob(kind=DARCY, gamma=np.zeros(8))
    assert abs(p.C).max() == 0.0


def test_approx_schur_entries_and_m_matrix():
    """Entries of S~ from Eq. approx-schur-entries; S~ is an M-matrix."""
    p = _prob(n=2, k=3)
    S, Mt, Ct = approx_schur(p)
    S = S.tocsr()
    lat = p.lat
    Sd = S.toarray()
    off = Sd - np.diag(np.diag(Sd))
    assert off.max() <= 0.0
    assert np.all(np.diag(Sd) > 0)
    assert np.all(Sd.sum(axis=1) >= -1e-12 * np.abs(Sd).max())
    # explicit entries: shared x-face between cells (I,J,K) and (I+1,J,K)
    for (I, J, K) in [(0, 0, 0), (2, 3, 1), (4, 5, 5)]:
        i, j = lat.cell(I, J, K), lat.cell(I + 1, J, K)
        f = lat.xface(I + 1, J, K)
        assert np.isclose(Sd[i, j], -1.0 / Mt[f], rtol=1e-14)
        faces = [lat.xface(I, J, K), lat.xface(I + 1, J, K), lat.yface(I, J, K), lat.yface(I, J + 1, K),
                 lat.zface(I, J, K), lat.zface(I, J, K + 1)]
        diag = Ct[i] + sum(1.0 / Mt[g] for g in faces if p.free[g])
        assert np.isclose(Sd[i, i], diag, rtol=1e-13)


def test_singular_schur_has_constant_kernel():
    p = _prob(kind=DARCY, gamma=np.zeros(8), ess=63)
    prec = BlockPrec(p)
    assert prec.singular
    assert np.abs(prec.S @ np.ones(p.lat.n_l2)).max() < 1e-12 * abs(prec.S).max()
    q = _prob(kind=DARCY, gamma=np.zeros(8), ess=62)
    assert not BlockPrec(q).singular


def test_galerkin_coarse_is_face_weight_sum():
    """P^T A P of a 7-point graph Laplacian + diagonal is again 7-point; each coarse
    face weight is the sum of the fine face weights across it."""
    rng = np.random.Generator(np.random.PCG64(1))
    dims = (5, 4, 3)
    X, Y, Z = dims
    n = X * Y * Z
    cell = lambda I, J, K: I + X * (J + Y * K)
    A = sp.lil_matrix((n, n))
    wx = rng.uniform(0.5, 2, (X + 1, Y, Z))
    mass = rng.uniform(0.1, 1, n)
    for i in range(n):
        A[i, i] += mass[i]
    for K in range(Z):
        for J in range(Y):
            for I in range(X - 1):
                a, b, w = cell(I, J, K), cell(I + 1, J, K), wx[I + 1, J, K]
                A[a, a] += w; A[b, b] += w; A[a, b] -= w; A[b, a] -= w
    P, cd = aggregation(dims)
    assert cd == (3, 2, 2)
    Ac = (P.T @ A.tocsr() @ P).toarray()
    cX, cY = cd[0], cd[1]
    ccell = lambda I, J, K: I + cX * (J + cY * K)
    # coarse x-face between coarse cells (0,0,0) and (1,0,0) = fine faces at I=2
    w = sum(wx[2, J, K] for J in range(2) for K in range(2))
    assert np.isclose(Ac[ccell(0, 0, 0), ccell(1, 0, 0)], -w)
    assert np.isclose(Ac[ccell(0, 0, 0), ccell(0, 1, 0)], 0.0)     # no y weights in this A
    assert np.isclose(Ac[ccell(0, 0, 0), ccell(1, 1, 0)], 0.0)


@pytest.mark.parametrize("singular", [False, True])
def test_vcycle_symmetric_positive(singular):
    p = _prob(n=4, k=2, kind=DARCY, gamma=np.zeros(64) if singular else np.ones(64), ess=63)
    prec = BlockPrec(p, nu=2, coarse_max=8)
    assert prec.vc.n_levels >= 3
    rng = np.random.Generator(np.random.PCG64(3))
    x, y = rng.standard_normal((2, p.lat.n_l2))
    if singular:
        x -= x.mean(); y -= y.mean()
    Vx, Vy = prec.vc.apply(x), prec.vc.apply(y)
    assert abs(x @ Vy - y @ Vx) < 1e-12 * np.linalg.norm(x) * np.linalg.norm(Vy)
    assert x @ Vx > 0


def test_vcycle_one_level_is_exact():
    p = _prob(n=2, k=2)
    prec = BlockPrec(p, coarse_max=10 ** 6)
    assert prec.vc.n_levels == 1
    r = np.random.Generator(np.random.PCG64(4)).standard_normal(p.lat.n_l2)
    z = prec.vc.apply(r)
    assert np.allclose(prec.S @ z, r, atol=1e-12)


@pytest.mark.parametrize("kind", [GRAD_DIV, DARCY])
def test_minres_matches_dense_solve(kind):
    p = _prob(n=2, k=2, kind=kind, ess=63 if kind == GRAD_DIV else 0)
    prec = BlockPrec(p, coarse_max=8)
    b = synth.uniform(p.n, seed=8)
    b[p.lat.n_rt:][:] = 0.0 if kind == GRAD_DIV else b[p.lat.n_rt:]
    x, info = minres(p.apply_op, prec.apply, b, rtol=1e-13, maxit=500)
    xd = np.linalg.solve(p.matrix().toarray(), b)
    assert info["converged"]
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)
    eta = np.array(info["eta"])
    assert np.all(np.diff(eta) <= 1e-12 * eta[0])        # MINRES residual is monotone


def test_manufactured_convergence_rate():
    """Grad-div with u = (s, s, s): L2 errors of u and div u fall like h^k (k = 2)."""
    errs = []
    for n in (2, 4, 8):
        vx, vy, vz = synth.lattice_vertices(n, n, n)
        p = Problem(n, n, n, 2, vx, vy, vz, 1.0, 1.0, kind=GRAD_DIV, ess_mask=63, affine=True)
        f = manufactured.rt_load(p, lambda X: manufactured.sinusoid_field(X)[2])
        f[~p.free] = 0.0
        b = np.concatenate([f, np.zeros(p.lat.n_l2)])
        x = sp.linalg.spsolve(p.matrix().tocsc(), b)
        u, qt = p.split(x)
        q = p.C @ qt
        errs.append(manufactured.l2_errors(p, u, q, manufactured.sinusoid_field))
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    assert np.all(rates[-1] > 1.8), rates


def test_manufactured_convergence_rate_k3():
    """The same field at k = 3: the errors fall like h^3 (2^3 -> 4^3 elements; a finer
    mesh is minutes of sparse direct solve)."""
    errs = []
    for n in (2, 4):
        vx, vy, vz = synth.lattice_vertices(n, n, n)
        p = Problem(n, n, n, 3, vx, vy, vz, 1.0, 1.0, kind=GRAD_DIV, ess_mask=63, affine=True)
        f = manufactured.rt_load(p, lambda X: manufactured.sinusoid_field(X)[2])
        f[~p.free] = 0.0
        b = np.concatenate([f, np.zeros(p.lat.n_l2)])
        x = sp.linalg.spsolve(p.matrix().tocsc(), b)
        u, qt = p.split(x)
        errs.append(manufactured.l2_errors(p, u, p.C @ qt, manufactured.sinusoid_field))
    rates = np.log2(np.array(errs[0]) / np.array(errs[1]))
    assert np.all(rates > 2.8), rates


def test_sampled_rows_match_assembled():
    n, k = 3, 2
    vx, vy, vz = synth.lattice_vertices(n, n, n, perturb=0.15)
    c0 = synth.lognormal(n ** 3, 1.0, seed=1)
    c1 = synth.lognormal(n ** 3, 1.0, seed=2)
    p = Problem(n, n, n, k, vx, vy, vz, c0, c1, ess_mask=5)
    s = SampledOperator(n, n, n, k, vx, vy, vz, c0, c1, ess_mask=5)
    x = synth.uniform(p.n, seed=3)
    y = p.apply_op(x)
    rng = np.random.Generator(np.random.PCG64(0))
    rt = np.concatenate([rng.choice(p.lat.n_rt, 25, replace=False), p.ess[:3]])
    l2 = rng.choice(p.lat.n_l2, 15, replace=False)
    assert np.allclose(s.rt_rows(x, rt), y[rt], rtol=1e-13, atol=1e-13)
    assert np.allclose(s.l2_rows(x, l2), y[p.lat.n_rt + l2], rtol=1e-13, atol=1e-13)

"""Pins of the oracle's element matrices (Sec. 2, Eq. matrices)."""
import numpy as np
import pytest

import synth
from oracle import basis1d, element
from oracle.lattice import Lattice


def _one_element(perturb, seed=7):
    """A single distorted hex: corners of the unit cube moved by U(-p, p)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    V = np.zeros((1, 2, 2, 2, 3))
    for c in range(2):
        for b in range(2):
            for a in range(2):
                V[0, c, b, a] = [a, b, c] + rng.uniform(-perturb, perturb, 3)
    return V


def _local_incidence(k):
    lat = Lattice(1, 1, 1, k)
    r, c, v = lat.divergence_incidence()
    D = np.zeros((lat.n_l2, lat.n_rt))
    D[r, c] = v
    # reorder columns from global face ids to element-local ids
    m = lat.e2d_map()[0]
    Dl = D[:, m]
    ml2 = lat.e2l2_map()[0]
    return Dl[ml2]


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_D_equals_Winv_B_on_distorted_element(k):
    """D = W_alpha^-1 B_alpha is the +-1 lattice incidence, independent of geometry
    and coefficient (Sec. 2.1 third property, Eq. transformed-system)."""
    V = _one_element(0.2)
    m = element.element_matrices(V, k, k + 3, np.array([1.0]), np.array([3.7]), want=("W", "B"))
    D = np.linalg.solve(m["W"][0], m["B"][0])
    Dref = _local_incidence(k)
    assert np.allclose(D, Dref, atol=1e-10)
    nz = np.abs(Dref) > 0.5
    assert np.all(nz.sum(axis=0)[(nz.sum(axis=0) > 0)] <= 2)
    assert set(np.unique(Dref)) <= {-1.0, 0.0, 1.0}


@pytest.mark.parametrize("k", [1, 2, 3])
def test_mass_symmetric_spd(k):
    V = _one_element(0.2, seed=3)
    M = element.element_matrices(V, k, k + 2, np.array([2.0]), np.array([1.0]), want=("M",))["M"][0]
    assert np.allclose(M, M.T, rtol=0, atol=1e-15 * np.abs(M).max())
    np.linalg.cholesky(M)


def _mass_1d(k, which):
    # 1D mass matrices with an independent 20-point Gauss rule
    t, w = np.polynomial.legendre.leggauss(20)
    x, w = 0.5 * (t + 1), 0.5 * w
    B = basis1d.interp_basis(k, x) if which == "I" else basis1d.histo_basis(k, x)
    return (B * w) @ B.T


def _mixed_1d(k):
    # C[i, j] = int l_i h_j with the same independent rule
    t, w = np.polynomial.legendre.leggauss(20)
    x, w = 0.5 * (t + 1), 0.5 * w
    return (basis1d.interp_basis(k, x) * w) @ basis1d.histo_basis(k, x).T


@pytest.mark.parametrize("k", [2, 3, 4])
def test_parallelepiped_closed_form(k):
    """On the image of the unit cube under x = A xi + t (J = A constant): every block of M
    is a Kronecker product of 1D matrices, M[(d, n), (d', n')] = G_dd' prod_c X_c with
    G = beta A^T A / det A and X_c = M_I, M_H or the mixed int l_i h_j along each axis
    (Piola map, Sec. 2); W = alpha / det A (M_H x M_H x M_H), so W^-1 = det A / alpha
    (M_H^-1 x M_H^-1 x M_H^-1): the forms the affine fast path of the GPU apply uses."""
    A = np.array([[0.9, 0.25, -0.1], [0.15, 1.2, 0.2], [-0.05, 0.3, 0.8]])
    t0 = np.array([0.3, -0.2, 0.5])
    V = np.zeros((1, 2, 2, 2, 3))
    for c in range(2):
        for b in range(2):
            for a in range(2):
                V[0, c, b, a] = A @ np.array([a, b, c]) + t0
    beta, alpha = 1.7, 0.6
    m = element.element_matrices(V, k, k + 1, np.array([beta]), np.array([alpha]), want=("M", "W"))
    det = np.linalg.det(A)
    G = beta * A.T @ A / det
    MI, MH, C = _mass_1d(k, "I"), _mass_1d(k, "H"), _mixed_1d(k)

    def axis_matrix(c, d, dp):
        if c == d and c == dp:
            return MI
        if c == d:
            return C
        if c == dp:
            return C.T
        return MH

    n1 = (k + 1) * k * k
    M = np.zeros((3 * n1, 3 * n1))
    for d in range(3):
        for dp in range(3):
            X = [axis_matrix(c, d, dp) for c in range(3)]
            M[d * n1:(d + 1) * n1, dp * n1:(dp + 1) * n1] = G[d, dp] * np.kron(X[2], np.kron(X[1], X[0]))
    assert np.abs(m["M"][0] - M).max() <= 1e-13 * np.abs(M).max()
    W = alpha / det * np.kron(MH, np.kron(MH, MH))
    assert np.abs(m["W"][0] - W).max() <= 1e-13 * np.abs(W).max()
    Hi = np.linalg.inv(MH)
    Winv = det / alpha * np.kron(Hi, np.kron(Hi, Hi))
    assert np.abs(np.linalg.inv(m["W"][0]) - Winv).max() <= 1e-12 * np.abs(Winv).max()


@pytest.mark.parametrize("k", [2, 3, 4])
def test_reference_mass_blocks_give_the_parallelepiped_mass(k):
    """M_e = sum_ab G_ab K_ab on a parallelepiped (the form of a batched, shared-matrix
    element contraction); the diagonal blocks K_aa are symmetric positive definite and
    K_ab = K_ba^T."""
    A = np.array([[1.1, -0.2, 0.15], [0.1, 0.7, 0.3], [0.2, 0.05, 0.9]])
    V = np.zeros((1, 2, 2, 2, 3))
    for c in range(2):
        for b in range(2):
            for a in range(2):
                V[0, c, b, a] = A @ np.array([a, b, c]) - 0.4
    beta = 2.3
    M = element.element_matrices(V, k, k + 1, np.array([beta]), np.array([1.0]), want=("M",))["M"][0]
    K = element.reference_mass_blocks(k, k + 1)
    G = beta * A.T @ A / np.linalg.det(A)
    Ms = np.einsum("ab,abnm->nm", G, K)
    assert np.abs(Ms - M).max() <= 1e-13 * np.abs(M).max()
    for a in range(3):
        assert np.all(np.linalg.eigvalsh(K[a, a]) > -1e-14)
        for b in range(3):
            assert np.allclose(K[a, b], K[b, a].T, atol=1e-15)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_cartesian_closed_form(k):
    """On a box hx x hy x hz: M_xx = beta hx/(hy hz) (M_I x M_H x M_H), no coupling
    between components; W = alpha/(hx hy hz) (M_H x M_H x M_H)."""
    hx, hy, hz = 0.7, 1.3, 0.4
    V = np.zeros((1, 2, 2, 2, 3))
    for c in range(2):
        for b in range(2):
            for a in range(2):
                V[0, c, b, a] = [a * hx, b * hy, c * hz]
    beta, alpha = 2.5, 0.3
    m = element.element_matrices(V, k, k + 1, np.array([beta]), np.array([alpha]), want=("M", "W"))
    MI, MH = _mass_1d(k, "I"), _mass_1d(k, "H")
    n1 = (k + 1) * k * k
    Mxx = beta * hx / (hy * hz) * np.kron(MH, np.kron(MH, MI))
    Myy = beta * hy / (hx * hz) * np.kron(MH, np.kron(MI, MH))
    Mzz = beta * hz / (hx * hy) * np.kron(MI, np.kron(MH, MH))
    M = m["M"][0]
    assert np.allclose(M[:n1, :n1], Mxx, atol=1e-13)
    assert np.allclose(M[n1:2 * n1, n1:2 * n1], Myy, atol=1e-13)
    assert np.allclose(M[2 * n1:, 2 * n1:], Mzz, atol=1e-13)
    assert np.allclose(M[:n1, n1:], 0, atol=1e-14)
    assert np.allclose(M[n1:2 * n1, 2 * n1:], 0, atol=1e-14)
    W = alpha / (hx * hy * hz) * np.kron(MH, np.kron(MH, MH))
    assert np.allclose(m["W"][0], W, atol=1e-13)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_rt_polynomial_reproduction(k):
    """A field in Q_{k,k-1,k-1} x ... is reproduced exactly from its subface fluxes
    (the RT dofs of Sec. 2.1) on the reference element."""
    rng = np.random.Generator(np.random.PCG64(11))
    ca = rng.standard_normal((k + 1, k, k))
    cb = rng.standard_normal((k, k + 1, k))
    cc = rng.standard_normal((k, k, k + 1))

    def field(x, y, z):
        ux = np.einsum("ijl,i...,j...,l...->...", ca, np.array([x ** i for i in range(k + 1)]),
                       np.array([y ** j for j in range(k)]), np.array([z ** l for l in range(k)]))
        uy = np.einsum("ijl,i...,j...,l...->...", cb, np.array([x ** i for i in range(k)]),
                       np.array([y ** j for j in range(k + 1)]), np.array([z ** l for l in range(k)]))
        uz = np.einsum("ijl,i...,j...,l...->...", cc, np.array([x ** i for i in range(k)]),
                       np.array([y ** j for j in range(k)]), np.array([z ** l for l in range(k + 1)]))
        return ux, uy, uz

    xi = basis1d.gll_nodes(k)
    t, w = np.polynomial.legendre.leggauss(k + 2)
    lat = Lattice(1, 1, 1, k)
    dofs = []
    for (d, i, j, l) in lat.local_rt():
        idx = [i, j, l]
        ranges = []
        for a in range(3):
            if a == d:
                ranges.append(None)
            else:
                lo, hi = xi[idx[a]], xi[idx[a] + 1]
                ranges.append((0.5 * (hi - lo) * t + 0.5 * (hi + lo), 0.5 * (hi - lo) * w))
        (p1, w1), (p2, w2) = [r for r in ranges if r is not None]
        P1, P2 = np.meshgrid(p1, p2, indexing="ij")
        W12 = np.outer(w1, w2)
        coords = [None, None, None]
        others = [a for a in range(3) if a != d]
        coords[d] = np.full(P1.shape, xi[idx[d]])
        coords[others[0]], coords[others[1]] = P1, P2
        dofs.append(np.sum(field(*coords)[d] * W12))
    dofs = np.array(dofs)
    pts = np.random.Generator(np.random.PCG64(5)).uniform(0, 1, (30, 3))
    Phi, _ = element.rt_basis(k, pts)
    uh = np.einsum("pnd,n->pd", Phi, dofs)
    ux, uy, uz = field(pts[:, 0], pts[:, 1], pts[:, 2])
    assert np.allclose(uh, np.stack([ux, uy, uz], axis=1), atol=1e-11)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_divdiv_equals_DtWD(k):
    """The Schur complement of the saddle-point matrix w.r.t. its (2,2) block is the
    H(div) matrix (Sec. 2): B^T W^-1 B = D^T W D equals the div-div matrix."""
    V = _one_element(0.15, seed=9)
    q = k + 3
    pts, w = element.quad_rule(q)
    J = element.jacobian(V, pts)
    detJ = np.linalg.det(J)[0]
    _, Div = element.rt_basis(k, pts)
    alpha = 1.9
    K = np.einsum("pn,p,pm->nm", Div, alpha * w / detJ, Div)
    m = element.element_matrices(V, k, q, np.array([1.0]), np.array([alpha]), want=("W", "B"))
    D = np.linalg.solve(m["W"][0], m["B"][0])
    assert np.allclose(D.T @ m["W"][0] @ D, K, atol=1e-11 * np.abs(K).max())


def test_gl_mass_diagonal_on_parallelepiped():
    """The L2 mass in the Gauss-Legendre nodal basis is diagonal when det J is
    constant (Sec. 2.5)."""
    k = 3
    A = np.array([[1.0, 0.3, 0.1], [0.2, 0.9, -0.2], [0.05, 0.1, 1.1]])
    V = np.zeros((1, 2, 2, 2, 3))
    for c in range(2):
        for b in range(2):
            for a in range(2):
                V[0, c, b, a] = A @ np.array([a, b, c])
    W = element.element_matrices(V, k, k + 2, np.array([1.0]), np.array([1.0]), want=("W",))["W"][0]
    g, _ = basis1d.gl_points(k)
    # S[j, m]: subcell integral j of the GL Lagrange polynomial m (GL nodal -> histopolation)
    xi = basis1d.gll_nodes(k)
    t, w = np.polynomial.legendre.leggauss(k + 2)
    S1 = np.zeros((k, k))
    for j in range(k):
        a, b = xi[j], xi[j + 1]
        x = 0.5 * (b - a) * t + 0.5 * (a + b)
        S1[j] = basis1d.lagrange(g, x) @ (0.5 * (b - a) * w)
    S = np.kron(S1, np.kron(S1, S1))
    WGL = S.T @ W @ S
    off = WGL - np.diag(np.diag(WGL))
    assert np.abs(off).max() < 1e-13 * np.abs(WGL).max()


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_gl_basis_is_better_conditioned_on_a_perturbed_element(k):
    """Sec. 3.1: the local CG changes to the Gauss-Legendre nodal basis because the
    Jacobi-scaled L2 mass is better conditioned there than in the histopolation basis
    (on a perturbed, non-affine element: close to 1 against several units)."""
    V = _one_element(0.15, seed=11)
    W = element.element_matrices(V, k, k + 2, np.array([1.0]), np.array([1.0]), want=("W",))["W"][0]
    g, _ = basis1d.gl_points(k)
    xi = basis1d.gll_nodes(k)
    t, w = np.polynomial.legendre.leggauss(k + 2)
    S1 = np.zeros((k, k))
    for j in range(k):
        a, b = xi[j], xi[j + 1]
        x = 0.5 * (b - a) * t + 0.5 * (a + b)
        S1[j] = basis1d.lagrange(g, x) @ (0.5 * (b - a) * w)
    S = np.kron(S1, np.kron(S1, S1))

    def scaled_cond(A):
        d = 1.0 / np.sqrt(np.diag(A))
        return np.linalg.cond(A * np.outer(d, d))

    k_hist, k_gl = scaled_cond(W), scaled_cond(S.T @ W @ S)
    assert k_gl < 1.5 < k_hist, (k_gl, k_hist)

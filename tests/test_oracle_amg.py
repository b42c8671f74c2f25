"""Pins of the oracle's smoothed-aggregation option of the Schur V-cycle.

The paper preconditions S~ with one AMG V-cycle and relies on its
mesh-independent convergence (Sec. 3.2, Sec. 4). The oracle's hierarchy is
geometric 2x2x2 aggregation; with smooth = omega the prolongator of the first
level is P = (I - omega D_l1^-1 A) P0 (smoothed aggregation). These tests pin
that construction with brute-force loops, algebraic identities and a
convergence check on lattice Laplacians with log-normal face weights."""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.precond import VCycle, aggregation

OMEGA = 4.0 / 3.0


def lattice_laplacian(dims, sigma=2.0, shift=1e-3, seed=0, singular=False):
    """7-point graph Laplacian on an X x Y x Z cell lattice with log-normal face
    weights, plus a small positive diagonal (none when singular)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    X, Y, Z = dims
    n = X * Y * Z
    cell = lambda I, J, K: I + X * (J + Y * K)
    rows, cols, vals = [], [], []
    diag = np.zeros(n) if singular else shift * rng.uniform(0.5, 1.5, n)
    for K, J, I in itertools.product(range(Z), range(Y), range(X)):
        a = cell(I, J, K)
        for d, (di, dj, dk) in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
            if I + di < X and J + dj < Y and K + dk < Z:
                b = cell(I + di, J + dj, K + dk)
                w = float(np.exp(sigma * rng.standard_normal()))
                rows += [a, b]; cols += [b, a]; vals += [-w, -w]
                diag[a] += w; diag[b] += w
    A = sp.coo_matrix((vals + list(diag), (rows + list(range(n)), cols + list(range(n)))), shape=(n, n))
    return A.tocsr()


def test_smoothed_prolongator_entries_brute_force():
    """P[i, C] = [i in C] - omega / D_l1[i] * sum_{j in C} A[i, j], by loops."""
    dims = (5, 4, 3)
    A = lattice_laplacian(dims, seed=1)
    vc = VCycle(A, dims, coarse_max=1, smooth=OMEGA, sa_levels=1, max_levels=2)
    P = vc.P[0].toarray()
    P0, cd = aggregation(dims)
    P0 = P0.toarray()
    Ad = A.toarray()
    dl1 = np.abs(Ad).sum(axis=1)
    n, nc = P0.shape
    for i in range(n):
        for C in range(nc):
            members = [j for j in range(n) if P0[j, C] == 1.0]
            expect = (1.0 if P0[i, C] == 1.0 else 0.0) - OMEGA / dl1[i] * sum(Ad[i, j] for j in members)
            assert abs(P[i, C] - expect) <= 1e-14 * max(1.0, abs(expect))
    # deeper levels keep piecewise-constant aggregation
    vc3 = VCycle(lattice_laplacian((8, 8, 8), seed=2), (8, 8, 8), coarse_max=1, smooth=OMEGA, sa_levels=1)
    assert vc3.n_levels >= 3
    assert set(np.unique(vc3.P[1].toarray())) <= {0.0, 1.0}


def test_zero_smoothing_is_plain_aggregation():
    dims = (6, 5, 4)
    A = lattice_laplacian(dims, seed=3)
    a = VCycle(A, dims, coarse_max=8)
    b = VCycle(A, dims, coarse_max=8, smooth=0.0, sa_levels=3)
    for Pa, Pb in zip(a.P, b.P):
        assert (Pa != Pb).nnz == 0
    r = np.random.Generator(np.random.PCG64(0)).standard_normal(A.shape[0])
    assert np.array_equal(a.apply(r), b.apply(r))


def test_smoothed_prolongator_keeps_constants_in_the_kernel():
    """When A 1 = 0 (pure-Neumann Schur complement) P maps coarse constants to
    fine constants, so the coarse operator keeps the same one-dimensional kernel."""
    dims = (6, 6, 5)
    A = lattice_laplacian(dims, seed=4, singular=True)
    assert np.abs(A @ np.ones(A.shape[0])).max() < 1e-10
    vc = VCycle(A, dims, coarse_max=8, smooth=OMEGA, sa_levels=1, singular=True)
    P = vc.P[0]
    assert np.allclose(P @ np.ones(P.shape[1]), 1.0, atol=1e-13)
    assert np.abs(vc.A[1] @ np.ones(P.shape[1])).max() < 1e-10 * abs(vc.A[1]).max()


def test_two_grid_correction_is_an_A_orthogonal_projector():
    """E = I - P (P^T A P)^-1 P^T A satisfies E^2 = E and A E = (A E)^T: this fails
    for any coarse operator other than the Galerkin product with the same P."""
    dims = (6, 5, 4)
    A = lattice_laplacian(dims, seed=5)
    vc = VCycle(A, dims, coarse_max=1, smooth=OMEGA, sa_levels=1, max_levels=2)
    P, Ac = vc.P[0].toarray(), vc.A[1].toarray()
    Ad = A.toarray()
    E = np.eye(Ad.shape[0]) - P @ np.linalg.solve(Ac, P.T @ Ad)
    assert np.abs(E @ E - E).max() < 1e-10
    AE = Ad @ E
    assert np.abs(AE - AE.T).max() < 1e-10 * np.abs(Ad).max()
    # the unsmoothed coarse operator with the smoothed P is not a projector
    P0 = aggregation(dims)[0].toarray()
    Ebad = np.eye(Ad.shape[0]) - P @ np.linalg.solve(P0.T @ Ad @ P0, P.T @ Ad)
    assert np.abs(Ebad @ Ebad - Ebad).max() > 1e-3


def test_first_coarse_level_has_the_33_point_stencil():
    """Interior rows of A_1 couple a coarse cell to its 3x3x3 box and to the six
    cells two steps away along an axis, and to nothing else."""
    dims = (12, 12, 12)
    A = lattice_laplacian(dims, seed=6)
    vc = VCycle(A, dims, coarse_max=1, smooth=OMEGA, sa_levels=1, max_levels=2)
    A1 = vc.A[1].tocoo()
    c = vc.dims[1][0]
    xyz = lambda i: np.stack([i % c, (i // c) % c, i // (c * c)])
    off = (xyz(A1.col) - xyz(A1.row)).T
    found = {tuple(o) for o in off[np.abs(A1.data) > 0]}
    box = {o for o in itertools.product((-1, 0, 1), repeat=3)}
    axis2 = {(2, 0, 0), (-2, 0, 0), (0, 2, 0), (0, -2, 0), (0, 0, 2), (0, 0, -2)}
    assert found == box | axis2
    # deeper (unsmoothed) levels: 3x3x3 box
    vc3 = VCycle(A, dims, coarse_max=1, smooth=OMEGA, sa_levels=1, max_levels=3)
    A2 = vc3.A[2].tocoo()
    c2 = vc3.dims[2][0]
    xyz2 = lambda i: np.stack([i % c2, (i // c2) % c2, i // (c2 * c2)])
    off2 = {tuple(o) for o in (xyz2(A2.col) - xyz2(A2.row)).T}
    assert off2 <= box


@pytest.mark.parametrize("cycle", [1, 2])
@pytest.mark.parametrize("singular", [False, True])
def test_smoothed_cycle_symmetric_positive(cycle, singular):
    dims = (8, 7, 6)
    A = lattice_laplacian(dims, seed=7, singular=singular)
    vc = VCycle(A, dims, coarse_max=8, smooth=OMEGA, sa_levels=1, cycle=cycle, singular=singular)
    assert vc.n_levels >= 3
    rng = np.random.Generator(np.random.PCG64(8))
    x, y = rng.standard_normal((2, A.shape[0]))
    if singular:
        x -= x.mean(); y -= y.mean()
    Vx, Vy = vc.apply(x), vc.apply(y)
    assert abs(x @ Vy - y @ Vx) < 1e-11 * np.linalg.norm(x) * np.linalg.norm(Vy)
    assert x @ Vx > 0


def _pcg_iterations(A, M, rtol=1e-8, maxit=500):
    b = np.random.Generator(np.random.PCG64(9)).uniform(-1, 1, A.shape[0])
    x = np.zeros_like(b); r = b.copy(); z = M(r); p = z.copy(); rz = r @ z; r0 = np.sqrt(rz)
    for it in range(1, maxit + 1):
        q = A @ p
        a = rz / (p @ q)
        x += a * p; r -= a * q
        z = M(r); rz2 = r @ z
        if np.sqrt(rz2) <= rtol * r0:
            return it
        p = z + (rz2 / rz) * p; rz = rz2
    return maxit


def block_laplacian(dims, block=4, sigma=2.0, shift=1e-3, seed=0):
    """Lattice Laplacian whose coefficient is log-normal per block of block^3 cells
    (as the Schur complement's is per element), face weight = harmonic mean of
    the two cells' coefficients, plus a small positive diagonal."""
    rng = np.random.Generator(np.random.PCG64(seed))
    X, Y, Z = dims
    nb = [-(-d // block) for d in dims]
    kap = np.exp(sigma * rng.standard_normal(nb[0] * nb[1] * nb[2]))
    coef = lambda I, J, K: kap[I // block + nb[0] * (J // block + nb[1] * (K // block))]
    n = X * Y * Z
    cell = lambda I, J, K: I + X * (J + Y * K)
    rows, cols, vals = [], [], []
    diag = shift * rng.uniform(0.5, 1.5, n)
    for K, J, I in itertools.product(range(Z), range(Y), range(X)):
        a = cell(I, J, K)
        for di, dj, dk in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
            if I + di < X and J + dj < Y and K + dk < Z:
                b = cell(I + di, J + dj, K + dk)
                ka, kb = coef(I, J, K), coef(I + di, J + dj, K + dk)
                w = 2.0 * ka * kb / (ka + kb)
                rows += [a, b]; cols += [b, a]; vals += [-w, -w]
                diag[a] += w; diag[b] += w
    A = sp.coo_matrix((vals + list(diag), (rows + list(range(n)), cols + list(range(n)))), shape=(n, n))
    return A.tocsr()


def test_smoothed_w_cycle_iterations_do_not_grow_with_the_lattice():
    """Log-normal block coefficients (sigma = 2): PCG preconditioned by the smoothed
    W-cycle needs the same number of iterations (within one) on 16^3 and 32^3
    cells, and fewer than the plain-aggregation V- and W-cycles on 32^3."""
    its = {}
    for m in (16, 32):
        dims = (m, m, m)
        A = block_laplacian(dims, seed=10)
        sa = VCycle(A, dims, coarse_max=512, smooth=OMEGA, sa_levels=1, cycle=2)
        its[m] = _pcg_iterations(A, sa.apply)
    its_ua_w = _pcg_iterations(A, VCycle(A, dims, coarse_max=512, cycle=2).apply)
    its_ua_v = _pcg_iterations(A, VCycle(A, dims, coarse_max=512).apply)
    assert abs(its[32] - its[16]) <= 1, its
    assert its[32] < its_ua_w < its_ua_v, (its, its_ua_w, its_ua_v)


def test_w_recursion_limited_to_the_first_levels():
    """cycle = 2 with w_levels = 1: level 0 makes two coarse corrections, each one
    V-cycle of the hierarchy from level 1 down (rebuilt here by hand); w_levels at
    or above the number of levels is the full W-cycle."""
    dims = (16, 12, 10)
    A = block_laplacian(dims, seed=11)
    kw = dict(coarse_max=8, smooth=OMEGA, sa_levels=1)
    w1 = VCycle(A, dims, cycle=2, w_levels=1, **kw)
    v = VCycle(A, dims, cycle=1, **kw)
    assert w1.n_levels >= 4
    b = np.random.Generator(np.random.PCG64(12)).standard_normal(A.shape[0])
    A0, d, P = v.A[0], v.dl1[0], v.P[0]
    x = np.zeros_like(b)
    for _ in range(2):
        x = x + (b - A0 @ x) / d
    for _ in range(2):
        x = x + P @ v._cycle(1, P.T @ (b - A0 @ x))
    for _ in range(2):
        x = x + (b - A0 @ x) / d
    assert np.allclose(w1._cycle(0, b), x, rtol=1e-13, atol=1e-13 * np.abs(x).max())
    full = VCycle(A, dims, cycle=2, **kw)
    deep = VCycle(A, dims, cycle=2, w_levels=w1.n_levels, **kw)
    assert np.array_equal(full._cycle(0, b), deep._cycle(0, b))
    assert not np.allclose(full._cycle(0, b), w1._cycle(0, b))


# -- smoothed prolongator on the second level as well (sa_levels = 2) ----------------

def _block_laplacian_fast(m, block=4, sigma=2.0, shift=1e-3, seed=0):
    """block_laplacian on an m^3 lattice, assembled with array operations (same
    definition: harmonic-mean face weights of log-normal per-block coefficients)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nb = -(-m // block)
    kap = np.exp(sigma * rng.standard_normal(nb ** 3))
    c = np.arange(m ** 3)
    I, J, K = c % m, (c // m) % m, c // (m * m)
    coef = kap[I // block + nb * (J // block + nb * (K // block))]
    diag = shift * rng.uniform(0.5, 1.5, m ** 3)
    rows, cols, vals = [], [], []
    for di, dj, dk in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
        a = c[(I + di < m) & (J + dj < m) & (K + dk < m)]
        b = a + di + m * (dj + m * dk)
        w = 2.0 * coef[a] * coef[b] / (coef[a] + coef[b])
        rows += [a, b]; cols += [b, a]; vals += [-w, -w]
        np.add.at(diag, a, w); np.add.at(diag, b, w)
    rows, cols = np.concatenate(rows + [c]), np.concatenate(cols + [c])
    return sp.csr_matrix((np.concatenate(vals + [diag]), (rows, cols)), shape=(m ** 3, m ** 3))


def _offsets(A, dims, radius_margin):
    """Offsets of the rows of A whose cell lies at least radius_margin from every side."""
    X, Y, Z = dims
    A = A.tocoo()
    keep = np.abs(A.data) > 0
    r, c = A.row[keep], A.col[keep]
    xyz = lambda i: np.stack([i % X, (i // X) % Y, i // (X * Y)])
    pr = xyz(r)
    inner = np.all((pr >= radius_margin) & (pr < np.array(dims)[:, None] - radius_margin), axis=0)
    return {tuple(o) for o in (xyz(c) - pr).T[inner]}


def _shape(box, axial, lateral):
    """The box of radius `box` and the cells `axial` steps away along an axis whose
    offsets across it are at most `lateral`."""
    out = set(itertools.product(range(-box, box + 1), repeat=3))
    for d in range(3):
        for v in (axial, -axial):
            for u, w in itertools.product(range(-lateral, lateral + 1), repeat=2):
                o = [u, w]
                o.insert(d, v)
                out.add(tuple(o))
    return out


def test_second_smoothed_prolongator_entries_brute_force():
    """P_1[i, C] = [i in C] - omega / D_l1(A_1)[i] * sum_{j in C} A_1[i, j] on the
    first coarse level (A_1 = P_0^T A P_0 with the smoothed P_0), by loops."""
    dims = (10, 8, 6)
    A = lattice_laplacian(dims, seed=21)
    vc = VCycle(A, dims, coarse_max=1, smooth=OMEGA, sa_levels=2, max_levels=3)
    assert vc.n_levels == 3
    A1 = vc.A[1].toarray()
    P1 = vc.P[1].toarray()
    Q, _ = aggregation(vc.dims[1])
    Q = Q.toarray()
    dl1 = np.abs(A1).sum(axis=1)
    for i in range(A1.shape[0]):
        for C in range(Q.shape[1]):
            members = np.nonzero(Q[:, C])[0]
            expect = Q[i, C] - OMEGA / dl1[i] * A1[i, members].sum()
            assert abs(P1[i, C] - expect) <= 1e-14 * max(1.0, abs(expect))
    # sa_levels = 1 leaves the second prolongator piecewise constant
    vc1 = VCycle(A, dims, coarse_max=1, smooth=OMEGA, sa_levels=1, max_levels=3)
    assert set(np.unique(vc1.P[1].toarray())) <= {0.0, 1.0}
    assert np.array_equal(vc1.P[0].toarray(), vc.P[0].toarray())


def test_second_prolongator_row_pattern():
    """A row of P_1 has nonzeros only at the aggregates agg(i) + (b_x s_x, b_y s_y,
    b_z s_z), b in {0,1}^3, and agg(i) - s_d e_d, where s = +1 on an odd and -1 on
    an even fine coordinate: at most 11 per row (the slots the kernels store)."""
    dims = (16, 14, 12)
    A = lattice_laplacian(dims, seed=22)
    vc = VCycle(A, dims, coarse_max=1, smooth=OMEGA, sa_levels=2, max_levels=3)
    P1 = vc.P[1].tocoo()
    (X, Y, Z), (cx, cy, _) = vc.dims[1], vc.dims[2]
    keep = np.abs(P1.data) > 0
    most = 0
    for i, C in zip(P1.row[keep], P1.col[keep]):
        f = np.array([i % X, (i // X) % Y, i // (X * Y)])
        s = np.where(f % 2 == 1, 1, -1)
        D = np.array([C % cx, (C // cx) % cy, C // (cx * cy)]) - f // 2
        box = all(D[d] in (0, s[d]) for d in range(3))
        far = sum(D[d] == -s[d] for d in range(3)) == 1 and sum(D != 0) == 1
        assert box or far, (i, C, D, s)
    counts = np.bincount(P1.row[keep], minlength=P1.shape[0])
    assert counts.max() == 11


def test_second_smoothed_level_shapes():
    """Interior stencils: level 1 the 33-point shape, level 2 the 5x5x5 box plus
    the cells 3 steps away along an axis with at most 1 across (179), level 3 the
    3x3x3 box plus 2 steps along an axis with at most 1 across (81), level 4 the
    3x3x3 box."""
    m = 48
    A = lattice_laplacian((m, m, m), seed=23)
    vc = VCycle(A, (m, m, m), coarse_max=1, smooth=OMEGA, sa_levels=2, max_levels=5)
    assert vc.n_levels == 5
    s33 = _shape(1, 2, 0)
    s179, s81, s27 = _shape(2, 3, 1), _shape(1, 2, 1), _shape(1, 1, 1)
    assert (len(s33), len(s179), len(s81), len(s27)) == (33, 179, 81, 27)
    assert _offsets(vc.A[1], vc.dims[1], 2) == s33
    assert _offsets(vc.A[2], vc.dims[2], 3) == s179
    assert _offsets(vc.A[3], vc.dims[3], 2) == s81
    assert _offsets(vc.A[4], vc.dims[4], 1) == s27


def test_second_level_two_grid_correction_is_an_A_orthogonal_projector():
    """E = I - P_1 (P_1^T A_1 P_1)^-1 P_1^T A_1 on the first coarse level."""
    dims = (12, 10, 8)
    A = lattice_laplacian(dims, seed=24)
    vc = VCycle(A, dims, coarse_max=1, smooth=OMEGA, sa_levels=2, max_levels=3)
    A1, P1, A2 = vc.A[1].toarray(), vc.P[1].toarray(), vc.A[2].toarray()
    E = np.eye(A1.shape[0]) - P1 @ np.linalg.solve(A2, P1.T @ A1)
    assert np.abs(E @ E - E).max() < 1e-10
    AE = A1 @ E
    assert np.abs(AE - AE.T).max() < 1e-10 * np.abs(A1).max()
    Q = aggregation(vc.dims[1])[0].toarray()
    Ebad = np.eye(A1.shape[0]) - P1 @ np.linalg.solve(Q.T @ A1 @ Q, P1.T @ A1)
    assert np.abs(Ebad @ Ebad - Ebad).max() > 1e-3


@pytest.mark.parametrize("cycle", [1, 2])
@pytest.mark.parametrize("singular", [False, True])
def test_second_smoothed_cycle_symmetric_positive(cycle, singular):
    dims = (12, 10, 9)
    A = lattice_laplacian(dims, seed=25, singular=singular)
    vc = VCycle(A, dims, coarse_max=8, smooth=OMEGA, sa_levels=2, cycle=cycle, singular=singular)
    assert vc.n_levels >= 4
    if singular:
        assert np.abs(vc.A[2] @ np.ones(vc.A[2].shape[0])).max() < 1e-10 * abs(vc.A[2]).max()
    rng = np.random.Generator(np.random.PCG64(26))
    x, y = rng.standard_normal((2, A.shape[0]))
    if singular:
        x -= x.mean(); y -= y.mean()
    Vx, Vy = vc.apply(x), vc.apply(y)
    assert abs(x @ Vy - y @ Vx) < 1e-11 * np.linalg.norm(x) * np.linalg.norm(Vy)
    assert x @ Vx > 0


def test_second_smoothed_w_cycle_iterations_flat():
    """Log-normal block coefficients: with both prolongators smoothed, PCG needs the
    same iterations (within one) on 32^3 and 64^3 cells, and fewer than with the
    first one smoothed alone on 64^3 (whose count grows)."""
    its2, its1 = {}, {}
    for m in (32, 64):
        A = _block_laplacian_fast(m, seed=27)
        its2[m] = _pcg_iterations(A, VCycle(A, (m,) * 3, coarse_max=512, smooth=OMEGA, sa_levels=2, cycle=2).apply)
        its1[m] = _pcg_iterations(A, VCycle(A, (m,) * 3, coarse_max=512, smooth=OMEGA, sa_levels=1, cycle=2).apply)
    assert abs(its2[64] - its2[32]) <= 1, its2
    assert its2[64] <= its1[64] - 2, (its1, its2)

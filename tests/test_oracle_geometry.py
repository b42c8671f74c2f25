"""Oracle pins on genuinely trilinear (non-affine) elements.

* The trilinear map (element.physical_points) takes the element's 8 vertices at the
  reference corners and is affine along every reference axis; its Jacobian
  (element.jacobian) equals central differences of that map, which are exact up to
  rounding for a map affine in each variable separately.
* The commuting property of the interpolation-histopolation pair (Sec. 2.1, the
  divergence theorem on every subcell): for a smooth non-polynomial field u, the
  face fluxes F (the RT degrees of freedom, integrals of u.n over the physical
  subcell faces, computed here by a high-order Gauss rule on each face) and the
  cell integrals G of div u (the L2 degrees of freedom) satisfy D F = G, and on
  every element the divergence of the RT interpolant equals the histopolant of
  div u pointwise: sum_n F_n div_hat(phi_n)(xi) = sum_a G_a psi_hat_a(xi).
* Constant fields on a trilinear element: the RT interpolant of a constant vector
  c is exact for k >= 2 (the Piola pull-back cof(J)^T c lies in Q_{k,k-1,k-1} x ...),
  so F^T M_e F = beta |c|^2 vol(e); the L2 interpolant of a constant is exact for
  k >= 3 (det J in Q_2), so G^T W_e G = alpha c^2 vol(e). The volume comes from
  the boundary fluxes of x/3 (faces only, no det J).

A dropped bilinear or trilinear term of the map, a wrong sign or index in the
lattice divergence or the local numbering, or a wrong basis derivative fails one
of these.
"""
import numpy as np
import pytest

import synth
from oracle import basis1d, element
from oracle.assembly import GRAD_DIV, Problem

GAUSS = 10  # Gauss points per direction on a subface / subcell (smooth integrands)


def _trilinear_patch(n, seed):
    """Unit-cube lattice of n^3 elements with every vertex (boundary too) moved by up
    to 15% of h: the elements are genuinely trilinear."""
    vx, vy, vz = synth.lattice_vertices(n, n, n)
    rng = np.random.Generator(np.random.PCG64(seed))
    h = 1.0 / n
    vx = vx + rng.uniform(-0.15 * h, 0.15 * h, vx.shape)
    vy = vy + rng.uniform(-0.15 * h, 0.15 * h, vy.shape)
    vz = vz + rng.uniform(-0.15 * h, 0.15 * h, vz.shape)
    return vx, vy, vz


def _field(X):
    x, y, z = X[..., 0], X[..., 1], X[..., 2]
    u = np.stack([np.sin(1.3 * x + 0.7 * y) * np.exp(0.5 * z),
                  np.cos(0.9 * x * z) + y * y,
                  np.exp(0.3 * x * y) * np.sin(z + 0.2)], axis=-1)
    div = (1.3 * np.cos(1.3 * x + 0.7 * y) * np.exp(0.5 * z) + 2.0 * y + np.exp(0.3 * x * y) * np.cos(z + 0.2))
    return u, div


def _gauss(a, b, m=GAUSS):
    t, w = np.polynomial.legendre.leggauss(m)
    return 0.5 * (a + b) + 0.5 * (b - a) * t, 0.5 * (b - a) * w


def _face_flux(V1, k, d, i, j, l, field):
    """Integral of field(x).n over the physical image of the reference subface of local
    RT dof (d, i, j, l) of one element (V1: its corners), n along +xi_d (area vector =
    the cross product of the two tangents in cyclic order)."""
    g = basis1d.gll_nodes(k)
    if d == 0:
        s, ws = _gauss(g[j], g[j + 1])
        t, wt = _gauss(g[l], g[l + 1])
        S, T = np.meshgrid(s, t, indexing="ij")
        pts = np.stack([np.full(S.size, g[i]), S.ravel(), T.ravel()], axis=1)
        a, b = 1, 2
    elif d == 1:
        s, ws = _gauss(g[l], g[l + 1])       # xi_3 first, then xi_1: cyclic (xi_3, xi_1)
        t, wt = _gauss(g[i], g[i + 1])
        S, T = np.meshgrid(s, t, indexing="ij")
        pts = np.stack([T.ravel(), np.full(S.size, g[j]), S.ravel()], axis=1)
        a, b = 2, 0
    else:
        s, ws = _gauss(g[i], g[i + 1])
        t, wt = _gauss(g[j], g[j + 1])
        S, T = np.meshgrid(s, t, indexing="ij")
        pts = np.stack([S.ravel(), T.ravel(), np.full(S.size, g[l])], axis=1)
        a, b = 0, 1
    W = np.outer(ws, wt).ravel()
    J = element.jacobian(V1[None], pts)[0]                      # (P, 3, 3): J[p, i, d] = dx_i/dxi_d
    nrm = np.cross(J[:, :, a], J[:, :, b])
    X = element.physical_points(V1[None], pts)[0]
    u = field(X)
    return float(np.sum(W * np.einsum("pi,pi->p", u, nrm)))


def _cell_integral(V1, k, a, b, c, fn):
    """Integral of fn(x) over the physical image of reference subcell (a, b, c)."""
    g = basis1d.gll_nodes(k)
    xs, wx = _gauss(g[a], g[a + 1])
    ys, wy = _gauss(g[b], g[b + 1])
    zs, wz = _gauss(g[c], g[c + 1])
    Z, Y, Xg = np.meshgrid(zs, ys, xs, indexing="ij")
    pts = np.stack([Xg.ravel(), Y.ravel(), Z.ravel()], axis=1)
    W = np.einsum("k,j,i->kji", wz, wy, wx).ravel()
    J = element.jacobian(V1[None], pts)[0]
    X = element.physical_points(V1[None], pts)[0]
    return float(np.sum(W * np.linalg.det(J) * fn(X)))


def _dofs(prob, V, field, div=None):
    """Global face fluxes F (each face from every element that has it; the copies must
    agree) and, when div is given, the cell integrals G of div."""
    lat, k = prob.lat, prob.k
    F = np.full(lat.n_rt, np.nan)
    loc = lat.local_rt()
    for e in range(lat.n_elem):
        for n, (d, i, j, l) in enumerate(loc):
            gid, sgn = prob.e2d_idx[e, n], prob.e2d_sign[e, n]
            f = sgn * _face_flux(V[e], k, d, i, j, l, field)
            if np.isnan(F[gid]):
                F[gid] = f
            else:  # a face shared by two elements: both parametrisations give the same flux
                assert abs(F[gid] - f) <= 1e-13 * max(1.0, abs(f))
                F[gid] = f
    assert not np.isnan(F).any()
    if div is None:
        return F
    G = np.zeros(lat.n_l2)
    for e in range(lat.n_elem):
        for m, (a, b, c) in enumerate(lat.local_l2()):
            G[prob.e2l[e, m]] = _cell_integral(V[e], k, a, b, c, div)
    return F, G


def test_trilinear_map_corners_axis_affinity_and_jacobian_by_central_differences():
    vx, vy, vz = _trilinear_patch(1, seed=31)
    V = element.element_vertices(1, 1, 1, vx, vy, vz)
    # genuinely trilinear: the twist (v000 - v100 - v010 + v110 ...) combinations are not zero
    tw = V[0, 0, 0, 0] - V[0, 0, 0, 1] - V[0, 0, 1, 0] + V[0, 0, 1, 1]
    tri = (V[0, 1, 1, 1] - V[0, 1, 1, 0] - V[0, 1, 0, 1] - V[0, 0, 1, 1]
           + V[0, 1, 0, 0] + V[0, 0, 1, 0] + V[0, 0, 0, 1] - V[0, 0, 0, 0])
    assert np.abs(tw).max() > 1e-3 and np.abs(tri).max() > 1e-3
    corners = np.array([[a, b, c] for c in (0, 1) for b in (0, 1) for a in (0, 1)], dtype=float)
    X = element.physical_points(V, corners)[0]
    for m, (a, b, c) in enumerate(corners.astype(int)):
        assert np.array_equal(X[m], V[0, c, b, a])
    rng = np.random.Generator(np.random.PCG64(32))
    P = rng.uniform(0.05, 0.95, (40, 3))
    h = 1e-3
    J = element.jacobian(V, P)[0]
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        xp = element.physical_points(V, P + e)[0]
        xm = element.physical_points(V, P - e)[0]
        x0 = element.physical_points(V, P)[0]
        # affine along the axis: equal steps give equal increments
        assert np.abs(xp - 2 * x0 + xm).max() <= 1e-14
        fd = (xp - xm) / (2 * h)
        assert np.abs(J[:, :, d] - fd).max() <= 1e-9
    # det J is the triple product of the columns and positive
    detJ = np.linalg.det(J)
    trip = np.einsum("pi,pi->p", J[:, :, 0], np.cross(J[:, :, 1], J[:, :, 2]))
    assert np.allclose(detJ, trip, rtol=1e-13) and (detJ > 0).all()


@pytest.mark.parametrize("n,k", [(1, 2), (1, 3), (1, 4), (2, 2), (2, 3), (2, 4)])
def test_commuting_identity_div_of_rt_interpolant_is_histopolant_of_div(n, k):
    vx, vy, vz = _trilinear_patch(n, seed=40 + 10 * n + k)
    prob = Problem(n, n, n, k, vx, vy, vz, np.ones(n ** 3), np.ones(n ** 3), kind=GRAD_DIV, ess_mask=0)
    V = prob.V
    F, G = _dofs(prob, V, lambda X: _field(X)[0], lambda X: _field(X)[1])
    # global: the lattice divergence of the face fluxes is the cell integrals of div u
    DF = prob.D_full @ F
    assert np.abs(DF - G).max() <= 1e-12 * np.abs(G).max()
    # element-local and pointwise, through the reference bases: div_hat(Pi_RT u) = Pi_L2(div_hat u)
    rng = np.random.Generator(np.random.PCG64(7))
    pts = rng.uniform(0, 1, (25, 3))
    _, Div = element.rt_basis(k, pts)
    Psi = element.l2_basis(k, pts)
    for e in range(prob.lat.n_elem):
        lhs = Div @ (F[prob.e2d_idx[e]] * prob.e2d_sign[e])
        rhs = Psi @ G[prob.e2l[e]]
        assert np.abs(lhs - rhs).max() <= 1e-11 * np.abs(rhs).max()


def test_commuting_identity_fails_for_a_planted_sign_slip():
    """A flipped +-1 in one cell's row of D breaks D F = G at that cell."""
    n, k = 1, 3
    vx, vy, vz = _trilinear_patch(n, seed=44)
    prob = Problem(n, n, n, k, vx, vy, vz, np.ones(1), np.ones(1), kind=GRAD_DIV, ess_mask=0)
    F, G = _dofs(prob, prob.V, lambda X: _field(X)[0], lambda X: _field(X)[1])
    D = prob.D_full.tolil()
    row = 5
    cols = D.rows[row]
    D[row, cols[0]] = -D[row, cols[0]]
    assert np.abs(D.tocsr() @ F - G).max() > 1e-6


@pytest.mark.parametrize("k", [2, 3, 4])
def test_constant_fields_give_exact_mass_on_a_trilinear_element(k):
    vx, vy, vz = _trilinear_patch(1, seed=50 + k)
    alpha, beta = 1.7, 0.6
    prob = Problem(1, 1, 1, k, vx, vy, vz, [alpha], [beta], kind=GRAD_DIV, ess_mask=0)
    V = prob.V
    # volume from the boundary fluxes of x/3 (faces only)
    Fx = _dofs(prob, V, lambda X: X / 3.0)
    cells = prob.D_full @ Fx          # subcell volumes (divergence theorem, div(x/3) = 1)
    vol = cells.sum()
    detJ_vol = sum(_cell_integral(V[0], k, a, b, c, lambda X: np.ones(X.shape[0]))
                   for (a, b, c) in prob.lat.local_l2())
    assert abs(vol - detJ_vol) <= 1e-13 * vol
    c = np.array([0.3, -1.1, 0.8])
    Fc = _dofs(prob, V, lambda X: np.broadcast_to(c, X.shape))
    Me = prob.Me[0]
    u = Fc[prob.e2d_idx[0]] * prob.e2d_sign[0]
    assert abs(u @ Me @ u - beta * (c @ c) * vol) <= 1e-12 * beta * (c @ c) * vol
    if k >= 3:
        gq = 2.5 * cells[prob.e2l[0]]   # L2 dofs of the constant 2.5: its integrals over the subcells
        We = prob.We[0]
        assert abs(gq @ We @ gq - alpha * 2.5 ** 2 * vol) <= 1e-12 * alpha * 2.5 ** 2 * vol

"""Reference bases, trilinear geometry and element matrices by full quadrature.

Sec. 2: each hex element is the image of [0,1]^3 under a trilinear map T. The
RT space uses the H(div) Piola map u = J u_hat / det J; the L2 space the
integral-preserving map w = w_hat / det J (Sec. 2, after Eq. block-variational).
The reference RT space is Q_{k,k-1,k-1} x Q_{k-1,k,k-1} x Q_{k-1,k-1,k} with the
interpolation-histopolation basis (Sec. 2.1):

  x-component dof (i,j,l):  phi = (l_i(x) h_j(y) h_l(z), 0, 0),

and y, z cyclically; the L2 basis is psi_(a,b,c) = h_a(x) h_b(y) h_c(z).

Element matrices (Eq. matrices), with the Piola maps pulled back:

  M_e[n,m] = int beta (J phi_n) . (J phi_m) / det J   dxi
  W_e[a,b] = int alpha psi_a psi_b / det J            dxi
  B_e[a,n] = int alpha psi_a div_hat(phi_n) / det J   dxi   (div u = div_hat u_hat / det J)

all evaluated with a q^3 tensor Gauss-Legendre rule: the full quadrature sum,
no sum factorisation.
"""
import numpy as np

from . import basis1d, lattice


def element_vertices(nx, ny, nz, vx, vy, vz, elems=None):
    """Corner coordinates V[e, c, b, a, dim] of elements e (vertex (ex+a, ey+b, ez+c))."""
    vx, vy, vz = (np.asarray(v, dtype=np.float64) for v in (vx, vy, vz))
    E = nx * ny * nz
    elems = np.arange(E) if elems is None else np.asarray(elems)
    ex = elems % nx
    ey = (elems // nx) % ny
    ez = elems // (nx * ny)
    V = np.zeros((len(elems), 2, 2, 2, 3))
    for c in range(2):
        for b in range(2):
            for a in range(2):
                vid = (ex + a) + (nx + 1) * ((ey + b) + (ny + 1) * (ez + c))
                V[:, c, b, a, 0] = vx[vid]
                V[:, c, b, a, 1] = vy[vid]
                V[:, c, b, a, 2] = vz[vid]
    return V


def rotate_vertices(V, rot):
    """Corner coordinates V[e, c, b, a, dim] in each element's own reference frame:
    with the rotation code rot[e] (oracle.lattice), the reference corner (a, b, c)
    is the lattice-aligned corner eta = 1/2 + R ((a, b, c) - 1/2), so the element's
    trilinear map is the lattice-aligned one composed with xi -> eta."""
    out = np.empty_like(V)
    for e in range(V.shape[0]):
        perm, sgn = lattice.rotation(int(rot[e]))
        for c in range(2):
            for b in range(2):
                for a in range(2):
                    eta = [0, 0, 0]
                    for d, t in enumerate((a, b, c)):
                        eta[perm[d]] = t if sgn[d] > 0 else 1 - t
                    out[e, c, b, a] = V[e, eta[2], eta[1], eta[0]]
    return out


def quad_rule(q):
    """Tensor GL rule: points P[p, 3] and weights w[p], p = px + q(py + q pz)."""
    x, w = basis1d.gl_points(q)
    pz, py, px = np.meshgrid(np.arange(q), np.arange(q), np.arange(q), indexing="ij")
    px, py, pz = px.ravel(), py.ravel(), pz.ravel()
    pts = np.stack([x[px], x[py], x[pz]], axis=1)
    return pts, w[px] * w[py] * w[pz]


def jacobian(V, pts):
    """J[e, p, i, d] = d x_i / d xi_d of the trilinear map at reference points."""
    xi = pts
    N = [1.0 - xi, xi]            # N_0, N_1 per coordinate: arrays (P, 3)
    dN = [-np.ones_like(xi), np.ones_like(xi)]
    J = np.zeros((V.shape[0], len(pts), 3, 3))
    for c in range(2):
        for b in range(2):
            for a in range(2):
                Xv = V[:, c, b, a, :]                       # (E, 3)
                g = np.stack([dN[a][:, 0] * N[b][:, 1] * N[c][:, 2],
                              N[a][:, 0] * dN[b][:, 1] * N[c][:, 2],
                              N[a][:, 0] * N[b][:, 1] * dN[c][:, 2]], axis=1)  # (P, 3)
                J += Xv[:, None, :, None] * g[None, :, None, :]
    return J


def physical_points(V, pts):
    N = [1.0 - pts, pts]
    X = np.zeros((V.shape[0], len(pts), 3))
    for c in range(2):
        for b in range(2):
            for a in range(2):
                X += V[:, None, c, b, a, :] * (N[a][:, 0] * N[b][:, 1] * N[c][:, 2])[None, :, None]
    return X


def rt_basis(k, pts):
    """Reference RT basis values Phi[p, n, 3] and divergences Div[p, n] at pts,
    in the local dof order of oracle.lattice."""
    P = len(pts)
    I = [basis1d.interp_basis(k, pts[:, d]) for d in range(3)]
    dI = [basis1d.interp_basis_deriv(k, pts[:, d]) for d in range(3)]
    H = [basis1d.histo_basis(k, pts[:, d]) for d in range(3)]
    n = 3 * (k + 1) * k * k
    Phi = np.zeros((P, n, 3))
    Div = np.zeros((P, n))
    m = 0
    for l in range(k):
        for j in range(k):
            for i in range(k + 1):
                Phi[:, m, 0] = I[0][i] * H[1][j] * H[2][l]
                Div[:, m] = dI[0][i] * H[1][j] * H[2][l]
                m += 1
    for l in range(k):
        for j in range(k + 1):
            for i in range(k):
                Phi[:, m, 1] = H[0][i] * I[1][j] * H[2][l]
                Div[:, m] = H[0][i] * dI[1][j] * H[2][l]
                m += 1
    for l in range(k + 1):
        for j in range(k):
            for i in range(k):
                Phi[:, m, 2] = H[0][i] * H[1][j] * I[2][l]
                Div[:, m] = H[0][i] * H[1][j] * dI[2][l]
                m += 1
    return Phi, Div


def l2_basis(k, pts):
    """Reference L2 basis Psi[p, a], local order a + k(b + k c)."""
    H = [basis1d.histo_basis(k, pts[:, d]) for d in range(3)]
    out = np.zeros((len(pts), k ** 3))
    m = 0
    for c in range(k):
        for b in range(k):
            for a in range(k):
                out[:, m] = H[0][a] * H[1][b] * H[2][c]
                m += 1
    return out


_TABLES = {}


def reference_tables(k, q):
    """Quadrature rule and reference basis values for (k, q), evaluated once."""
    key = (k, q)
    if key not in _TABLES:
        pts, w = quad_rule(q)
        Phi, Div = rt_basis(k, pts)
        _TABLES[key] = (pts, w, Phi, Div, l2_basis(k, pts))
    return _TABLES[key]


def reference_mass_blocks(k, q):
    """K[a, b] (a, b = 0..2): the reference-cube matrices K_ab[n, m] = int phi_hat_n,a
    phi_hat_m,b dxi by the q^3 Gauss rule. On a parallelepiped (J = A constant) the
    Piola-mapped mass is M_e = sum_ab G_ab K_ab with G = beta A^T A / det A (Eq. matrices
    with the geometric factor taken out of the integral)."""
    pts, w, Phi, _, _ = reference_tables(k, q)
    return np.einsum("p,pna,pmb->abnm", w, Phi, Phi)


def element_matrices(V, k, q, beta, alpha, want=("M", "W", "B")):
    """Element matrices for elements with corner coordinates V (see module doc).

    beta, alpha: per-element coefficients (arrays of length E).
    Returns a dict with the requested 'M' (E, n, n), 'W' (E, k^3, k^3),
    'B' (E, k^3, n)."""
    pts, w, Phi, Div, Psi = reference_tables(k, q)
    J = jacobian(V, pts)
    detJ = np.linalg.det(J)
    if np.any(detJ <= 0):
        raise ValueError("inverted element (det J <= 0)")
    beta = np.asarray(beta, dtype=np.float64)
    alpha = np.asarray(alpha, dtype=np.float64)
    out = {}
    if "M" in want:
        A = np.einsum("epid,pnd->epin", J, Phi)                  # J phi at points
        s = np.sqrt(w[None, :] * beta[:, None] / detJ)           # (E, P)
        A = A * s[:, :, None, None]
        A = A.reshape(A.shape[0], -1, A.shape[-1])                # (E, 3P, n)
        out["M"] = np.matmul(A.transpose(0, 2, 1), A)
    if "W" in want or "B" in want:
        wt = w[None, :] * alpha[:, None] / detJ                  # (E, P)
        if "W" in want:
            out["W"] = np.einsum("pa,ep,pb->eab", Psi, wt, Psi)
        if "B" in want:
            out["B"] = np.einsum("pa,ep,pn->ean", Psi, wt, Div)
    return out

"""Assembled global matrices and the transformed block operator.

Grad-div (Eq. saddle-point, Eq. transformed-system):

    AA = [[ M_beta, D^T        ],
          [ D,      -W_alpha^-1 ]],   D = W_alpha^-1 B_alpha (the lattice incidence).

Darcy (Eq. darcy-nonzero, Eq. transformed-system-darcy):

    AA' = [[ M_{1/eps}, D^T                  ],
           [ D,         -W^-1 W_gamma W^-1 ]],   (2,2) block zero when gamma = 0.

Coefficients are per element: grad-div (coef0, coef1) = (alpha, beta); Darcy
(coef0, coef1) = (eps, gamma).

Essential (u.n prescribed) RT dofs are eliminated as a constrained identity: the
rows and columns of M and the columns of D belonging to them are dropped and the
diagonal of AA is 1 there, so (AA x)_ess = x_ess.

Elements may carry rotation codes (oracle.lattice): element matrices are then
computed in each element's own reference frame and assembled through the rotated
signed maps, and D is built by Algorithm 1 from those maps.

Everything is assembled with scipy.sparse from element matrices computed by full
quadrature (oracle.element); (2,2) blocks use dense per-element inverses
(numpy.linalg.inv). This is the plain definition; it is slow by design.
"""
import numpy as np
import scipy.sparse as sp

from . import element
from .lattice import Lattice, algorithm1_divergence

GRAD_DIV, DARCY = 0, 1


def default_q(k, affine):
    """Quadrature points per direction: k+1 on affine meshes, k+2 otherwise."""
    return k + 1 if affine else k + 2


class Problem:
    """A discretised grad-div or Darcy problem on a structured hex mesh."""

    def __init__(self, nx, ny, nz, k, vx, vy, vz, coef0, coef1, kind=GRAD_DIV,
                 ess_mask=0, q=None, affine=False, batch=64, rot=None):
        self.lat = Lattice(nx, ny, nz, k)
        self.rot = None if rot is None else np.asarray(rot, dtype=np.int64)
        self.k, self.kind = k, kind
        self.q = default_q(k, affine) if q is None else q
        self.vx, self.vy, self.vz = (np.asarray(v, dtype=np.float64) for v in (vx, vy, vz))
        E = self.lat.n_elem
        self.coef0 = np.broadcast_to(np.asarray(coef0, dtype=np.float64), (E,)).copy()
        self.coef1 = np.broadcast_to(np.asarray(coef1, dtype=np.float64), (E,)).copy()
        if kind == GRAD_DIV:
            self.alpha, self.beta = self.coef0, self.coef1
        else:
            self.eps, self.gamma = self.coef0, self.coef1
            self.beta = 1.0 / self.eps
        self.ess = self.lat.ess_dofs(ess_mask)
        self.free = np.ones(self.lat.n_rt, dtype=bool)
        self.free[self.ess] = False
        self._batch = batch
        self._build()

    # -- assembly -----------------------------------------------------------
    def _build(self):
        lat, k, q = self.lat, self.k, self.q
        E = lat.n_elem
        nloc, wloc = lat.n_rt_loc, lat.n_l2_loc
        self.e2d = lat.e2d_map(self.rot)
        self.e2l = lat.e2l2_map(self.rot)
        V = element.element_vertices(lat.nx, lat.ny, lat.nz, self.vx, self.vy, self.vz)
        if self.rot is not None:
            V = element.rotate_vertices(V, self.rot)
        self.V = V
        Me = np.zeros((E, nloc, nloc))
        We = np.zeros((E, wloc, wloc))           # unweighted or alpha-weighted L2 mass
        Ce = np.zeros((E, wloc, wloc))           # the (2,2) block C (AA has -C)
        ones = np.ones(E)
        for s in range(0, E, self._batch):
            sl = slice(s, min(E, s + self._batch))
            if self.kind == GRAD_DIV:
                m = element.element_matrices(V[sl], k, q, self.beta[sl], self.alpha[sl], want=("M", "W"))
                Me[sl], We[sl] = m["M"], m["W"]
                Ce[sl] = np.linalg.inv(m["W"])                         # W_alpha^-1
            else:
                m = element.element_matrices(V[sl], k, q, self.beta[sl], ones[sl], want=("M", "W"))
                Me[sl], We[sl] = m["M"], m["W"]
                g = element.element_matrices(V[sl], k, q, ones[sl], self.gamma[sl], want=("W",))["W"]
                Winv = np.linalg.inv(m["W"])
                Ce[sl] = Winv @ g @ Winv                               # W^-1 W_gamma W^-1
        self.Me, self.We, self.Ce = Me, We, Ce
        # signed map -> (index, sign)
        sign = np.where(self.e2d < 0, -1.0, 1.0)
        idx = np.where(self.e2d < 0, -1 - self.e2d, self.e2d)
        self.e2d_idx, self.e2d_sign = idx, sign
        rows = np.repeat(idx[:, :, None], nloc, axis=2)
        cols = np.repeat(idx[:, None, :], nloc, axis=1)
        vals = Me * sign[:, :, None] * sign[:, None, :]
        M = sp.coo_matrix((vals.ravel(), (rows.ravel(), cols.ravel())),
                          shape=(lat.n_rt, lat.n_rt)).tocsr()
        self.M_full = M
        if self.rot is None:
            r, c, v = lat.divergence_incidence()
            self.D_full = sp.coo_matrix((v, (r, c)), shape=(lat.n_l2, lat.n_rt)).tocsr()
        else:
            ip, ix, dv = algorithm1_divergence(lat, self.e2d, self.e2l)
            self.D_full = sp.csr_matrix((dv, ix, ip), shape=(lat.n_l2, lat.n_rt))
        # constrained versions: drop essential rows/cols of M, essential cols of D
        Pf = sp.diags(self.free.astype(np.float64))
        Pe = sp.diags((~self.free).astype(np.float64))
        self.M = (Pf @ M @ Pf + Pe).tocsr()
        self.D = (self.D_full @ Pf).tocsr()
        # (2,2) block as a block-diagonal CSR
        rows = np.repeat(self.e2l[:, :, None], wloc, axis=2)
        cols = np.repeat(self.e2l[:, None, :], wloc, axis=1)
        self.C = sp.coo_matrix((Ce.ravel(), (rows.ravel(), cols.ravel())),
                               shape=(lat.n_l2, lat.n_l2)).tocsr()

    # -- operators ------------------------------------------------------------
    @property
    def n(self):
        return self.lat.n_rt + self.lat.n_l2

    def split(self, x):
        return x[: self.lat.n_rt], x[self.lat.n_rt:]

    def apply_A(self, u):
        """M_beta u (constrained)."""
        return self.M @ u

    def apply_B(self, u):
        """D u (lattice divergence, essential columns dropped)."""
        return self.D @ u

    def apply_Bt(self, q):
        """D^T q, with zero on essential rows."""
        return self.D.T @ q

    def apply_C(self, q):
        """The (2,2) block C: W_alpha^-1 q (grad-div) or W^-1 W_gamma W^-1 q (Darcy)."""
        return self.C @ q

    def apply_op(self, x):
        """AA x for x = [u; q_tilde] (Eq. transformed-saddle-point)."""
        u, qt = self.split(x)
        yu = self.M @ u + self.D.T @ qt
        yq = self.D @ u - self.C @ qt
        return np.concatenate([yu, yq])

    def matrix(self):
        """The assembled AA as CSR."""
        return sp.bmat([[self.M, self.D.T], [self.D, -self.C]]).tocsr()

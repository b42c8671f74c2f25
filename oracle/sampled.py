"""Single rows of the block operator AA x at any mesh size.

Each RT row is the sum over the (one or two) elements that contain the subcell
face of (M_e u_e) at that face, plus (D^T q)_face = q_low - q_high; each L2 row
is (D u)_cell - (C_e q_e)_cell of the one element owning the cell. Only the
elements touching the requested rows are integrated (oracle.element), so rows
of a full-size problem can be checked one by one.
"""
import numpy as np

from . import element
from .assembly import GRAD_DIV, default_q
from .lattice import Lattice


class SampledOperator:
    def __init__(self, nx, ny, nz, k, vx, vy, vz, coef0, coef1, kind=GRAD_DIV,
                 ess_mask=0, q=None, affine=False):
        self.lat = Lattice(nx, ny, nz, k)
        self.k, self.kind = k, kind
        self.q = default_q(k, affine) if q is None else q
        self.v = (np.asarray(vx), np.asarray(vy), np.asarray(vz))
        E = self.lat.n_elem
        self.coef0 = np.broadcast_to(np.asarray(coef0, dtype=np.float64), (E,))
        self.coef1 = np.broadcast_to(np.asarray(coef1, dtype=np.float64), (E,))
        self.ess = self.lat.ess_dofs(ess_mask)
        self._ess_set = set(self.ess.tolist())
        self._loc_rt = {t: n for n, t in enumerate(self.lat.local_rt())}
        self._loc_l2 = {t: n for n, t in enumerate(self.lat.local_l2())}

    # -- geometry of a dof -----------------------------------------------------
    def _face(self, g):
        lat = self.lat
        X, Y = lat.X, lat.Y
        if g < lat.n_xf:
            d, r = 0, g
            I = r % (X + 1); r //= (X + 1); J = r % Y; K = r // Y
        elif g < lat.n_xf + lat.n_yf:
            d, r = 1, g - lat.n_xf
            I = r % X; r //= X; J = r % (Y + 1); K = r // (Y + 1)
        else:
            d, r = 2, g - lat.n_xf - lat.n_yf
            I = r % X; r //= X; J = r % Y; K = r // Y
        return d, I, J, K

    def _elements_of_face(self, d, I, J, K):
        """(element id, local RT index) pairs containing face (d, I, J, K)."""
        lat, k = self.lat, self.k
        c = [I, J, K]
        n = [lat.nx, lat.ny, lat.nz]
        choices = []
        for a in range(3):
            if a != d:
                choices.append([c[a] // k])
            else:
                opts = []
                if c[a] % k == 0:
                    if c[a] // k - 1 >= 0:
                        opts.append(c[a] // k - 1)
                    if c[a] // k < n[a]:
                        opts.append(c[a] // k)
                else:
                    opts.append(c[a] // k)
                choices.append(opts)
        out = []
        for ex in choices[0]:
            for ey in choices[1]:
                for ez in choices[2]:
                    e = ex + lat.nx * (ey + lat.ny * ez)
                    loc = (d, I - ex * k, J - ey * k, K - ez * k)
                    out.append((e, self._loc_rt[loc]))
        return out

    def _elem_mats(self, elems):
        lat = self.lat
        V = element.element_vertices(lat.nx, lat.ny, lat.nz, *self.v, elems=elems)
        ones = np.ones(len(elems))
        if self.kind == GRAD_DIV:
            m = element.element_matrices(V, self.k, self.q, self.coef1[elems], self.coef0[elems],
                                         want=("M", "W"))
            return m["M"], np.linalg.inv(m["W"])
        m = element.element_matrices(V, self.k, self.q, 1.0 / self.coef0[elems], ones, want=("M", "W"))
        g = element.element_matrices(V, self.k, self.q, ones, self.coef1[elems], want=("W",))["W"]
        Wi = np.linalg.inv(m["W"])
        return m["M"], Wi @ g @ Wi

    def _gather_u(self, e, u):
        lat, k = self.lat, self.k
        ex, ey, ez = lat.elem_coords(e)
        ue = np.zeros(lat.n_rt_loc)
        for n, (d, i, j, l) in enumerate(lat.local_rt()):
            I, J, K = ex * k + i, ey * k + j, ez * k + l
            g = (lat.xface, lat.yface, lat.zface)[d](I, J, K)
            ue[n] = 0.0 if g in self._ess_set else u[g]
        return ue

    def _gather_q(self, e, q):
        lat, k = self.lat, self.k
        ex, ey, ez = lat.elem_coords(e)
        return np.array([q[lat.cell(ex * k + a, ey * k + b, ez * k + c)]
                         for (a, b, c) in lat.local_l2()])

    # -- rows ---------------------------------------------------------------------
    def rt_rows(self, x, rows):
        lat = self.lat
        u, q = x[: lat.n_rt], x[lat.n_rt:]
        out = np.zeros(len(rows))
        for r, g in enumerate(rows):
            g = int(g)
            if g in self._ess_set:
                out[r] = u[g]
                continue
            d, I, J, K = self._face(g)
            pairs = self._elements_of_face(d, I, J, K)
            Me, _ = self._elem_mats(np.array([e for e, _ in pairs]))
            val = 0.0
            for t, (e, n) in enumerate(pairs):
                val += Me[t][n] @ self._gather_u(e, u)
            c = [I, J, K]
            N = [lat.X, lat.Y, lat.Z]
            if c[d] > 0:                       # low-side cell: this face is its high face
                lo = list(c); lo[d] -= 1
                val += q[lat.cell(*lo)]
            if c[d] < N[d]:                    # high-side cell: this face is its low face
                val -= q[lat.cell(*c)]
            out[r] = val
        return out

    def l2_rows(self, x, rows):
        lat, k = self.lat, self.k
        u, q = x[: lat.n_rt], x[lat.n_rt:]
        out = np.zeros(len(rows))
        for r, c in enumerate(rows):
            c = int(c)
            I = c % lat.X; J = (c // lat.X) % lat.Y; K = c // (lat.X * lat.Y)
            div = 0.0
            for d in range(3):
                lo = [I, J, K]
                hi = [I, J, K]; hi[d] += 1
                f = (lat.xface, lat.yface, lat.zface)[d]
                glo, ghi = f(*lo), f(*hi)
                div += (0.0 if ghi in self._ess_set else u[ghi]) - (0.0 if glo in self._ess_set else u[glo])
            e = (I // k) + lat.nx * ((J // k) + lat.ny * (K // k))
            _, Ce = self._elem_mats(np.array([e]))
            a = self._loc_l2[(I - (I // k) * k, J - (J // k) * k, K - (K // k) * k)]
            out[r] = div - Ce[0][a] @ self._gather_q(e, q)
        return out

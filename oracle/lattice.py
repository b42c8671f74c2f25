"""Global numbering of the refined subcell lattice and the element-to-dof maps.

Sec. 2.1: every RT dof is a subcell face of the Gauss-Lobatto subcell mesh and
every L2 dof a subcell volume. On a structured nx x ny x nz hex mesh with k
subcells per direction per element, the subcells form an X x Y x Z lattice
(X = nx k, ...). Algorithm 1 names the arrays (element map, local-to-global map,
local and global orientations) but not a convention; this module fixes one:

* element e = ex + nx (ey + ny ez);
* lattice cell (I, J, K) -> I + X (J + Y K)                    (L2 dof);
* x-face (I, J, K), I in [0, X]          -> I + (X+1)(J + Y K)
  y-face (I, J, K), J in [0, Y]          -> NX + I + X (J + (Y+1) K)
  z-face (I, J, K), K in [0, Z]          -> NX + NY + I + X (J + Y K)
  (NX, NY = number of x-, y-faces); global orientation +x, +y, +z;
* element-local RT dof (component d, indices i, j, l along x, y, z):
  d=0: i in [0,k], j,l in [0,k)   -> i + (k+1)(j + k l)
  d=1: j in [0,k], i,l in [0,k)   -> (k+1)k^2 + i + k (j + (k+1) l)
  d=2: l in [0,k], i,j in [0,k)   -> 2(k+1)k^2 + i + k (j + k l)
  local orientation +xi_d, the same as global for unrotated elements;
* element-local L2 dof (a, b, c) -> a + k (b + k c).

The signed map stores the global id g where the local and global orientations
agree and ~g = -1-g where they are opposite (sigma_loc * sigma_glob of
Algorithm 1). On this lattice all elements are unrotated, so every sign is +1.
"""
import numpy as np

SIDE_X0, SIDE_X1, SIDE_Y0, SIDE_Y1, SIDE_Z0, SIDE_Z1 = 1, 2, 4, 8, 16, 32


class Lattice:
    def __init__(self, nx, ny, nz, k):
        self.nx, self.ny, self.nz, self.k = int(nx), int(ny), int(nz), int(k)
        self.X, self.Y, self.Z = nx * k, ny * k, nz * k
        X, Y, Z = self.X, self.Y, self.Z
        self.n_xf = (X + 1) * Y * Z
        self.n_yf = X * (Y + 1) * Z
        self.n_zf = X * Y * (Z + 1)
        self.n_rt = self.n_xf + self.n_yf + self.n_zf
        self.n_l2 = X * Y * Z
        self.n_elem = nx * ny * nz
        self.n_rt_loc = 3 * (k + 1) * k * k
        self.n_l2_loc = k ** 3

    # -- global ids -------------------------------------------------------
    def xface(self, I, J, K):
        return I + (self.X + 1) * (J + self.Y * K)

    def yface(self, I, J, K):
        return self.n_xf + I + self.X * (J + (self.Y + 1) * K)

    def zface(self, I, J, K):
        return self.n_xf + self.n_yf + I + self.X * (J + self.Y * K)

    def cell(self, I, J, K):
        return I + self.X * (J + self.Y * K)

    # -- element-local ordering -------------------------------------------
    def local_rt(self):
        """List of (d, i, j, l) for local RT dofs in local-id order."""
        k = self.k
        out = []
        for l in range(k):
            for j in range(k):
                for i in range(k + 1):
                    out.append((0, i, j, l))
        for l in range(k):
            for j in range(k + 1):
                for i in range(k):
                    out.append((1, i, j, l))
        for l in range(k + 1):
            for j in range(k):
                for i in range(k):
                    out.append((2, i, j, l))
        return out

    def local_l2(self):
        k = self.k
        return [(a, b, c) for c in range(k) for b in range(k) for a in range(k)]

    def elem_coords(self, e):
        ex = e % self.nx
        ey = (e // self.nx) % self.ny
        ez = e // (self.nx * self.ny)
        return ex, ey, ez

    def e2d_map(self):
        """Signed element-to-RT-dof map, shape (E, 3(k+1)k^2), int64."""
        k = self.k
        loc = self.local_rt()
        m = np.zeros((self.n_elem, len(loc)), dtype=np.int64)
        for e in range(self.n_elem):
            ex, ey, ez = self.elem_coords(e)
            ox, oy, oz = ex * k, ey * k, ez * k
            for n, (d, i, j, l) in enumerate(loc):
                if d == 0:
                    g = self.xface(ox + i, oy + j, oz + l)
                elif d == 1:
                    g = self.yface(ox + i, oy + j, oz + l)
                else:
                    g = self.zface(ox + i, oy + j, oz + l)
                m[e, n] = g  # orientation +1 everywhere on an unrotated lattice
        return m

    def e2l2_map(self):
        """Element-to-L2-dof map, shape (E, k^3)."""
        k = self.k
        loc = self.local_l2()
        m = np.zeros((self.n_elem, len(loc)), dtype=np.int64)
        for e in range(self.n_elem):
            ex, ey, ez = self.elem_coords(e)
            for n, (a, b, c) in enumerate(loc):
                m[e, n] = self.cell(ex * k + a, ey * k + b, ez * k + c)
        return m

    def ess_dofs(self, side_mask):
        """Ascending global ids of the RT dofs on the domain sides in side_mask."""
        X, Y, Z = self.X, self.Y, self.Z
        out = []
        J, K = np.meshgrid(np.arange(Y), np.arange(Z), indexing="ij")
        if side_mask & SIDE_X0:
            out.append(self.xface(0, J, K).ravel())
        if side_mask & SIDE_X1:
            out.append(self.xface(X, J, K).ravel())
        I, K = np.meshgrid(np.arange(X), np.arange(Z), indexing="ij")
        if side_mask & SIDE_Y0:
            out.append(self.yface(I, 0, K).ravel())
        if side_mask & SIDE_Y1:
            out.append(self.yface(I, Y, K).ravel())
        I, J = np.meshgrid(np.arange(X), np.arange(Y), indexing="ij")
        if side_mask & SIDE_Z0:
            out.append(self.zface(I, J, 0).ravel())
        if side_mask & SIDE_Z1:
            out.append(self.zface(I, J, Z).ravel())
        if not out:
            return np.zeros(0, dtype=np.int64)
        return np.unique(np.concatenate(out).astype(np.int64))

    def divergence_incidence(self):
        """Rows = cells, columns = faces: +1 on a cell's high faces, -1 on its
        low faces (outward flux with global orientation +x/+y/+z). Returns
        (rows, cols, vals) triplets, 6 per cell."""
        X, Y, Z = self.X, self.Y, self.Z
        I, J, K = np.meshgrid(np.arange(X), np.arange(Y), np.arange(Z), indexing="ij")
        I, J, K = I.ravel(), J.ravel(), K.ravel()
        c = self.cell(I, J, K)
        rows, cols, vals = [], [], []
        for lo, hi in ((self.xface(I, J, K), self.xface(I + 1, J, K)),
                       (self.yface(I, J, K), self.yface(I, J + 1, K)),
                       (self.zface(I, J, K), self.zface(I, J, K + 1))):
            rows += [c, c]
            cols += [lo, hi]
            vals += [-np.ones(len(c)), np.ones(len(c))]
        return np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)

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
Algorithm 1).

Element rotations. An element's reference axes need not be the lattice axes:
its reference cube may be placed by any of the 24 proper symmetries R of the
cube, xi -> eta = 1/2 + R (xi - 1/2) (eta: the lattice-aligned coordinates of
the element). R sends reference axis d to lattice axis perm[d] with sign
sgn[d]; a node index t in [0, k] along axis d becomes t or k - t, an interval
index t in [0, k) becomes t or k - 1 - t, and the RT basis function of
reference component d has the orientation sgn[d] against the global +axis
(the Piola map u = J u_hat / det J with J = J_lattice R). The rotation code is
4 p + t: p indexes the 6 permutations of (0, 1, 2) in lexicographic order, t the
4 sign patterns with det R = +1 in increasing order of the bit pattern
[sgn0 < 0] + 2 [sgn1 < 0] + 4 [sgn2 < 0]; code 0 is the identity.
"""
import itertools

import numpy as np

SIDE_X0, SIDE_X1, SIDE_Y0, SIDE_Y1, SIDE_Z0, SIDE_Z1 = 1, 2, 4, 8, 16, 32


def _parity(perm):
    inv = sum(1 for a in range(3) for b in range(a + 1, 3) if perm[a] > perm[b])
    return -1 if inv % 2 else 1


def rotation(code):
    """(perm, sgn) of the cube symmetry with the given code (module doc)."""
    if not 0 <= code < 24:
        raise ValueError("rotation code must be in 0..23")
    perm = list(itertools.permutations(range(3)))[code // 4]
    pats = []
    for bits in range(8):
        sgn = tuple(-1 if bits >> d & 1 else 1 for d in range(3))
        if _parity(perm) * sgn[0] * sgn[1] * sgn[2] == 1:
            pats.append(sgn)
    return perm, pats[code % 4]


def rotation_matrix(code):
    """R with R e_d = sgn[d] e_perm[d] (columns are the images of the reference axes)."""
    perm, sgn = rotation(code)
    R = np.zeros((3, 3))
    for d in range(3):
        R[perm[d], d] = sgn[d]
    return R


def _to_lattice(t, s, n):
    """Index t along a reference axis with sign s, on an axis of n positions."""
    return t if s > 0 else n - 1 - t


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

    def local_to_lattice(self, rot, idx, node_axis):
        """Lattice-aligned indices (along x, y, z) of the local subcell entity with
        reference indices idx; idx[node_axis] is a node index in [0, k] (an RT face)
        and the others interval indices in [0, k); node_axis None for a cell."""
        perm, sgn = rotation(rot)
        k = self.k
        L = [0, 0, 0]
        for c in range(3):
            n = k + 1 if c == node_axis else k
            L[perm[c]] = _to_lattice(idx[c], sgn[c], n)
        return L

    def e2d_map(self, rot=None):
        """Signed element-to-RT-dof map, shape (E, 3(k+1)k^2), int64; rot: rotation
        code per element (None: all 0)."""
        k = self.k
        loc = self.local_rt()
        rot = np.zeros(self.n_elem, dtype=np.int64) if rot is None else np.asarray(rot)
        face = (self.xface, self.yface, self.zface)
        m = np.zeros((self.n_elem, len(loc)), dtype=np.int64)
        for e in range(self.n_elem):
            ex, ey, ez = self.elem_coords(e)
            perm, sgn = rotation(int(rot[e]))
            for n, (d, i, j, l) in enumerate(loc):
                L = self.local_to_lattice(int(rot[e]), (i, j, l), d)
                g = face[perm[d]](ex * k + L[0], ey * k + L[1], ez * k + L[2])
                m[e, n] = g if sgn[d] > 0 else -1 - g
        return m

    def e2l2_map(self, rot=None):
        """Element-to-L2-dof map, shape (E, k^3); rot as for e2d_map."""
        k = self.k
        loc = self.local_l2()
        rot = np.zeros(self.n_elem, dtype=np.int64) if rot is None else np.asarray(rot)
        m = np.zeros((self.n_elem, len(loc)), dtype=np.int64)
        for e in range(self.n_elem):
            ex, ey, ez = self.elem_coords(e)
            for n, (a, b, c) in enumerate(loc):
                L = self.local_to_lattice(int(rot[e]), (a, b, c), None)
                m[e, n] = self.cell(ex * k + L[0], ey * k + L[1], ez * k + L[2])
        return m

    def volume_to_face(self):
        """For each local L2 dof, its 2d local subcell faces as (local RT id, sigma_loc):
        the low then the high face along reference axes 0, 1, 2; sigma_loc = -1 on the
        low face (the basis function points into the subcell) and +1 on the high face."""
        k = self.k
        off = (0, (k + 1) * k * k, 2 * (k + 1) * k * k)
        out = []
        for (a, b, c) in self.local_l2():
            faces = []
            for d in range(3):
                for hi in (0, 1):
                    i, j, l = a + (hi if d == 0 else 0), b + (hi if d == 1 else 0), c + (hi if d == 2 else 0)
                    if d == 0:
                        jl = off[0] + i + (k + 1) * (j + k * l)
                    elif d == 1:
                        jl = off[1] + i + k * (j + (k + 1) * l)
                    else:
                        jl = off[2] + i + k * (j + k * l)
                    faces.append((jl, 1 if hi else -1))
            out.append(faces)
        return out

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


def algorithm1_divergence(lat, e2d, e2l):
    """The discrete divergence D in CSR form by Algorithm 1 (Sec. 3.2): row i (an L2
    dof, a subcell volume) has 2d = 6 entries at I[i] = 6 i; for each subcell face of
    the volume, the local RT dof j_loc and its reference orientation sigma_loc, the
    global dof j and the orientation sigma_glob of j relative to j_loc (both read from
    the signed map), and the entry sigma_loc * sigma_glob. element_map and
    l2_global_to_local are the inverse of the element-to-L2 map e2l.
    Returns (indptr, indices, data)."""
    N = lat.n_l2
    element_map = np.zeros(N, dtype=np.int64)
    l2_global_to_local = np.zeros(N, dtype=np.int64)
    for e in range(e2l.shape[0]):
        for a in range(e2l.shape[1]):
            element_map[e2l[e, a]] = e
            l2_global_to_local[e2l[e, a]] = a
    v2f = lat.volume_to_face()
    indptr = 6 * np.arange(N + 1, dtype=np.int64)
    indices = np.zeros(6 * N, dtype=np.int64)
    data = np.zeros(6 * N)
    for i in range(N):
        e, iloc = element_map[i], l2_global_to_local[i]
        for f, (jloc, sigma_loc) in enumerate(v2f[iloc]):
            s = e2d[e, jloc]
            j, sigma_glob = (s, 1) if s >= 0 else (-1 - s, -1)
            indices[6 * i + f] = j
            data[6 * i + f] = sigma_loc * sigma_glob
    return indptr, indices, data

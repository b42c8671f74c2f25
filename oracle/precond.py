"""Block-diagonal preconditioner: diag(M) for the (1,1) block and a geometric
V-cycle on the approximate Schur complement (Sec. 2.3-2.4).

* M~ = diag(M_beta) (Sec. 2.3), applied as z_u = r_u / (tau M~); tau = 1 by
  default (final proposition of Sec. 2.3; tau = 2 is Prop. 2's optimal scaling
  for exact blocks). Essential dofs: z = r.
* C~ approximates the (2,2) block: 1/diag(W_alpha) for grad-div; for Darcy the
  product of the diagonals diag(W)^-1 diag(W_gamma) diag(W)^-1 (Sec. 2.4), zero
  when gamma = 0.
* S~ = C~ + D M~^-1 D^T (Eq. approx-schur; the paper's Sec. 2.3 prints W_alpha
  where its own definitions give W_alpha^-1, see Eq. approx-schur-entries).
* S^-1 is approximated by one V-cycle (the paper uses one BoomerAMG V-cycle,
  Sec. 3.2). The geometric V-cycle used here:
    - levels: piecewise-constant aggregation of 2 cells per direction (a trailing
      odd cell is its own aggregate; a direction of length 1 is not coarsened),
      until at most `coarse_max` cells remain; `aligned` = True groups the cells
      inside each element instead (element_groups: for odd k the pairs cannot all
      follow the element boundaries, and aggregates that straddle them slow the
      cycle down);
    - prolongation: piecewise constant P0 on the aggregates, or, on the first
      `sa_levels` levels when `smooth` = omega > 0, the smoothed-aggregation
      prolongator P = (I - omega D_l1^-1 A_l) P0 (one damped l1-Jacobi step
      applied to P0; omega = 4/3 is the customary choice);
    - Galerkin coarse operators A_{l+1} = P^T A_l P;
    - nu pre- and nu post-sweeps of l1-Jacobi (D_l1 = sum_j |A_ij|, omega = 1),
      zero initial guess on every level, coarse correction added unscaled;
    - cycle = 1 (V-cycle) or 2 (W-cycle: the coarse correction is computed
      twice, each time from the current residual, on every level whose coarse
      level is not the coarsest; above the coarsest one exact correction);
      `w_levels` = k > 0 limits the repetition to levels 0..k-1 (V below);
    - coarsest level: dense Cholesky; when S~ is singular (pure Neumann Darcy
      with gamma = 0) it factors A + s 1 1^T with s = mean(diag A)/n;
    - singular case: the result is projected to zero mean (Sec. 4.2).
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .assembly import GRAD_DIV


def approx_schur(prob):
    """Returns (S~ as CSR, M~ diagonal (1 on essential dofs), C~ diagonal)."""
    Mt = prob.M.diagonal().copy()
    E = prob.lat.n_elem
    wdiag = np.einsum("eaa->ea", prob.We)                 # (E, k^3)
    if prob.kind == GRAD_DIV:
        ct_loc = 1.0 / wdiag
    else:
        gdiag = prob.gamma[:, None] * wdiag               # diag(W_gamma) for per-element gamma
        ct_loc = gdiag / (wdiag * wdiag)
    Ct = np.zeros(prob.lat.n_l2)
    Ct[prob.e2l.ravel()] = ct_loc.ravel()
    S = (sp.diags(Ct) + prob.D @ sp.diags(1.0 / Mt) @ prob.D.T).tocsr()
    return S, Mt, Ct


def element_groups(c):
    """Aggregate index of each of the c cells that one element holds along an axis, for
    element-aligned aggregation: pairs taken alternately from the two ends of the element
    (the first from its low end), an odd count leaving one single cell in the middle;
    c = 3 gives groups [2, 1], c = 5 gives [2, 1, 2], c = 4 gives [2, 2]."""
    lo, hi, sizes_lo, sizes_hi = 0, c, [], []
    take_low = True
    while hi - lo >= 2:
        if take_low:
            sizes_lo.append(2)
            lo += 2
        else:
            sizes_hi.append(2)
            hi -= 2
        take_low = not take_low
    sizes = sizes_lo + ([1] if hi - lo == 1 else []) + sizes_hi[::-1]
    return np.repeat(np.arange(len(sizes)), sizes), len(sizes)


def aggregation(dims, elems=None):
    """P (fine cells x coarse cells) for 2-per-direction aggregation; coarse dims.

    elems = (nx, ny, nz) element counts selects element-aligned aggregation: along an
    axis whose length is c > 1 cells per element, the aggregates are element_groups(c)
    inside each element, so that no aggregate straddles an element boundary; an axis
    with one cell per element (or not a multiple of its element count) takes the pairs
    of the default."""
    X, Y, Z = dims
    maps = []
    for n, ne in zip(dims, elems if elems is not None else (None,) * 3):
        if n == 1:
            maps.append((np.zeros(1, dtype=np.int64), 1))
        elif ne is not None and n % ne == 0 and n // ne > 1:
            g, m = element_groups(n // ne)
            maps.append((np.arange(n) // (n // ne) * m + np.tile(g, ne), ne * m))
        else:
            maps.append((np.arange(n) // 2, (n + 1) // 2))
    (ix, cx), (iy, cy), (iz, cz) = maps
    I, J, K = np.meshgrid(np.arange(X), np.arange(Y), np.arange(Z), indexing="ij")
    fine = (I + X * (J + Y * K)).ravel()
    coarse = (ix[I] + cx * (iy[J] + cy * iz[K])).ravel()
    P = sp.coo_matrix((np.ones(fine.size), (fine, coarse)), shape=(X * Y * Z, cx * cy * cz)).tocsr()
    return P, (cx, cy, cz)


def l1_diag(A):
    """l1-Jacobi diagonal: D_l1 = sum_j |A_ij|."""
    return np.asarray(abs(A).sum(axis=1)).ravel()


class VCycle:
    def __init__(self, A0, dims, nu=2, coarse_max=512, singular=False, max_levels=20, cycle=1,
                 smooth=0.0, sa_levels=1, w_levels=0, elems=None):
        self.nu, self.singular, self.cycle, self.w_levels = nu, singular, cycle, w_levels
        self.A, self.P, self.dims, self.dl1 = [A0.tocsr()], [], [tuple(dims)], []
        while np.prod(self.dims[-1]) > coarse_max and len(self.A) < max_levels:
            P, cd = aggregation(self.dims[-1], elems)
            if cd == self.dims[-1]:
                break
            if smooth and len(self.P) < sa_levels:
                A = self.A[-1]
                P = (P - smooth * sp.diags(1.0 / l1_diag(A)) @ (A @ P)).tocsr()
            self.P.append(P)
            self.A.append((P.T @ self.A[-1] @ P).tocsr())
            self.dims.append(cd)
        for A in self.A:
            self.dl1.append(l1_diag(A))
        Ac = self.A[-1].toarray()
        if singular:
            n = Ac.shape[0]
            Ac = Ac + (np.mean(np.diag(Ac)) / n) * np.ones((n, n))
        self.chol = sla.cho_factor(Ac, lower=True)

    @property
    def n_levels(self):
        return len(self.A)

    def _cycle(self, l, b):
        if l == len(self.A) - 1:
            return sla.cho_solve(self.chol, b)
        A, d = self.A[l], self.dl1[l]
        x = np.zeros_like(b)
        for _ in range(self.nu):
            x = x + (b - A @ x) / d
        repeats = self.cycle if (l + 1 < len(self.A) - 1 and (self.w_levels <= 0 or l < self.w_levels)) else 1
        for _ in range(repeats):
            r = b - A @ x
            x = x + self.P[l] @ self._cycle(l + 1, self.P[l].T @ r)
        for _ in range(self.nu):
            x = x + (b - A @ x) / d
        return x

    def apply(self, b):
        z = self._cycle(0, np.asarray(b, dtype=np.float64))
        if self.singular:
            z = z - z.mean()
        return z


def is_singular(prob, Ct):
    """S~ is singular (constants in its kernel) exactly when C~ vanishes and no
    boundary face is free: every row of D M~^-1 D^T then sums to zero."""
    boundary = prob.lat.ess_dofs(63)
    return bool(np.all(Ct == 0.0)) and bool(np.all(~prob.free[boundary]))


class BlockPrec:
    """z = B^-1 r with B = diag(tau M~, S^)."""

    def __init__(self, prob, tau=1.0, nu=2, coarse_max=512, cycle=1, smooth=0.0, sa_levels=1, w_levels=0,
                 aligned=False):
        self.prob, self.tau = prob, tau
        self.S, self.Mt, self.Ct = approx_schur(prob)
        self.singular = is_singular(prob, self.Ct)
        lat = prob.lat
        self.vc = VCycle(self.S, (lat.X, lat.Y, lat.Z), nu=nu, coarse_max=coarse_max,
                         singular=self.singular, cycle=cycle, smooth=smooth, sa_levels=sa_levels,
                         w_levels=w_levels, elems=(lat.nx, lat.ny, lat.nz) if aligned else None)

    def apply(self, r):
        nrt = self.prob.lat.n_rt
        ru, rq = r[:nrt], r[nrt:]
        zu = np.where(self.prob.free, ru / (self.tau * self.Mt), ru)
        zq = self.vc.apply(rq)
        return np.concatenate([zu, zq])


class BlockTriPrec(BlockPrec):
    """z = P^-1 r with the block upper-triangular P = [[tau M~, D^T], [0, -S^]]
    (the remark on block-triangular preconditioners in Sec. 2.3), for GMRES:
    z_q = -S^-1 r_q (the V/W-cycle of BlockPrec), then
    z_u = (r_u - D^T z_q) / (tau M~) on free dofs and z_u = r_u on essential dofs
    (D has no columns for them, so D^T z_q vanishes there)."""

    def apply(self, r):
        nrt = self.prob.lat.n_rt
        ru, rq = r[:nrt], r[nrt:]
        zq = -self.vc.apply(rq)
        zu = np.where(self.prob.free, (ru - self.prob.apply_Bt(zq)) / (self.tau * self.Mt), ru)
        return np.concatenate([zu, zq])

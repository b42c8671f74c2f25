"""1D points and bases of the interpolation-histopolation basis (Sec. 2.1).

The reference interval is [0, 1]. With k = the paper's degree p (number of
subcells per direction):

* Gauss-Lobatto (GLL) nodes xi_0 = 0 < ... < xi_k = 1: the endpoints plus the
  roots of P_k' (Legendre), mapped from [-1, 1]. They are the subcell vertices
  (Fig. lor-cube).
* l_i, i = 0..k: the degree-k Lagrange polynomials at the GLL nodes (the
  interpolation basis: l_i(xi_m) = delta_im).
* h_j, j = 0..k-1: the degree-(k-1) histopolation basis, defined by the DOFs
  "integral over subcell m": int_{xi_m}^{xi_{m+1}} h_j = delta_mj. It equals
  sum_{i>j} l_i', because int_{xi_m}^{xi_{m+1}} l_i' = delta_{i,m+1} - delta_{i,m}.
* Gauss-Legendre (GL) points and weights on [0, 1] (quadrature; also the nodal
  basis used for the local L2 mass solve, Sec. 2.5).
"""
import numpy as np


def legendre_and_derivs(n, x):
    """P_n(x), P_n'(x), P_n''(x) on [-1, 1] by the three-term recurrence."""
    x = np.asarray(x, dtype=np.float64)
    p0 = np.ones_like(x)
    if n == 0:
        return p0, np.zeros_like(x), np.zeros_like(x)
    p1 = x.copy()
    d0, d1 = np.zeros_like(x), np.ones_like(x)
    dd0, dd1 = np.zeros_like(x), np.zeros_like(x)
    for m in range(1, n):
        # (m+1) P_{m+1} = (2m+1) x P_m - m P_{m-1}, differentiated twice
        p2 = ((2 * m + 1) * x * p1 - m * p0) / (m + 1)
        d2 = ((2 * m + 1) * (p1 + x * d1) - m * d0) / (m + 1)
        dd2 = ((2 * m + 1) * (2 * d1 + x * dd1) - m * dd0) / (m + 1)
        p0, p1, d0, d1, dd0, dd1 = p1, p2, d1, d2, dd1, dd2
    return p1, d1, dd1


def gll_nodes(k):
    """k+1 Gauss-Lobatto nodes on [0, 1]: 0, 1 and the roots of P_k' (Newton)."""
    if k < 1:
        raise ValueError("k >= 1")
    t = -np.cos(np.pi * np.arange(k + 1) / k)  # Chebyshev-Gauss-Lobatto start
    inner = t[1:-1].copy()
    for _ in range(100):
        _, d, dd = legendre_and_derivs(k, inner)
        step = d / dd
        inner -= step
        if np.max(np.abs(step), initial=0.0) < 1e-16:
            break
    t[1:-1] = inner
    t[0], t[-1] = -1.0, 1.0
    return 0.5 * (t + 1.0)


def gl_points(q):
    """q Gauss-Legendre points and weights on [0, 1] (library routine, rescaled)."""
    t, w = np.polynomial.legendre.leggauss(q)
    return 0.5 * (t + 1.0), 0.5 * w


def lagrange(nodes, x):
    """Values L[i, m] = l_i(x_m) of the Lagrange basis on `nodes` (product formula)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    L = np.ones((n, len(x)))
    for i in range(n):
        for m in range(n):
            if m != i:
                L[i] *= (x - nodes[m]) / (nodes[i] - nodes[m])
    return L


def lagrange_deriv(nodes, x):
    """Derivatives dL[i, m] = l_i'(x_m): sum over the dropped factor of the product."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    dL = np.zeros((n, len(x)))
    for i in range(n):
        for m in range(n):
            if m == i:
                continue
            term = np.full(len(x), 1.0 / (nodes[i] - nodes[m]))
            for r in range(n):
                if r != i and r != m:
                    term = term * (x - nodes[r]) / (nodes[i] - nodes[r])
            dL[i] += term
    return dL


def interp_basis(k, x):
    """I[i, m] = l_i(x_m), i = 0..k, Lagrange at the GLL nodes."""
    return lagrange(gll_nodes(k), x)


def interp_basis_deriv(k, x):
    return lagrange_deriv(gll_nodes(k), x)


def histo_basis(k, x):
    """H[j, m] = h_j(x_m) = sum_{i>j} l_i'(x_m), j = 0..k-1."""
    dL = interp_basis_deriv(k, x)
    H = np.zeros((k, dL.shape[1]))
    for j in range(k):
        H[j] = dL[j + 1:].sum(axis=0)
    return H

"""Condition-number studies of Sec. 2.5 (the L2 mass in three bases) and of the
transformed versus the untransformed Schur complement (the notes on the
untransformed system), by dense eigenvalues on single elements.

Test infrastructure: only tests/ use it.

* l2_mass_conditions: the L2 mass W_e of one element (histopolation basis, full
  quadrature) changed to the Gauss-Lobatto and the Gauss-Legendre nodal bases of the
  same space Q_{k-1}, each scaled by its diagonal: kappa(D^-1/2 W D^-1/2).
* schur_conditions: for the transformed system, kappa(S~^-1 S) with
  S = W^-1 + D M^-1 D^T and S~ = diag(W)^-1 + D diag(M)^-1 D^T; for the
  untransformed one, kappa(S~'^-1 S') with S' = W + W D M^-1 D^T W and
  S~' = diag(W) + diag(W) D diag(M)^-1 D^T diag(W) (every factor replaced by its
  diagonal). Grad-div with alpha = beta = 1 on one element, natural boundary
  conditions (every RT dof free).
"""
import numpy as np
import scipy.linalg as sla

from . import basis1d, element
from .assembly import GRAD_DIV, Problem


def _subcell_integrals(nodes, k):
    """T[j, m] = integral over subcell j (between consecutive Gauss-Lobatto points of
    the k + 1 subcell boundaries) of the Lagrange polynomial m on `nodes` (k points):
    the histopolation coefficients of that nodal basis function."""
    xi = basis1d.gll_nodes(k)
    t, w = np.polynomial.legendre.leggauss(k + 2)
    T = np.zeros((k, k))
    for j in range(k):
        a, b = xi[j], xi[j + 1]
        x = 0.5 * (b - a) * t + 0.5 * (a + b)
        T[j] = basis1d.lagrange(nodes, x) @ (0.5 * (b - a) * w)
    return T


def _scaled_cond(A):
    d = 1.0 / np.sqrt(np.diag(A))
    ev = np.linalg.eigvalsh(A * np.outer(d, d))
    return ev[-1] / ev[0]


def l2_mass_conditions(V, k, q=None):
    """{'histopolation', 'gauss_lobatto', 'gauss_legendre'} -> condition number of the
    diagonally scaled L2 mass of the element with corners V (shape (1, 2, 2, 2, 3))."""
    q = q or k + 2
    W = element.element_matrices(V, k, q, np.array([1.0]), np.array([1.0]), want=("W",))["W"][0]
    out = {"histopolation": _scaled_cond(W)}
    for name, nodes in (("gauss_lobatto", basis1d.gll_nodes(k - 1) if k > 1 else np.array([0.5])),
                        ("gauss_legendre", basis1d.gl_points(k)[0])):
        T1 = _subcell_integrals(nodes, k)
        T = np.kron(T1, np.kron(T1, T1))
        out[name] = _scaled_cond(T.T @ W @ T)
    return out


def _generalised_cond(A, B):
    ev = sla.eigh(A, B, eigvals_only=True)
    return ev[-1] / ev[0]


def schur_conditions(vx, vy, vz, k, q=None):
    """(kappa(S~^-1 S), kappa(S~'^-1 S')) on the single element with vertex arrays
    vx, vy, vz (2 x 2 x 2 lattice vertices)."""
    q = q or k + 2
    prob = Problem(1, 1, 1, k, vx, vy, vz, np.ones(1), np.ones(1), kind=GRAD_DIV, ess_mask=0, q=q)
    M = prob.M.toarray()
    D = prob.D.toarray()
    C = prob.C.toarray()                 # W_alpha^-1
    W = np.linalg.inv(C)
    Mi = np.linalg.inv(M)
    S = C + D @ Mi @ D.T
    St = np.diag(1.0 / np.diag(W)) + D @ np.diag(1.0 / np.diag(M)) @ D.T
    Sp = W + W @ D @ Mi @ D.T @ W
    dW = np.diag(np.diag(W))
    Stp = dW + dW @ D @ np.diag(1.0 / np.diag(M)) @ D.T @ dW
    return _generalised_cond(S, St), _generalised_cond(Sp, Stp)

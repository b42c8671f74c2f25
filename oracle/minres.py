"""Preconditioned MINRES (Paige & Saunders 1975) in FP64.

The paper solves the transformed system with block-diagonally preconditioned
MINRES (Sec. 3) but prints no listing. This is the textbook method: a
preconditioned Lanczos process for the symmetric operator A with SPD
preconditioner B (applied as B^-1), and a QR factorisation of the Lanczos
tridiagonal by Givens rotations, updated one column per iteration.

Stopping: eta_j <= rtol * eta_0, where eta_j is the B^-1-norm of the residual
that the recurrence carries (the paper states only "relative tolerance").
"""
import numpy as np


def minres(apply_A, apply_Binv, b, x0=None, rtol=1e-8, maxit=1000):
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    r_prev = b - apply_A(x) if x0 is not None else b.copy()   # unpreconditioned Lanczos vector
    z = apply_Binv(r_prev)
    beta = np.sqrt(r_prev @ z)                 # beta_1 = ||r_0||_{B^-1}
    eta0 = beta
    hist = [eta0]
    if beta == 0.0:
        return x, {"iterations": 0, "eta": hist, "converged": True}
    r_prevprev = np.zeros(n)
    beta_prev = 0.0
    # Givens state and the two previous search directions
    c_prev, s_prev = -1.0, 0.0
    d_bar, eps_next = 0.0, 0.0
    phi_bar = beta
    w, w_prev = np.zeros(n), np.zeros(n)
    converged = False
    it = 0
    for it in range(1, maxit + 1):
        # Lanczos step: v_j = z / beta_j, new unpreconditioned vector
        v = z / beta
        y = apply_A(v)
        if it > 1:
            y = y - (beta / beta_prev) * r_prevprev
        alpha = v @ y
        y = y - (alpha / beta) * r_prev
        r_prevprev, r_prev = r_prev, y
        z = apply_Binv(r_prev)
        beta_prev, beta = beta, np.sqrt(r_prev @ z)
        # apply the previous rotation to the new column, then make a new one
        eps = eps_next
        delta = c_prev * d_bar + s_prev * alpha
        g_bar = s_prev * d_bar - c_prev * alpha
        eps_next = s_prev * beta
        d_bar = -c_prev * beta
        gamma = np.hypot(g_bar, beta)
        c_prev, s_prev = g_bar / gamma, beta / gamma
        phi = c_prev * phi_bar
        phi_bar = s_prev * phi_bar
        # search direction and solution update
        w_prevprev, w_prev = w_prev, w
        w = (v - eps * w_prevprev - delta * w_prev) / gamma
        x = x + phi * w
        hist.append(abs(phi_bar))
        if abs(phi_bar) <= rtol * eta0:
            converged = True
            break
    return x, {"iterations": it, "eta": hist, "converged": converged}

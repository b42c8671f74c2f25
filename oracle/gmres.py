"""Restarted, right-preconditioned GMRES (Saad & Schultz 1986) in FP64.

Test infrastructure: the CPU reference for the GPU GMRES; only tests/, smoke() and
the benchmark's CPU baseline use it.

The paper remarks (Sec. 2.3) that the block upper-triangular preconditioner
[[M, D^T], [0, -S]] makes the preconditioned saddle-point operator have the single
eigenvalue 1 with a minimal polynomial of degree two, so that GMRES converges in
at most two iterations with exact blocks; being non-symmetric it needs GMRES
instead of MINRES. It prints no listing. This is the textbook method:

* right preconditioning: x = x0 + P^-1 V_j y minimises ||b - A x||_2 over the
  Krylov space K_j(A P^-1, r0), so the recurrence estimates the true residual;
* Arnoldi with classical Gram-Schmidt applied twice per step (the two-pass
  orthogonalisation, stable like modified Gram-Schmidt);
* the Hessenberg least-squares problem by Givens rotations, one column per step;
* restart after `restart` steps from the true residual; stop when the estimate
  reaches rtol ||b||_2 and confirm with the true residual (else restart).
"""
import numpy as np


def gmres(apply_A, apply_Pinv, b, x0=None, rtol=1e-8, maxit=1000, restart=50):
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bn = np.linalg.norm(b)
    its, cycles = 0, 0
    hist = []
    converged = bn == 0.0
    while not converged and its < maxit:
        r = b - apply_A(x)
        beta = np.linalg.norm(r)
        hist.append(beta / bn)
        if beta <= rtol * bn:
            converged = True
            break
        cycles += 1
        m = min(restart, maxit - its)
        V = np.zeros((m + 1, n))
        V[0] = r / beta
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        j = 0
        while j < m:
            w = apply_A(apply_Pinv(V[j]))
            for _ in range(2):
                h = V[:j + 1] @ w
                w = w - V[:j + 1].T @ h
                H[:j + 1, j] += h
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):          # previous rotations on the new column
                a, c = H[i, j], H[i + 1, j]
                H[i, j], H[i + 1, j] = cs[i] * a + sn[i] * c, -sn[i] * a + cs[i] * c
            d = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / d, H[j + 1, j] / d
            H[j, j], H[j + 1, j] = d, 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            j += 1
            its += 1
            hist.append(abs(g[j]) / bn)
            if abs(g[j]) <= rtol * bn:
                break
        y = np.linalg.solve(np.triu(H[:j, :j]), g[:j])
        x = x + apply_Pinv(V[:j].T @ y)
        converged = np.linalg.norm(b - apply_A(x)) <= rtol * bn
    relres = np.linalg.norm(b - apply_A(x)) / bn if bn > 0 else 0.0
    return x, {"iterations": its, "cycles": cycles, "estimate": hist, "true_relres": relres,
               "converged": bool(converged)}

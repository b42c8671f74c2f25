"""A manufactured solution of the grey radiation-diffusion equations (Sec. 4.3, Eq.
rad-diff-e, rad-diff-E, rad-diff-F) on the unit cube, and the sources that make it exact.

The paper's own manufactured solution is not available here, so this one stands in for it:

    g(x)   = cos(pi x) cos(pi y) cos(pi z)
    T(x,t) = 1 + A_T g(x) exp(-t),           e = Cv T
    E(x,t) = a (1 + A_E g(x) exp(-2 t))
    F      = -(c / (3 sigma)) grad E          (F.n = 0 on every face of the cube)
    Q      = rho de/dt + c sigma (a T^4 - E)
    S      = dE/dt + div F - c sigma (a T^4 - E)

with constant rho, Cv, a, c and sigma. These are closed-form problem data: the module holds
none of the discretisation's arithmetic, so the CUDA path and the oracle both sample it.
"""
import numpy as np

A_T, A_E = 0.3, 0.5


def fields(X, t, rho=1.0, cv=1.0, a=1.0, c=1.0, sigma=1.0):
    """(e, E, F, Q, S) at the points X (..., 3) and time t."""
    x, y, z = X[..., 0], X[..., 1], X[..., 2]
    pi = np.pi
    cx, cy, cz = np.cos(pi * x), np.cos(pi * y), np.cos(pi * z)
    sx, sy, sz = np.sin(pi * x), np.sin(pi * y), np.sin(pi * z)
    g = cx * cy * cz
    et, e2t = np.exp(-t), np.exp(-2.0 * t)
    T = 1.0 + A_T * g * et
    e = cv * T
    E = a * (1.0 + A_E * g * e2t)
    grad_g = np.stack([-pi * sx * cy * cz, -pi * cx * sy * cz, -pi * cx * cy * sz], axis=-1)
    kappa = c / (3.0 * sigma)
    F = -kappa * a * A_E * e2t * grad_g
    lap_g = -3.0 * pi * pi * g
    div_F = -kappa * a * A_E * e2t * lap_g
    de_dt = -cv * A_T * g * et
    dE_dt = -2.0 * a * A_E * g * e2t
    coupling = c * sigma * (a * T ** 4 - E)
    Q = rho * de_dt + coupling
    S = dE_dt + div_F - coupling
    return e, E, F, Q, S

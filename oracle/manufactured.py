"""Right-hand sides and errors for manufactured solutions (grad-div).

The grad-div problem -grad(alpha div u) + beta u = f (Eq. grad-div) becomes the
transformed system [[M, D^T], [D, -W_alpha^-1]] [u; q~] = [f_h; 0] (Eq.
transformed-saddle-point) with (f_h)_n = (f, phi_n) = int f(T(xi)) . J phi_hat_n dxi
(the Piola-mapped basis times det J). Essential dofs carry the prescribed
normal flux, here zero.
"""
import numpy as np

from . import element


def sinusoid_field(X):
    """u = (s, s, s), s = sin(pi x) sin(pi y) sin(pi z); its divergence and
    f = -grad(div u) + u for alpha = beta = 1."""
    x, y, z = X[..., 0], X[..., 1], X[..., 2]
    pi = np.pi
    sx, sy, sz = np.sin(pi * x), np.sin(pi * y), np.sin(pi * z)
    cx, cy, cz = np.cos(pi * x), np.cos(pi * y), np.cos(pi * z)
    s = sx * sy * sz
    u = np.stack([s, s, s], axis=-1)
    div = pi * (cx * sy * sz + sx * cy * sz + sx * sy * cz)
    # grad(div u)
    gx = pi * pi * (-sx * sy * sz + cx * cy * sz + cx * sy * cz)
    gy = pi * pi * (cx * cy * sz - sx * sy * sz + sx * cy * cz)
    gz = pi * pi * (cx * sy * cz + sx * cy * cz - sx * sy * sz)
    f = u - np.stack([gx, gy, gz], axis=-1)
    return u, div, f


def rt_load(prob, f_fn, qf=None):
    """(f, phi_n) assembled over elements with a qf^3 Gauss rule."""
    lat, k = prob.lat, prob.k
    qf = k + 2 if qf is None else qf
    pts, w = element.quad_rule(qf)
    V = prob.V
    J = element.jacobian(V, pts)
    Xp = element.physical_points(V, pts)
    Phi, _ = element.rt_basis(k, pts)
    f = f_fn(Xp)                                            # (E, P, 3)
    Jphi = np.einsum("epid,pnd->epni", J, Phi)
    loc = np.einsum("epi,epni,p->en", f, Jphi, w)
    b = np.zeros(lat.n_rt)
    np.add.at(b, prob.e2d_idx.ravel(), (loc * prob.e2d_sign).ravel())
    return b


def l2_errors(prob, u_h, q_h, u_fn, qe=None):
    """||u - u_h||_L2 and ||div u - div u_h||_L2 with a qe^3 Gauss rule; q_h holds the
    L2 dofs of div u_h (q = W^-1 q~)."""
    lat, k = prob.lat, prob.k
    qe = k + 3 if qe is None else qe
    pts, w = element.quad_rule(qe)
    V = prob.V
    J = element.jacobian(V, pts)
    detJ = np.linalg.det(J)
    Xp = element.physical_points(V, pts)
    Phi, _ = element.rt_basis(k, pts)
    Psi = element.l2_basis(k, pts)
    ue = u_h[prob.e2d_idx] * prob.e2d_sign                     # (E, n)
    uh_hat = np.einsum("pnd,en->epd", Phi, ue)
    uh = np.einsum("epid,epd->epi", J, uh_hat) / detJ[..., None]
    qh = np.einsum("pa,ea->ep", Psi, q_h[prob.e2l]) / detJ
    u, div, _ = u_fn(Xp)
    eu = np.sqrt(np.sum(np.sum((u - uh) ** 2, axis=-1) * detJ * w))
    ed = np.sqrt(np.sum((div - qh) ** 2 * detJ * w))
    return eu, ed

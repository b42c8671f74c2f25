"""Grey nonlinear radiation diffusion (Sec. 4.3): the three-stage SDIRK time integrator,
the outer fixed-point iteration and the element-wise Newton solve that drive the repeated
Darcy-type solves of Eq. darcy-nonzero.

TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's CPU legs use this
module. It is the plain, slow FP64 statement of what the GPU path computes and shares no
code with it.

Equations (Eq. rad-diff-e, rad-diff-E, rad-diff-F), with T = e / Cv:

    rho de/dt     = -c sigma (a T^4 - E) + Q
    dE/dt + div F =  c sigma (a T^4 - E) + S
    F             = -(c / (3 sigma)) grad E

e and E lie in the L2 space W_h, and F lies in the RT space V_h. The walls reflect
(F.n = 0 on every side, as essential RT faces), so the boundary term of E vanishes and
(3 sigma / c) (F, v) - (E, div v) = 0. The opacity sigma is constant on each element.

Unknowns. E is carried as Eh = W E, with W the L2 mass. This is the transformed L2 unknown
of Eq. transformed-system-darcy up to its sign. A stage with diagonal coefficient a_ii and
beta = 1 / (dt a_ii) solves the following, for stage-start values (e*, Eh*) and source
loads Q_j = (Q, psi_j), S_j = (S, psi_j):

    R1 = rho beta W (e - e*) + c sigma (a N(e) - Eh) - Q            = 0
    R2 = beta (Eh - Eh*) + W D F - c sigma (a N(e) - Eh) - S        = 0
    R3 = M_{3 sigma / c} F - D^T Eh                                  = 0

Here N(e)_j = (T(e)^4, psi_j) by the element quadrature (q^3 Gauss points). D is the
lattice divergence, so that (div F, psi_j) = (W D F)_j. The essential rows of R3 are F.

The stage iteration follows Sec. 4.3. First F is lagged and (R1, R2) are solved for
(e, Eh), element by element, by Newton's method on the coupled 2n x 2n element system.
Then e is fixed and (R2, R3) are solved for (Eh, F). That is the Darcy system of Eq.
transformed-system-darcy with eps = c / (3 sigma), gamma = beta + c sigma, x = [F; -Eh]
and right-hand side [0; W^-1 G], where G = S + c sigma a N(e) + beta Eh*. The two steps
repeat until ||(R1, R2, R3)|| <= outer_rtol times its value at the stage's initial guess,
or until the residual, already below 1e3 outer_rtol times that value, no longer halves
from one pass to the next (its rounding floor, which lies above 1e-12 on finer meshes). The Newton solve stops per element once
||(R1_e, R2_e)|| <= newton_rtol times its first value, or <= 1e-14 times the size of the
element's leading terms ||(rho beta W e_e, beta Eh_e)|| (the rounding floor: later passes
start close to it). Here the Newton systems are solved densely and the Darcy system
directly (sparse LU): the plain definitions of both steps.
"""

import numpy as np
import scipy.sparse.linalg as spla

from . import element
from .assembly import DARCY, Problem

ALL_WALLS = 63
NEWTON_FLOOR = 1e-14


def sdirk3():
    """Alexander's three-stage, L-stable, stiffly accurate SDIRK method (order 3):
    (A, b, c). The diagonal gamma is the root in (1/6, 1/2) of 6x^3 - 18x^2 + 9x - 1,
    c = (gamma, (1 + gamma) / 2, 1), a21 = (1 - gamma) / 2, and the last row of A is b
    with b1 = -(6 gamma^2 - 16 gamma + 1) / 4, b2 = (6 gamma^2 - 20 gamma + 5) / 4,
    b3 = gamma."""
    r = np.roots([6.0, -18.0, 9.0, -1.0])
    r = np.real(r[np.abs(np.imag(r)) < 1e-12])
    g = float(r[(r > 1.0 / 6.0) & (r < 0.5)][0])
    b1 = -(6 * g * g - 16 * g + 1) / 4.0
    b2 = (6 * g * g - 20 * g + 5) / 4.0
    A = np.array([[g, 0.0, 0.0], [(1 - g) / 2.0, g, 0.0], [b1, b2, g]])
    return A, A[2].copy(), np.array([g, (1 + g) / 2.0, 1.0])


class RadDiff:
    """The discretised radiation-diffusion system on a structured hex mesh."""

    def __init__(self, nx, ny, nz, k, vx, vy, vz, sigma, dt, rho=1.0, cv=1.0, a=1.0, c=1.0, q=None):
        A, _, _ = sdirk3()
        self.dt, self.rho, self.cv, self.a, self.c = float(dt), float(rho), float(cv), float(a), float(c)
        self.beta = 1.0 / (self.dt * A[0, 0])
        E = nx * ny * nz
        self.sigma = np.broadcast_to(np.asarray(sigma, dtype=np.float64), (E,)).copy()
        eps = self.c / (3.0 * self.sigma)
        gam = self.beta + self.c * self.sigma
        self.prob = p = Problem(nx, ny, nz, k, vx, vy, vz, eps, gam, kind=DARCY, ess_mask=ALL_WALLS, q=q)
        self.k, self.q = k, p.q
        self.pts, self.w = element.quad_rule(p.q)
        self.Psi = element.l2_basis(k, self.pts)                        # (P, n)
        self.detJ = np.linalg.det(element.jacobian(p.V, self.pts))      # (E, P)
        self.e2l = p.e2l                                                # (E, n)
        self.We = p.We                                                  # unweighted L2 mass
        self.Winv = np.linalg.inv(p.We)
        self.cs = self.c * self.sigma                                   # per element
        self.AA = spla.splu(p.matrix().tocsc())  # the same matrix for every stage (a_ii is constant)
        self.n_l2, self.n_rt = p.lat.n_l2, p.lat.n_rt

    # -- element-local helpers ------------------------------------------------
    def _loc(self, v):
        return v[self.e2l]

    def _glob(self, v_loc):
        out = np.zeros(self.n_l2)
        out[self.e2l] = v_loc
        return out

    def temperature(self, e_loc, sel=slice(None)):
        """T at the quadrature points (E, P) from local coefficients (of the elements sel)."""
        return np.einsum("pa,ea->ep", self.Psi, e_loc) / self.detJ[sel] / self.cv

    def emission(self, e_loc):
        """N(e)_j = sum_p w_p T_p^4 psi_j(p), local (E, n)."""
        T = self.temperature(e_loc)
        return np.einsum("ep,pj->ej", self.w[None, :] * T ** 4, self.Psi)

    def emission_jacobian(self, e_loc, sel=slice(None)):
        """dN_j / de_a = sum_p w_p 4 T_p^3 psi_a psi_j / (Cv det J_p), (E, n, n)."""
        T = self.temperature(e_loc, sel)
        wt = self.w[None, :] * 4.0 * T ** 3 / (self.cv * self.detJ[sel])
        return np.einsum("pa,ep,pb->eab", self.Psi, wt, self.Psi)

    def mass(self, v_loc):
        return np.einsum("eab,eb->ea", self.We, v_loc)

    # -- residuals ---------------------------------------------------------------
    def residual_12(self, e, Eh, F, e_star, Eh_star, Ql, Sl):
        """(R1, R2) as local arrays (E, n)."""
        el, Ehl = self._loc(e), self._loc(Eh)
        WDF = self.mass(self._loc(self.prob.apply_B(F)))
        aN = self.a * self.emission(el)
        cs = self.cs[:, None]
        R1 = self.rho * self.beta * self.mass(el - self._loc(e_star)) + cs * (aN - Ehl) - self._loc(Ql)
        R2 = self.beta * (Ehl - self._loc(Eh_star)) + WDF - cs * (aN - Ehl) - self._loc(Sl)
        return R1, R2

    def residual(self, e, Eh, F, e_star, Eh_star, Ql, Sl):
        """The full stage residual (R1, R2, R3) as one vector: R1, R2 in L2 lattice order,
        then R3 (RT order)."""
        R1, R2 = self.residual_12(e, Eh, F, e_star, Eh_star, Ql, Sl)
        R3 = self.prob.apply_op(np.concatenate([F, -Eh]))[: self.n_rt]
        return np.concatenate([self._glob(R1), self._glob(R2), R3])

    # -- the two steps of the stage iteration ------------------------------------------
    def newton(self, e, Eh, F, e_star, Eh_star, Ql, Sl, rtol=1e-8, maxit=30):
        """F fixed: Newton on (R1, R2) for (e, Eh), each element on its own 2n x 2n system.
        Returns (e, Eh, the largest number of Newton steps an element took)."""
        e, Eh = e.copy(), Eh.copy()
        E, n = self.e2l.shape
        cs = self.cs[:, None, None]
        I = np.eye(n)[None]
        r0 = None
        steps = 0
        for it in range(maxit + 1):
            R1, R2 = self.residual_12(e, Eh, F, e_star, Eh_star, Ql, Sl)
            rn = np.sqrt(np.sum(R1 * R1 + R2 * R2, axis=1))
            if r0 is None:
                r0 = rn
            el, Ehl = self._loc(e), self._loc(Eh)
            scale = np.sqrt(np.sum((self.rho * self.beta * self.mass(el)) ** 2 + (self.beta * Ehl) ** 2, axis=1))
            act = (rn > rtol * r0) & (rn > NEWTON_FLOOR * scale)
            if not act.any() or it == maxit:
                break
            dN = self.a * self.emission_jacobian(el[act], act)
            J11 = self.rho * self.beta * self.We[act] + cs[act] * dN
            J12 = -cs[act] * I
            J21 = -cs[act] * dN
            J22 = (self.beta + cs[act]) * I
            Jac = np.concatenate([np.concatenate([J11, J12], axis=2), np.concatenate([J21, J22], axis=2)], axis=1)
            rhs = -np.concatenate([R1[act], R2[act]], axis=1)
            d = np.linalg.solve(Jac, rhs[..., None])[..., 0]
            idx = self.e2l[act]
            e[idx] += d[:, :n]
            Eh[idx] += d[:, n:]
            steps = it + 1
        return e, Eh, steps

    def darcy(self, e, Eh_star, Sl):
        """e fixed: (R2, R3) = 0 for (Eh, F) by a direct solve of the transformed Darcy system."""
        G = self._loc(Sl) + self.cs[:, None] * self.a * self.emission(self._loc(e)) + self.beta * self._loc(Eh_star)
        rhs = np.concatenate([np.zeros(self.n_rt), self._glob(np.einsum("eab,eb->ea", self.Winv, G))])
        x = self.AA.solve(rhs)
        return -x[self.n_rt:], x[: self.n_rt]

    def stage(self, e_star, Eh_star, Ql, Sl, e, Eh, F, outer_rtol=1e-12, outer_maxit=10, newton_rtol=1e-8,
              newton_maxit=30):
        """One stage: the outer iteration from the initial guess (e, Eh, F). Returns
        (e, Eh, F, info) with info = {outer, newton_max, relres}."""
        Ql = np.zeros(self.n_l2) if Ql is None else Ql
        Sl = np.zeros(self.n_l2) if Sl is None else Sl
        r0 = np.linalg.norm(self.residual(e, Eh, F, e_star, Eh_star, Ql, Sl))
        info = {"outer": 0, "newton_max": 0, "relres": 0.0}
        if r0 == 0.0:
            return e.copy(), Eh.copy(), F.copy(), info
        r_prev = r0
        for m in range(outer_maxit):
            e, Eh, s = self.newton(e, Eh, F, e_star, Eh_star, Ql, Sl, newton_rtol, newton_maxit)
            Eh, F = self.darcy(e, Eh_star, Sl)
            r = np.linalg.norm(self.residual(e, Eh, F, e_star, Eh_star, Ql, Sl))
            info["outer"] = m + 1
            info["newton_max"] = max(info["newton_max"], s)
            info["relres"] = r / r0
            if r <= outer_rtol * r0 or (r > 0.5 * r_prev and r <= 1e3 * outer_rtol * r0):
                break
            r_prev = r
        return e, Eh, F, info

    def step(self, e, Eh, F, loads=None, **kw):
        """One SDIRK3 step of size dt from (e, Eh, F). loads: None (no sources) or three
        (Q_load, S_load) pairs, at the stage times t + c_i dt. Returns (e, Eh, F, infos)."""
        A, _, _ = sdirk3()
        e_n, Eh_n = e.copy(), Eh.copy()
        ke, kE, infos = [], [], []
        for i in range(3):
            e_star = e_n + self.dt * sum(A[i, j] * ke[j] for j in range(i))
            Eh_star = Eh_n + self.dt * sum(A[i, j] * kE[j] for j in range(i))
            Ql, Sl = (None, None) if loads is None else loads[i]
            e, Eh, F, info = self.stage(e_star, Eh_star, Ql, Sl, e, Eh, F, **kw)
            ke.append((e - e_star) / (self.dt * A[i, i]))
            kE.append((Eh - Eh_star) / (self.dt * A[i, i]))
            infos.append(info)
        return e, Eh, F, infos

    # -- data in and out ---------------------------------------------------------------
    def points(self):
        """Physical coordinates of the quadrature points, (E, P, 3)."""
        return element.physical_points(self.prob.V, self.pts)

    def load(self, values):
        """(v, psi_j) for point values v (E, P): sum_p w_p v_p psi_j(p) (det J cancels)."""
        return self._glob(np.einsum("ep,pj->ej", self.w[None, :] * values, self.Psi))

    def project(self, values):
        """The L2 projection onto W_h of a field given at the points (E, P)."""
        return self.winv(self.load(values))

    def winv(self, v):
        return self._glob(np.einsum("eab,eb->ea", self.Winv, self._loc(v)))

    def total_energy(self, e, Eh):
        """int (rho e + E): the histopolation coefficients of an element sum to its integral."""
        return self.rho * e.sum() + self.winv(Eh).sum()

    def l2_error(self, coef, values):
        """||u_h - u||_L2 for L2 coefficients and exact point values (E, P)."""
        uh = np.einsum("pa,ea->ep", self.Psi, self._loc(coef)) / self.detJ
        return np.sqrt(np.sum(self.w[None, :] * self.detJ * (uh - values) ** 2))

"""Seeded test problems shared by the parity tests: each case builds the oracle
problem and describes the same inputs for the CUDA library."""
import numpy as np

import synth

GRAD_DIV, DARCY = 0, 1

# name: (kind, (nx, ny, nz), k, q, perturb, ess_mask, coefficient recipe)
CASES = {
    # C1 shape: unit cube, k = 2, alpha = beta = 1, u.n = 0 everywhere, affine
    "c1": (GRAD_DIV, (4, 4, 4), 2, 3, 0.0, 63, "ones"),
    # grad-div, k = 4, perturbed, ragged element count (18, not a multiple of 8), mixed BCs
    "gd_k4_ragged": (GRAD_DIV, (3, 2, 3), 4, 6, 0.15, 5, "lognormal1"),
    # C2 shape (small): Darcy gamma = 0, k = 3, perturbed, eps log-normal sigma = 2, natural BC
    "darcy_k3": (DARCY, (3, 3, 3), 3, 5, 0.15, 0, "darcy_sigma2"),
    # Darcy with piecewise-constant gamma > 0, k = 2, q = k+2
    "darcy_gamma": (DARCY, (2, 3, 2), 2, 4, 0.15, 12, "darcy_gamma"),
    # pure-Neumann Darcy, gamma = 0: singular Schur complement
    "darcy_neumann": (DARCY, (4, 2, 2), 2, 4, 0.1, 63, "darcy_sigma2"),
    # k = 5, q = k+1 (affine rule on a perturbed mesh is allowed: q is a parameter)
    "gd_k5": (GRAD_DIV, (1, 2, 1), 5, 6, 0.1, 3, "lognormal1"),
    # k = 3, q = k+1, grad-div, more elements than one CTA batch plus a tail
    "gd_k3": (GRAD_DIV, (3, 3, 2), 3, 4, 0.12, 48, "lognormal1"),
    # tall grad-div column, 11 element layers: the host-buffer apply's slabs are uneven
    "gd_tall": (GRAD_DIV, (2, 3, 11), 2, 4, 0.1, 21, "lognormal1"),
    # one element layer in y (a lattice 2 cells thick): a coarse level of extent 1 that
    # the next aggregation leaves unsplit
    "gd_flat": (GRAD_DIV, (4, 1, 5), 2, 4, 0.1, 12, "lognormal1"),
}


def inputs(name, seed=2304):
    kind, (nx, ny, nz), k, q, perturb, ess, recipe = CASES[name]
    vx, vy, vz = synth.lattice_vertices(nx, ny, nz, perturb=perturb, seed=seed)
    E = nx * ny * nz
    if recipe == "ones":
        c0, c1 = np.ones(E), np.ones(E)
    elif recipe == "lognormal1":
        c0, c1 = synth.lognormal(E, 1.0, seed=seed + 1), synth.lognormal(E, 1.0, seed=seed + 2)
    elif recipe == "darcy_sigma2":
        c0, c1 = synth.lognormal(E, 2.0, seed=seed + 1), np.zeros(E)
    elif recipe == "darcy_gamma":
        c0, c1 = synth.lognormal(E, 1.0, seed=seed + 1), synth.lognormal(E, 1.0, seed=seed + 3)
    else:
        raise KeyError(recipe)
    return dict(kind=kind, nx=nx, ny=ny, nz=nz, k=k, q=q, vx=vx, vy=vy, vz=vz, coef0=c0, coef1=c1,
                ess_mask=ess, affine=perturb == 0.0)


def oracle_problem(d):
    from oracle.assembly import Problem
    return Problem(d["nx"], d["ny"], d["nz"], d["k"], d["vx"], d["vy"], d["vz"], d["coef0"], d["coef1"],
                   kind=d["kind"], ess_mask=d["ess_mask"], q=d["q"])


def gpu_operator(d, **kw):
    import paper_2304_12387_gb300 as hd
    return hd.Operator(d["nx"], d["ny"], d["nz"], d["k"], d["vx"], d["vy"], d["vz"], d["coef0"], d["coef1"],
                       kind=d["kind"], ess_mask=d["ess_mask"], q=d["q"], affine=d["affine"], **kw)


def close(a, b, rtol):
    """Componentwise |a - b| <= rtol * max|b| (norm-scaled: entries near zero are
    compared at the scale of the whole vector). Returns the observed ratio."""
    a, b = np.asarray(a), np.asarray(b)
    scale = max(np.abs(b).max(initial=0.0), 1e-300)
    return np.abs(a - b).max(initial=0.0) / scale


# Full-size workloads (parity on sampled rows). name: builder returning the input dict.
def fullsize(name, seed=2304):
    if name == "m64":      # the bench workload: grad-div 64^3, k=4, q=6, beta = exp(2Z), u.n = 0
        n = 64
        vx, vy, vz = synth.lattice_vertices(n, n, n, perturb=0.15, seed=seed)
        return dict(kind=GRAD_DIV, nx=n, ny=n, nz=n, k=4, q=6, vx=vx, vy=vy, vz=vz, coef0=np.ones(n ** 3),
                    coef1=synth.lognormal(n ** 3, 2.0, seed=seed + 1), ess_mask=63, affine=False)
    if name == "c2":       # Darcy 32^3, perturbed, k=3, gamma=0, eps = exp(2Z), natural BC
        n = 32
        vx, vy, vz = synth.lattice_vertices(n, n, n, perturb=0.15, seed=seed)
        return dict(kind=DARCY, nx=n, ny=n, nz=n, k=3, q=5, vx=vx, vy=vy, vz=vz,
                    coef0=synth.lognormal(n ** 3, 2.0, seed=seed + 1), coef1=np.zeros(n ** 3), ess_mask=0,
                    affine=False)
    if name == "c3":       # layered reservoir, 60 x 220 x 85 cells on [0,1200]x[0,2200]x[0,170], k=2
        nx, ny, nz = 60, 220, 85
        vx, vy, vz = synth.lattice_vertices(nx, ny, nz, extent=(1200.0, 2200.0, 170.0))
        eps = synth.layered_permeability(nx, ny, nz, sigma=3.0, corr_len=10.0, seed=seed)
        return dict(kind=DARCY, nx=nx, ny=ny, nz=nz, k=2, q=3, vx=vx, vy=vy, vz=vz, coef0=eps,
                    coef1=np.zeros(nx * ny * nz), ess_mask=63, affine=True)
    if name == "c4":       # bent two-material tube, grad-div 48^3, k=4
        n = 48
        vx, vy, vz = synth.lattice_vertices(n, n, n)
        inside = synth.bent_tube_mask(n, n, n, seed=seed)
        alpha = np.where(inside, 1e3, 1.0)
        beta = np.where(inside, 1.0, 1e-3)
        return dict(kind=GRAD_DIV, nx=n, ny=n, nz=n, k=4, q=5, vx=vx, vy=vy, vz=vz, coef0=alpha, coef1=beta,
                    ess_mask=63, affine=True)
    if name == "c5":       # evaluation size of the learned-preconditioner study: Darcy 96^3, k=3
        n = 96
        vx, vy, vz = synth.lattice_vertices(n, n, n, perturb=0.15, seed=seed)
        return dict(kind=DARCY, nx=n, ny=n, nz=n, k=3, q=5, vx=vx, vy=vy, vz=vz,
                    coef0=synth.lognormal(n ** 3, 2.0, seed=seed + 1), coef1=np.zeros(n ** 3), ess_mask=0,
                    affine=False)
    raise KeyError(name)

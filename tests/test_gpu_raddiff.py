"""Radiation diffusion (hd_rad_*, Sec. 4.3) through the C ABI against the oracle.

Parity bars.
- Loads, W^-1 and the stage residual are direct evaluations: 1e-12 of the largest entry
  (the CG inside W^-1 stops at a relative residual of 1e-14).
- A stage and an SDIRK step: the oracle solves each Newton system densely and the Darcy
  system by LU. The CUDA path uses CG and MINRES to 1e-8 per pass, warm-started. Both
  drive ||(R1, R2, R3)|| to 1e-12 of its initial value or to its rounding floor (a few
  1e-13 at these sizes). The stage Jacobian's condition number is below 1e3 here, so the
  solutions agree to 1e-9 of their largest entry.
- Energy: with no sources and reflecting walls, int(rho e + E) is conserved to 1e-11 over
  whole steps, also at sizes the oracle does not reach.
"""
import numpy as np
import pytest

import synth
from synth import raddiff as mms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RHO, CV, A_RAD, C = 1.1, 0.8, 0.5, 1.0


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _mesh(nx, ny, nz, seed=11):
    return synth.lattice_vertices(nx, ny, nz, perturb=0.2, seed=seed)


def _pair(nx, ny, nz, k, sigma, dt, emul=1, **kw):
    import paper_2304_12387_gb300 as hd
    from oracle.raddiff import RadDiff
    v = _mesh(nx, ny, nz)
    ora = RadDiff(nx, ny, nz, k, *v, sigma, dt, rho=RHO, cv=CV, a=A_RAD, c=C)
    gpu = hd.RadDiff(nx, ny, nz, k, *v, sigma, dt, rho=RHO, cv=CV, a=A_RAD, c=C, fp64_emulation=emul, **kw)
    assert (gpu.n_rt, gpu.n_l2, gpu.q) == (ora.n_rt, ora.n_l2, ora.q)
    return ora, gpu


def _state(ora, seed):
    """A positive state away from equilibrium, as point values projected by the oracle's
    own routines (the CUDA side gets the same coefficients)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = ora.detJ.shape
    e = ora.project(CV * (1.0 + 0.5 * rng.uniform(0, 1, shape)))
    Eh = ora.load(A_RAD * (1.0 + 0.8 * rng.uniform(0, 1, shape)))
    return e, Eh


def _d(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _close(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def test_points_load_and_mass_inverse_match_the_oracle():
    _need_gpu()
    ora, gpu = _pair(3, 2, 2, 3, 1.0, 0.05)
    X = gpu.points()
    assert np.abs(X - ora.points()).max() <= 1e-14
    vals = np.random.Generator(np.random.PCG64(3)).uniform(-1, 1, X.shape[:2])
    ld = torch.empty(gpu.n_l2, dtype=torch.float64, device="cuda")
    gpu.load(_d(vals), ld)
    assert _close(ld.cpu().numpy(), ora.load(vals)) <= 1e-12
    y = torch.empty_like(ld)
    gpu.winv(ld, y)
    torch.cuda.synchronize()
    assert _close(y.cpu().numpy(), ora.winv(ora.load(vals))) <= 1e-12


@pytest.mark.parametrize("k", [2, 3, 4])
def test_stage_residual_matches_the_oracle(k):
    _need_gpu()
    sigma = synth.lognormal(12, 0.5, seed=12)
    ora, gpu = _pair(3, 2, 2, k, sigma, 0.05)
    e_s, Eh_s = _state(ora, 20)
    e, Eh = _state(ora, 21)
    rng = np.random.Generator(np.random.PCG64(22))
    F = rng.uniform(-1, 1, ora.n_rt)
    F[ora.prob.ess] = 0.0
    Ql, Sl = ora.load(rng.uniform(-1, 1, ora.detJ.shape)), ora.load(rng.uniform(-1, 1, ora.detJ.shape))
    ref = ora.residual(e, Eh, F, e_s, Eh_s, Ql, Sl)
    r = torch.empty(2 * ora.n_l2 + ora.n_rt, dtype=torch.float64, device="cuda")
    nrm = gpu.residual(*[_d(x) for x in (e_s, Eh_s, Ql, Sl, e, Eh, F)], r)
    assert _close(r.cpu().numpy(), ref) <= 1e-12
    assert abs(nrm - np.linalg.norm(ref)) <= 1e-12 * np.linalg.norm(ref)
    # loads left out count as zero
    ref0 = ora.residual(e, Eh, F, e_s, Eh_s, 0 * Ql, 0 * Sl)
    nrm0 = gpu.residual(*[_d(x) for x in (e_s, Eh_s)], None, None, *[_d(x) for x in (e, Eh, F)])
    assert abs(nrm0 - np.linalg.norm(ref0)) <= 1e-12 * np.linalg.norm(ref0)


@pytest.mark.parametrize("k,emul,lp", [(2, 0, 0), (3, 1, 0), (4, 1, 0), (3, 2, 0), (3, 1, 1), (4, 1, 1)])
def test_stage_matches_the_oracle(k, emul, lp):
    """lp = 1: the Darcy step by the mixed-precision solve (FP32 operator and cycle inside the
    FP64 residual correction); the stage converges to the same solution."""
    _need_gpu()
    sigma = synth.lognormal(12, 0.5, seed=13)
    ora, gpu = _pair(3, 2, 2, k, sigma, 0.05, emul=emul, linear_precision=lp)
    e_s, Eh_s = _state(ora, 30)
    rng = np.random.Generator(np.random.PCG64(31))
    Ql, Sl = ora.load(rng.uniform(0, 1, ora.detJ.shape)), ora.load(rng.uniform(0, 1, ora.detJ.shape))
    F0 = np.zeros(ora.n_rt)
    e_r, Eh_r, F_r, inf_r = ora.stage(e_s, Eh_s, Ql, Sl, e_s.copy(), Eh_s.copy(), F0)
    e, Eh, F = _d(e_s.copy()), _d(Eh_s.copy()), _d(F0)
    info = gpu.stage(*[_d(x) for x in (e_s, Eh_s, Ql, Sl)], e, Eh, F)
    torch.cuda.synchronize()
    assert info["status"] == 0 and info["stages"] == 1
    assert info["relres"] <= max(1e-12, 10 * inf_r["relres"]), (info, inf_r)
    assert 1 <= info["newton_max"] <= 6, info
    assert _close(e.cpu().numpy(), e_r) <= 1e-9
    assert _close(Eh.cpu().numpy(), Eh_r) <= 1e-9
    assert _close(F.cpu().numpy(), F_r) <= 1e-9


def test_sdirk_step_on_the_manufactured_solution_matches_the_oracle():
    _need_gpu()
    from oracle.raddiff import sdirk3
    sigma, dt, n, k = 2.0, 0.02, 2, 3
    import paper_2304_12387_gb300 as hd
    from oracle.raddiff import RadDiff
    v = synth.lattice_vertices(n, n, n, perturb=0.1, seed=5)
    ora = RadDiff(n, n, n, k, *v, sigma, dt)
    gpu = hd.RadDiff(n, n, n, k, *v, sigma, dt)
    _, _, c = sdirk3()
    Xo, Xg = ora.points(), gpu.points()
    e0o, E0o, _, _, _ = mms.fields(Xo, 0.0, sigma=sigma)
    e0g, E0g, _, _, _ = mms.fields(Xg, 0.0, sigma=sigma)
    # oracle side
    e_r, Eh_r, F_r = ora.project(e0o), ora.load(E0o), np.zeros(ora.n_rt)
    loads = [tuple(ora.load(f) for f in mms.fields(Xo, ci * dt, sigma=sigma)[3:]) for ci in c]
    e_r, Eh_r, F_r, _ = ora.step(e_r, Eh_r, F_r, loads)
    # CUDA side: its own points, loads and projection
    nl = gpu.n_l2
    e, Eh, tmp = (torch.empty(nl, dtype=torch.float64, device="cuda") for _ in range(3))
    gpu.load(_d(e0g), tmp)
    gpu.winv(tmp, e)
    gpu.load(_d(E0g), Eh)
    F = torch.zeros(gpu.n_rt, dtype=torch.float64, device="cuda")
    ql = torch.empty(3 * nl, dtype=torch.float64, device="cuda")
    sl = torch.empty(3 * nl, dtype=torch.float64, device="cuda")
    for i, ci in enumerate(c):
        _, _, _, Q, S = mms.fields(Xg, ci * dt, sigma=sigma)
        gpu.load(_d(Q), ql[i * nl:(i + 1) * nl])
        gpu.load(_d(S), sl[i * nl:(i + 1) * nl])
    info = gpu.step(e, Eh, F, ql, sl)
    assert info["status"] == 0 and info["stages"] == 3, info
    assert _close(e.cpu().numpy(), e_r) <= 1e-9
    assert _close(Eh.cpu().numpy(), Eh_r) <= 1e-9
    assert _close(F.cpu().numpy(), F_r) <= 1e-9
    # and close to the exact solution at t = dt (the 2^3 mesh's discretisation error, ~2e-3)
    ee, EE, _, _, _ = mms.fields(Xo, dt, sigma=sigma)
    E_h = torch.empty_like(Eh)
    gpu.winv(Eh, E_h)
    assert ora.l2_error(e.cpu().numpy(), ee) < 5e-3
    assert ora.l2_error(E_h.cpu().numpy(), EE) < 5e-3


@pytest.mark.parametrize("dims,k", [((8, 8, 8), 4), ((12, 10, 6), 3)])
def test_energy_is_conserved_at_larger_sizes(dims, k):
    """No oracle here: total energy, and the stage residual the CUDA path reports."""
    _need_gpu()
    import paper_2304_12387_gb300 as hd
    nx, ny, nz = dims
    v = _mesh(nx, ny, nz, seed=41)
    sigma = synth.lognormal(nx * ny * nz, 0.5, seed=42)
    gpu = hd.RadDiff(nx, ny, nz, k, *v, sigma, 0.05, rho=RHO, cv=CV, a=A_RAD, c=C)
    X = gpu.points()
    rng = np.random.Generator(np.random.PCG64(43))
    nl = gpu.n_l2
    e, Eh, tmp, E = (torch.empty(nl, dtype=torch.float64, device="cuda") for _ in range(4))
    hot = np.exp(-20.0 * np.sum((X - 0.5) ** 2, axis=-1))   # a hot spot in the middle
    gpu.load(_d(CV * (1.0 + hot + 0.1 * rng.uniform(0, 1, X.shape[:2]))), tmp)
    gpu.winv(tmp, e)
    gpu.load(_d(A_RAD * (1.0 + 0.2 * rng.uniform(0, 1, X.shape[:2]))), Eh)
    F = torch.zeros(gpu.n_rt, dtype=torch.float64, device="cuda")

    def energy():
        gpu.winv(Eh, E)
        return RHO * e.sum().item() + E.sum().item()

    W0 = energy()
    for _ in range(2):
        info = gpu.step(e, Eh, F)
        assert info["status"] == 0 and info["relres"] <= 1e-10, info
    assert abs(energy() - W0) <= 1e-11 * abs(W0)
    assert F.abs().max().item() > 0.0


def test_invalid_input_is_refused():
    import paper_2304_12387_gb300 as hd
    v = _mesh(2, 2, 2)
    for kw in (dict(sigma=-1.0), dict(dt=0.0), dict(rho=0.0), dict(cv=-1.0), dict(a=0.0), dict(c=0.0),
               dict(linear_precision=2)):
        args = dict(sigma=1.0, dt=0.1)
        args.update(kw)
        sigma, dt = args.pop("sigma"), args.pop("dt")
        with pytest.raises(hd.HdError) as e:
            hd.RadDiff(2, 2, 2, 3, *v, sigma, dt, **args)
        assert e.value.status == hd.HD_ERR_INVALID_ARG

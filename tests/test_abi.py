"""CPU checks of the C ABI: the library loads, exports every declared entry point,
and its host-side index maps equal the oracle's bit for bit."""
import os
import re

import numpy as np
import pytest

import paper_2304_12387_gb300 as hd
from oracle.lattice import Lattice

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hdivsp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hd_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = hd.lib()
    names = _declared()
    assert "hd_create" in names and "hd_minres_solve" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol():
    names = set(_declared())
    wrapped = set(hd._SIGS) | {"hd_last_error", "hd_rad_last_error"}
    assert names <= wrapped, names - wrapped


@pytest.mark.parametrize("dims,k", [((1, 1, 1), 2), ((2, 3, 1), 3), ((3, 2, 2), 4), ((1, 2, 1), 5)])
def test_e2d_map_bit_exact(dims, k):
    lat = Lattice(*dims, k)
    ref = lat.e2d_map()
    got = hd.hd_lattice_e2d_map(*dims, k)
    assert got.dtype == np.int32
    assert np.array_equal(got.astype(np.int64), ref)


@pytest.mark.parametrize("dims,k", [((1, 1, 1), 2), ((2, 3, 1), 3), ((3, 2, 2), 4), ((1, 2, 1), 5)])
def test_rotated_maps_bit_exact(dims, k):
    """Algorithm 1's signed maps for rotated elements: every one of the 24 codes."""
    lat = Lattice(*dims, k)
    E = lat.n_elem
    for shift in range(0, 24, E):
        rot = (np.arange(E) + shift) % 24
        got = hd.hd_lattice_e2d_map_rot(*dims, k, rot)
        assert np.array_equal(got.astype(np.int64), lat.e2d_map(rot))
        got = hd.hd_lattice_e2l_map(*dims, k, rot)
        assert np.array_equal(got.astype(np.int64), lat.e2l2_map(rot))
    assert np.array_equal(hd.hd_lattice_e2l_map(*dims, k).astype(np.int64), lat.e2l2_map())


def test_bad_rotation_codes_are_rejected():
    for bad in (24, -1, 100):
        with pytest.raises(hd.HdError):
            hd.hd_lattice_e2d_map_rot(2, 1, 1, 2, [0, bad])
        with pytest.raises(hd.HdError):
            hd.hd_lattice_e2l_map(2, 1, 1, 2, [bad, 3])


@pytest.mark.parametrize("mask", [0, 1, 2, 5, 12, 48, 63, 42])
def test_ess_dofs_bit_exact(mask):
    lat = Lattice(3, 2, 2, 3)
    assert np.array_equal(hd.hd_lattice_ess_dofs(3, 2, 2, 3, mask), lat.ess_dofs(mask))


def test_bad_arguments_are_rejected():
    with pytest.raises(hd.HdError):
        hd.hd_lattice_e2d_map(0, 1, 1, 2)
    with pytest.raises(hd.HdError):
        hd.hd_lattice_ess_dofs(1, 1, 1, 2, 64)


def test_affine_mesh_test():
    """The host-side test that selects the affine fast path: parallelepiped meshes
    (uniform, graded and sheared, translated to large coordinates) pass; a perturbed
    mesh, or one vertex moved by 1e-9 of the element size, does not."""
    import synth
    A = np.array([[1.0, 0.3, 0.1], [0.05, 0.8, 0.2], [0.1, -0.1, 1.2]])
    for dims in ((1, 1, 1), (3, 2, 4)):
        vx, vy, vz = synth.lattice_vertices(*dims)
        assert hd.hd_lattice_is_affine(*dims, vx, vy, vz)
        X = A @ (np.stack([vx, vy, vz]) ** 1.3)
        assert hd.hd_lattice_is_affine(*dims, *X)
        vx2, vy2, vz2 = synth.lattice_vertices(*dims, extent=(1200.0, 2200.0, 170.0))
        assert hd.hd_lattice_is_affine(*dims, vx2 + 5e3, vy2 - 7e3, vz2 + 1e4)
        if min(dims) > 1:  # the perturbation moves interior vertices only
            assert not hd.hd_lattice_is_affine(*dims, *synth.lattice_vertices(*dims, perturb=0.01))
        bumped = vx.copy()
        bumped[-1] += 1e-9 / max(dims)
        assert not hd.hd_lattice_is_affine(*dims, bumped, vy, vz)
    with pytest.raises(ValueError):
        hd.hd_lattice_is_affine(2, 2, 2, np.zeros(3), np.zeros(3), np.zeros(3))


def test_radiation_diffusion_create_refuses_invalid_input_on_the_host():
    """hd_rad_create checks its descriptor before any device work: a non-positive opacity,
    constant or time step, or an unknown linear_precision, is HD_ERR_INVALID_ARG."""
    import synth
    v = synth.lattice_vertices(2, 2, 2, perturb=0.1, seed=3)
    sigma = np.ones(8)
    sigma[5] = 0.0
    cases = [dict(sigma=sigma), dict(dt=-0.1), dict(rho=0.0), dict(cv=-2.0), dict(a=0.0), dict(c=0.0),
             dict(linear_precision=3), dict(outer_rtol=-1.0), dict(newton_maxit=-1)]
    for kw in cases:
        args = dict(sigma=1.0, dt=0.1)
        args.update(kw)
        sg, dt = args.pop("sigma"), args.pop("dt")
        with pytest.raises(hd.HdError) as e:
            hd.RadDiff(2, 2, 2, 3, *v, sg, dt, **args)
        assert e.value.status == hd.HD_ERR_INVALID_ARG, kw

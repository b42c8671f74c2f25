"""Pins of the oracle's element rotations and of Algorithm 1 (Sec. 3.2).

An element of a hex mesh may place its reference cube by any of the 24 proper
symmetries of the cube. The global RT and L2 bases do not depend on that choice:
rotating an element only renumbers its local dofs and flips the orientation of the
RT functions whose reference axis lands on a negative lattice axis (the
sigma_loc * sigma_glob signs of Algorithm 1). So, whatever the rotations:

* Algorithm 1 gives exactly the lattice divergence (two +-1 per cell and face pair);
* the assembled M, D, C and the whole block operator equal the unrotated ones up
  to rounding (the quadrature points are the same physical points);
* the assembled load vector of a manufactured field is the same.

A wrong mirror index, a wrong sign or a transposed axis in the rotated maps or in
the rotated vertex order breaks one of these.
"""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import manufactured
from oracle.assembly import DARCY, GRAD_DIV, Problem
from oracle.lattice import Lattice, algorithm1_divergence, rotation, rotation_matrix


def test_rotation_codes_form_the_proper_cube_group():
    Rs = [rotation_matrix(c) for c in range(24)]
    keys = {tuple(R.ravel()) for R in Rs}
    assert len(keys) == 24
    assert np.array_equal(Rs[0], np.eye(3))
    for R in Rs:
        assert np.array_equal(R @ R.T, np.eye(3))
        assert round(np.linalg.det(R)) == 1
        assert np.count_nonzero(R) == 3
    for A, B in itertools.product(Rs, Rs):       # closed under composition
        assert tuple((A @ B).ravel()) in keys
    with pytest.raises(ValueError):
        rotation(24)


@pytest.mark.parametrize("k", [2, 3])
def test_rotated_maps_renumber_and_flip(k):
    lat = Lattice(2, 2, 3, k)
    rot = np.arange(lat.n_elem) % 24
    m0, m1 = lat.e2d_map(), lat.e2d_map(rot)
    l0, l1 = lat.e2l2_map(), lat.e2l2_map(rot)
    per_comp = (k + 1) * k * k
    for e in range(lat.n_elem):
        ids = np.where(m1[e] < 0, -1 - m1[e], m1[e])
        assert sorted(ids) == sorted(m0[e])
        assert sorted(l1[e]) == sorted(l0[e])
        perm, sgn = rotation(int(rot[e]))
        neg = m1[e] < 0
        for d in range(3):
            block = neg[d * per_comp:(d + 1) * per_comp]
            assert block.all() if sgn[d] < 0 else not block.any()
            # component d lands on faces normal to lattice axis perm[d]
            g = ids[d * per_comp:(d + 1) * per_comp]
            lo = (0, lat.n_xf, lat.n_xf + lat.n_yf)[perm[d]]
            hi = (lat.n_xf, lat.n_xf + lat.n_yf, lat.n_rt)[perm[d]]
            assert ((g >= lo) & (g < hi)).all()


@pytest.mark.parametrize("dims,k", [((1, 1, 1), 2), ((2, 3, 2), 3), ((3, 1, 2), 4)])
def test_algorithm1_divergence_is_the_lattice_divergence(dims, k):
    lat = Lattice(*dims, k)
    r, c, v = lat.divergence_incidence()
    Dinc = sp.coo_matrix((v, (r, c)), shape=(lat.n_l2, lat.n_rt)).toarray()
    rng = np.random.Generator(np.random.PCG64(7))
    for rot in (None, rng.integers(0, 24, lat.n_elem)):
        ip, ix, dv = algorithm1_divergence(lat, lat.e2d_map(rot), lat.e2l2_map(rot))
        D = sp.csr_matrix((dv, ix, ip), shape=(lat.n_l2, lat.n_rt)).toarray()
        assert np.array_equal(D, Dinc)


def test_algorithm1_catches_a_flipped_orientation():
    lat = Lattice(2, 1, 1, 2)
    rot = np.array([5, 17])
    m = lat.e2d_map(rot)
    m[1, 3] = -1 - m[1, 3]                        # planted: one sigma_glob flipped
    ip, ix, dv = algorithm1_divergence(lat, m, lat.e2l2_map(rot))
    r, c, v = lat.divergence_incidence()
    Dinc = sp.coo_matrix((v, (r, c)), shape=(lat.n_l2, lat.n_rt)).toarray()
    assert not np.array_equal(sp.csr_matrix((dv, ix, ip), shape=Dinc.shape).toarray(), Dinc)


CASES = [
    # kind, dims, k, q, perturb, ess_mask
    (GRAD_DIV, (2, 2, 2), 2, 4, 0.15, 5),
    (DARCY, (2, 1, 2), 3, 5, 0.12, 12),
    (GRAD_DIV, (1, 2, 1), 4, 5, 0.1, 63),
]


@pytest.mark.parametrize("case", CASES, ids=["gd_k2", "darcy_k3_gamma", "gd_k4"])
def test_assembled_operator_is_rotation_invariant(case):
    kind, (nx, ny, nz), k, q, perturb, ess = case
    vx, vy, vz = synth.lattice_vertices(nx, ny, nz, perturb=perturb, seed=2304)
    E = nx * ny * nz
    c0 = synth.lognormal(E, 1.0, seed=2305)
    c1 = synth.lognormal(E, 1.0, seed=2306)
    rot = np.random.Generator(np.random.PCG64(11)).integers(0, 24, E)
    p0 = Problem(nx, ny, nz, k, vx, vy, vz, c0, c1, kind=kind, ess_mask=ess, q=q)
    p1 = Problem(nx, ny, nz, k, vx, vy, vz, c0, c1, kind=kind, ess_mask=ess, q=q, rot=rot)
    assert (p1.e2d < 0).any()                     # some orientations are flipped
    for A0, A1 in ((p0.M, p1.M), (p0.C, p1.C), (p0.matrix(), p1.matrix())):
        a0, a1 = A0.toarray(), A1.toarray()
        assert np.abs(a1 - a0).max() <= 1e-13 * np.abs(a0).max()
    assert np.array_equal(p1.D.toarray(), p0.D.toarray())
    def f(X):  # no symmetry between the components, so a swapped axis shows
        x, y, z = X[..., 0], X[..., 1], X[..., 2]
        return np.stack([1.0 + x * x, y * z - 0.3, np.sin(2.0 * z) + x], axis=-1)
    b0, b1 = manufactured.rt_load(p0, f), manufactured.rt_load(p1, f)
    assert np.abs(b1 - b0).max() <= 1e-13 * np.abs(b0).max()

"""Aggregation of the Schur V/W-cycle and the element boundaries (oracle only, no GPU).

The lattice of S~ has k cells per element along each axis, of GLL widths (thin at the
element ends). Pairwise aggregation follows the element boundaries when k is even and
cannot when k is odd. The tests pin the element-aligned aggregation map (element_groups:
pairs from both ends of the element, an odd middle cell alone; for even k the default
pairs exactly) and measure what alignment does to the cycle: preconditioned CG on S~ of
the metric recipe (perturbed mesh, beta = exp(2Z), u.n = 0), one W-cycle per step with
one smoothed level. Shifting the pairs by one cell, so that they straddle every element
boundary, makes even k much slower, odd k hardly changes (its pairs straddle half the
boundaries either way), and the element-aligned map makes odd k as fast as even k."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import precond
from oracle.assembly import GRAD_DIV, Problem
from oracle.precond import VCycle, aggregation, approx_schur, element_groups


@pytest.mark.parametrize("c,sizes", [(1, [1]), (2, [2]), (3, [2, 1]), (4, [2, 2]), (5, [2, 1, 2]), (6, [2, 2, 2]),
                                     (7, [2, 2, 1, 2])])
def test_element_groups(c, sizes):
    g, m = element_groups(c)
    assert m == len(sizes)
    assert np.array_equal(np.bincount(g), sizes)
    assert np.all(np.diff(g) >= 0)


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_aligned_aggregates_stay_inside_elements(k):
    ne = (3, 2, 4)
    dims = tuple(n * k for n in ne)
    P, cd = aggregation(dims, ne)
    P0, cd0 = aggregation(dims)
    if k % 2 == 0:
        assert cd == cd0 and (P != P0).nnz == 0       # even k: the default pairs
    coarse = P.tocoo()
    X, Y, _ = dims
    f = coarse.row
    ix, iy, iz = f % X, (f // X) % Y, f // (X * Y)
    elem = (ix // k) + ne[0] * ((iy // k) + ne[1] * (iz // k))
    for J in range(P.shape[1]):
        assert np.unique(elem[coarse.col == J]).size == 1
    assert np.all(np.asarray(P.sum(axis=1)).ravel() == 1.0)


def _shifted(dims, elems=None):
    """Pairs shifted by one cell: the first cell alone, then (1, 2), (3, 4), ..."""
    maps = []
    for n in dims:
        if n == 1:
            maps.append((np.zeros(1, dtype=np.int64), 1))
        else:
            i = (np.arange(n) + 1) // 2
            maps.append((i, int(i[-1]) + 1))
    (ix, cx), (iy, cy), (iz, cz) = maps
    X, Y, Z = dims
    I, J, K = np.meshgrid(np.arange(X), np.arange(Y), np.arange(Z), indexing="ij")
    P = sp.coo_matrix((np.ones(X * Y * Z), ((I + X * (J + Y * K)).ravel(), (ix[I] + cx * (iy[J] + cy * iz[K])).ravel())),
                      shape=(X * Y * Z, cx * cy * cz)).tocsr()
    return P, (cx, cy, cz)


def _pcg_steps(S, apply_m, b, rtol=1e-8, maxit=500):
    x, r = np.zeros_like(b), b.copy()
    z = apply_m(r)
    p, rz, nb = z.copy(), r @ z, np.linalg.norm(b)
    for it in range(1, maxit + 1):
        Ap = S @ p
        a = rz / (p @ Ap)
        x += a * p
        r -= a * Ap
        if np.linalg.norm(r) <= rtol * nb:
            return it
        z = apply_m(r)
        rz, rz_old = r @ z, rz
        p = z + (rz / rz_old) * p
    return maxit


def _counts(k, monkeypatch, n=6):
    vx, vy, vz = synth.lattice_vertices(n, n, n, perturb=0.15, seed=2304)
    E = n ** 3
    prob = Problem(n, n, n, k, vx, vy, vz, np.ones(E), synth.lognormal(E, 2.0, seed=2305), kind=GRAD_DIV,
                   ess_mask=63, q=k + 2)
    S, _, _ = approx_schur(prob)
    dims = (prob.lat.X, prob.lat.Y, prob.lat.Z)
    b = synth.uniform(S.shape[0], seed=2306)
    kw = dict(nu=2, coarse_max=64, cycle=2, smooth=4.0 / 3.0, sa_levels=1)
    out = {"default": _pcg_steps(S, VCycle(S, dims, **kw).apply, b),
           "aligned": _pcg_steps(S, VCycle(S, dims, elems=(n, n, n), **kw).apply, b)}
    with monkeypatch.context() as m:
        m.setattr(precond, "aggregation", _shifted)
        out["shifted"] = _pcg_steps(S, VCycle(S, dims, **kw).apply, b)
    return out


def test_aggregates_across_element_boundaries_slow_the_cycle(monkeypatch):
    c = {k: _counts(k, monkeypatch) for k in (2, 3, 4, 5)}
    print(c)
    for k in (2, 4):
        assert c[k]["aligned"] == c[k]["default"]
        assert c[k]["shifted"] >= 1.4 * c[k]["default"], c[k]
    for k in (3, 5):
        assert abs(c[k]["shifted"] - c[k]["default"]) <= 0.2 * c[k]["default"], c[k]
        assert c[k]["aligned"] <= 0.85 * c[k]["default"], c[k]
    aligned = [c[k]["aligned"] for k in (2, 3, 4, 5)]
    assert max(aligned) <= 1.3 * min(aligned), aligned

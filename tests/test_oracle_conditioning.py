"""Condition-number studies on single elements (oracle only): the diagonally scaled
L2 mass in three bases on a skewed hexahedron (Sec. 2.5) and the transformed against
the untransformed preconditioned Schur complement (the notes on the untransformed
system). Pinned to what the paper states about them."""
import numpy as np
import pytest

from oracle.conditioning import l2_mass_conditions, schur_conditions


def _skewed(a, b, c):
    """A skewed, non-affine hexahedron (det J varies, between 0.46 and 1)."""
    return np.array([a + 0.6 * b * c, b + 0.3 * a * c, c + 0.4 * a * b])


def _element(f):
    V = np.zeros((1, 2, 2, 2, 3))
    vx, vy, vz = np.zeros(8), np.zeros(8), np.zeros(8)
    for c in range(2):
        for b in range(2):
            for a in range(2):
                p = f(a, b, c)
                V[0, c, b, a] = p
                i = a + 2 * (b + 2 * c)
                vx[i], vy[i], vz[i] = p
    return V, vx, vy, vz


def test_l2_mass_conditioning_in_three_bases():
    """Gauss-Legendre nodal: close to 1 for every degree (the paper: at most about 1.12
    in its tests); Gauss-Lobatto nodal: improves with the degree; histopolation:
    grows before it levels off (pre-asymptotic), below Gauss-Lobatto at these degrees
    and above Gauss-Legendre; all bounded."""
    V, *_ = _element(_skewed)
    r = {k: l2_mass_conditions(V, k) for k in range(2, 7)}
    gl = [r[k]["gauss_legendre"] for k in r]
    gll = [r[k]["gauss_lobatto"] for k in r]
    hist = [r[k]["histopolation"] for k in r]
    assert max(gl) < 1.12 and min(gl) >= 1.0
    assert all(a > b for a, b in zip(gll, gll[1:])), gll
    assert all(a < b for a, b in zip(hist, hist[1:])), hist
    assert all(g < h < l < 30 for g, h, l in zip(gl, hist, gll)), (gl, hist, gll)


@pytest.mark.parametrize("shape", ["unit_cube", "skewed"])
def test_transformed_schur_complement_is_better_conditioned(shape):
    """kappa(S~^-1 S) of the transformed system is well below kappa(S~'^-1 S') of the
    untransformed one (three diagonal approximations in its second term instead of
    one), at every degree k = 2..5."""
    f = (lambda a, b, c: np.array([a, b, c], dtype=float)) if shape == "unit_cube" else _skewed
    _, vx, vy, vz = _element(f)
    for k in range(2, 6):
        kt, ku = schur_conditions(vx, vy, vz, k)
        assert 1.0 <= kt < 0.5 * ku, (k, kt, ku)

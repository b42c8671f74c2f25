"""Pins of the oracle's 1D bases against closed forms and their DOF definitions (Sec. 2.1)."""
import numpy as np
import pytest

from oracle import basis1d


def test_gll_closed_forms():
    assert np.allclose(basis1d.gll_nodes(1), [0, 1], atol=0, rtol=0)
    assert np.allclose(basis1d.gll_nodes(2), [0, 0.5, 1], atol=1e-16)
    # P_3' roots are +-1/sqrt(5); P_4' roots are 0, +-sqrt(3/7)
    assert np.allclose(basis1d.gll_nodes(3), [0, 0.5 - 0.5 / np.sqrt(5), 0.5 + 0.5 / np.sqrt(5), 1], atol=1e-15)
    r = 0.5 * np.sqrt(3.0 / 7.0)
    assert np.allclose(basis1d.gll_nodes(4), [0, 0.5 - r, 0.5, 0.5 + r, 1], atol=1e-15)


@pytest.mark.parametrize("k", range(2, 11))
def test_gll_against_library_roots(k):
    roots = np.sort(np.polynomial.legendre.Legendre.basis(k).deriv().roots().real)
    ref = np.concatenate([[0.0], 0.5 * (roots + 1.0), [1.0]])
    assert np.allclose(basis1d.gll_nodes(k), ref, atol=1e-13)


@pytest.mark.parametrize("q", range(1, 9))
def test_gl_exactness(q):
    x, w = basis1d.gl_points(q)
    for deg in range(2 * q):
        assert abs(np.sum(w * x ** deg) - 1.0 / (deg + 1)) < 1e-14


@pytest.mark.parametrize("k", range(1, 9))
def test_lagrange_kronecker_and_partition(k):
    xi = basis1d.gll_nodes(k)
    L = basis1d.interp_basis(k, xi)
    assert np.allclose(L, np.eye(k + 1), atol=1e-13)
    x = np.linspace(0, 1, 37)
    assert np.allclose(basis1d.interp_basis(k, x).sum(axis=0), 1.0, atol=1e-12)
    # derivative against central differences
    h = 1e-6
    fd = (basis1d.interp_basis(k, x + h) - basis1d.interp_basis(k, x - h)) / (2 * h)
    assert np.allclose(basis1d.interp_basis_deriv(k, x), fd, atol=1e-6 * max(1, k ** 2))


@pytest.mark.parametrize("k", range(1, 9))
def test_histopolation_dofs(k):
    """int_{xi_m}^{xi_{m+1}} h_j = delta_mj, integrated by an independent Gauss rule."""
    xi = basis1d.gll_nodes(k)
    t, w = np.polynomial.legendre.leggauss(k + 2)
    I = np.zeros((k, k))
    for m in range(k):
        a, b = xi[m], xi[m + 1]
        x = 0.5 * (b - a) * t + 0.5 * (a + b)
        I[m] = basis1d.histo_basis(k, x) @ (0.5 * (b - a) * w)
    assert np.allclose(I, np.eye(k), atol=1e-13)


@pytest.mark.parametrize("k", range(1, 7))
def test_histopolation_symmetry(k):
    """h_j(1 - x) = h_{k-1-j}(x) from the symmetric GLL nodes."""
    x = np.linspace(0, 1, 23)
    H = basis1d.histo_basis(k, x)
    Hr = basis1d.histo_basis(k, 1 - x)
    assert np.allclose(Hr, H[::-1], atol=1e-11)

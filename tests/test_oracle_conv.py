"""Pins of the FP64 reference of the learned Schur preconditioner (oracle.conv):
adjointness of each convolution, symmetry and positivity of the net, the
delta-input closed form and the hand-derived gradient against central finite
differences."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import conv

DIMS = (5, 4, 3)        # X, Y, Z
NC = 4


def _rand(shape, seed):
    return np.random.Generator(np.random.PCG64(seed)).standard_normal(shape)


def test_conv1_delta_gives_kernel():
    X, Y, Z = DIMS
    W1 = _rand((NC, 27), 1)
    x = np.zeros((Z, Y, X))
    x[1, 2, 2] = 1.0
    out = conv.conv1(W1, x)
    # out[co](p) = W1[co, t] where p + off_t = (2, 2, 1) (x, y, z)
    for t, (ox, oy, oz) in enumerate(conv.TAPS):
        assert np.allclose(out[:, 1 - oz, 2 - oy, 2 - ox], W1[:, t])


def test_adjoints():
    X, Y, Z = DIMS
    W1, W2 = _rand((NC, 27), 2), _rand((NC, NC, 27), 3)
    x, g1 = _rand((Z, Y, X), 4), _rand((NC, Z, Y, X), 5)
    assert np.isclose(np.sum(conv.conv1(W1, x) * g1), np.sum(x * conv.conv1_T(W1, g1)), rtol=1e-13)
    a, g2 = _rand((NC, Z, Y, X), 6), _rand((NC, Z, Y, X), 7)
    assert np.isclose(np.sum(conv.conv2(W2, a) * g2), np.sum(a * conv.conv2_T(W2, g2)), rtol=1e-13)


def test_net_symmetric_positive():
    X, Y, Z = DIMS
    n = X * Y * Z
    W1, W2 = _rand((NC, 27), 8), _rand((NC, NC, 27), 9)
    d = 1.0 + np.abs(_rand(n, 10))
    a, b = _rand(n, 11), _rand(n, 12)
    Pa = conv.apply_net(W1, W2, a, d, DIMS, 1e-3)
    Pb = conv.apply_net(W1, W2, b, d, DIMS, 1e-3)
    assert np.isclose(Pa @ b, a @ Pb, rtol=1e-12)
    assert a @ Pa > 0


def _spd(n, seed):
    A = sp.random(n, n, density=0.05, random_state=seed)
    A = A + A.T
    return (A + sp.diags(np.abs(A).sum(axis=1).A1 + 1.0)).tocsr()


def test_gradient_matches_finite_differences():
    X, Y, Z = DIMS
    n = X * Y * Z
    S = _spd(n, 13)
    d = S.diagonal()
    W1, W2 = conv.init_weights(NC, seed=14)
    pairs = []
    for s in range(2):
        r = _rand(n, 20 + s)
        e = np.linalg.solve(S.toarray(), r)
        pairs.append((r, e, 0.1 * _rand(n, 30 + s)))
    g1, g2 = conv.grad(W1, W2, pairs, S, d, DIMS, 1e-3)
    h = 1e-6
    rng = np.random.Generator(np.random.PCG64(40))
    for _ in range(6):
        co, t = rng.integers(NC), rng.integers(27)
        Wp, Wm = W1.copy(), W1.copy()
        Wp[co, t] += h
        Wm[co, t] -= h
        fd = (conv.loss(Wp, W2, pairs, S, d, DIMS, 1e-3) - conv.loss(Wm, W2, pairs, S, d, DIMS, 1e-3)) / (2 * h)
        assert np.isclose(g1[co, t], fd, rtol=1e-6, atol=1e-9)
        co, ci, t = rng.integers(NC), rng.integers(NC), rng.integers(27)
        Wp, Wm = W2.copy(), W2.copy()
        Wp[co, ci, t] += h
        Wm[co, ci, t] -= h
        fd = (conv.loss(W1, Wp, pairs, S, d, DIMS, 1e-3) - conv.loss(W1, Wm, pairs, S, d, DIMS, 1e-3)) / (2 * h)
        assert np.isclose(g2[co, ci, t], fd, rtol=1e-6, atol=1e-9)

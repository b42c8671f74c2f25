"""FP64 reference of the learned Schur-complement preconditioner.

The paper preconditions S~ with one AMG V-cycle (Sec. 3.2). The learned variant
adds to a fixed symmetric positive definite part Q (the library uses its V/W-cycle)
a small linear convolutional network on the L2 cell lattice, positive semi-definite
by construction, so that P stays SPD and MINRES stays valid:

    P r = d^-1/2 C1^T C2^T C2 C1 d^-1/2 r  +  delta d^-1 r  +  Q r,

  d      = diag(S~),
  C1     = 3x3x3 convolution, 1 -> nc channels (weights W1[co, t]),
  C2     = 3x3x3 convolution, nc -> nc channels (weights W2[co, ci, t]),
  ^T     = the adjoint convolutions (flipped taps, transposed channels),
  Q      = the fixed part, given per pair as the vector Q r.

Taps t = dx + 3 (dy + 3 dz) address the neighbour at offset (dx-1, dy-1, dz-1);
outside the lattice the field is zero. Fields are stored in lattice order
c = I + X (J + Y K) and reshaped to (Z, Y, X) here.

Training loss over pairs (r, e = S~^-1 r):

    L = sum_pairs ||e - P r||_S^2 / ||e||_S^2,   ||v||_S^2 = v . S~ v.

Everything here is plain loops over taps and numpy; `grad` is the hand-derived
adjoint of `apply_net`, pinned by finite differences in the tests.
"""
import numpy as np

TAPS = [(dx - 1, dy - 1, dz - 1) for dz in range(3) for dy in range(3) for dx in range(3)]


def _shift(a, off):
    """b[..., z, y, x] = a[..., z+oz, y+oy, x+ox] (zero outside)."""
    ox, oy, oz = off
    b = np.zeros_like(a)
    Z, Y, X = a.shape[-3:]
    zs, zd = (slice(oz, Z), slice(0, Z - oz)) if oz >= 0 else (slice(0, Z + oz), slice(-oz, Z))
    ys, yd = (slice(oy, Y), slice(0, Y - oy)) if oy >= 0 else (slice(0, Y + oy), slice(-oy, Y))
    xs, xd = (slice(ox, X), slice(0, X - ox)) if ox >= 0 else (slice(0, X + ox), slice(-ox, X))
    b[..., zd, yd, xd] = a[..., zs, ys, xs]
    return b


def conv1(W1, x):
    """(nc, Z, Y, X) <- (Z, Y, X): out[co] = sum_t W1[co,t] x(. + off_t)."""
    out = np.zeros((W1.shape[0],) + x.shape)
    for t, off in enumerate(TAPS):
        out += W1[:, t, None, None, None] * _shift(x, off)[None]
    return out


def conv1_T(W1, g):
    """Adjoint of conv1: (Z, Y, X) <- (nc, Z, Y, X)."""
    out = np.zeros(g.shape[1:])
    for t, off in enumerate(TAPS):
        neg = (-off[0], -off[1], -off[2])
        out += np.einsum("c,czyx->zyx", W1[:, t], _shift(g, neg))
    return out


def conv2(W2, a):
    """(nc, ...) <- (nc, ...): out[co] = sum_{ci,t} W2[co,ci,t] a[ci](. + off_t)."""
    out = np.zeros((W2.shape[0],) + a.shape[1:])
    for t, off in enumerate(TAPS):
        out += np.einsum("oi,izyx->ozyx", W2[:, :, t], _shift(a, off))
    return out


def conv2_T(W2, g):
    """Adjoint of conv2."""
    out = np.zeros((W2.shape[1],) + g.shape[1:])
    for t, off in enumerate(TAPS):
        neg = (-off[0], -off[1], -off[2])
        out += np.einsum("oi,ozyx->izyx", W2[:, :, t], _shift(g, neg))
    return out


def apply_net(W1, W2, r, d, dims, delta):
    """P_L r = d^-1/2 C1^T C2^T C2 C1 d^-1/2 r + delta r / d (lattice-order vectors)."""
    X, Y, Z = dims
    s = 1.0 / np.sqrt(d)
    u = (s * r).reshape(Z, Y, X)
    a1 = conv1(W1, u)
    a2 = conv2(W2, a1)
    a3 = conv2_T(W2, a2)
    a4 = conv1_T(W1, a3)
    return s * a4.ravel() + delta * r / d


def loss(W1, W2, pairs, S, d, dims, delta):
    """sum over (r, e, Qr) of ||e - P r||_S^2 / ||e||_S^2 with P = P_L + Q."""
    L = 0.0
    for r, e, Qr in pairs:
        err = e - apply_net(W1, W2, r, d, dims, delta) - Qr
        L += (err @ (S @ err)) / (e @ (S @ e))
    return L


def grad(W1, W2, pairs, S, d, dims, delta):
    """(dL/dW1, dL/dW2) by the adjoint of apply_net."""
    X, Y, Z = dims
    s = 1.0 / np.sqrt(d)
    g1 = np.zeros_like(W1)
    g2 = np.zeros_like(W2)
    for r, e, Qr in pairs:
        u = (s * r).reshape(Z, Y, X)
        a1 = conv1(W1, u)
        a2 = conv2(W2, a1)
        a3 = conv2_T(W2, a2)
        a4 = conv1_T(W1, a3)
        y = s * a4.ravel() + delta * r / d
        err = e - y - Qr
        gy = -2.0 * (S @ err) / (e @ (S @ e))           # dL/dy
        b4 = (s * gy).reshape(Z, Y, X)                   # dL/da4
        b3 = conv1(W1, b4)                               # dL/da3 (adjoint of conv1_T is conv1)
        b2 = conv2(W2, b3)                               # dL/da2
        b1 = conv2_T(W2, b2)                             # dL/da1
        # weight gradients of the four uses:
        #   a1 = conv1(W1, u):     d/dW1[co,t] += sum b1[co] * u(. + off_t)
        #   a4 = conv1_T(W1, a3):  d/dW1[co,t] += sum a3[co] * b4(. + off_t)
        #   a2 = conv2(W2, a1):    d/dW2[co,ci,t] += sum b2[co] * a1[ci](. + off_t)
        #   a3 = conv2_T(W2, a2):  d/dW2[co,ci,t] += sum a2[co] * b3[ci](. + off_t)
        for t, off in enumerate(TAPS):
            g1[:, t] += np.einsum("czyx,zyx->c", b1, _shift(u, off))
            g1[:, t] += np.einsum("czyx,zyx->c", a3, _shift(b4, off))
            g2[:, :, t] += np.einsum("ozyx,izyx->oi", b2, _shift(a1, off))
            g2[:, :, t] += np.einsum("ozyx,izyx->oi", a2, _shift(b3, off))
    return g1, g2


def init_weights(nc, seed=2304):
    """Seeded small initial weights (scaled so that C2 C1 starts near a smoothing average)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    W1 = rng.standard_normal((nc, 27)) / np.sqrt(27.0)
    W2 = rng.standard_normal((nc, nc, 27)) / np.sqrt(27.0 * nc)
    return W1, W2

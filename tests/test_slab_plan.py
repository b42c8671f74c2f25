"""The z-slab partition plan (hd_slab_plan, host only) against the lattice numbering.

For several meshes, degrees and partition counts (ragged splits included): the owned
ranges of the P partitions tile [0, n_rt + n_l2) exactly once; every RT and L2 dof
that an element of slab p touches (the oracle's element maps) is owned by p or lies in
p's halo; the halo is the z-face layer at the top of the slab, owned by p + 1 and of
size X Y; the element layers tile [0, nz) with sizes that differ by at most one."""
import numpy as np
import pytest

import paper_2304_12387_gb300 as hd
from oracle.lattice import Lattice


@pytest.mark.parametrize("dims,k,P", [((3, 2, 4), 2, 2), ((2, 3, 11), 2, 3), ((2, 2, 7), 3, 4), ((1, 2, 5), 4, 5),
                                      ((3, 3, 3), 2, 1)])
def test_slab_plan_tiles_the_dofs_and_covers_each_slab(dims, k, P):
    nx, ny, nz = dims
    lat = Lattice(nx, ny, nz, k)
    n = lat.n_rt + lat.n_l2
    owner = np.full(n, -1)
    plans = [hd.hd_slab_plan(nx, ny, nz, k, P, p) for p in range(P)]
    layers = []
    for p, s in enumerate(plans):
        for key in ("xf", "yf", "zf", "cell"):
            lo, hi = s[key]
            assert lo <= hi
            assert (owner[lo:hi] == -1).all()
            owner[lo:hi] = p
        layers.append(s["ez"])
    assert (owner >= 0).all()
    # element layers: a balanced tiling of [0, nz)
    assert layers[0][0] == 0 and layers[-1][1] == nz
    assert all(layers[i][1] == layers[i + 1][0] for i in range(P - 1))
    sizes = [b - a for a, b in layers]
    assert max(sizes) - min(sizes) <= 1
    e2d = lat.e2d_map()
    e2d = np.where(e2d < 0, -1 - e2d, e2d)
    e2l = lat.e2l2_map() + lat.n_rt
    X, Y = lat.X, lat.Y
    for p, s in enumerate(plans):
        h0, h1 = s["halo"]
        if p == P - 1:
            assert h0 == h1
        else:
            assert h1 - h0 == X * Y
            assert (owner[h0:h1] == p + 1).all()
            # the halo is the z-face layer K = k ez1
            Kh = k * s["ez"][1]
            I, J = np.meshgrid(np.arange(X), np.arange(Y), indexing="ij")
            assert set(lat.zface(I, J, Kh).ravel()) == set(range(h0, h1))
        ez = np.arange(nx * ny * nz) // (nx * ny)
        elems = np.nonzero((ez >= s["ez"][0]) & (ez < s["ez"][1]))[0]
        touched = np.unique(np.concatenate([e2d[elems].ravel(), e2l[elems].ravel()]))
        halo = np.zeros(n, dtype=bool)
        halo[h0:h1] = True
        ok = (owner[touched] == p) | halo[touched]
        assert ok.all(), touched[~ok][:10]
        # and every halo face is touched (the halo is not larger than needed)
        assert set(range(h0, h1)) <= set(touched.tolist())


def test_slab_plan_rejects_bad_arguments():
    for args in ((2, 2, 3, 2, 4, 0), (2, 2, 3, 2, 2, 2), (2, 2, 3, 2, 0, 0), (0, 2, 3, 2, 1, 0)):
        with pytest.raises(hd.HdError) as e:
            hd.hd_slab_plan(*args)
        assert e.value.status == hd.HD_ERR_INVALID_ARG

"""The z-slab exchange protocol (paper_2304_12387_gb300.slab) on CPU ranks with gloo.

World sizes 2 and 3 (ragged slabs): every rank holds only its owned entries and its
halo, applies the block operator of its own element layers (element matrices of the
oracle, assembled element by element in the test), and the two neighbour exchanges
(halo values in, interface partial sums out) plus a scalar allreduce must reproduce
the assembled global operator (1e-13) and the global inner product. A rank that reads
an entry it does not hold sees NaN there, so a missing exchange fails the test. No GPU.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DIMS, K = (3, 2, 5), 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    import synth
    from oracle.assembly import GRAD_DIV, Problem
    nx, ny, nz = DIMS
    vx, vy, vz = synth.lattice_vertices(nx, ny, nz, perturb=0.1, seed=71)
    E = nx * ny * nz
    return Problem(nx, ny, nz, K, vx, vy, vz, synth.lognormal(E, 1.0, seed=72), synth.lognormal(E, 1.0, seed=73),
                   kind=GRAD_DIV, ess_mask=63)


def _local_apply(prob, elems, xg):
    """Element-by-element block apply of the given elements on a global-indexed vector xg
    (NaN where the rank holds nothing): the RT mass, the element's own cells' D and D^T
    parts, C, and the constrained identity on essential faces."""
    lat = prob.lat
    n_rt = lat.n_rt
    y = np.zeros_like(xg)
    v2f = lat.volume_to_face()
    ess = np.zeros(n_rt, dtype=bool)
    ess[prob.ess] = True
    for e in elems:
        g, sg = prob.e2d_idx[e], prob.e2d_sign[e]
        cells = prob.e2l[e] + n_rt
        u = np.where(ess[g], 0.0, xg[g] * sg)
        q = xg[cells]
        De = np.zeros((lat.n_l2_loc, lat.n_rt_loc))  # element-local divergence (local orientation)
        for a, faces in enumerate(v2f):
            for jloc, s in faces:
                De[a, jloc] = s
        yu = prob.Me[e] @ u + De.T @ q
        y[g] += np.where(ess[g], 0.0, yu * sg)
        y[g[ess[g]]] += xg[g[ess[g]]]  # each essential face belongs to one element
        y[cells] += De @ u - prob.Ce[e] @ q
    return y


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from paper_2304_12387_gb300.slab import SlabExchange, SlabLayout
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        prob = _problem()
        n = prob.n
        xg = np.random.Generator(np.random.PCG64(74)).uniform(-1, 1, n)
        L = SlabLayout(*DIMS, K, world, rank)
        ex = SlabExchange(L)
        x = L.to_local(torch.from_numpy(xg))
        ex.halo_in(x)
        # the rank's view of the global vector: its owned entries and halo, NaN elsewhere
        view = np.full(n, np.nan)
        for gs, ls in L.owned_pairs():
            view[gs] = x[ls].numpy()
        h0, h1 = L.plan["halo"]
        view[h0:h1] = x[L.halo_slice()].numpy()
        nx, ny, _ = DIMS
        ez = np.arange(prob.lat.n_elem) // (nx * ny)
        elems = np.nonzero((ez >= L.plan["ez"][0]) & (ez < L.plan["ez"][1]))[0]
        yv = _local_apply(prob, elems, view)
        y = torch.zeros(L.n_local, dtype=torch.float64)
        for gs, ls in L.owned_pairs():
            y[ls] = torch.from_numpy(yv[gs])
        y[L.halo_slice()] = torch.from_numpy(yv[h0:h1])
        ex.interface_sum(y)
        # global inner product by the allreduce of the owned partial sums
        d = ex.allreduce(torch.tensor([float((x[:L.n_owned] * y[:L.n_owned]).sum())], dtype=torch.float64))
        out.put((rank, [(gs.start, gs.stop, y[ls].numpy()) for gs, ls in L.owned_pairs()], float(d[0]),
                 bool(np.isfinite(yv[np.concatenate([np.arange(gs.start, gs.stop) for gs, _ in L.owned_pairs()])]).all())))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slab_exchange_reproduces_the_global_operator(world):
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    prob = _problem()
    xg = np.random.Generator(np.random.PCG64(74)).uniform(-1, 1, prob.n)
    ref = prob.apply_op(xg)
    y = np.full(prob.n, np.nan)
    for _, parts, _, finite in res:
        assert finite
        for lo, hi, v in parts:
            y[lo:hi] = v
    assert np.isfinite(y).all()
    assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max()
    for _, _, d, _ in res:
        assert abs(d - xg @ ref) <= 1e-12 * abs(xg @ ref)

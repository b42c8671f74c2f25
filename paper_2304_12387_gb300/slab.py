"""Exchange protocol of the z-slab partition over torch.distributed.

Partition p of P keeps, as one local vector, its owned entries of a block vector (its
x-faces, y-faces, z-faces and cells, the id ranges of hd_slab_plan, in that order)
followed by its halo: the z-face layer at the top of the slab, owned by p + 1. The
operator apply of a distributed solve then runs

    halo_in(x)          # x on the halo from p + 1 (X Y values per interface)
    local element loop  # the partition's element layers, into y (owned + halo)
    interface_sum(y)    # p's partial sums on its halo added to p + 1's own entries

and a MINRES iteration adds allreduce() of two scalars. The lower interface layer of
p (its first X Y owned z-faces) is the halo of p - 1. The calls are collective over the
P ranks of the process group; the local vectors are torch tensors on the device the
backend serves (CPU tensors for gloo).
"""
import torch
import torch.distributed as dist

from . import hd_slab_plan


class SlabLayout:
    """Local storage of partition p: owned ranges then the halo layer."""

    def __init__(self, nx, ny, nz, k, P, p):
        self.plan = hd_slab_plan(nx, ny, nz, k, P, p)
        self.p, self.P = p, P
        self.iface = (nx * k) * (ny * k)  # X Y values per interface layer
        self.ranges = [self.plan[key] for key in ("xf", "yf", "zf", "cell")]
        off, self.offsets = 0, []
        for lo, hi in self.ranges:
            self.offsets.append(off)
            off += hi - lo
        self.n_owned = off
        h0, h1 = self.plan["halo"]
        self.n_halo = h1 - h0
        self.n_local = off + self.n_halo
        self.zf_off = self.offsets[2]

    def to_local(self, x_global):
        """Owned entries of a global vector (halo left zero)."""
        out = torch.zeros(self.n_local, dtype=x_global.dtype, device=x_global.device)
        for (lo, hi), o in zip(self.ranges, self.offsets):
            out[o:o + hi - lo] = x_global[lo:hi]
        return out

    def owned_pairs(self):
        """(global slice, local slice) of each owned range."""
        return [(slice(lo, hi), slice(o, o + hi - lo)) for (lo, hi), o in zip(self.ranges, self.offsets)]

    def halo_slice(self):
        return slice(self.n_owned, self.n_local)

    def lower_interface_slice(self):
        """The first X Y owned z-faces: the layer that is the halo of p - 1."""
        return slice(self.zf_off, self.zf_off + self.iface)


class SlabExchange:
    """The two neighbour exchanges and the scalar allreduce of the partitioned apply."""

    def __init__(self, layout, group=None):
        self.L, self.group = layout, group

    def _peer(self, q):
        return q if self.group is None else dist.get_global_rank(self.group, q)

    def halo_in(self, x_local):
        """x_local's halo <- the lower interface layer of partition p + 1."""
        L, reqs = self.L, []
        if L.p > 0:
            reqs.append(dist.isend(x_local[L.lower_interface_slice()].contiguous(), self._peer(L.p - 1),
                                   group=self.group))
        if L.p < L.P - 1:
            buf = torch.empty(L.n_halo, dtype=x_local.dtype, device=x_local.device)
            reqs.append(dist.irecv(buf, self._peer(L.p + 1), group=self.group))
        for r in reqs:
            r.wait()
        if L.p < L.P - 1:
            x_local[L.halo_slice()] = buf

    def interface_sum(self, y_local):
        """p's partial sums on its halo are added to partition p + 1's lower interface layer."""
        L, reqs = self.L, []
        if L.p < L.P - 1:
            reqs.append(dist.isend(y_local[L.halo_slice()].contiguous(), self._peer(L.p + 1), group=self.group))
        if L.p > 0:
            buf = torch.empty(L.iface, dtype=y_local.dtype, device=y_local.device)
            reqs.append(dist.irecv(buf, self._peer(L.p - 1), group=self.group))
        for r in reqs:
            r.wait()
        if L.p > 0:
            y_local[L.lower_interface_slice()] += buf

    def allreduce(self, values):
        """Sum of a few scalars (a tensor) over the partitions, in place."""
        dist.all_reduce(values, op=dist.ReduceOp.SUM, group=self.group)
        return values

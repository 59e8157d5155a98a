"""Multi-GPU sharding of the hot path: x slabs with an x halo.

The cube is cut along x (the major axis, as the paper's node and section
decomposition cuts it, Sec. 3.1) into slabs whose boundaries fall on
multiples of the statistics window wx, so every window lives on one rank.
The only exchange is before the x pass: each rank needs `halo` = max R_xy
planes of its neighbours on each side (zeros beyond the cube edge).  The y/z
passes, the statistics, the threshold and the mask are then local, and the
global mask is the concatenation of the slab masks along x.

The exchange uses torch.distributed point-to-point send/recv (gloo on CPU,
NCCL on GPU), each rank receiving into its own memory.
"""
from __future__ import annotations

import math


def halo_width(bank, truncation: float) -> int:
    """Largest spatial radius of the bank: planes needed from each neighbour."""
    r = 0
    for sxy, _ in bank:
        if sxy > 0:
            r = max(r, int(math.ceil(truncation * sxy)))
    return r


def plan_slabs(nx: int, wx: int, world: int) -> list[tuple[int, int]]:
    """[x_begin, x_end) per rank: whole windows, as even as the window count allows."""
    nwin = -(-nx // wx)
    base, extra = divmod(nwin, world)
    out, w0 = [], 0
    for r in range(world):
        nw = base + (1 if r < extra else 0)
        x0 = min(nx, w0 * wx)
        x1 = min(nx, (w0 + nw) * wx)
        out.append((x0, x1))
        w0 += nw
    return out


def exchange_halo(slab, rank: int, world: int, halo: int, group=None):
    """Return (left, right) halo tensors of `halo` x-planes from the neighbours.

    slab is this rank's [x_end - x_begin][ny][nz] tensor.  A neighbour that
    does not exist contributes zeros (the image is zero outside the cube).  A
    slab thinner than the halo sends what it has, padded with zeros on the
    far side (its own neighbours' planes are not forwarded; plan_slabs keeps
    slabs at least one window thick).
    """
    import torch
    import torch.distributed as dist

    ny, nz = slab.shape[1], slab.shape[2]
    zeros = lambda: torch.zeros((halo, ny, nz), dtype=slab.dtype, device=slab.device)  # noqa: E731
    left, right = zeros(), zeros()
    if halo == 0 or world == 1:
        return left, right

    def edge(first: bool):
        n = min(halo, slab.shape[0])
        buf = zeros()
        if first:
            buf[:n] = slab[:n]
        else:
            buf[halo - n:] = slab[slab.shape[0] - n:]
        return buf.contiguous()

    ops = []
    if rank > 0:
        ops.append(dist.P2POp(dist.isend, edge(True), rank - 1, group))
        ops.append(dist.P2POp(dist.irecv, left, rank - 1, group))
    if rank < world - 1:
        ops.append(dist.P2POp(dist.isend, edge(False), rank + 1, group))
        ops.append(dist.P2POp(dist.irecv, right, rank + 1, group))
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    return left, right


def exchange_halo_into(ext, halo: int, rank: int, world: int, group=None):
    """In-place exchange on a preallocated extended slab ext = [halo | slab |
    halo] (x the major axis, so every part is a contiguous view): this rank's
    first and last `halo` slab planes go to its neighbours, whose planes are
    received straight into ext[:halo] and ext[-halo:].  Halo planes without a
    neighbour are left as they are (zeros, set once by the caller).  Slabs
    must be at least `halo` planes thick."""
    import torch.distributed as dist

    if halo == 0 or world == 1:
        return
    s = ext.shape[0] - 2 * halo
    if s < halo:
        raise ValueError("slab thinner than its halo")
    ops = []
    if rank > 0:
        ops.append(dist.P2POp(dist.isend, ext[halo:2 * halo], rank - 1, group))
        ops.append(dist.P2POp(dist.irecv, ext[:halo], rank - 1, group))
    if rank < world - 1:
        ops.append(dist.P2POp(dist.isend, ext[s:s + halo], rank + 1, group))
        ops.append(dist.P2POp(dist.irecv, ext[s + halo:], rank + 1, group))
    for req in dist.batch_isend_irecv(ops):
        req.wait()


def extended_slab(slab, left, right):
    """Halo + slab + halo along x, the input of the x pass for this rank."""
    import torch
    return torch.cat([left, slab, right], dim=0).contiguous()

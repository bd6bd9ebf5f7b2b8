"""Slice sharding across GPUs.

In parallel geometry each reconstructed slice depends on one detector row
only (Sec. 2.3: a reconstructed line depends on one and only one sinogram),
so several GPUs share a volume by taking contiguous ranges of slices, with no
exchange on the data path.  The only collective is the reduction of timings
and counts at the end of a measurement (or an optional gather of results).
"""
from __future__ import annotations

import torch


def slice_shard(n_slices: int, world: int, rank: int):
    """Contiguous range [z0, z1) of slices for ``rank`` of ``world``: the
    first n_slices % world ranks take one extra slice."""
    if world < 1 or not 0 <= rank < world or n_slices < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n_slices, world)
    z0 = rank * base + min(rank, extra)
    return z0, z0 + base + (1 if rank < extra else 0)


def reduce_throughput(elapsed_ms: float, units: float, device=None):
    """Max of the per-rank elapsed times and sum of the per-rank work units
    over the default process group (identity without one)."""
    import torch.distributed as dist
    t = torch.tensor([elapsed_ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return t.item(), u.item()


def fbp_shard(geom, data, kind, flat=None, dark=None, world: int = 1, rank: int = 0, out=None, **kw):
    """Reconstruct this rank's contiguous share of a raw stack
    [n_angles, n_slices, n_bins] (read in place) with pyhst_fbp; returns
    (z0, z1, images [z1 - z0, ny, nx])."""
    from . import pyhst_fbp
    ns = data.shape[1] if data.dim() == 3 else 1
    z0, z1 = slice_shard(ns, world, rank)
    if z1 == z0:
        return z0, z1, None
    return z0, z1, pyhst_fbp(geom, data, kind, flat, dark, out=out, slices=(z0, z1), **kw)

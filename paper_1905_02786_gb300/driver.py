"""Expansion driver over the C ABI, optionally sharded over processes.

The tuples of one order are independent CASCI problems (Sec. 2; the paper
farms them out to MPI workers, Sec. 4.2.3).  With ``world > 1`` every
process generates the same order-k tuple list on its GPU, solves the tuples
i with i % world == rank, the energies are all-gathered (the one exchange
per order), and every process then assembles the increments of the whole
order (Eq. 3) so that all hashes stay identical for the next order.
"""
from __future__ import annotations

import numpy as np

from . import _binding as B


def shard_indices(n: int, rank: int, world: int) -> np.ndarray:
    """Round-robin share of rank: tuples of similar size are interleaved in
    lexicographic order, so every rank gets a similar mix."""
    return np.arange(rank, n, world, dtype=np.int64)


def merge_shards(parts, n: int, world: int) -> np.ndarray:
    """Inverse of shard_indices: parts[r] holds the values of rank r's share."""
    out = np.empty(n)
    for r in range(world):
        out[shard_indices(n, r, world)] = parts[r]
    return out


def torch_allgather(group=None):
    """all-gather of float64 arrays of different lengths over torch.distributed."""
    import torch
    import torch.distributed as dist

    def gather(local: np.ndarray, counts):
        world = dist.get_world_size(group)
        dev = torch.device("cuda", torch.cuda.current_device()) \
            if dist.get_backend(group) == "nccl" else torch.device("cpu")
        mx = max(max(counts), 1)
        buf = torch.zeros(mx, dtype=torch.float64, device=dev)
        buf[: local.size] = torch.from_numpy(local).to(dev)
        outs = [torch.empty(mx, dtype=torch.float64, device=dev) for _ in range(world)]
        dist.all_gather(outs, buf, group=group)
        return [outs[r][: counts[r]].cpu().numpy() for r in range(world)]
    return gather


def run_expansion(ctx, ref, exp, max_order, thr=0.0, rank=0, world=1, allgather=None,
                  solve=None, callback=None):
    """Run orders 1..max_order; returns dict(eps_ref, orders, total, ntup).

    ``solve(ctx, tuples, k) -> eps`` defaults to mbe_solve_tuples; tests may
    pass a host solver to exercise the sharding logic without a GPU."""
    if solve is None:
        def solve(c, t, k):
            return B.mbe_solve_tuples(c, t, k)[0]
    e_ref = B.mbe_set_reference(ctx, ref, exp)
    orders = []
    total = e_ref
    ntot = 0
    for k in range(1, max_order + 1):
        tuples = B.mbe_next_tuples(ctx, k)
        n = len(tuples)
        if n == 0:
            break
        mine = shard_indices(n, rank, world)
        eps_local = solve(ctx, tuples[mine], k) if len(mine) else np.zeros(0)
        if world > 1:
            counts = [len(shard_indices(n, r, world)) for r in range(world)]
            eps = merge_shards(allgather(np.asarray(eps_local, dtype=np.float64), counts), n, world)
            B.mbe_set_order_energies(ctx, tuples, eps, k)
        else:
            eps = eps_local
        inc, keep, e_order, total = B.mbe_increments(ctx, k, thr, n)
        ntot += n
        rec = dict(order=k, tuples=tuples, eps=eps, inc=inc, keep=keep, E_order=e_order)
        orders.append(rec)
        if callback:
            callback(rec)
    return dict(eps_ref=e_ref, orders=orders, total=total, ntup=ntot)

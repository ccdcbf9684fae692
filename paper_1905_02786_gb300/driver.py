"""Expansion driver over the C ABI, optionally sharded over processes.

The tuples of one order are independent CASCI problems (Sec. 2; the paper
farms them out to MPI workers, Sec. 4.2.3).  With ``world > 1`` every
process generates the same order-k tuple list on its GPU, solves its share
of the tuples, the energies are all-gathered (the one exchange per order),
and every process then assembles the increments of the whole order (Eq. 3)
so that all hashes stay identical for the next order.

Shares: with per-tuple work estimates (the determinant count of the tuple's
CASCI, which sets the cost of its sigma vectors; the iteration counts are
alike) the tuples are dealt heaviest first to the least loaded rank, so the
ranks carry equal work and each holds a share of every bin of equal size;
without them, round-robin in lexicographic order.
"""
from __future__ import annotations

import math

import numpy as np

from . import _binding as B


def shard_indices(n: int, rank: int, world: int, weights=None) -> np.ndarray:
    """Indices (ascending) of the tuples that rank solves.  Deterministic:
    every rank computes the same assignment from the same inputs."""
    if weights is None or world == 1:
        return np.arange(rank, n, world, dtype=np.int64)
    return np.flatnonzero(shard_owner(np.asarray(weights, dtype=np.float64), world) == rank)


def shard_owner(weights: np.ndarray, world: int) -> np.ndarray:
    """Owner rank of every tuple: heaviest first (stable), each to the rank
    with the least load so far (lowest rank on ties)."""
    order = np.argsort(-weights, kind="stable")
    load = np.zeros(world)
    owner = np.empty(len(weights), dtype=np.int64)
    for i in order:
        r = int(np.argmin(load))
        owner[i] = r
        load[r] += weights[i]
    return owner


def merge_shards(parts, n: int, world: int, weights=None) -> np.ndarray:
    """Inverse of shard_indices: parts[r] holds the values of rank r's share."""
    out = np.empty(n)
    for r in range(world):
        out[shard_indices(n, r, world, weights)] = parts[r]
    return out


def tuple_weights(tuples: np.ndarray, ref, nocc) -> np.ndarray:
    """Work estimate of each tuple's CASCI: its determinant count
    C(n, n_alpha) C(n, n_beta), n = |Pi| + order active orbitals, n_alpha and
    n_beta the occupied orbitals of each spin among them.  ``nocc``: an int
    (closed shell) or (n_alpha, n_beta) occupied orbitals (high spin)."""
    na, nb = (int(nocc[0]), int(nocc[1])) if isinstance(nocc, (tuple, list)) else (nocc, nocc)
    n = len(ref) + tuples.shape[1]
    cnt = []
    for occ in (na, nb):
        base = sum(1 for r in ref if r < occ)
        cnt.append(base + (tuples < occ).sum(axis=1))
    return np.array([float(math.comb(n, int(a)) * math.comb(n, int(b)))
                     for a, b in zip(*cnt)])


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


def torch_allreduce_sum(group=None):
    """sum of float64 arrays over torch.distributed (same shape on all ranks)."""
    import torch
    import torch.distributed as dist

    def reduce(a: np.ndarray) -> np.ndarray:
        dev = torch.device("cuda", torch.cuda.current_device()) \
            if dist.get_backend(group) == "nccl" else torch.device("cpu")
        t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)
        dist.all_reduce(t, group=group)
        return t.cpu().numpy()
    return reduce


def run_expansion(ctx, ref, exp, max_order, thr=0.0, rank=0, world=1, allgather=None,
                  solve=None, callback=None, api=None, nocc=None, pairs=None):
    """Run orders 1..max_order; returns dict(eps_ref, orders, total, ntup).

    ``api`` is the module of C-ABI wrappers (default: the binding);
    ``solve(ctx, tuples, k) -> eps`` defaults to its mbe_solve_tuples.  Tests
    pass a host stand-in for both to exercise the sharding logic without a
    GPU.  With ``nocc`` (occupied orbitals of the reference determinant) the
    shares are weighted by the tuples' determinant counts.  ``pairs`` of
    degenerate expansion orbitals switch on pi-pruning (Sec. 3)."""
    B_ = api or B
    if solve is None:
        def solve(c, t, k):
            return B_.mbe_solve_tuples(c, t, k)[0]
    e_ref = B_.mbe_set_reference(ctx, ref, exp)
    if pairs:
        B_.mbe_set_pruning_pairs(ctx, pairs)
    orders = []
    total = e_ref
    ntot = 0
    empty_run = 0
    for k in range(1, max_order + 1):
        tuples = B_.mbe_next_tuples(ctx, k).reshape(-1, k)
        n = len(tuples)
        if n == 0:
            # with pruning an empty order can precede a non-empty one (a pair
            # adds two orbitals); two empty orders end the expansion
            empty_run += 1
            if empty_run >= (2 if pairs else 1):
                break
        else:
            empty_run = 0
        wts = tuple_weights(tuples, ref, nocc) if (nocc is not None and world > 1) else None
        mine = shard_indices(n, rank, world, wts)
        eps_local = solve(ctx, tuples[mine], k) if len(mine) else np.zeros(0)
        if world > 1:
            counts = [len(shard_indices(n, r, world, wts)) for r in range(world)]
            eps = merge_shards(allgather(np.asarray(eps_local, dtype=np.float64), counts), n,
                               world, wts)
            B_.mbe_set_order_energies(ctx, tuples, eps, k)
        else:
            eps = eps_local
        inc, keep, e_order, total = B_.mbe_increments(ctx, k, thr, n)
        ntot += n
        rec = dict(order=k, tuples=tuples, eps=eps, inc=inc, keep=keep, E_order=e_order)
        orders.append(rec)
        if callback:
            callback(rec)
    return dict(eps_ref=e_ref, orders=orders, total=total, ntup=ntot)


def sharded_backward(ctx, norb, rank=0, world=1, allreduce=None, api=None):
    """Gradient of a sharded expansion: each context sums the weighted RDMs
    of the CASCIs it solved (created with backward_share = 2 on rank 0 and 1
    on the others, so the reference term is counted once) and the shares are
    summed over the ranks."""
    B_ = api or B
    dh, deri = B_.mbe_energy_backward(ctx, norb)
    if world > 1:
        dh, deri = allreduce(dh), allreduce(deri)
    return dh, deri

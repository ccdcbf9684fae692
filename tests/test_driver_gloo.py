"""Sharded expansion driver over torch.distributed (gloo, world size 2, CPU).

The tuples of one order are split round-robin over the ranks, each rank
solves its share, the energies are all-gathered and every rank assembles the
increments of the whole order.  Here the C-ABI calls are replaced by a host
stand-in built on the oracle (same contract: the order-k tuples from the
screening rule, Eq. 3 increments, the backward of the held CI vectors), so
the sharding logic itself runs without a GPU.
"""
import multiprocessing as mp
import os
import math
import socket

import numpy as np
import pytest

import mbe_synth as ms
from oracle import casci as oc
from oracle import mbe as om

NORB, NOCC, SEED = 6, 2, 17
REF, EXP, MAX_ORDER, THR = [1, 2], [0, 3, 4, 5], 3, 2e-3


class HostAPI:
    """Oracle-backed stand-in for the binding's mbe_* wrappers."""

    def __init__(self, h, eri, nocc, share):
        self.h, self.eri, self.nocc, self.share = h, eri, nocc, share
        self.inc, self.prev, self.thr = {}, {}, 0.0
        self.held = {}                       # tuples solved by this rank
        self.sums = []

    def mbe_set_reference(self, ctx, ref, exp):
        self.ref, self.exp = list(ref), list(exp)
        self.e_ref = oc.casci(self.h, self.eri, self.nocc, sorted(ref))
        return self.e_ref

    def mbe_next_tuples(self, ctx, k):
        t = om.next_order_tuples(self.exp, self.prev, self.thr, k)
        return np.array(t, dtype=np.int32).reshape(len(t), k)

    def mbe_solve_tuples(self, ctx, tuples, k):
        eps = []
        for row in tuples:
            t = tuple(int(x) for x in row)
            eps.append(oc.casci(self.h, self.eri, self.nocc, om.active_space(self.ref, t)))
            self.held[t] = True
        self.cur = (np.asarray(tuples), np.array(eps))
        return np.array(eps), np.zeros(len(eps), dtype=np.int32)

    def mbe_set_order_energies(self, ctx, tuples, eps, k):
        self.cur = (np.asarray(tuples), np.asarray(eps))

    def mbe_increments(self, ctx, k, thr, n):
        tuples, eps = self.cur
        lvl, incs = {}, []
        for row, e in zip(tuples, eps):
            t = tuple(int(x) for x in row)
            d = om.increment_recursive(t, float(e), self.e_ref, self.inc)
            self.inc[t] = d
            lvl[t] = d
            incs.append(d)
        self.prev, self.thr = lvl, thr
        e_order = om.kahan_sum(incs)
        self.sums.append(e_order)
        keep = np.array([abs(d) >= thr if thr > 0 else True for d in incs])
        return np.array(incs), keep, e_order, om.kahan_sum([self.e_ref] + self.sums)

    def mbe_energy_backward(self, ctx, norb, scale=1.0):
        coef = om.mbe_coefficients(list(self.inc.keys()))
        n = self.h.shape[0]
        dh = np.zeros((n, n))
        dg = np.zeros((n, n, n, n))
        for s, c in coef.items():
            if c == 0 or (s == () and self.share == 1) or (s != () and s not in self.held):
                continue
            e, vec, sp = oc.casci(self.h, self.eri, self.nocc, om.active_space(self.ref, s),
                                  want_vector=True)
            g1, g2 = sp.rdm12(vec)
            dh += c * g1
            dg += c * 0.5 * g2
        return scale * dh, scale * om.pack_eri_gradient(dg, n)


def _worker(rank, world, port, q):
    import torch.distributed as dist
    from paper_1905_02786_gb300 import driver
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        h, eri, _ = ms.gen_integrals(NORB, NOCC, SEED)
        api = HostAPI(h, eri, NOCC, share=2 if rank == 0 else 1)
        res = driver.run_expansion(None, REF, EXP, MAX_ORDER, THR, rank=rank, world=world,
                                   allgather=driver.torch_allgather(), api=api, nocc=NOCC)
        dh, dg = driver.sharded_backward(None, NORB, rank, world,
                                         driver.torch_allreduce_sum(), api=api)
        q.put((rank, res["total"], res["ntup"], len(api.held), dh, dg))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_indices_partition():
    from paper_1905_02786_gb300 import driver
    rng = np.random.default_rng(3)
    for n in (0, 1, 5, 17, 200):
        for world in (1, 2, 3, 8):
            for weights in (None, rng.choice([48400.0, 245025.0, 108900.0], size=n)):
                parts = [driver.shard_indices(n, r, world, weights) for r in range(world)]
                assert sorted(np.concatenate(parts).tolist()) == list(range(n))
                vals = np.arange(n, dtype=np.float64) * 1.5
                got = driver.merge_shards([vals[p] for p in parts], n, world, weights)
                assert np.array_equal(got, vals)
                if weights is not None and n:
                    # greedy heaviest-first: loads differ by at most one tuple's weight
                    loads = [weights[p].sum() for p in parts]
                    assert max(loads) - min(loads) <= weights.max()


def test_tuple_weights_are_determinant_counts():
    """The work estimate of a tuple is the determinant count of its CASCI:
    Pi = {1..6} with orbitals 0-3 occupied (CAS(6e,6o)); adding occupied
    orbital 0 gives 8 electrons, a virtual keeps 6."""
    from paper_1905_02786_gb300 import driver
    t = np.array([[0, 7, 8], [7, 8, 9]], dtype=np.int32)
    w = driver.tuple_weights(t, [1, 2, 3, 4, 5, 6], 4)
    assert w[0] == float(math.comb(9, 4)) ** 2 and w[1] == float(math.comb(9, 3)) ** 2


@pytest.mark.timeout(600)
def test_sharded_expansion_gloo_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=500) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    h, eri, _ = ms.gen_integrals(NORB, NOCC, SEED)
    ref = om.run_mbe(h, eri, NOCC, REF, EXP, MAX_ORDER, THR)
    ntup = sum(len(o["tuples"]) for o in ref["orders"])
    odh, odg, _ = om.mbe_gradient(h, eri, NOCC, REF, list(ref["inc"].keys()))
    for rank, total, nt, held, dh, dg in out:
        # every rank assembles the same total from the gathered energies
        assert abs(total - ref["total"]) < 1e-12
        assert nt == ntup
        # shares weighted by determinant counts: each rank solved a part
        assert 0 < held < ntup
        # the summed shares are the whole gradient
        assert np.max(np.abs(dh - odh)) < 1e-12
        assert np.max(np.abs(dg - odg)) < 1e-12

"""Oracle (test infrastructure only): the many-body expansion bookkeeping.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs may import this package.

Follows Sec. 2 of the paper:
* Eq. 1: E = sum of the increments of all orders (here plus the order-0
  reference-space energy, because with a CAS reference the reference
  CASCI is not zero; Eq. 3).
* Eq. 2 / Eq. 3: the increment of a tuple is its CASCI energy minus the
  reference-space energy minus the increments of all of its proper,
  non-empty subtuples (S_m = all unique subtuples of length m, 1 <= m < n).
* Fig. 2: the CASCI of a tuple correlates the reference space plus the
  tuple; other occupied orbitals are inactive, other virtuals deleted.

Screening: the paper defines its threshold ``a`` in Part I of the series,
which is not reproduced; this oracle uses the downward-closed rule on
increment magnitudes: at order k >= 2 a tuple is formed iff every one of its
(k-1)-subtuples was formed at order k-1 and at least one of those has
|increment| >= thr.  A screened tuple still contributes its own increment;
it only cannot spawn children on its own.  thr = 0 means no screening.

The energies used are total electronic energies (the paper's correlation
energies differ from them by a constant, which changes only the order-0
term).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from .casci import casci, Space


def kahan_sum(values) -> float:
    """Compensated (Kahan) summation."""
    s = 0.0
    comp = 0.0
    for v in values:
        y = v - comp
        t = s + y
        comp = (t - s) - y
        s = t
    return s


def next_order_tuples(exp, prev: dict, thr: float, k: int):
    """Order-k tuples (sorted, lexicographic) from the order-(k-1) level
    ``prev`` = {tuple: increment} by the downward-closed screening rule."""
    exp = sorted(exp)
    if k == 1:
        return [(o,) for o in exp]
    out = []
    for t in itertools.combinations(exp, k):
        subs = [t[:i] + t[i + 1:] for i in range(k)]
        if not all(s in prev for s in subs):
            continue
        if thr > 0.0 and not any(abs(prev[s]) >= thr for s in subs):
            continue
        out.append(t)
    return out


def increment_recursive(t, eps_t: float, eps_ref: float, inc: dict) -> float:
    """Eq. 3: eps_T - eps_Pi - sum over proper non-empty subtuples of their
    increments (looked up in ``inc``, which holds all lower orders)."""
    d = eps_t - eps_ref
    for m in range(1, len(t)):
        for s in itertools.combinations(t, m):
            d -= inc[s]
    return d


def increment_mobius(t, eps: dict, eps_ref: float) -> float:
    """Closed form of the recursion (Moebius inversion over the subset
    lattice): sum_{S subset T} (-1)^{|T|-|S|} eps_S, with eps_{} = eps_Pi."""
    d = 0.0
    n = len(t)
    for m in range(0, n + 1):
        sg = -1.0 if (n - m) % 2 else 1.0
        for s in itertools.combinations(t, m):
            d += sg * (eps[s] if m else eps_ref)
    return d


def active_space(ref, t):
    return sorted(set(ref) | set(t))


def run_mbe(h, eri, nocc, ref, exp, max_order, thr=0.0, solver=None, keep_vectors=False):
    """Run the expansion.  Returns a dict with the reference energy, per
    order lists (tuples, eps, inc, keep, E_order) and the total (Kahan)."""
    if solver is None:
        def solver(act):
            return casci(h, eri, nocc, act)
    eps_ref = solver(sorted(ref))
    eps, inc = {}, {}
    orders = []
    prev = None
    for k in range(1, max_order + 1):
        tuples = next_order_tuples(exp, prev or {}, thr, k)
        if not tuples:
            break
        lvl = {}
        rec = dict(tuples=tuples, eps=[], inc=[], keep=[])
        for t in tuples:
            e = solver(active_space(ref, t))
            eps[t] = e
            d = increment_recursive(t, e, eps_ref, inc)
            inc[t] = d
            lvl[t] = d
            rec["eps"].append(e)
            rec["inc"].append(d)
            rec["keep"].append(abs(d) >= thr if thr > 0.0 else True)
        rec["E_order"] = kahan_sum(rec["inc"])
        orders.append(rec)
        prev = lvl
    total = kahan_sum([eps_ref] + [o["E_order"] for o in orders])
    return dict(eps_ref=eps_ref, orders=orders, total=total, eps=eps, inc=inc)


def mbe_coefficients(tuples):
    """c_S = sum_{T in set, T >= S} (-1)^{|T|-|S|} over the tuple set plus the
    empty tuple (the reference space), so that E_MBE = sum_S c_S eps_S."""
    tset = set(tuples) | {()}
    coef = {}
    for s in tset:
        c = 0
        ss = set(s)
        for t in tset:
            if len(t) >= len(s) and ss.issubset(t):
                c += -1 if (len(t) - len(s)) % 2 else 1
        coef[s] = c
    return coef


def pack_eri_gradient(g2_half, norb):
    """Gradient w.r.t. the symmetric packed ERI matrix eri[P, Q]:
    sum of dE/d(pq|rs) over the full-tensor images of (P, Q), symmetrised
    over P <-> Q."""
    npair = norb * (norb + 1) // 2
    G = np.zeros((npair, npair))
    pairs = [(p, q) for p in range(norb) for q in range(p + 1)]
    for P, (p, q) in enumerate(pairs):
        imgs_pq = [(p, q)] if p == q else [(p, q), (q, p)]
        for Q, (r, s) in enumerate(pairs):
            imgs_rs = [(r, s)] if r == s else [(r, s), (s, r)]
            G[P, Q] = sum(g2_half[a, b, c, d] for a, b in imgs_pq for c, d in imgs_rs)
    return 0.5 * (G + G.T)


def mbe_gradient(h, eri, nocc, ref, tuples):
    """dE_MBE/dh (n x n) and dE_MBE/d eri_packed (npair x npair) for the given
    tuple set (assumed downward closed), via Hellmann-Feynman:
    dE_T/dh_pq = gamma^T_pq and dE_T/d(pq|rs) = 1/2 Gamma^T_pqrs (full-space
    spin-summed RDMs), summed with the coefficients of ``mbe_coefficients``."""
    n = h.shape[0]
    coef = mbe_coefficients(tuples)
    dh = np.zeros((n, n))
    dg = np.zeros((n, n, n, n))
    for s, c in coef.items():
        if c == 0:
            continue
        e, vec, sp = casci(h, eri, nocc, active_space(ref, s), want_vector=True)
        g1, g2 = sp.rdm12(vec)
        dh += c * g1
        dg += c * 0.5 * g2
    return dh, pack_eri_gradient(dg, n), coef

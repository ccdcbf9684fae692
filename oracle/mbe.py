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

pi-pruning (Sec. 3): given pairs of degenerate expansion orbitals, only
tuples that hold both orbitals of a pair or neither are formed.  The
expansion then runs over "units" (a single orbital, or a pair taken
together): a tuple is a union of units, its order is its orbital count, its
parents are the tuples with one unit removed (one or two orbitals fewer),
and Eq. 3 subtracts the increments of its proper non-empty sub-unions of
units.  The Moebius form counts units.  Unscreened and taken to all orders
it still sums to the FCI energy of the whole space.
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


# ----------------------------------------------------------- pi-pruning
def expansion_units(exp, pairs):
    """Units of the pruned expansion: tuples of one orbital (no partner) or
    two orbitals (a degenerate pair), sorted by their lowest orbital."""
    paired = {}
    for a, b in pairs:
        paired[a], paired[b] = b, a
    units = []
    for o in sorted(exp):
        if o not in paired:
            units.append((o,))
        elif o < paired[o]:
            units.append((o, paired[o]))
    return sorted(units)


def _unit_split(t, units):
    """The units whose union is t (t must be such a union)."""
    ts = set(t)
    us = [u for u in units if ts.issuperset(u)]
    if sum(len(u) for u in us) != len(t):
        raise ValueError(f"tuple {t} is not a union of units")
    return us


def next_order_tuples_pruned(exp, pairs, formed: dict, thr: float, k: int):
    """Order-k tuples (orbital count k, lexicographic) of the pruned
    expansion: unions of units of k orbitals whose every one-unit-removed
    subtuple was formed (the empty tuple, i.e. the reference space, counts as
    formed and kept) and, with screening, at least one of them has
    |increment| >= thr.  ``formed`` = {tuple: increment} of all lower orders."""
    units = expansion_units(exp, pairs)
    out = []
    for r in range(1, len(units) + 1):
        for us in itertools.combinations(units, r):
            if sum(len(u) for u in us) != k:
                continue
            t = tuple(sorted(o for u in us for o in u))
            subs = []
            for i in range(r):
                subs.append(tuple(sorted(o for j, u in enumerate(us) if j != i for o in u)))
            if not all(s == () or s in formed for s in subs):
                continue
            if thr > 0.0 and not any(s == () or abs(formed[s]) >= thr for s in subs):
                continue
            out.append(t)
    return sorted(out)


def increment_recursive_units(t, eps_t: float, eps_ref: float, inc: dict, units) -> float:
    """Eq. 3 over units: eps_T - eps_Pi - sum over the proper non-empty
    sub-unions of units of T of their increments."""
    us = _unit_split(t, units)
    d = eps_t - eps_ref
    for m in range(1, len(us)):
        for sub in itertools.combinations(us, m):
            d -= inc[tuple(sorted(o for u in sub for o in u))]
    return d


def increment_mobius_units(t, eps: dict, eps_ref: float, units) -> float:
    """Closed form over the lattice of unit sets: sum over sub-unions S of T
    of (-1)^(units(T) - units(S)) eps_S, eps_{} = eps_Pi."""
    us = _unit_split(t, units)
    n = len(us)
    d = 0.0
    for m in range(0, n + 1):
        sg = -1.0 if (n - m) % 2 else 1.0
        for sub in itertools.combinations(us, m):
            key = tuple(sorted(o for u in sub for o in u))
            d += sg * (eps[key] if m else eps_ref)
    return d


def run_mbe(h, eri, nocc, ref, exp, max_order, thr=0.0, solver=None, keep_vectors=False,
            pairs=None):
    """Run the expansion (pi-pruned over ``pairs`` of degenerate expansion
    orbitals if given); ``nocc`` is an int (closed-shell reference) or
    (n_alpha, n_beta) for a high-spin one (Fig. 2 case (b)).  Returns a dict with the reference energy, per
    order lists (tuples, eps, inc, keep, E_order) and the total (Kahan)."""
    if solver is None:
        def solver(act):
            return casci(h, eri, nocc, act)
    eps_ref = solver(sorted(ref))
    eps, inc = {}, {}
    orders = []
    prev = None
    units = expansion_units(exp, pairs) if pairs else None
    empty_run = 0
    for k in range(1, max_order + 1):
        if pairs:
            tuples = next_order_tuples_pruned(exp, pairs, inc, thr, k)
        else:
            tuples = next_order_tuples(exp, prev or {}, thr, k)
        if not tuples:
            # a unit holds one or two orbitals: after two empty orders no
            # tuple can be formed any more (after one without pruning)
            empty_run += 1
            if empty_run >= (2 if pairs else 1):
                break
            orders.append(dict(tuples=[], eps=[], inc=[], keep=[], E_order=0.0))
            continue
        empty_run = 0
        lvl = {}
        rec = dict(tuples=tuples, eps=[], inc=[], keep=[])
        for t in tuples:
            e = solver(active_space(ref, t))
            eps[t] = e
            if pairs:
                d = increment_recursive_units(t, e, eps_ref, inc, units)
            else:
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


def mbe_coefficients(tuples, units=None):
    """c_S = sum_{T in set, T >= S} (-1)^{|T|-|S|} over the tuple set plus the
    empty tuple (the reference space), so that E_MBE = sum_S c_S eps_S; with
    the units of a pruned expansion |.| counts units."""
    tset = set(tuples) | {()}

    def size(t):
        return len(_unit_split(t, units)) if units else len(t)
    coef = {}
    for s in tset:
        c = 0
        ss = set(s)
        for t in tset:
            if len(t) >= len(s) and ss.issubset(t):
                c += -1 if (size(t) - size(s)) % 2 else 1
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


def mbe_gradient(h, eri, nocc, ref, tuples, units=None):
    """dE_MBE/dh (n x n) and dE_MBE/d eri_packed (npair x npair) for the given
    tuple set (assumed downward closed), via Hellmann-Feynman:
    dE_T/dh_pq = gamma^T_pq and dE_T/d(pq|rs) = 1/2 Gamma^T_pqrs (full-space
    spin-summed RDMs), summed with the coefficients of ``mbe_coefficients``
    (over units for a pruned expansion)."""
    n = h.shape[0]
    coef = mbe_coefficients(tuples, units)
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

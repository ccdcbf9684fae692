"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds only input recipes (integral generators and the workload
definitions); none of the MBE-FCI arithmetic lives here.  Both the oracle
(``oracle/``) and the CUDA path's tests and benchmark draw their inputs from
it, so both sides see bit-identical integrals.

Integral recipe (stand-in for the molecular MO integrals of the paper's
H2O / N2 / C2 / H10 systems, Sec. 4):

* orbital energies ``eps``: the occupied values uniform in ``eps_occ``, the
  virtual values uniform in ``eps_vir``, drawn in that order, then sorted
  ascending (occupied below virtual, so the lowest ``nocc`` orbitals are the
  RHF-occupied ones);
* one-electron integrals ``h_pq = delta_pq eps_p + h_noise * S_pq`` with ``S``
  symmetric, upper triangle (diagonal included) N(0,1), mirrored, / sqrt(n);
* two-electron integrals in chemists' notation
  ``(pq|rs) = sum_{L=1..2n} B^L_pq B^L_rs`` with every ``B^L`` symmetric,
  upper triangle N(0,1), mirrored, then all ``B`` scaled by one ``s`` so that
  the mean of ``(pp|pp)`` over p equals ``mean_pppp``.  This gives the full
  8-fold permutational symmetry and a positive semi-definite ERI matrix.

The ERI tensor is returned packed 4-fold as an ``npair x npair`` matrix
``eri[P, Q]`` with ``P = pair(p, q) = p(p+1)/2 + q`` for ``p >= q``.
"""
from __future__ import annotations

import numpy as np

__all__ = ["pair_index", "npair", "gen_integrals", "unpack_eri", "WORKLOADS",
           "workload", "workload_integrals", "random_symmetric_ci",
           "sample_tuples"]


def npair(n: int) -> int:
    return n * (n + 1) // 2


def pair_index(p: int, q: int) -> int:
    if p < q:
        p, q = q, p
    return p * (p + 1) // 2 + q


def gen_integrals(norb: int, nocc: int, seed: int,
                  eps_occ=(-1.5, -0.4), eps_vir=(0.05, 3.0),
                  mean_pppp: float = 0.5, h_noise: float = 0.05):
    """Return ``(h, eri_packed, eps)``; see the module docstring."""
    rng = np.random.default_rng(seed)
    eo = rng.uniform(eps_occ[0], eps_occ[1], size=nocc)
    ev = rng.uniform(eps_vir[0], eps_vir[1], size=norb - nocc)
    eps = np.sort(np.concatenate([eo, ev]))
    iu = np.triu_indices(norb)
    S = np.zeros((norb, norb))
    S[iu] = rng.standard_normal(iu[0].size)
    S = S + np.triu(S, 1).T
    S /= np.sqrt(norb)
    h = np.diag(eps) + h_noise * S
    nL = 2 * norb
    # B^L packed over pairs: column L holds B^L_pq for p >= q in pair order.
    il = np.tril_indices(norb)          # (p, q) with p >= q, row-major = pair order
    Bp = np.empty((npair(norb), nL))
    for L in range(nL):
        B = np.zeros((norb, norb))
        B[iu] = rng.standard_normal(iu[0].size)
        B = B + np.triu(B, 1).T
        Bp[:, L] = B[il]
    diag = np.array([pair_index(p, p) for p in range(norb)])
    s2 = mean_pppp / np.mean(np.sum(Bp[diag] ** 2, axis=1))
    Bp *= np.sqrt(s2)
    eri = Bp @ Bp.T
    eri = 0.5 * (eri + eri.T)
    return np.ascontiguousarray(h), np.ascontiguousarray(eri), eps


def unpack_eri(eri_packed: np.ndarray, norb: int) -> np.ndarray:
    """Expand a packed ``npair x npair`` ERI matrix to a full ``n^4`` array."""
    idx = np.empty((norb, norb), dtype=np.int64)
    for p in range(norb):
        for q in range(norb):
            idx[p, q] = pair_index(p, q)
    return eri_packed[idx[:, :, None, None], idx[None, None, :, :]]


# Workload definitions (sizes, seeds, reference and expansion spaces).
# Orbital indices are 0-based; the occupied orbitals are 0 .. nocc-1.
WORKLOADS = {
    # 8e/12o, all orders, no screening: sum of increments = full FCI.
    "fci8e12o_allorder": dict(norb=12, nel=8, seed=0, eps_occ=(-1.5, -0.4),
                              eps_vir=(0.05, 3.0), mean_pppp=0.5,
                              ref=[2, 3, 4, 5], exp=[0, 1, 6, 7, 8, 9, 10, 11],
                              max_order=8, thr=0.0),
    # 8e/23o water-double-zeta-shaped, CAS(6e,6o), order <= 6, screened.
    "h2o_dz_8e23o": dict(norb=23, nel=8, seed=1, eps_occ=(-1.5, -0.4),
                         eps_vir=(0.05, 3.0), mean_pppp=0.5,
                         ref=[1, 2, 3, 4, 5, 6], exp=[0] + list(range(7, 23)),
                         max_order=6, thr=1e-6),
    "h2o_dz_8e23o_stretched": dict(norb=23, nel=8, seed=1, eps_occ=(-1.5, -0.4),
                                   eps_vir=(0.02, 0.6), mean_pppp=0.5,
                                   ref=[1, 2, 3, 4, 5, 6],
                                   exp=[0] + list(range(7, 23)),
                                   max_order=6, thr=1e-6),
    # 10e/60o hydrogen-chain-shaped, CAS(10e,10o), order <= 4, screened.
    "h10_chain_10e60o": dict(norb=60, nel=10, seed=2, eps_occ=(-0.6, -0.3),
                             eps_vir=(0.0, 1.5), mean_pppp=0.6,
                             ref=list(range(10)), exp=list(range(10, 60)),
                             max_order=4, thr=1e-6),
    # 8e/20o, CAS(4e,4o), unscreened to order 4 (energy gradient workload).
    "grad_8e20o": dict(norb=20, nel=8, seed=3, eps_occ=(-1.5, -0.4),
                       eps_vir=(0.05, 3.0), mean_pppp=0.5,
                       ref=[2, 3, 4, 5], exp=[0, 1] + list(range(6, 20)),
                       max_order=4, thr=0.0),
    # 8e/114o water-quadruple-zeta-shaped, CAS(8e,8o), order <= 5, screened.
    "h2o_qz_8e114o": dict(norb=114, nel=8, seed=4, eps_occ=(-1.5, -0.4),
                          eps_vir=(0.05, 3.0), mean_pppp=0.5,
                          ref=list(range(8)), exp=list(range(8, 114)),
                          max_order=5, thr=1e-6),
}


def workload(name: str) -> dict:
    w = dict(WORKLOADS[name])
    w["name"] = name
    w["nocc"] = w["nel"] // 2
    return w


def workload_integrals(name: str):
    w = workload(name)
    return gen_integrals(w["norb"], w["nocc"], w["seed"], w["eps_occ"],
                         w["eps_vir"], w["mean_pppp"])


def random_symmetric_ci(nstr: int, seed: int, batch: int = 1) -> np.ndarray:
    """Seeded random CI matrices C[b, Ia, Ib] with C = C^T (singlet sector)."""
    rng = np.random.default_rng(seed)
    c = rng.standard_normal((batch, nstr, nstr))
    c = 0.5 * (c + np.swapaxes(c, 1, 2))
    return c


def sample_tuples(exp, order: int, count: int, seed: int):
    """Seeded sample of distinct sorted tuples of ``order`` expansion orbitals."""
    rng = np.random.default_rng(seed)
    exp = np.asarray(sorted(exp))
    seen, out = set(), []
    while len(out) < count:
        t = tuple(sorted(rng.choice(exp, size=order, replace=False).tolist()))
        if t not in seen:
            seen.add(t)
            out.append(t)
    return out

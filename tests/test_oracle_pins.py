"""Pins of the oracle against facts fixed by the paper and by mathematics.

None of these tests compares the oracle with itself: each checks it against
a closed form, a library routine on an independent formulation, a printed
count of the paper, or an exact identity.
"""
import itertools
import math
import os

import numpy as np
import pytest

import mbe_synth as ms
from oracle import casci as oc
from oracle import mbe as om

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def pack(eri_full, n):
    P = ms.npair(n)
    out = np.empty((P, P))
    pairs = [(p, q) for p in range(n) for q in range(p + 1)]
    for a, (p, q) in enumerate(pairs):
        for b, (r, s) in enumerate(pairs):
            out[a, b] = eri_full[p, q, r, s]
    return out


def two_orbital_system(h11, h22, J11, J22, J12, K12):
    h = np.diag([h11, h22]).astype(float)
    e = np.zeros((3, 3))          # pairs: (0,0)=0, (1,0)=1, (1,1)=2
    e[0, 0], e[2, 2] = J11, J22
    e[0, 2] = e[2, 0] = J12
    e[1, 1] = K12
    return h, e


@pytest.mark.parametrize("vals", [
    (-1.0, -0.3, 0.7, 0.6, 0.4, 0.15),   # closed-shell pair lowest
    (-1.0, -0.9, 1.0, 1.0, 0.2, 0.05),   # open-shell singlet lowest
])
def test_two_electron_closed_form(vals):
    """2 electrons in 2 orbitals with h12 = (11|12) = (22|12) = 0: the
    singlet energies are the lower eigenvalue of the closed-shell 2x2 block
    [[2h11+J11, K12], [K12, 2h22+J22]] and the open-shell singlet
    h11+h22+J12+K12 (Szabo & Ostlund, Sec. 4.1 and Exercise 4.x)."""
    h11, h22, J11, J22, J12, K12 = vals
    h, eri = two_orbital_system(*vals)
    a, b = 2 * h11 + J11, 2 * h22 + J22
    e_cs = 0.5 * (a + b) - math.sqrt(0.25 * (a - b) ** 2 + K12 ** 2)
    e_os = h11 + h22 + J12 + K12
    e = oc.casci(h, eri, 1, [0, 1])
    assert abs(e - min(e_cs, e_os)) < 1e-13


def test_two_electron_first_quantization():
    """2 electrons in n orbitals: the singlet spectrum of the Slater-Condon
    oracle equals numpy eigh of H in the first-quantised spatial basis
    (phi_p phi_q + phi_q phi_p)/norm, <pq|H|rs> = h_pr d_qs + d_pr h_qs + (pr|qs)."""
    n = 5
    h, eri, _ = ms.gen_integrals(n, 1, 11)
    G = ms.unpack_eri(eri, n)
    prod = np.zeros((n * n, n * n))
    I = np.eye(n)
    for p, q, r, s in itertools.product(range(n), repeat=4):
        prod[p * n + q, r * n + s] = h[p, r] * I[q, s] + I[p, r] * h[q, s] + G[p, r, q, s]
    basis = []
    for p in range(n):
        for q in range(p + 1):
            v = np.zeros(n * n)
            v[p * n + q] += 1.0
            v[q * n + p] += 1.0
            basis.append(v / np.linalg.norm(v))
    B = np.array(basis).T
    e_ref = np.linalg.eigvalsh(B.T @ prod @ B)[0]
    assert abs(oc.casci(h, eri, 1, range(n)) - e_ref) < 1e-12


def test_noninteracting_limit():
    """g = 0: eps_T = 2 sum_core h_ii + 2 sum of the lowest n_sigma eigenvalues
    of h restricted to the active orbitals (inactive core, deleted virtuals)."""
    n, nocc = 10, 4
    h, eri, _ = ms.gen_integrals(n, nocc, 5)
    act = [1, 3, 4, 6, 7, 9]
    core = [i for i in range(nocc) if i not in act]
    nsig = sum(1 for a in act if a < nocc)
    w = np.linalg.eigvalsh(h[np.ix_(act, act)])
    expect = 2 * sum(h[i, i] for i in core) + 2 * w[:nsig].sum()
    e = oc.casci(h, np.zeros_like(eri), nocc, act)
    assert abs(e - expect) < 1e-12


def test_hermitian_s2_and_spin_algebra():
    """H is symmetric; S^2 in the symmetric subspace has eigenvalues S(S+1)
    with even S only, commutes with H, and the C implementation agrees with
    an independent pure-Python S- S+ loop; the selected root is a singlet."""
    n, nocc = 6, 2
    h, eri, _ = ms.gen_integrals(n, nocc, 3)
    sp = oc.Space(h, eri, nocc, range(n))
    H = sp.hdense()
    assert np.abs(H - H.T).max() < 1e-13 * np.abs(H).max()
    S2 = np.array([sp.s2(col) for col in np.eye(sp.ndet)]).T
    assert np.abs(S2 - S2.T).max() < 1e-14
    P = sp.sym_basis()
    ev = np.linalg.eigvalsh(P.T @ S2 @ P)
    allowed = np.array([S * (S + 1) for S in (0, 2, 4)])
    assert np.abs(ev[:, None] - allowed[None, :]).min(axis=1).max() < 1e-10
    Hs = 0.5 * (H + H.T)
    assert np.abs(Hs @ S2 - S2 @ Hs).max() < 1e-11
    rng = np.random.default_rng(0)
    v = rng.standard_normal(sp.ndet)
    v /= np.linalg.norm(v)
    assert abs(v @ sp.s2(v) - oc.spin_square(sp, v)) < 1e-12
    e, c, _ = oc.casci(h, eri, nocc, range(n), want_vector=True)
    assert abs(oc.spin_square(sp, c)) < 1e-10
    # the singlet is an eigenvector of the symmetric H
    assert np.linalg.norm(Hs @ c - e * c) < 1e-10


def test_dense_equals_davidson():
    """Dense eigh (singlet selected by <S^2>) and the spin-shifted Davidson
    give the same energy and state on a 3136-determinant space."""
    w = ms.workload("h2o_dz_8e23o")
    h, eri, _ = ms.workload_integrals("h2o_dz_8e23o")
    act = sorted(set(w["ref"]) | {7, 8})
    e, c, sp = oc.casci(h, eri, w["nocc"], act, want_vector=True)
    ed, cd, _ = oc.davidson(sp)
    assert sp.ndet == 3136
    assert abs(e - ed) < 1e-11
    assert abs(abs(c @ cd) - 1.0) < 1e-10


def _rotate(h, eri, n, idx, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((len(idx), len(idx))))
    U = np.eye(n)
    U[np.ix_(idx, idx)] = Q
    G = ms.unpack_eri(eri, n)
    h2 = U.T @ h @ U
    G2 = np.einsum("pqrs,pa,qb,rc,sd->abcd", G, U, U, U, U, optimize=True)
    return h2, pack(G2, n)


@pytest.mark.parametrize("which", ["active", "core", "deleted"])
def test_rotation_invariance(which):
    """The CASCI energy is invariant under orthogonal rotations among the
    active orbitals, among the inactive core orbitals, and among the deleted
    virtuals (each block separately)."""
    n, nocc = 9, 3
    h, eri, _ = ms.gen_integrals(n, nocc, 8)
    act = [1, 2, 3, 4, 5]
    blocks = {"active": act, "core": [0, 6][:1] + [], "deleted": [6, 7, 8]}
    idx = blocks[which]
    if which == "core":
        act = [2, 3, 4, 5]       # core = {0, 1}
        idx = [0, 1]
    e0 = oc.casci(h, eri, nocc, act)
    h2, eri2 = _rotate(h, eri, n, idx, 1)
    assert abs(oc.casci(h2, eri2, nocc, act) - e0) < 1e-11


def _small_mbe(thr=0.0, max_order=None):
    n, nocc = 8, 3
    h, eri, _ = ms.gen_integrals(n, nocc, 21)
    ref = [2, 3]
    exp = [0, 1, 4, 5, 6, 7]
    res = om.run_mbe(h, eri, nocc, ref, exp, max_order or len(exp), thr)
    return h, eri, nocc, ref, exp, res


def test_allorder_unscreened_identity():
    """Unscreened and to all orders, eps_Pi + sum of all increments equals
    the FCI energy of the full space (Eqs. 1-3 telescope exactly)."""
    h, eri, nocc, ref, exp, res = _small_mbe()
    e_fci = oc.casci(h, eri, nocc, range(h.shape[0]))
    assert abs(res["total"] - e_fci) < 1e-11
    # ...and the last order holds exactly one tuple: the full space.
    assert len(res["orders"][-1]["tuples"]) == 1


def test_recursion_equals_mobius():
    """The recursion of Eq. 3 equals the closed-form inclusion-exclusion sum
    over all subtuples."""
    h, eri, nocc, ref, exp, res = _small_mbe()
    for t, d in res["inc"].items():
        assert abs(d - om.increment_mobius(t, res["eps"], res["eps_ref"])) < 1e-11


def test_tuple_counts_match_paper():
    """Enumeration and tuple -> CASCI(nel, norb) map reproduce the counts of
    Fig. 2 (cases a, c) and Table 2 (standard, orders 1-4)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "paper_tuple_counts.txt"))
            if l.strip() and not l.startswith("#")]
    for case, norb, nocc, ref, exp, order, count, nel_c, norb_c in rows:
        norb, nocc, order, count = int(norb), int(nocc), int(order), int(count)
        ref = [int(x) for x in ref.split(",")]
        exp = [int(x) for x in exp.split(",")]
        prev = {}
        for k in range(1, order + 1):
            tuples = om.next_order_tuples(exp, prev, 0.0, k)
            prev = {t: 1.0 for t in tuples}
        assert len(tuples) == count, (case, order)
        for t in tuples[:3]:
            act = om.active_space(ref, t)
            strs, nsig = oc.tuple_strings(nocc, act)
            assert (2 * nsig, len(act)) == (int(nel_c), int(norb_c)), (case, t)


def test_screening_rule_downward_closed():
    """A tuple is formed iff all its (k-1)-subtuples exist and at least one of
    them is at or above the threshold."""
    exp = [0, 1, 2, 3]
    prev = {(0, 1): 1e-3, (0, 2): 1e-9, (1, 2): 1e-9, (0, 3): 1e-9, (1, 3): 1e-9}
    got = om.next_order_tuples(exp, prev, 1e-6, 3)
    # (0,1,2): parents (0,1) kept -> in. (0,1,3): parents (0,1),(0,3),(1,3) -> in.
    # (0,2,3): parent (2,3) missing -> out. (1,2,3): (2,3) missing -> out.
    assert got == [(0, 1, 2), (0, 1, 3)]
    prev[(0, 1)] = 1e-9
    assert om.next_order_tuples(exp, prev, 1e-6, 3) == []
    assert om.next_order_tuples(exp, prev, 0.0, 3) == [(0, 1, 2), (0, 1, 3)]


def test_kahan_sum_matches_fsum():
    rng = np.random.default_rng(4)
    vals = list(rng.standard_normal(2000) * 10.0 ** rng.integers(-12, 4, 2000))
    assert abs(om.kahan_sum(vals) - math.fsum(vals)) <= 1e-15 * sum(abs(v) for v in vals)


def test_rdm_traces_and_energy():
    """tr gamma = N, sum_pq Gamma_ppqq = N(N-1), and
    E = sum h gamma + 1/2 sum (pq|rs) Gamma for the full-space RDMs
    (core included)."""
    n, nocc = 8, 3
    h, eri, _ = ms.gen_integrals(n, nocc, 13)
    act = [1, 2, 3, 4, 6]
    e, c, sp = oc.casci(h, eri, nocc, act, want_vector=True)
    g1, g2 = sp.rdm12(c)
    N = 2 * nocc
    assert abs(np.trace(g1) - N) < 1e-12
    assert abs(np.einsum("ppqq", g2) - N * (N - 1)) < 1e-11
    G = ms.unpack_eri(eri, n)
    assert abs(np.einsum("pq,pq", h, g1) + 0.5 * np.einsum("pqrs,pqrs", G, g2) - e) < 1e-11


def test_mbe_coefficients_allorder():
    """For the complete unscreened set the coefficients vanish except for the
    full tuple (c = 1), so the assembled RDMs are the full-space FCI RDMs."""
    exp = [0, 1, 2, 3]
    tuples = [t for k in range(1, 5) for t in itertools.combinations(exp, k)]
    coef = om.mbe_coefficients(tuples)
    for t, c in coef.items():
        assert c == (1 if t == (0, 1, 2, 3) else 0)


@pytest.mark.parametrize("nocc", [2, (3, 1)])
def test_gradient_central_fd(nocc):
    """Oracle Hellmann-Feynman gradient vs central finite differences of the
    whole MBE energy (step 1e-5) on random unique integrals; closed-shell and
    high-spin (triplet) references."""
    n = 6
    h, eri, _ = ms.gen_integrals(n, 2, 17)
    ref, exp = [1, 2], [0, 3, 4, 5]
    tuples = [t for k in range(1, 3) for t in itertools.combinations(exp, k)]
    dh, dg, _ = om.mbe_gradient(h, eri, nocc, ref, tuples)

    def energy(h_, e_):
        return om.run_mbe(h_, e_, nocc, ref, exp, 2, 0.0)["total"]

    rng = np.random.default_rng(3)
    step = 1e-5
    for _ in range(4):
        p, q = sorted(rng.integers(0, n, 2))
        hp, hm = h.copy(), h.copy()
        for M, s in ((hp, step), (hm, -step)):
            M[p, q] += s
            if p != q:
                M[q, p] += s
        fd = (energy(hp, eri) - energy(hm, eri)) / (2 * step)
        an = dh[p, q] * (1 if p == q else 2)
        assert abs(fd - an) <= 1e-6 * abs(an) + 1e-8
    P = ms.npair(n)
    for _ in range(4):
        a, b = sorted(rng.integers(0, P, 2))
        ep, em = eri.copy(), eri.copy()
        for M, s in ((ep, step), (em, -step)):
            M[a, b] += s
            if a != b:
                M[b, a] += s
        fd = (energy(h, ep) - energy(h, em)) / (2 * step)
        an = dg[a, b] * (1 if a == b else 2)
        assert abs(fd - an) <= 1e-6 * abs(an) + 1e-8


def test_sigma_rows_equals_dense_rows():
    """The oracle's sigma on a listed set of determinants equals the same
    rows of the dense Slater-Condon matrix times c (Sec. 2: the CASCI
    Hamiltonian of one tuple, inactive core and deleted virtuals included),
    and the full-vector sigma at those rows; a row index outside the space
    is rejected."""
    n, nocc = 7, 3
    h, eri, _ = ms.gen_integrals(n, nocc, 11)
    act = [1, 2, 3, 4, 6]                      # orbital 0 inactive, 5 deleted
    sp = oc.Space(h, eri, nocc, act)
    rng = np.random.default_rng(4)
    c = rng.standard_normal(sp.ndet)
    rows = rng.choice(sp.ndet, size=min(40, sp.ndet), replace=False)
    rows = np.concatenate([rows, [0, sp.ndet - 1]])
    H = sp.hdense()
    got = sp.sigma_rows(c, rows)
    assert np.abs(got - H[rows] @ c).max() < 1e-12 * max(1.0, np.abs(H).max())
    assert np.array_equal(got, sp.sigma(c)[rows])
    assert sp.sigma_rows(c, np.array([], dtype=np.int64)).size == 0
    with pytest.raises(ValueError):
        sp.sigma_rows(c, [sp.ndet])


def _pruned_counts(nsingle, npairs, max_order):
    """Unscreened tuple counts of a pi-pruned expansion (tuple enumeration of
    the oracle, no energies needed)."""
    exp = list(range(nsingle + 2 * npairs))
    pairs = [(nsingle + 2 * i, nsingle + 2 * i + 1) for i in range(npairs)]
    formed, counts = {}, []
    for k in range(1, max_order + 1):
        t = om.next_order_tuples_pruned(exp, pairs, formed, 0.0, k)
        formed.update({x: 1.0 for x in t})
        counts.append(len(t))
    return counts


def test_pi_pruned_counts_match_paper():
    """Table 2 (pi-pruned columns): 6, 21, 56, 120, 216 tuples at orders 1-5
    for 6 single orbitals and 6 degenerate pairs; the same counts follow from
    the closed form sum_j C(6, k - 2j) C(6, j)."""
    gold = {}
    with open(os.path.join(GOLDEN, "paper_pi_pruned_counts.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, c = line.split()
                gold[int(k)] = int(c)
    counts = _pruned_counts(6, 6, max(gold))
    assert {k: counts[k - 1] for k in gold} == gold
    closed = [sum(math.comb(6, k - 2 * j) * math.comb(6, j) for j in range(k // 2 + 1)
                  if k - 2 * j >= 0) for k in range(1, max(gold) + 1)]
    assert counts == closed


def test_pi_pruned_allorder_equals_fci_and_mobius():
    """Unscreened and to all orders the pruned expansion (units: single
    orbitals and degenerate pairs) sums to the FCI energy of the whole space;
    every increment equals its Moebius form over the unit lattice; without
    pairs the pruned bookkeeping reproduces the standard expansion."""
    n, nocc = 9, 3
    h, eri, _ = ms.gen_integrals(n, nocc, 5)
    ref, exp, pairs = [1, 2], [0, 3, 4, 5, 6, 7, 8], [(3, 4), (6, 8)]
    res = om.run_mbe(h, eri, nocc, ref, exp, 7, 0.0, pairs=pairs)
    assert abs(res["total"] - oc.casci(h, eri, nocc, list(range(n)))) < 1e-10
    # no tuple splits a pair; order 2 holds the two pairs alone
    for o in res["orders"]:
        for t in o["tuples"]:
            for a, b in pairs:
                assert (a in t) == (b in t)
    assert (3, 4) in res["orders"][1]["tuples"] and (6, 8) in res["orders"][1]["tuples"]
    units = om.expansion_units(exp, pairs)
    for t, d in res["inc"].items():
        assert abs(d - om.increment_mobius_units(t, res["eps"], res["eps_ref"], units)) < 1e-10
    # E = sum_S c_S eps_S with coefficients that count units
    coef = om.mbe_coefficients(list(res["inc"].keys()), units)
    e = coef[()] * res["eps_ref"] + sum(c * res["eps"][s] for s, c in coef.items() if s)
    assert abs(e - res["total"]) < 1e-10
    # without pairs every unit is one orbital: the unit enumeration gives the
    # standard tuples of the screened expansion order by order
    std = om.run_mbe(h, eri, nocc, ref, exp, 4, 1e-3)
    formed = {}
    for k, o in enumerate(std["orders"], start=1):
        assert om.next_order_tuples_pruned(exp, [], formed, 1e-3, k) == o["tuples"]
        formed.update(dict(zip(o["tuples"], o["inc"])))


# ---------------------------------------------------------------- open shell
# High-spin references (Fig. 2 case (b)): nocc = (n_alpha, n_beta).

@pytest.mark.parametrize("seed,norb,nocc,act", [
    (3, 6, (3, 1), list(range(6))),
    (7, 7, (4, 2), [1, 2, 3, 4, 5, 6]),      # orbital 0: inactive core
    (11, 7, (4, 1), list(range(7))),          # quartet (Ms = 3/2)
])
def test_open_shell_energy_is_ms0_spin_eigenvalue(seed, norb, nocc, act):
    """The lowest S = Ms state of the Ms = (na - nb)/2 space is an eigenvalue
    of the same Hamiltonian in the Ms = 0 (or 1/2) space of the same electron
    count: dense diagonalisation of the whole lower-Ms space (no symmetry
    restriction), the lowest eigenvalue whose <S^2> is S(S+1)."""
    na, nb = nocc
    h, eri, _ = ms.gen_integrals(norb, nb, seed)
    e_hs = oc.casci(h, eri, nocc, act)
    ntot = na + nb
    lo = (ntot // 2 + ntot % 2, ntot // 2)
    sp = oc.Space(h, eri, lo, act)
    H = sp.hdense()
    w, U = np.linalg.eigh(0.5 * (H + H.T))
    S = 0.5 * (na - nb)
    for k in range(len(w)):
        c = U[:, k]
        if abs(c @ sp.s2(c) - S * (S + 1)) < 1e-6:
            assert abs(w[k] - e_hs) < 1e-10
            break
    else:
        raise AssertionError("no S = Ms state in the lower-Ms space")


def test_open_shell_single_determinant_closed_forms():
    """Spaces of one determinant: the energy is the textbook sum over the
    occupied spin-orbitals, h_ii once per electron, Coulomb for every pair,
    exchange only between equal spins."""
    n = 5
    h, eri, _ = ms.gen_integrals(n, 1, 17)
    G = ms.unpack_eri(eri, n)
    J = lambda p, q: G[p, p, q, q]
    K = lambda p, q: G[p, q, q, p]
    # alpha {0, 1, 2}, beta {0}: core orbital 0, act {1, 2} singly occupied
    e = oc.casci(h, eri, (3, 1), [1, 2])
    ref = (2 * h[0, 0] + h[1, 1] + h[2, 2] + J(0, 0) + 2 * J(0, 1) - K(0, 1)
           + 2 * J(0, 2) - K(0, 2) + J(1, 2) - K(1, 2))
    assert abs(e - ref) < 1e-12
    # doublet: alpha {0, 1}, beta {0}
    e = oc.casci(h, eri, (2, 1), [1])
    assert abs(e - (2 * h[0, 0] + h[1, 1] + J(0, 0) + 2 * J(0, 1) - K(0, 1))) < 1e-12
    # two alpha electrons in orbitals 0 and 1, no beta electron
    e = oc.casci(h, eri, (2, 0), [0, 1])
    assert abs(e - (h[0, 0] + h[1, 1] + J(0, 1) - K(0, 1))) < 1e-12


def test_open_shell_rdm_energy_and_traces():
    """tr gamma = N, sum Gamma_ppqq = N(N-1), E = h.gamma + 1/2 (pq|rs).Gamma
    for a high-spin CASCI with an inactive core."""
    n, nocc = 7, (4, 2)
    h, eri, _ = ms.gen_integrals(n, 2, 23)
    e, c, sp = oc.casci(h, eri, nocc, [1, 2, 3, 4, 6], want_vector=True)
    g1, g2 = sp.rdm12(c)
    N = 6
    assert abs(np.trace(g1) - N) < 1e-12
    assert abs(np.einsum("ppqq", g2) - N * (N - 1)) < 1e-11
    G = ms.unpack_eri(eri, n)
    assert abs(np.einsum("pq,pq", h, g1) + 0.5 * np.einsum("pqrs,pqrs", G, g2) - e) < 1e-11
    assert abs(c @ sp.s2(c) - 2.0) < 1e-8


def test_open_shell_allorder_mbe_is_fci():
    """Unscreened to all orders the expansion around a high-spin CAS
    reference telescopes to the CASCI of the whole space (Eq. 3)."""
    n, nocc = 7, (3, 1)
    h, eri, _ = ms.gen_integrals(n, 1, 29)
    ref, exp = [1, 2], [0, 3, 4, 5, 6]
    res = om.run_mbe(h, eri, nocc, ref, exp, len(exp))
    assert abs(res["total"] - oc.casci(h, eri, nocc, list(range(n)))) < 1e-10

"""Energy backward on the GPU (mbe_energy_backward) against the oracle.

dE/dh and dE/d eri_packed of the whole MBE energy: the MBE-weighted sum of
the tuples' full-space RDMs (Hellmann-Feynman).  Pinned three ways: against
the oracle's gradient, against the full-space FCI RDMs for the complete
unscreened expansion, and against central finite differences of the GPU's
own energies.  Tolerance 1e-9 (FP64 path; RDM elements are O(1)).  RDMs are
first order in the CI-vector error (energies are second order), so the
backward runs converge the Davidson residual to 1e-11 (vector error
~1e-11 / gap) instead of the default 1e-8.
"""
import itertools

import numpy as np
import pytest

import mbe_synth as ms
from oracle import casci as oc
from oracle import mbe as om

pytestmark = pytest.mark.gpu

TOL = 1e-9
TIGHT = dict(conv_tol_r=1e-11, conv_tol_e=1e-14)


@pytest.fixture(scope="module")
def lib():
    from paper_1905_02786_gb300 import build, _binding
    build.build()
    _binding.load_library()
    return _binding


def gpu_grad(lib, h, eri, nocc, ref, exp, max_order, thr, **opts):
    m = lib.MBE(0, keep_ci=1, **{**TIGHT, **opts})
    m.load(h, eri, 2 * nocc)
    res = m.run(ref, exp, max_order, thr)
    dh, dg = m.backward()
    m.close()
    return res, dh, dg


def processed_tuples(res):
    return [tuple(int(x) for x in t) for o in res["orders"] for t in o["tuples"]]


@pytest.mark.parametrize("case", [
    # norb, nocc, seed, ref, exp, max_order, thr
    (10, 3, 5, [2, 3], [0, 1, 4, 5, 6, 7, 8, 9], 3, 0.0),
    (10, 3, 5, [2, 3], [0, 1, 4, 5, 6, 7, 8, 9], 4, 3e-4),    # screened set
    (9, 4, 2, [3, 4, 5], [0, 1, 2, 6, 7, 8], 3, 0.0),
    (7, 2, 3, [], list(range(7)), 2, 0.0),                    # empty reference
])
def test_backward_matches_oracle(lib, case):
    norb, nocc, seed, ref, exp, max_order, thr = case
    h, eri, _ = ms.gen_integrals(norb, nocc, seed)
    res, dh, dg = gpu_grad(lib, h, eri, nocc, ref, exp, max_order, thr)
    tuples = processed_tuples(res)
    ores = om.run_mbe(h, eri, nocc, ref, exp, max_order, thr)
    assert sorted(tuples) == sorted(ores["inc"].keys())
    odh, odg, _ = om.mbe_gradient(h, eri, nocc, ref, tuples)
    assert np.max(np.abs(dh - odh)) < TOL
    assert np.max(np.abs(dg - odg)) < TOL
    assert np.allclose(dh, dh.T, atol=0) and np.allclose(dg, dg.T, atol=0)


def test_allorder_gradient_is_fci_rdm(lib):
    """Complete unscreened expansion: all coefficients vanish but the full
    tuple's, so the gradient is the full-space FCI RDM pair."""
    n, nocc = 8, 3
    h, eri, _ = ms.gen_integrals(n, nocc, 21)
    ref, exp = [2, 3], [0, 1, 4, 5, 6, 7]
    res, dh, dg = gpu_grad(lib, h, eri, nocc, ref, exp, len(exp), 0.0)
    e, c, sp = oc.casci(h, eri, nocc, range(n), want_vector=True)
    g1, g2 = sp.rdm12(c)
    assert abs(res["total"] - e) < 1e-10
    assert np.max(np.abs(dh - g1)) < TOL
    assert np.max(np.abs(dg - om.pack_eri_gradient(0.5 * g2, n))) < TOL
    # trace of the one-particle density: the electron number
    assert abs(np.trace(dh) - 2 * nocc) < 1e-10


def test_backward_central_fd(lib):
    """Directional derivative of the GPU energy (central differences, step
    1e-6 along a random symmetric direction with O(1) entries in every h and
    eri element) equals <grad, direction>."""
    n, nocc = 9, 3
    h, eri, _ = ms.gen_integrals(n, nocc, 7)
    ref, exp = [2, 3], [0, 1, 4, 5, 6, 7, 8]
    _, dh, dg = gpu_grad(lib, h, eri, nocc, ref, exp, 3, 0.0)
    rng = np.random.default_rng(11)
    vh = rng.standard_normal(h.shape)
    vh = 0.5 * (vh + vh.T)
    ve = rng.standard_normal(eri.shape)
    ve = 0.5 * (ve + ve.T)
    an = np.sum(dh * vh) + np.sum(dg * ve)

    def energy(t):
        m = lib.MBE(0)
        m.load(h + t * vh, eri + t * ve, 2 * nocc)
        e = m.run(ref, exp, 3, 0.0)["total"]
        m.close()
        return e

    step = 1e-6
    fd = (energy(step) - energy(-step)) / (2 * step)
    assert abs(fd - an) <= 1e-6 * abs(an) + 1e-8


def test_backward_sharded_contexts_sum(lib):
    """Tuples of each order split over two contexts (as over two GPUs): the
    shares (reference term on one of them) sum to the single-context
    gradient; a context asked for the whole gradient without holding every
    CI vector refuses."""
    n, nocc = 9, 3
    h, eri, _ = ms.gen_integrals(n, nocc, 4)
    ref, exp = [2, 3], [0, 1, 4, 5, 6, 7, 8]
    _, dh, dg = gpu_grad(lib, h, eri, nocc, ref, exp, 3, 1e-4)
    ctxs = [lib.MBE(0, keep_ci=1, backward_share=2, **TIGHT),
            lib.MBE(0, keep_ci=1, backward_share=1, **TIGHT)]
    for m in ctxs:
        m.load(h, eri, 2 * nocc)
        lib.mbe_set_reference(m.ctx, ref, exp)
    for k in range(1, 4):
        tuples = lib.mbe_next_tuples(ctxs[0].ctx, k)
        if len(tuples) == 0:
            break
        eps = np.zeros(len(tuples))
        for r, m in enumerate(ctxs):
            idx = np.arange(r, len(tuples), 2)
            if len(idx):
                eps[idx], _ = lib.mbe_solve_tuples(m.ctx, tuples[idx], k)
        for m in ctxs:
            lib.mbe_set_order_energies(m.ctx, tuples, eps, k)
            lib.mbe_increments(m.ctx, k, 1e-4, len(tuples))
    parts = [m.backward() for m in ctxs]
    assert np.max(np.abs(parts[0][0] + parts[1][0] - dh)) < TOL
    assert np.max(np.abs(parts[0][1] + parts[1][1] - dg)) < TOL
    whole = lib.MBE(0, keep_ci=1, backward_share=0)
    whole.load(h, eri, 2 * nocc)
    lib.mbe_set_reference(whole.ctx, ref, exp)
    t1 = lib.mbe_next_tuples(whole.ctx, 1)
    lib.mbe_set_order_energies(whole.ctx, t1, np.full(len(t1), -1.0), 1)
    lib.mbe_increments(whole.ctx, 1, 0.0, len(t1))
    with pytest.raises(lib.MBEError):
        whole.backward()
    for m in ctxs + [whole]:
        m.close()


def test_backward_needs_keep_ci(lib):
    n, nocc = 6, 2
    h, eri, _ = ms.gen_integrals(n, nocc, 1)
    m = lib.MBE(0)
    m.load(h, eri, 2 * nocc)
    m.run([1, 2], [0, 3, 4, 5], 2, 0.0)
    with pytest.raises(lib.MBEError):
        m.backward()
    m.close()


def test_autograd_function(lib):
    torch = pytest.importorskip("torch")
    from paper_1905_02786_gb300.autograd import mbe_energy
    n, nocc = 8, 3
    h, eri, _ = ms.gen_integrals(n, nocc, 9)
    ref, exp = [2, 3], [0, 1, 4, 5, 6, 7]
    ht = torch.tensor(h, requires_grad=True)
    et = torch.tensor(eri, requires_grad=True)
    e = mbe_energy(ht, et, 2 * nocc, ref, exp, 3, **TIGHT)
    (2.0 * e).backward()
    tuples = [t for k in range(1, 4) for t in itertools.combinations(exp, k)]
    odh, odg, _ = om.mbe_gradient(h, eri, nocc, ref, tuples)
    assert abs(e.item() - om.run_mbe(h, eri, nocc, ref, exp, 3, 0.0)["total"]) < 1e-10
    assert np.max(np.abs(ht.grad.numpy() - 2.0 * odh)) < 2 * TOL
    assert np.max(np.abs(et.grad.numpy() - 2.0 * odg)) < 2 * TOL


def test_grad_workload_fd_sample(lib):
    """8e/20o, CAS(4e,4o) reference over orbitals 2-5, unscreened to order 4
    (2,516 tuples): central differences (step 1e-5) of the GPU energy on a
    seeded sample of unique integrals, and the trace invariant
    tr dE/dh = N_el (the MBE coefficients sum to one).

    Tolerance 1e-6 |g| + 2e-7: the MBE weights the tuple energies with
    coefficients up to 1,365 (the reference space) and 364 (order-1 tuples)
    here, so FP64 rounding of
    ~1e-15 relative in the ~2,500 tuple energies leaves ~1e-12 Eh of noise in
    each total energy, i.e. ~1e-7 in a difference quotient with step 1e-5."""
    w = ms.workload("grad_8e20o")
    h, eri, _ = ms.workload_integrals("grad_8e20o")
    nocc, n = w["nocc"], w["norb"]
    _, dh, dg = gpu_grad(lib, h, eri, nocc, w["ref"], w["exp"], w["max_order"], 0.0)
    assert abs(np.trace(dh) - w["nel"]) < 1e-9

    def energy(h_, e_):
        m = lib.MBE(0)
        m.load(h_, e_, w["nel"])
        e = m.run(w["ref"], w["exp"], w["max_order"], 0.0)["total"]
        m.close()
        return e

    rng = np.random.default_rng(3)
    step = 1e-5
    for _ in range(3):
        p, q = sorted(rng.integers(0, n, 2))
        hp, hm = h.copy(), h.copy()
        for M, s in ((hp, step), (hm, -step)):
            M[p, q] += s
            if p != q:
                M[q, p] += s
        fd = (energy(hp, eri) - energy(hm, eri)) / (2 * step)
        an = dh[p, q] * (1 if p == q else 2)
        assert abs(fd - an) <= 1e-6 * abs(an) + 2e-7, (p, q, fd, an)
    P = ms.npair(n)
    for _ in range(3):
        a, b = sorted(rng.integers(0, P, 2))
        ep, em = eri.copy(), eri.copy()
        for M, s in ((ep, step), (em, -step)):
            M[a, b] += s
            if a != b:
                M[b, a] += s
        fd = (energy(h, ep) - energy(h, em)) / (2 * step)
        an = dg[a, b] * (1 if a == b else 2)
        assert abs(fd - an) <= 1e-6 * abs(an) + 2e-7, (a, b, fd, an)


def test_backward_mixed_path_matches_oracle(lib):
    """The backward of the mixed-precision path (the production workload asks
    for it there).  Its RDMs come from the FP32 exact-point vectors, converged
    to the mixed path's relative residual (mixed_rel_tol, 2e-7); an RDM is
    first order in the vector error (residual / gap), so each CASCI carries
    ~1e-6 relative error, and the MBE coefficients of an order-3 expansion over
    8 orbitals (|c_T| up to 35) add those of ~100 CASCIs.  Bound: 2e-5 of the
    largest gradient entry (measured 6e-6 and 7e-6 of it; the FP64 path meets
    1e-9 absolute)."""
    norb, nocc, seed = 10, 3, 5
    ref, exp = [2, 3], [0, 1, 4, 5, 6, 7, 8, 9]
    h, eri, _ = ms.gen_integrals(norb, nocc, seed)
    m = lib.MBE(0, keep_ci=1, precision=lib.MBE_MIXED_BF16X3)
    m.load(h, eri, 2 * nocc)
    res = m.run(ref, exp, 3, 0.0)
    dh, dg = m.backward()
    m.close()
    odh, odg, _ = om.mbe_gradient(h, eri, nocc, ref, processed_tuples(res))
    eh, eg = np.abs(dh - odh).max(), np.abs(dg - odg).max()
    mh, mg = np.abs(odh).max(), np.abs(odg).max()
    print(f"\n[parity] mixed-path backward: max |dE/dh - oracle| = {eh:.3e} "
          f"({eh / mh:.2e} of the largest entry {mh:.2f}), max |dE/d(pq|rs) - oracle| = "
          f"{eg:.3e} ({eg / mg:.2e} of {mg:.2f})")
    assert eh < 2e-5 * mh and eg < 2e-5 * mg, (eh, eg, mh, mg)

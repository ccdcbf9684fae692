"""GPU parity of high-spin open-shell references (Fig. 2 case (b)) against
the oracle, through the C ABI.

A reference determinant with n_alpha > n_beta (mbe_set_spin): orbitals below
n_beta doubly occupied, n_beta .. n_alpha - 1 singly occupied and part of the
reference space.  Every CASCI is solved for its lowest S = Ms state in the
Ms = (n_alpha - n_beta) / 2 determinant space.  Tolerances as for the closed
shell: sigma 1e-11 of the largest element, energies and increments 1e-10 Eh,
gradient 1e-9.
"""
import itertools

import numpy as np
import pytest

import mbe_synth as ms
from oracle import casci as oc
from oracle import mbe as om

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10
TIGHT = dict(conv_tol_r=1e-11, conv_tol_e=1e-14)


@pytest.fixture(scope="module")
def lib():
    from paper_1905_02786_gb300 import build, _binding
    build.build()
    _binding.load_library()
    return _binding


def string_signs(strs, core, act):
    """+-1 per string: parity of the (active electron, core orbital) pairs
    with the active orbital below the core orbital (the oracle interleaves
    core and active creation operators in ascending order; the CUDA path
    keeps core operators in front)."""
    out = []
    for lo, hi in strs:
        m = int(lo) | (int(hi) << 64)
        cnt = sum(1 for p in act if (m >> p) & 1 for c in core if p < c)
        out.append(-1.0 if cnt % 2 else 1.0)
    return np.array(out)


def core_signs(sp, nb, act):
    core = [i for i in range(nb) if i not in act]
    return np.outer(string_signs(sp.astrs, core, act), string_signs(sp.bstrs, core, act)).ravel()


def make(lib, h, eri, nocc, **opts):
    na, nb = nocc
    m = lib.MBE(0, **opts)
    m.load(h, eri, na + nb, two_sz=na - nb)
    return m


SIGMA_CASES = [
    # norb, (n_alpha, n_beta), seed, active orbitals
    (6, (3, 1), 3, [0, 1, 2, 3, 4, 5]),             # triplet, no core
    (7, (4, 2), 7, [1, 2, 3, 4, 5, 6]),             # triplet, core orbital 0
    (8, (4, 3), 9, [1, 2, 3, 5, 6, 7]),             # doublet, core 0, deleted 4
    (9, (5, 2), 11, [0, 2, 3, 4, 6, 8]),            # quartet, core 1 between actives
    (12, (5, 3), 13, list(range(1, 12))),           # 330 x 55 strings, ragged tiles
]


@pytest.mark.parametrize("case", SIGMA_CASES)
@pytest.mark.parametrize("shift", [0.0, 0.5])
def test_open_shell_sigma_elementwise(lib, case, shift):
    """(H_active + shift S^2) c on a random (non-symmetric) vector of the
    n_alpha x n_beta string space, element by element against the oracle's
    Slater-Condon sigma plus shift times its S^2 = S-S+ + Ms(Ms+1)."""
    norb, nocc, seed, act = case
    na, nb = nocc
    h, eri, _ = ms.gen_integrals(norb, nb, seed)
    sp = oc.Space(h, eri, nocc, act)
    m = make(lib, h, eri, nocc, spin_shift=shift)
    rng = np.random.default_rng(seed)
    c = rng.standard_normal((sp.nstr, sp.nstrb))
    sig, ecore = lib.mbe_sigma(m.ctx, act, c)
    m.close()
    S = core_signs(sp, nb, act)
    cs = S * c.ravel()
    ref = S * (sp.sigma(cs) + shift * sp.s2(cs) - ecore * cs)
    scale = max(1.0, np.abs(ref).max())
    assert sig.shape == ref.shape
    assert np.abs(sig - ref).max() <= 1e-11 * scale


def test_open_shell_casci_energies(lib):
    """Reference and tuple CASCIs of orders 1-3 (triplet, core orbital 0)."""
    norb, nocc = 9, (4, 2)
    h, eri, _ = ms.gen_integrals(norb, 2, 21)
    ref, exp = [1, 2, 3], [0, 4, 5, 6, 7, 8]
    m = make(lib, h, eri, nocc)
    e_ref = lib.mbe_set_reference(m.ctx, ref, exp)
    assert abs(e_ref - oc.casci(h, eri, nocc, ref)) < TOL_FP64
    for k, tk in ((1, [(0,), (4,), (8,)]), (2, [(0, 4), (5, 8), (6, 7)]),
                  (3, [(0, 4, 5), (4, 6, 8)])):
        eps, st = lib.mbe_solve_tuples(m.ctx, np.array(tk), k)
        assert np.all(st == 0)
        for t, e in zip(tk, eps):
            e_or = oc.casci(h, eri, nocc, om.active_space(ref, t))
            assert abs(e - e_or) < TOL_FP64, (t, e, e_or)
    m.close()


def _cmp_expansion(res, ores, tol):
    assert abs(res["eps_ref"] - ores["eps_ref"]) < tol
    assert len(res["orders"]) == len(ores["orders"])
    for g, o in zip(res["orders"], ores["orders"]):
        assert [tuple(int(x) for x in t) for t in g["tuples"]] == o["tuples"]
        if o["tuples"]:
            assert np.abs(g["inc"] - np.array(o["inc"])).max() < tol
            assert list(g["keep"]) == o["keep"]
        assert abs(g["E_order"] - o["E_order"]) < tol
    assert abs(res["total"] - ores["total"]) < tol


@pytest.mark.parametrize("thr", [0.0, 1e-4])
def test_open_shell_expansion_vs_oracle(lib, thr):
    """Expansion around a high-spin CAS reference (Eq. 3 with a non-zero
    order-0 correlation energy): tuple sets, increments, keep flags and order
    sums equal to the oracle's; unscreened it reaches the whole-space CASCI."""
    norb, nocc = 9, (4, 2)
    h, eri, _ = ms.gen_integrals(norb, 2, 33, eps_vir=(0.05, 3.0))
    ref, exp = [1, 2, 3], [0, 4, 5, 6, 7, 8]
    max_order = len(exp) if thr == 0.0 else 4
    ores = om.run_mbe(h, eri, nocc, ref, exp, max_order, thr)
    m = make(lib, h, eri, nocc)
    res = m.run(ref, exp, max_order, thr)
    m.close()
    _cmp_expansion(res, ores, TOL_FP64)
    if thr == 0.0:
        assert abs(res["total"] - oc.casci(h, eri, nocc, list(range(norb)))) < 1e-9


def test_open_shell_mixed_mode_runs_fp64_grade(lib):
    """The mixed mode sends open-shell spaces through the FP64 Davidson with
    the FP64-grade emulated contraction: FP64 tolerances hold."""
    norb, nocc = 8, (3, 1)
    h, eri, _ = ms.gen_integrals(norb, 1, 41)
    ref, exp = [1, 2], [0, 3, 4, 5, 6, 7]
    ores = om.run_mbe(h, eri, nocc, ref, exp, 3, 0.0)
    m = make(lib, h, eri, nocc, precision=lib.MBE_MIXED_BF16X3)
    res = m.run(ref, exp, 3, 0.0)
    m.close()
    _cmp_expansion(res, ores, 1e-9)


def test_open_shell_backward_vs_oracle(lib):
    """Energy gradient of an open-shell expansion (RDMs over separate alpha
    and beta strings, closed-shell inactive core) against the oracle's."""
    norb, nocc = 8, (4, 2)
    h, eri, _ = ms.gen_integrals(norb, 2, 43)
    ref, exp = [1, 2, 3], [0, 4, 5, 6, 7]
    m = make(lib, h, eri, nocc, keep_ci=1, **TIGHT)
    res = m.run(ref, exp, 3, 0.0)
    dh, dg = m.backward()
    m.close()
    tuples = [tuple(int(x) for x in t) for o in res["orders"] for t in o["tuples"]]
    odh, odg, _ = om.mbe_gradient(h, eri, nocc, ref, tuples)
    assert abs(np.trace(dh) - np.trace(odh)) < 1e-9
    assert np.abs(dh - odh).max() < 1e-9
    assert np.abs(dg - odg).max() < 1e-9


def test_odd_electron_count_defaults_to_doublet(lib):
    """nelec odd with no mbe_set_spin: the doublet reference (n_alpha =
    n_beta + 1), the singly occupied orbital in the reference space."""
    norb = 7
    h, eri, _ = ms.gen_integrals(norb, 2, 47)
    m = lib.MBE(0)
    m.load(h, eri, 5)
    ref, exp = [1, 2], [0, 3, 4, 5, 6]
    e_ref = lib.mbe_set_reference(m.ctx, ref, exp)
    assert abs(e_ref - oc.casci(h, eri, (3, 2), ref)) < TOL_FP64
    eps, st = lib.mbe_solve_tuples(m.ctx, np.array([[0, 4], [3, 6]]), 2)
    for t, e in zip([(0, 4), (3, 6)], eps):
        assert abs(e - oc.casci(h, eri, (3, 2), om.active_space(ref, t))) < TOL_FP64
    m.close()


def test_open_shell_errors(lib):
    h, eri, _ = ms.gen_integrals(7, 2, 49)
    m = lib.MBE(0)
    with pytest.raises(lib.MBEError) as ei:
        lib.mbe_set_spin(m.ctx, 2)                     # before the integrals
    assert ei.value.code == lib.MBE_ESTATE
    m.load(h, eri, 6)
    for bad in (-2, 1, 8):                            # sign, parity, beyond nelec
        with pytest.raises(lib.MBEError) as ei:
            lib.mbe_set_spin(m.ctx, bad)
        assert ei.value.code == lib.MBE_EINVAL
    lib.mbe_set_spin(m.ctx, 2)                        # n_alpha 4, n_beta 2
    with pytest.raises(lib.MBEError) as ei:           # orbital 3 singly occupied
        lib.mbe_set_reference(m.ctx, [1, 2], [0, 3, 4, 5, 6])
    assert ei.value.code == lib.MBE_EINVAL
    with pytest.raises(lib.MBEError) as ei:           # mbe_sigma without orbital 2
        lib.mbe_sigma(m.ctx, [1, 3, 4], np.zeros(1))
    assert ei.value.code == lib.MBE_EINVAL
    lib.mbe_set_reference(m.ctx, [2, 3], [0, 1, 4, 5, 6])
    lib.mbe_set_spin(m.ctx, 0)                        # back to the closed shell
    e0 = lib.mbe_set_reference(m.ctx, [1, 2], [0, 3, 4, 5, 6])
    assert abs(e0 - oc.casci(h, eri, 3, [1, 2])) < TOL_FP64
    m.close()

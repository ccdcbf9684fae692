"""GPU parity of the CUDA path (through the C ABI) against the oracle.

Tolerances: FP64 path 1e-10 Eh per energy / increment; sigma vectors
element by element to 1e-11 relative to the largest element.
"""
import itertools
import os

import numpy as np
import pytest

import mbe_synth as ms
from oracle import casci as oc
from oracle import mbe as om

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TOL_FP64 = 1e-10


@pytest.fixture(scope="module")
def lib():
    from paper_1905_02786_gb300 import build, _binding
    build.build()
    _binding.load_library()
    return _binding


def make(lib, **opts):
    return lib.MBE(0, **opts)


def core_signs(sp, nocc, act):
    """+-1 per determinant relating the oracle's full-space determinants
    (creation operators of core and active orbitals interleaved in ascending
    order) to active-space strings (core operators moved to the front): the
    parity of the number of (active electron, core orbital) pairs with the
    active orbital below the core orbital, for each spin string."""
    core = [i for i in range(nocc) if i not in act]
    s = []
    for lo, hi in sp.strs:
        m = int(lo) | (int(hi) << 64)
        cnt = sum(1 for p in act if (m >> p) & 1 for c in core if p < c)
        s.append(-1.0 if cnt % 2 else 1.0)
    s = np.array(s)
    return np.outer(s, s).ravel()


@pytest.mark.parametrize("case", [
    # (norb, nocc, seed, act) -- core orbitals and deleted virtuals included
    (8, 3, 1, [0, 1, 2, 3, 4, 5]),
    (10, 4, 2, [1, 3, 4, 5, 7, 8, 9]),
    (12, 4, 0, [0, 1, 2, 3, 4, 5, 6, 7, 8]),     # several tiles, ragged tail
    (9, 4, 3, [0, 1, 2, 3]),                      # all active orbitals occupied
    (9, 3, 4, [5, 6, 7]),                         # no active electrons
])
@pytest.mark.parametrize("shift", [0.0, 0.5])
def test_sigma_elementwise(lib, case, shift):
    norb, nocc, seed, act = case
    h, eri, _ = ms.gen_integrals(norb, nocc, seed)
    sp = oc.Space(h, eri, nocc, act)
    m = make(lib, spin_shift=shift)
    m.load(h, eri, 2 * nocc)
    rng = np.random.default_rng(seed)
    for sym in (True, False):
        c = rng.standard_normal((sp.nstr, sp.nstr))
        if sym:
            c = 0.5 * (c + c.T)
        sig, ecore = lib.mbe_sigma(m.ctx, act, c)
        S = core_signs(sp, nocc, act)
        cs = S * c.ravel()
        ref = S * (sp.sigma(cs) + shift * sp.s2(cs) - ecore * cs)
        scale = max(1.0, np.abs(ref).max())
        assert np.abs(sig - ref).max() <= 1e-11 * scale
    m.close()


def test_casci_energies_vs_oracle(lib):
    w = ms.workload("h2o_dz_8e23o")
    h, eri, _ = ms.workload_integrals("h2o_dz_8e23o")
    tuples = [(0,), (7,), (22,), (0, 7), (8, 9), (0, 7, 8), (9, 10, 11)]
    m = make(lib)
    m.load(h, eri, w["nel"])
    e_ref = lib.mbe_set_reference(m.ctx, w["ref"], w["exp"])
    assert abs(e_ref - oc.casci(h, eri, w["nocc"], w["ref"])) < TOL_FP64
    for k in (1, 2, 3):
        tk = [t for t in tuples if len(t) == k]
        eps, st = lib.mbe_solve_tuples(m.ctx, np.array(tk), k)
        assert np.all(st == 0)
        for t, e in zip(tk, eps):
            e_or = oc.casci(h, eri, w["nocc"], om.active_space(w["ref"], t))
            assert abs(e - e_or) < TOL_FP64, (t, e, e_or)
    m.close()


def _golden(name):
    rows = {}
    for line in open(os.path.join(GOLDEN, name + ".txt")):
        if line.startswith("#"):
            if "total MBE energy" in line:
                total = float(line.split()[-1])
            continue
        k, t, e = line.split()
        rows[() if t == "-" else tuple(int(x) for x in t.split(","))] = float(e)
    return rows, total


def test_allorder_fci8e12o_matches_golden(lib):
    """All 255 tuples + reference of the 8e/12o expansion, per-tuple energies
    against the stored oracle values, and the total against the full FCI."""
    name = "fci8e12o_allorder"
    w = ms.workload(name)
    h, eri, _ = ms.workload_integrals(name)
    gold, total = _golden(name)
    m = make(lib)
    m.load(h, eri, w["nel"])
    res = m.run(w["ref"], w["exp"], w["max_order"], 0.0)
    assert abs(res["eps_ref"] - gold[()]) < TOL_FP64
    n = 0
    for o in res["orders"]:
        assert np.all(o["status"] == 0)
        for t, e in zip(o["tuples"], o["eps"]):
            assert abs(e - gold[tuple(int(x) for x in t)]) < TOL_FP64
            n += 1
    assert n == 255
    assert abs(res["total"] - total) < 1e-9
    assert abs(res["total"] - gold[tuple(w["exp"])]) < 1e-9     # = full 8e/12o FCI
    m.close()


def test_screened_expansion_vs_oracle(lib):
    """Screened expansion (downward-closed rule, thr 1e-6): tuple sets,
    increments, keep flags and order sums identical to the oracle's."""
    n, nocc = 10, 3
    h, eri, _ = ms.gen_integrals(n, nocc, 31, eps_vir=(0.05, 3.0))
    ref, exp = [2, 3], [0, 1, 4, 5, 6, 7, 8, 9]
    thr = 1e-4
    ores = om.run_mbe(h, eri, nocc, ref, exp, 4, thr)
    m = make(lib)
    m.load(h, eri, 2 * nocc)
    res = m.run(ref, exp, 4, thr)
    assert abs(res["eps_ref"] - ores["eps_ref"]) < TOL_FP64
    assert len(res["orders"]) == len(ores["orders"])
    for g, o in zip(res["orders"], ores["orders"]):
        assert [tuple(int(x) for x in t) for t in g["tuples"]] == o["tuples"]
        assert np.abs(g["inc"] - np.array(o["inc"])).max() < TOL_FP64
        assert list(g["keep"]) == o["keep"]
        assert abs(g["E_order"] - o["E_order"]) < TOL_FP64
    assert abs(res["total"] - ores["total"]) < TOL_FP64
    m.close()


def test_tuple_generation_counts_fig2a(lib):
    """Device tuple generation, unscreened, reproduces Fig. 2 case (a):
    6, 15, 20, 15, 6, 1 tuples for a (6,9) system with the RHF reference."""
    h, eri, _ = ms.gen_integrals(9, 3, 5)
    m = make(lib)
    m.load(h, eri, 6)
    res = m.run([0, 1, 2], [3, 4, 5, 6, 7, 8], 6, 0.0)
    assert [len(o["tuples"]) for o in res["orders"]] == [6, 15, 20, 15, 6, 1]
    e_fci = oc.casci(h, eri, 3, range(9))
    assert abs(res["total"] - e_fci) < 1e-9
    m.close()


def test_empty_reference_and_degenerate_spaces(lib):
    """Empty reference space (HF determinant, Eq. 2), a tuple with no active
    electrons and an empty tuple list."""
    h, eri, _ = ms.gen_integrals(7, 2, 9)
    m = make(lib)
    m.load(h, eri, 4)
    e0 = lib.mbe_set_reference(m.ctx, [], list(range(7)))
    assert abs(e0 - oc.casci(h, eri, 2, [])) < TOL_FP64
    eps, st = lib.mbe_solve_tuples(m.ctx, np.array([[5], [1]]), 1)
    assert abs(eps[0] - oc.casci(h, eri, 2, [5])) < TOL_FP64
    assert abs(eps[1] - oc.casci(h, eri, 2, [1])) < TOL_FP64
    eps, st = lib.mbe_solve_tuples(m.ctx, np.zeros((0, 2), dtype=np.int32), 2)
    assert eps.size == 0
    m.close()


def test_invalid_inputs_rejected(lib):
    h, eri, _ = ms.gen_integrals(6, 2, 1)
    m = make(lib)
    bad = h.copy()
    bad[0, 1] = np.nan
    with pytest.raises(lib.MBEError) as ei:
        m.load(bad, eri, 4)
    assert ei.value.code == lib.MBE_EINVAL
    m.load(h, eri, 4)
    with pytest.raises(lib.MBEError) as ei:
        lib.mbe_solve_tuples(m.ctx, np.array([[3]]), 1)
    assert ei.value.code == lib.MBE_ESTATE
    lib.mbe_set_reference(m.ctx, [1, 2], [0, 3, 4, 5])
    with pytest.raises(lib.MBEError) as ei:
        lib.mbe_solve_tuples(m.ctx, np.array([[4, 3]]), 2)
    assert ei.value.code == lib.MBE_EINVAL
    lib.mbe_solve_tuples(m.ctx, np.array([[3, 4]]), 2)
    with pytest.raises(lib.MBEError) as ei:         # order 2 before order 1
        lib.mbe_increments(m.ctx, 2, 0.0, 1)
    assert ei.value.code == lib.MBE_ESTATE
    m.close()

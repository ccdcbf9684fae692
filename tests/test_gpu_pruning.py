"""GPU parity of pi-pruning (Sec. 3): tuples that hold both orbitals of a
degenerate pair or neither, the expansion run over units (single orbitals
and pairs).  Against the oracle's pruned expansion: identical tuple sets per
order (device generation from one-unit-smaller tuples, screening on the
one-unit-removed subtuples), increments of Eq. 3 over units (1e-10 Eh in
FP64, 1e-7 Eh mixed), the all-order unscreened sum equal to the FCI energy,
and the energy gradient with unit-counted MBE coefficients.
"""
import numpy as np
import pytest

import mbe_synth as ms
from oracle import casci as oc
from oracle import mbe as om

pytestmark = pytest.mark.gpu

NORB, NOCC, SEED = 10, 3, 31
REF = [2, 3]
EXP = [0, 1, 4, 5, 6, 7, 8, 9]
PAIRS = [(4, 5), (7, 9)]


@pytest.fixture(scope="module")
def lib():
    from paper_1905_02786_gb300 import build, _binding
    build.build()
    _binding.load_library()
    return _binding


def _cmp(res, ores, tol):
    assert len(res["orders"]) == len(ores["orders"])
    for g, o in zip(res["orders"], ores["orders"]):
        assert [tuple(int(x) for x in t) for t in g["tuples"]] == o["tuples"]
        if o["tuples"]:
            assert np.abs(np.asarray(g["inc"]) - np.array(o["inc"])).max() < tol
            assert [bool(x) for x in g["keep"]] == [bool(x) for x in o["keep"]]
    assert abs(res["total"] - ores["total"]) < tol


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-7)])
def test_pruned_screened_expansion_vs_oracle(lib, precision, tol):
    h, eri, _ = ms.gen_integrals(NORB, NOCC, SEED)
    thr = 1e-2
    ores = om.run_mbe(h, eri, NOCC, REF, EXP, 6, thr, pairs=PAIRS)
    prec = lib.MBE_FP64 if precision == "fp64" else lib.MBE_MIXED_BF16X3
    m = lib.MBE(0, precision=prec)
    m.load(h, eri, 2 * NOCC)
    res = m.run(REF, EXP, 6, thr, pairs=PAIRS)
    m.close()
    _cmp(res, ores, tol)
    for o in res["orders"]:
        for t in o["tuples"]:
            for a, b in PAIRS:
                assert (a in t) == (b in t)


def test_pruned_allorder_sum_is_fci_and_gradient(lib):
    """Unscreened to all orders (odd orders can be empty before even ones are
    not): the total is the FCI energy of the whole space; the gradient of the
    pruned expansion (MBE coefficients over units) equals the oracle's."""
    n, nocc = 8, 3
    h, eri, _ = ms.gen_integrals(n, nocc, 5)
    ref, exp, pairs = [1, 2], [0, 3, 4, 5, 6, 7], [(3, 4), (5, 7)]
    # RDMs are first order in the CI-vector error: converge the residual to
    # 1e-11 (the default 1e-8 leaves ~3e-9 in the gradient); 8 orbitals keep
    # every oracle CASCI on its dense eigensolver (3136 determinants at most),
    # whose vectors are exact to rounding
    m = lib.MBE(0, keep_ci=1, conv_tol_r=1e-11, conv_tol_e=1e-14)
    m.load(h, eri, 2 * nocc)
    res = m.run(ref, exp, len(exp), 0.0, pairs=pairs)
    assert abs(res["total"] - oc.casci(h, eri, nocc, list(range(n)))) < 1e-9
    dh, dg = m.backward()
    m.close()
    tuples = [tuple(int(x) for x in t) for o in res["orders"] for t in o["tuples"]]
    odh, odg, _ = om.mbe_gradient(h, eri, nocc, ref, tuples, om.expansion_units(exp, pairs))
    assert np.abs(dh - odh).max() < 1e-9
    assert np.abs(dg - odg).max() < 1e-9


def test_pruning_pairs_checked(lib):
    h, eri, _ = ms.gen_integrals(NORB, NOCC, SEED)
    m = lib.MBE(0)
    m.load(h, eri, 2 * NOCC)
    lib.mbe_set_reference(m.ctx, REF, EXP)
    for bad in ([(4, 4)], [(4, 2)], [(4, 5), (5, 6)], [(4, 11)]):
        with pytest.raises(lib.MBEError) as ei:
            lib.mbe_set_pruning_pairs(m.ctx, bad)
        assert ei.value.code == lib.MBE_EINVAL
    lib.mbe_set_pruning_pairs(m.ctx, PAIRS)
    t1 = lib.mbe_next_tuples(m.ctx, 1)
    assert sorted(int(x) for x in t1.ravel()) == [0, 1, 6, 8]
    eps, _ = lib.mbe_solve_tuples(m.ctx, t1, 1)
    lib.mbe_increments(m.ctx, 1, 0.0, len(t1))
    with pytest.raises(lib.MBEError) as ei:
        lib.mbe_set_pruning_pairs(m.ctx, PAIRS)
    assert ei.value.code == lib.MBE_ESTATE
    m.close()

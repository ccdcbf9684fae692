"""GPU parity of the mixed-precision path (tcgen05 split-BF16x3 sigma with
FP64 refinement) against the oracle.

Tolerances: sigma vectors element by element to 2e-4 of the largest element
(split-BF16x3 carries ~16 significant bits per operand); CASCI energies and
increments to 1e-7 Eh (the mixed-precision target), checked tighter (1e-8)
for the per-tuple energies because increments combine up to 2^n of them.
"""
import numpy as np
import pytest

import mbe_synth as ms
from oracle import casci as oc
from oracle import mbe as om

from test_gpu_parity import core_signs

pytestmark = pytest.mark.gpu
TOL_MIXED_INC = 1e-7
TOL_MIXED_EPS = 1e-8


@pytest.fixture(scope="module")
def lib():
    from paper_1905_02786_gb300 import build, _binding
    build.build()
    _binding.load_library()
    return _binding


def mixed(lib, **opts):
    return lib.MBE(0, precision=lib.MBE_MIXED_BF16X3, **opts)


@pytest.mark.parametrize("case", [
    (8, 3, 1, [0, 1, 2, 3, 4, 5]),                  # npair 21, one column tile
    (12, 4, 0, [0, 1, 2, 3, 4, 5, 6, 7, 8]),        # 126 strings, ragged tiles
    (14, 4, 2, list(range(12))),                    # 8e/12o: 495 strings, npair 78
    (16, 1, 3, list(range(14))),                    # 2e/14o: npair 105 (Kpad 112)
    (10, 4, 5, [1, 3, 4, 5, 7, 8, 9]),              # inactive core + deleted virtuals
])
@pytest.mark.parametrize("shift", [0.0, 0.5])
def test_sigma_tc_elementwise(lib, case, shift):
    norb, nocc, seed, act = case
    h, eri, _ = ms.gen_integrals(norb, nocc, seed)
    sp = oc.Space(h, eri, nocc, act)
    m = mixed(lib, spin_shift=shift)
    m.load(h, eri, 2 * nocc)
    c = ms.random_symmetric_ci(sp.nstr, seed)[0]
    sig, ecore = lib.mbe_sigma(m.ctx, act, c)
    S = core_signs(sp, nocc, act)
    cs = S * c.ravel()
    ref = S * (sp.sigma(cs) + shift * sp.s2(cs) - ecore * cs)
    scale = np.abs(ref).max()
    err = np.abs(sig - ref).max()
    assert err <= 2e-4 * scale, (err, scale)
    # and exactly symmetric (sigma = X + X^T, one value per element pair)
    s2 = sig.reshape(sp.nstr, sp.nstr)
    assert np.array_equal(s2, s2.T)
    m.close()


def test_sigma_tc_one_row_per_cta(lib):
    """12e/14o (3,003 strings, 9.0e6 determinants): above 2,048 strings the
    tensor-core sigma owns one row of X per CTA.  Too large for the oracle's
    determinant-driven sigma in test time, so compared with the FP64 GPU
    sigma, itself pinned to the oracle element by element above."""
    norb, nocc, seed = 14, 6, 7
    act = list(range(14))
    h, eri, _ = ms.gen_integrals(norb, nocc, seed)
    nstr = 3003
    c = ms.random_symmetric_ci(nstr, 5)[0]
    ref_ctx = lib.MBE(0)
    ref_ctx.load(h, eri, 2 * nocc)
    ref, ec_ref = lib.mbe_sigma(ref_ctx.ctx, act, c)
    ref_ctx.close()
    m = mixed(lib)
    m.load(h, eri, 2 * nocc)
    sig, ec = lib.mbe_sigma(m.ctx, act, c)
    m.close()
    assert abs(ec - ec_ref) < 1e-12 * max(1.0, abs(ec_ref))
    scale = np.abs(ref).max()
    assert np.abs(sig - ref).max() <= 2e-4 * scale


def test_mixed_casci_energies_vs_oracle(lib):
    w = ms.workload("h2o_dz_8e23o")
    h, eri, _ = ms.workload_integrals("h2o_dz_8e23o")
    m = mixed(lib)
    m.load(h, eri, w["nel"])
    e_ref = lib.mbe_set_reference(m.ctx, w["ref"], w["exp"])
    assert abs(e_ref - oc.casci(h, eri, w["nocc"], w["ref"])) < TOL_MIXED_EPS
    for k, tk in ((1, [(0,), (7,), (22,)]), (2, [(0, 7), (8, 9)]), (3, [(0, 7, 8), (9, 10, 11)])):
        eps, st = lib.mbe_solve_tuples(m.ctx, np.array(tk), k)
        assert np.all(st == 0)
        for t, e in zip(tk, eps):
            e_or = oc.casci(h, eri, w["nocc"], om.active_space(w["ref"], t))
            assert abs(e - e_or) < TOL_MIXED_EPS, (t, e, e_or)
    m.close()


def test_mixed_screened_expansion_vs_oracle(lib):
    n, nocc = 10, 3
    h, eri, _ = ms.gen_integrals(n, nocc, 31)
    ref, exp = [2, 3], [0, 1, 4, 5, 6, 7, 8, 9]
    thr = 1e-4
    ores = om.run_mbe(h, eri, nocc, ref, exp, 4, thr)
    m = mixed(lib)
    m.load(h, eri, 2 * nocc)
    res = m.run(ref, exp, 4, thr)
    for g, o in zip(res["orders"], ores["orders"]):
        assert [tuple(int(x) for x in t) for t in g["tuples"]] == o["tuples"]
        assert np.abs(g["inc"] - np.array(o["inc"])).max() < TOL_MIXED_INC
    assert abs(res["total"] - ores["total"]) < TOL_MIXED_INC
    m.close()


@pytest.mark.parametrize("case", [
    (8, 3, 1, [0, 1, 2, 3, 4, 5]),
    (14, 4, 2, list(range(12))),                    # 8e/12o, npair 78
    (16, 1, 3, list(range(14))),                    # npair 105 (Kpad 112)
    (10, 4, 5, [1, 3, 4, 5, 7, 8, 9]),
])
def test_sigma_emulated_fp64_elementwise(lib, case):
    """The sliced tensor-core contraction (exact 8-bit slices, grouped exact
    FP32 accumulators) gives sigma to ~1e-10 relative; checked at 1e-9 of
    the largest element, non-symmetric c included (pull scatter)."""
    norb, nocc, seed, act = case
    h, eri, _ = ms.gen_integrals(norb, nocc, seed)
    sp = oc.Space(h, eri, nocc, act)
    m = lib.MBE(0, precision=lib.MBE_EMULATED_FP64, spin_shift=0.5)
    m.load(h, eri, 2 * nocc)
    rng = np.random.default_rng(seed)
    c = rng.standard_normal((sp.nstr, sp.nstr))
    sig, ecore = lib.mbe_sigma(m.ctx, act, c)
    S = core_signs(sp, nocc, act)
    cs = S * c.ravel()
    ref = S * (sp.sigma(cs) + 0.5 * sp.s2(cs) - ecore * cs)
    scale = np.abs(ref).max()
    assert np.abs(sig - ref).max() <= 1e-9 * scale
    m.close()


def test_emulated_fp64_energies_vs_oracle(lib):
    w = ms.workload("h2o_dz_8e23o")
    h, eri, _ = ms.workload_integrals("h2o_dz_8e23o")
    m = lib.MBE(0, precision=lib.MBE_EMULATED_FP64)
    m.load(h, eri, w["nel"])
    lib.mbe_set_reference(m.ctx, w["ref"], w["exp"])
    tk = [(0, 7), (8, 9), (9, 10)]
    eps, st = lib.mbe_solve_tuples(m.ctx, np.array(tk), 2)
    assert np.all(st == 0)
    for t, e in zip(tk, eps):
        assert abs(e - oc.casci(h, eri, w["nocc"], om.active_space(w["ref"], t))) < 1e-9
    m.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_warm_start_same_increments(lib, precision):
    """Starting each tuple from its parent's converged vector (the tuple
    less one orbital, previous order; opt-in) reaches the same increments as
    the cold start, to the tolerance of the mode, on a system where the
    parent states lead to the ground-state root."""
    n, nocc = 12, 4
    h, eri, _ = ms.gen_integrals(n, nocc, 41)
    ref, exp = [2, 3, 4, 5], [0, 1, 6, 7, 8, 9, 10, 11]
    prec = lib.MBE_FP64 if precision == "fp64" else lib.MBE_MIXED_BF16X3
    tol = 1e-10 if precision == "fp64" else TOL_MIXED_INC
    runs = {}
    for warm in (0, 1):
        m = lib.MBE(0, precision=prec, warm_start=warm)
        m.load(h, eri, 2 * nocc)
        lib.mbe_reset_stats(m.ctx)
        res = m.run(ref, exp, 4, 0.0)
        runs[warm] = (res, lib.mbe_get_stats(m.ctx)["iters_total"])
        m.close()
    (cold, it_cold), (hot, it_hot) = runs[0], runs[1]
    for oc_, oh in zip(cold["orders"], hot["orders"]):
        assert np.array_equal(oc_["tuples"], oh["tuples"])
        assert np.max(np.abs(np.asarray(oc_["inc"]) - np.asarray(oh["inc"]))) < tol
    assert abs(cold["total"] - hot["total"]) < tol


@pytest.mark.parametrize("case", [
    (8, 3, 1, [0, 1, 2, 3, 4, 5]),
    (14, 4, 2, list(range(12))),                    # 8e/12o, npair 78 (kpad 80)
    (10, 4, 5, [1, 3, 4, 5, 7, 8, 9]),              # inactive core + deleted virtuals
    (12, 4, 0, [0, 1, 2, 3, 4, 5, 6, 7, 8]),        # ragged tiles
])
def test_sigma_exact_fused_elementwise(lib, case):
    """The fused exact-point sigma (gather, exact 8-bit digits of D and g',
    grouped exact FP32 accumulators in tensor memory, 64-bit fixed-point
    scatter) for symmetric vectors with FP32 values, as at the exact points
    of the mixed mode: element by element to 1e-9 of the largest element,
    and exactly symmetric."""
    norb, nocc, seed, act = case
    h, eri, _ = ms.gen_integrals(norb, nocc, seed)
    sp = oc.Space(h, eri, nocc, act)
    m = lib.MBE(0, precision=lib.MBE_EMULATED_FP64, spin_shift=0.5)
    m.load(h, eri, 2 * nocc)
    c = ms.random_symmetric_ci(sp.nstr, seed + 7)[0]
    c = (c / np.linalg.norm(c)).astype(np.float32).astype(np.float64)
    sig, ecore = lib.mbe_sigma(m.ctx, act, c)
    S = core_signs(sp, nocc, act)
    cs = S * c.ravel()
    ref = S * (sp.sigma(cs) + 0.5 * sp.s2(cs) - ecore * cs)
    scale = np.abs(ref).max()
    assert np.abs(sig - ref).max() <= 1e-9 * scale
    s2 = sig.reshape(sp.nstr, sp.nstr)
    assert np.array_equal(s2, s2.T)
    m.close()


def test_pspace_preconditioner_same_energies_fewer_iterations(lib):
    """The P-space block (the 128 lowest-diagonal symmetric functions solved
    exactly in the Davidson correction) changes the path of the iteration,
    not its limit: seeded order-4 tuples of the 8e/23o workload (8e/10o
    CASCIs) give the energies of the diagonal preconditioner and the
    oracle's, in fewer iterations."""
    w = ms.workload("h2o_dz_8e23o")
    h, eri, _ = ms.workload_integrals("h2o_dz_8e23o")
    rest = [o for o in w["exp"] if o != 0]
    tuples = np.array([(0,) + t for t in ms.sample_tuples(rest, 3, 12, 31)], dtype=np.int32)
    out = {}
    for psp in (0, 128):
        m = mixed(lib, pspace=psp)
        m.load(h, eri, w["nel"])
        lib.mbe_set_reference(m.ctx, w["ref"], w["exp"])
        lib.mbe_reset_stats(m.ctx)
        eps, st = lib.mbe_solve_tuples(m.ctx, tuples, 4)
        assert np.all(st == 0)
        out[psp] = (eps, lib.mbe_get_stats(m.ctx)["iters_total"])
        m.close()
    (e0, it0), (e1, it1) = out[0], out[128]
    assert np.max(np.abs(e0 - e1)) < 1e-9
    assert it1 < it0, (it1, it0)
    for t, e in list(zip(tuples, e1))[:3]:
        e_or = oc.casci(h, eri, w["nocc"], om.active_space(w["ref"], tuple(t)))
        assert abs(e - e_or) < TOL_MIXED_EPS, (t, e, e_or)

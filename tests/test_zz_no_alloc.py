"""mbe_sigma_noalloc (sigma with every intermediate in one fixed device
array, no allocation) against mbe_sigma, the pooled entry point.

Collected last (file name) and self-contained: it builds its own context and
inputs, so it passes alone and after the other GPU tests.  Both entry points
run the FP64 sigma; tolerance 1e-12 of the largest element.
"""
import math

import numpy as np
import pytest

import mbe_synth as ms

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def lib():
    from paper_1905_02786_gb300 import build, _binding
    build.build()
    _binding.load_library()
    return _binding


def _nstr(act, nocc):
    return math.comb(len(act), sum(1 for a in act if a < nocc))


def test_noalloc_matches_pooled_two_calls(lib):
    torch = pytest.importorskip("torch")
    norb, nocc = 10, 4
    h, eri, _ = ms.gen_integrals(norb, nocc, 6)
    m = lib.MBE(0)
    m.load(h, eri, 2 * nocc)
    for seed, act in enumerate([[0, 1, 3, 4, 5, 7, 8], [2, 3, 4, 6, 9]]):
        nstr = _nstr(act, nocc)
        c = ms.random_symmetric_ci(nstr, 30 + seed)[0].ravel()
        ref, ec_ref = lib.mbe_sigma(m.ctx, act, c)
        scale = np.max(np.abs(ref))
        cd = torch.tensor(c, dtype=torch.float64, device="cuda:0")
        # two calls in a row into the same output buffer; the second one
        # without the core energy (no wait inside the call)
        sd = torch.full_like(cd, float("nan"))
        ec = lib.mbe_sigma_noalloc(m.ctx, act, cd, sd)
        first = sd.cpu().numpy()
        assert lib.mbe_sigma_noalloc(m.ctx, act, cd, sd, want_core=False) is None
        torch.cuda.synchronize()
        second = sd.cpu().numpy()
        assert abs(ec - ec_ref) <= 1e-12 * max(1.0, abs(ec_ref))
        assert np.max(np.abs(first - ref)) <= TOL * scale
        assert np.max(np.abs(second - ref)) <= TOL * scale
    m.close()


def test_noalloc_rejects_oversize_and_bad_length(lib):
    torch = pytest.importorskip("torch")
    norb, nocc = 12, 4
    h, eri, _ = ms.gen_integrals(norb, nocc, 2)
    m = lib.MBE(0)
    m.load(h, eri, 2 * nocc)
    big = list(range(10))                        # 8e/10o: D and E need ~39 MB
    n = _nstr(big, nocc) ** 2
    cd = torch.zeros(n, dtype=torch.float64, device="cuda:0")
    sd = torch.full_like(cd, 7.0)
    with pytest.raises(lib.MBEError) as e:
        lib.mbe_sigma_noalloc(m.ctx, big, cd, sd)
    assert e.value.code == lib.MBE_EINVAL
    assert bool(torch.all(sd == 7.0))            # nothing was launched
    small = [0, 1, 4, 5]
    n = _nstr(small, nocc) ** 2
    cd = torch.zeros(n + 1, dtype=torch.float64, device="cuda:0")
    sd = torch.zeros_like(cd)
    with pytest.raises(lib.MBEError) as e:
        lib.mbe_sigma_noalloc(m.ctx, small, cd, sd)
    assert e.value.code == lib.MBE_EINVAL
    m.close()

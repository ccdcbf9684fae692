"""The operand-plan autotuner of the two-spin tensor-core sigma (mixed mode).

Every plan computes the same sums in the same order, so an autotuned run
gives the same bits as the default plan; the tuned plans are cached in the
file named by tune_file and read back by the next context.
"""
import numpy as np
import pytest

import mbe_synth as ms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1905_02786_gb300 import build, _binding
    build.build()
    _binding.load_library()
    return _binding


def _solve(lib, h, eri, nocc, ref, tuples, **opts):
    m = lib.MBE(0, precision=lib.MBE_MIXED_BF16X3, **opts)
    m.load(h, eri, 2 * nocc)
    lib.mbe_set_reference(m.ctx, ref, [o for o in range(h.shape[0]) if o not in ref])
    eps, st = lib.mbe_solve_tuples(m.ctx, np.array(tuples, dtype=np.int32), len(tuples[0]))
    m.close()
    return eps, st


def test_autotune_same_bits_and_cache(lib, tmp_path):
    n, nocc = 14, 4
    h, eri, _ = ms.gen_integrals(n, nocc, 7)
    ref = [2, 3, 4, 5, 6, 7]
    tuples = [(0, 1, 8, 9, 10, 11), (0, 8, 9, 10, 11, 12), (1, 9, 10, 11, 12, 13)]
    cache = tmp_path / "tune.txt"
    e_def, st_def = _solve(lib, h, eri, nocc, ref, tuples)
    e_tun, st_tun = _solve(lib, h, eri, nocc, ref, tuples, autotune=1,
                           tune_file=str(cache).encode())
    assert np.all(st_def == 0) and np.all(st_tun == 0)
    assert np.array_equal(e_def, e_tun)
    lines = [ln.split() for ln in cache.read_text().splitlines() if ln.strip()]
    assert lines and all(ln[0] == "sigma_ab" and len(ln) == 7 for ln in lines)
    shapes = {(int(ln[1]), int(ln[2])) for ln in lines}
    assert len(shapes) == len(lines)
    for ln in lines:
        assert 2 <= int(ln[3]) <= 4 and int(ln[4]) in (0, 1) and int(ln[5]) in (1, 2)
        assert float(ln[6]) > 0.0
    # a second context reads the cache: nothing is tuned again
    e_again, _ = _solve(lib, h, eri, nocc, ref, tuples, autotune=1,
                        tune_file=str(cache).encode())
    assert np.array_equal(e_again, e_def)
    assert len([ln for ln in cache.read_text().splitlines() if ln.strip()]) == len(lines)


def test_autotune_rejects_bad_flag(lib):
    with pytest.raises(lib.MBEError) as ei:
        lib.MBE(0, autotune=2)
    assert ei.value.code == lib.MBE_EINVAL

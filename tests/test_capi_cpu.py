"""Host-side checks of the C-ABI library (no GPU needed): it builds, loads and
exports every entry point that include/mbe.h declares; the synthetic-input
module holds the stated recipe."""
import os
import re

import numpy as np
import pytest

import mbe_synth as ms

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mbe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mbe_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_1905_02786_gb300 import build
    path = build.build()
    import ctypes
    lib = ctypes.CDLL(path)
    names = _declared()
    assert "mbe_solve_tuples" in names and "mbe_energy_backward" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_lists_every_declared_symbol():
    from paper_1905_02786_gb300 import _binding
    for n in _declared():
        assert n in _binding.EXPORTED, n


def test_options_struct_matches_header_defaults():
    from paper_1905_02786_gb300 import _binding
    o = _binding.mbe_default_options()
    assert o.precision == _binding.MBE_FP64
    assert o.max_subspace == 20 and o.spin_shift == 0.5 and o.deterministic == 1
    assert (o.mixed_stage_tol, o.mixed_round_drop, o.mixed_rel_tol) == (1e-5, 1e-2, 2e-7)
    assert o.pspace == 128
    assert o.autotune == 0 and o.graphs == 1 and o.wait_limit == 1 << 24


@pytest.mark.parametrize("field,value", [("mixed_stage_tol", 0.0), ("mixed_round_drop", 1.0),
                                         ("mixed_round_drop", 0.0), ("mixed_rel_tol", -1.0),
                                         ("max_subspace", 33), ("pspace", 129),
                                         ("pspace", -1), ("graphs", 2), ("graphs", -1),
                                         ("autotune", 3)])
def test_create_rejects_bad_options(field, value):
    """Options are checked before any device call, so this runs without a GPU."""
    from paper_1905_02786_gb300 import _binding
    with pytest.raises(_binding.MBEError) as e:
        _binding.mbe_create(0, _binding.mbe_default_options(**{field: value}))
    assert e.value.code == _binding.MBE_EINVAL


def test_create_without_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1905_02786_gb300 import _binding
    with pytest.raises(_binding.MBEError):
        _binding.mbe_create(0)


def test_generator_recipe():
    h, eri, eps = ms.gen_integrals(12, 4, 0)
    assert np.all(np.diff(eps) >= 0)
    assert np.all(eps[:4] < -0.39) and np.all(eps[4:] > 0.049)
    assert np.allclose(h, h.T) and np.allclose(eri, eri.T)
    d = [ms.pair_index(p, p) for p in range(12)]
    assert abs(eri[d, d].mean() - 0.5) < 1e-12
    assert np.linalg.eigvalsh(eri).min() > -1e-12      # sum of outer products
    G = ms.unpack_eri(eri, 12)
    assert np.allclose(G, G.transpose(1, 0, 2, 3)) and np.allclose(G, G.transpose(2, 3, 0, 1))

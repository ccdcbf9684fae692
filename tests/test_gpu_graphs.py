"""CUDA-graph replay of the mixed-precision Davidson iteration (opt.graphs).

Each iteration's launches (sigma vector, subspace row, Ritz step, residual,
correction and its orthogonalisation) are captured from the stream and
replayed as one graph.  The device runs the same kernels on the same data in
the same order, so energies, iteration counts and the number of kernels run
equal those of plain stream launches bit for bit, while the host makes one
launch per iteration instead of about twenty-five.
"""
import numpy as np
import pytest

import mbe_synth as ms
from oracle import casci as oc
from oracle import mbe as om

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1905_02786_gb300 import build, _binding
    build.build()
    _binding.load_library()
    return _binding


def _solve(lib, graphs, tuples, order, **opts):
    w = ms.workload("h2o_dz_8e23o")
    h, eri, _ = ms.workload_integrals("h2o_dz_8e23o")
    m = lib.MBE(0, precision=lib.MBE_MIXED_BF16X3, graphs=graphs, **opts)
    m.load(h, eri, w["nel"])
    lib.mbe_set_reference(m.ctx, w["ref"], w["exp"])
    lib.mbe_reset_stats(m.ctx)
    eps, st = lib.mbe_solve_tuples(m.ctx, tuples, order)
    stats = lib.mbe_get_stats(m.ctx)
    m.close()
    return eps, st, stats


def _tuples(order, count, seed):
    w = ms.workload("h2o_dz_8e23o")
    return np.array(ms.sample_tuples(w["exp"], order, count, seed), dtype=np.int32)


@pytest.mark.parametrize("order,count", [(3, 24), (5, 8)])
def test_graphs_same_bits_fewer_host_launches(lib, order, count):
    tuples = _tuples(order, count, 17 + order)
    e0, s0, st0 = _solve(lib, 0, tuples, order)
    e1, s1, st1 = _solve(lib, 1, tuples, order)
    assert np.all(s0 == 0) and np.all(s1 == 0)
    assert np.array_equal(e0, e1)
    assert st0["iters_total"] == st1["iters_total"]
    # the same kernels ran; the host launched far fewer times
    assert st0["launches"] == st1["launches"]
    assert st0["graph_launches"] == 0 and st1["graph_launches"] > 0
    assert st0["host_launches"] == st0["launches"]
    assert st1["host_launches"] < st1["launches"] // 3, st1
    # one executable graph per iteration shape and batch, updated in place
    # for the other iterations
    assert 3 * st1["graph_builds"] <= st1["graph_launches"], st1


def test_graphs_energies_vs_oracle(lib):
    """Order-4 tuples through the graph path against the oracle's CASCI at
    the mixed-mode tolerance of a tuple energy."""
    w = ms.workload("h2o_dz_8e23o")
    h, eri, _ = ms.workload_integrals("h2o_dz_8e23o")
    tuples = _tuples(4, 6, 5)
    eps, st, stats = _solve(lib, 1, tuples, 4)
    assert np.all(st == 0) and stats["graph_launches"] > 0
    for t, e in zip(tuples, eps):
        e_or = oc.casci(h, eri, w["nocc"], om.active_space(w["ref"], tuple(int(x) for x in t)))
        assert abs(e - e_or) < 1e-8, (t, e, e_or)


def test_graphs_keep_sigma_timing(lib):
    """The sigma-contraction CUDA events are graph nodes under replay: the
    timed total stays positive and close to the plain-launch one."""
    tuples = _tuples(5, 8, 23)
    _, _, st0 = _solve(lib, 0, tuples, 5, timing=1)
    _, _, st1 = _solve(lib, 1, tuples, 5, timing=1)
    assert st0["dom_ms"] > 0.0 and st1["dom_ms"] > 0.0
    assert 0.5 < st1["dom_ms"] / st0["dom_ms"] < 2.0, (st0["dom_ms"], st1["dom_ms"])
    assert st0["dom_launches"] == st1["dom_launches"]


def test_graphs_rejects_bad_flag(lib):
    with pytest.raises(lib.MBEError) as ei:
        lib.MBE(0, graphs=2)
    assert ei.value.code == lib.MBE_EINVAL

"""Write stored oracle values used by the GPU parity tests.

Calls only ``oracle/`` and the seeded input generator ``mbe_synth``.
Usage: python tests/golden/make_golden.py [name ...]
Writes tests/golden/<name>.txt with one line per tuple:
    order  comma-separated-tuple(or '-')  eps_T  (total electronic energy, Eh)
``name`` is a workload of ``mbe_synth`` (the whole expansion, all orders) or
one of the seeded tuple samples of ``SAMPLES`` (``<workload>_sampled``).
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import mbe_synth as ms                     # noqa: E402
from oracle import casci as oc             # noqa: E402
from oracle import mbe as om               # noqa: E402


def allorder(name):
    w = ms.workload(name)
    h, eri, _ = ms.workload_integrals(name)
    t0 = time.time()
    res = om.run_mbe(h, eri, w["nocc"], w["ref"], w["exp"], w["max_order"], w["thr"])
    path = os.path.join(HERE, name + ".txt")
    with open(path, "w") as f:
        f.write(f"# oracle CASCI energies for workload {name} (mbe_synth), "
                f"written by tests/golden/make_golden.py\n")
        f.write(f"# total MBE energy {res['total']!r}\n")
        f.write(f"0 - {res['eps_ref']!r}\n")
        for k, o in enumerate(res["orders"], start=1):
            for t, e in zip(o["tuples"], o["eps"]):
                f.write(f"{k} {','.join(map(str, t))} {e!r}\n")
    print(name, "done in", time.time() - t0, "s; total", res["total"])


# seeded tuples whose CASCIs are too large for the oracle's Davidson in test
# time: (order, count, seed, with orbital 0).  For the 8e/23o workload, with
# occupied orbital 0 in the tuple the CASCI has 8 electrons, else 6; None
# samples the whole expansion space (the 10e/60o and 8e/114o workloads, whose
# expansion spaces hold virtual orbitals only).
SAMPLES = {
    "h2o_dz_8e23o_sampled": ("h2o_dz_8e23o", [(5, 2, 61, True), (5, 1, 62, False),
                                              (6, 2, 63, True), (6, 2, 64, False)]),
    "h10_chain_10e60o_sampled": ("h10_chain_10e60o", [(1, 2, 71, None), (2, 1, 72, None)]),
    "h2o_qz_8e114o_sampled": ("h2o_qz_8e114o", [(1, 3, 73, None), (2, 3, 74, None)]),
}


def sample_tuples(w, spec):
    rest = [o for o in w["exp"] if o != 0]
    out = []
    for order, count, seed, with0 in spec:
        if with0 is None:
            for t in ms.sample_tuples(w["exp"], order, count, seed):
                out.append((order, tuple(sorted(t))))
            continue
        for t in ms.sample_tuples(rest, order - 1 if with0 else order, count, seed):
            out.append((order, tuple(sorted(((0,) if with0 else ()) + t))))
    return out


def sampled(name):
    wname, spec = SAMPLES[name]
    w = ms.workload(wname)
    h, eri, _ = ms.workload_integrals(wname)
    t0 = time.time()
    path = os.path.join(HERE, name + ".txt")
    with open(path, "w") as f:
        f.write(f"# oracle CASCI energies of seeded tuples of workload {wname} (mbe_synth), "
                f"written by tests/golden/make_golden.py\n")
        f.write(f"0 - {oc.casci(h, eri, w['nocc'], w['ref'])!r}\n")
        for order, t in sample_tuples(w, spec):
            e = oc.casci(h, eri, w["nocc"], om.active_space(w["ref"], t))
            f.write(f"{order} {','.join(map(str, t))} {e!r}\n")
            f.flush()
            print(order, t, e, round(time.time() - t0, 1), "s", flush=True)
    print(name, "done in", time.time() - t0, "s")


if __name__ == "__main__":
    for n in (sys.argv[1:] or ["fci8e12o_allorder"]):
        sampled(n) if n in SAMPLES else allorder(n)

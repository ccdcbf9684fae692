"""Write stored oracle values used by the GPU parity tests.

Calls only ``oracle/`` and the seeded input generator ``mbe_synth``.
Usage: python tests/golden/make_golden.py [name ...]
Writes tests/golden/<name>.txt with one line per tuple:
    order  comma-separated-tuple(or '-')  eps_T  (total electronic energy, Eh)
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


if __name__ == "__main__":
    for n in (sys.argv[1:] or ["fci8e12o_allorder"]):
        allorder(n)

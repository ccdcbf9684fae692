"""Benchmark of the MBE-FCI hot path on GB300.

One step = one complete many-body expansion of the workload (default: the
8e/23o water-double-zeta-shaped system, CAS(6e,6o) reference, 17 expansion
orbitals to order 6, screening 1e-6 Eh): tuple generation, every CASCI
(effective integrals, string tables, diagonal, Davidson with the
string-driven sigma), increment assembly by hash lookup, screening and
Kahan order sums, all through the C ABI of include/mbe.h.

Metric: CASCI increments per second (tuples solved and assembled per second)
over the whole job.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
  python bench.py --impl reference ...   # the CPU oracle on a bounded sample
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import mbe_synth as ms  # noqa: E402

METRIC = ("CASCI increments/sec and sigma TFLOP/s, mixed+batched vs plain FP64 GPU "
          "at 1e-7 Eh")
UNIT = "increments/s"
DEFAULT_WORKLOAD = "h2o_dz_8e23o"

# DRAM traffic per launch of the dominant kernels from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum), per algorithmic flop
# (2 N_det npair^2 per sigma vector), keyed by kernel; valid only while the
# kernel definition is unchanged (sha256 prefix of its source text).  From
# the captures of one launch over 64 active 8e/12o tuples (1.9081e+11 flop),
# profiles/k_sigma_ab_8e12o_batch64.md.
TRAFFIC = {"k_gemm_haa": {"bytes_per_flop": (126411008 + 33256448) / 1.9081e11,
                          "sha": "230b4e42ae85e619"},
           "k_sigma_ab": {"bytes_per_flop": (100085760 + 9144576) / 1.9081e11,
                          "sha": "b562c774055038dc"}}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def src_sha(path, kernel=None):
    """sha256 prefix of a source file, or of one kernel's definition in it
    (from its signature line to the first line that is a lone closing brace)
    together with the file's constexpr lines (tile sizes, stages, threads)."""
    text = open(os.path.join(ROOT, path)).read()
    if kernel:
        lines = text.splitlines()
        start = next(i for i, l in enumerate(lines) if l.startswith(kernel + "(")
                     or (" " + kernel + "(") in l and "__global__" in l)
        end = next(i for i in range(start, len(lines)) if lines[i] == "}")
        consts = [l for l in lines if l.startswith("constexpr")]
        text = "\n".join(lines[start:end + 1] + consts)
    return hashlib.sha256(text.encode()).hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample_rate(w, h, eri, ntup_per_order=2, orders=(1, 2, 3), seed=7):
    """The oracle (as it stands) on a seeded sample of the workload's tuples:
    returns (tuples/s, seconds, description, cores)."""
    from oracle import casci as oc
    from oracle import mbe as om
    cores = len(os.sched_getaffinity(0))
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    sample = []
    for k in orders:
        sample += ms.sample_tuples(w["exp"], k, ntup_per_order, seed + k)
    t0 = time.perf_counter()
    per_order = {}
    for t in sample:
        t1 = time.perf_counter()
        oc.casci(h, eri, w["nocc"], om.active_space(w["ref"], t))
        per_order.setdefault(len(t), []).append(time.perf_counter() - t1)
    dt = time.perf_counter() - t0
    desc = (f"{len(sample)} seeded random tuples ({ntup_per_order} each of orders "
            f"{list(orders)}) of {w['name']}, each CASCI solved by the oracle; higher orders "
            f"are larger, so the oracle's rate on the full expansion is lower")
    sec = {k: sum(v) / len(v) for k, v in per_order.items()}
    return len(sample) / dt, dt, desc, cores, sec


def oracle_sigma_seconds(w, h, eri, order, seed=5):
    """Seconds of one oracle sigma vector (Slater-Condon, determinant-driven,
    all host cores) on the CASCI of one seeded tuple of `order` containing
    orbital 0 (the largest bin of that order), and its determinant count."""
    from oracle import casci as oc
    from oracle import mbe as om
    rest = [o for o in w["exp"] if o != 0]
    t = (0,) + ms.sample_tuples(rest, order - 1, 1, seed)[0]
    sp = oc.Space(h, eri, w["nocc"], om.active_space(w["ref"], t))
    c = np.random.default_rng(seed).standard_normal(sp.ndet)
    t0 = time.perf_counter()
    sp.sigma(c)
    return time.perf_counter() - t0, sp.ndet


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = ms.workload(args.workload)
    h, eri, _ = ms.workload_integrals(args.workload)
    for _ in range(args.warmup):
        oracle_sample_rate(w, h, eri, ntup_per_order=1, orders=(1,))
    tot_t, tot_n, desc, cores = 0.0, 0, "", 1
    for s in range(args.steps):
        rate, dt, desc, cores, _ = oracle_sample_rate(w, h, eri, ntup_per_order=1,
                                                      orders=(1, 2, 3), seed=100 + s)
        tot_t += dt
        tot_n += int(round(rate * dt))
    value = tot_n / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_t / max(args.steps, 1), "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "sample": desc},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_fd_check(args):
    """Central differences of the GPU energy against the analytic gradient
    (mbe_energy_backward) on N seeded unique integrals of the differentiation
    workload (8e/20o, CAS(4e,4o) reference, unscreened to order 4, FP64):
    each entry h_pq (with h_qp) or (pq|rs) (with all its images) is moved by
    +-step and the difference quotient compared with the gradient entry.
    Prints one JSON line with the error distribution."""
    from paper_1905_02786_gb300 import build, _binding as B
    build.build()
    B.load_library()
    name = "grad_8e20o"
    w = ms.workload(name)
    h, eri, _ = ms.workload_integrals(name)
    n, P = w["norb"], ms.npair(w["norb"])
    tight = dict(conv_tol_r=1e-11, conv_tol_e=1e-14)
    m = B.MBE(0, keep_ci=1, **tight)
    m.load(h, eri, w["nel"])
    m.run(w["ref"], w["exp"], w["max_order"], 0.0)
    dh, dg = m.backward()
    m.close()
    e0 = B.MBE(0, **tight)

    def energy(h_, e_):
        e0.load(h_, e_, w["nel"])
        return e0.run(w["ref"], w["exp"], w["max_order"], 0.0)["total"]

    rng = np.random.default_rng(args.fd_seed)
    step = args.fd_step
    rows = []
    t0 = time.perf_counter()
    for i in range(args.fd_check):
        if i % 2 == 0:
            p, q = sorted(int(x) for x in rng.integers(0, n, 2))
            hp, hm = h.copy(), h.copy()
            for M, s in ((hp, step), (hm, -step)):
                M[p, q] += s
                if p != q:
                    M[q, p] += s
            fd = (energy(hp, eri) - energy(hm, eri)) / (2 * step)
            an = dh[p, q] * (1 if p == q else 2)
            rows.append(("h", p, q, fd, an))
        else:
            a, b = sorted(int(x) for x in rng.integers(0, P, 2))
            ep, em = eri.copy(), eri.copy()
            for M, s in ((ep, step), (em, -step)):
                M[a, b] += s
                if a != b:
                    M[b, a] += s
            fd = (energy(h, ep) - energy(h, em)) / (2 * step)
            an = dg[a, b] * (1 if a == b else 2)
            rows.append(("eri", a, b, fd, an))
    e0.close()
    err = np.array([abs(r[3] - r[4]) for r in rows])
    mag = np.array([abs(r[4]) for r in rows])
    big = mag >= 0.1
    rel_big = err[big] / mag[big] if big.any() else np.zeros(0)
    out = {"fd_check": len(rows), "workload": name, "step": step, "seed": args.fd_seed,
           "seconds": time.perf_counter() - t0,
           "max_abs_error": float(err.max()), "median_abs_error": float(np.median(err)),
           "entries_with_abs_grad_ge_0.1": int(big.sum()),
           "max_rel_error_abs_grad_ge_0.1": float(rel_big.max()) if big.any() else None,
           "within_1e-6_rel_plus_2e-7": int(np.sum(err <= 1e-6 * mag + 2e-7)),
           "within_1e-6_rel": int(np.sum(err <= 1e-6 * mag)),
           "max_abs_grad": float(mag.max()), "min_abs_grad": float(mag.min()),
           "trace_dh_minus_nel": float(np.trace(dh) - w["nel"])}
    print(json.dumps(out), flush=True)
    return 0


def transfer_bytes(res, h, eri):
    """Bytes that cross the C ABI per expansion: tuples out of next_tuples,
    tuples into solve, energies/status/increments/keep back."""
    h2d = d2h = 0
    for o in res["orders"]:
        n, k = o["tuples"].shape
        d2h += 4 * n * k          # mbe_next_tuples
        h2d += 4 * n * k          # mbe_solve_tuples input
        d2h += 8 * n + 4 * n      # energies + status
        d2h += 8 * n + n + 16     # increments + keep + sums
    return h2d, d2h


def mbe_opts(args) -> dict:
    """--mbe-opt name=value overrides of mbe_options fields (ints or floats);
    --tune-file PATH switches the autotuner on with that cache."""
    out = {}
    for item in args.mbe_opt or []:
        k, v = item.split("=", 1)
        out[k.strip()] = int(v) if v.strip().lstrip("-").isdigit() else float(v)
    if getattr(args, "tune_file", None):
        out["autotune"] = 1
        out["tune_file"] = args.tune_file.encode()
    return out


def opts_json(args) -> dict:
    return {k: (v.decode() if isinstance(v, bytes) else v) for k, v in mbe_opts(args).items()}


def run_profile_batch(args):
    """One mixed batch of seeded order-6 tuples of the 8e/23o workload (all
    with orbital 0: 8e/12o CASCIs, 245,025 determinants; or, with
    --profile-small, all without it: 6e/12o, 48,400), solved inside the NVTX
    range 'solve' after the reference space is set up, so that
    `ncu --nvtx --nvtx-include solve/` captures exactly this batch."""
    import torch
    from paper_1905_02786_gb300 import build, _binding as B
    build.build()
    B.load_library()
    name = "h2o_dz_8e23o"
    w = ms.workload(name)
    h, eri, _ = ms.workload_integrals(name)
    m = B.MBE(0, **{**dict(precision=B.MBE_MIXED_BF16X3, max_batch=4096, timing=1),
                    **mbe_opts(args)})
    m.load(h, eri, w["nel"])
    B.mbe_set_reference(m.ctx, w["ref"], w["exp"])
    rest = [o for o in w["exp"] if o != 0]
    n = args.profile_batch
    if args.profile_small:
        tuples = np.array(ms.sample_tuples(rest, 6, n, 13), dtype=np.int32)
    else:
        tuples = np.array([(0,) + t for t in ms.sample_tuples(rest, 5, n, 12)], dtype=np.int32)
    B.mbe_reset_stats(m.ctx)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("solve")
    t0 = time.perf_counter()
    eps, _ = B.mbe_solve_tuples(m.ctx, tuples, 6)
    dt = time.perf_counter() - t0
    torch.cuda.nvtx.range_pop()
    st = B.mbe_get_stats(m.ctx)
    print(json.dumps({"profile_batch": n, "cas": "6e/12o" if args.profile_small else "8e/12o",
                      "options": opts_json(args), "seconds": dt, "tuples_per_s": n / dt,
                      "eps": [float(e) for e in eps],
                      "tc_tflops": st["dom_flops"] / st["dom_ms"] / 1e9 if st["dom_ms"] else None,
                      "stats": st}))
    m.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--max-order", type=int, default=None)
    ap.add_argument("--max-batch", type=int, default=4096)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--mbe-opt", action="append", default=None, metavar="NAME=VALUE",
                    help="override an mbe_options field (repeatable), e.g. max_subspace=12")
    ap.add_argument("--tune-file", default=None,
                    help="autotune the two-spin tensor-core sigma, caching plans in this file")
    ap.add_argument("--fd-check", type=int, default=0,
                    help="finite-difference check of the energy gradient on this many "
                         "seeded unique integrals of the differentiation workload")
    ap.add_argument("--fd-step", type=float, default=1e-5)
    ap.add_argument("--fd-seed", type=int, default=3)
    ap.add_argument("--backward", action="store_true",
                    help="keep the CI vectors and run the energy backward (dE/dh, "
                         "dE/d(pq|rs)) inside every step")
    ap.add_argument("--profile-batch", type=int, default=0,
                    help="profiling case instead of the bench: solve this many seeded "
                         "order-6 tuples of the workload as one batch inside the NVTX "
                         "range 'solve' and print its counters")
    ap.add_argument("--profile-small", action="store_true",
                    help="with --profile-batch: tuples without orbital 0 (6e/12o "
                         "CASCIs) instead of tuples with it (8e/12o)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_batch:
        return run_profile_batch(args)
    if args.fd_check:
        return run_fd_check(args)

    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1905_02786_gb300 import build, _binding as B, driver
    build.build()
    B.load_library()

    w = ms.workload(args.workload)
    h, eri, _ = ms.workload_integrals(args.workload)
    max_order = args.max_order or w["max_order"]
    prec = B.MBE_MIXED_BF16X3 if args.precision == "mixed" else B.MBE_FP64
    m = B.MBE(local, **{**dict(precision=prec, max_batch=args.max_batch, timing=1,
                               keep_ci=1 if args.backward else 0,
                               backward_share=(2 if rank == 0 else 1) if world > 1 else 0),
                        **mbe_opts(args)})
    stream = torch.cuda.Stream()
    B.mbe_set_stream(m.ctx, stream.cuda_stream)
    m.load(h, eri, w["nel"])
    allgather = driver.torch_allgather() if world > 1 else None
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    order_s = []
    bwd_s = []

    def step():
        # host-side seconds per order (the solve returns its energies to the
        # host, so each order ends synchronised): a breakdown, not the metric
        order_s.clear()
        t_last = [time.perf_counter()]

        def mark(rec):
            t = time.perf_counter()
            order_s.append({"order": rec["order"], "tuples": len(rec["tuples"]),
                            "s": round(t - t_last[0], 4)})
            t_last[0] = t

        res = driver.run_expansion(m.ctx, w["ref"], w["exp"], max_order, w["thr"], rank, world,
                                   allgather, callback=mark, nocc=w["nocc"])
        if args.backward:
            t0 = time.perf_counter()
            driver.sharded_backward(m.ctx, w["norb"], rank, world,
                                    driver.torch_allreduce_sum() if world > 1 else None)
            bwd_s.append(time.perf_counter() - t0)
        return res

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        m.load(h, eri, w["nel"])
        res = step()
    # timed region: K steps.  A step uploads the integrals through the C ABI
    # (host buffers) and runs the whole expansion, whose per-order arrays
    # (tuples in, energies / increments out) cross to and from the host inside
    # it.  value = tuples / time from the end of the upload (inputs resident)
    # to the end of the step; e2e = tuples / time of the whole step.  The L2
    # is flushed before each step, outside both regions.
    B.mbe_reset_stats(m.ctx)
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    ntup = 0
    t_ms = 0.0
    e2e_ms = 0.0
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            flush.fill_(1.0)
            ea, eb, ec = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            torch.cuda.nvtx.range_push("timed_step")
            ea.record(stream)
            m.load(h, eri, w["nel"])
            eb.record(stream)
            res = step()
            ec.record(stream)
            torch.cuda.nvtx.range_pop()
            ntup += res["ntup"]
            ec.synchronize()
            t_ms += eb.elapsed_time(ec)
            e2e_ms += ea.elapsed_time(ec)
    barrier()
    clk = clocks.stop()
    if world > 1:
        t = torch.tensor([t_ms, e2e_ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_ms, e2e_ms = float(t[0].item()), float(t[1].item())
    st = B.mbe_get_stats(m.ctx)
    value = ntup / (t_ms / 1e3)
    h2d, d2h = transfer_bytes(res, h, eri)
    h2d += h.nbytes + eri.nbytes
    e2e = {"value": ntup / (e2e_ms / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    pk, pk_kind = peaks()
    # FP64 / FP32 FMA rates of this GPU, measured by the library's probe
    fp_peaks = B.mbe_measure_peaks(local)
    if prec == B.MBE_FP64:
        dom_ms_per = st["fp64_ms"] / max(st["fp64_launches"], 1)
        dom_flops_per = st["fp64_flops"] / max(st["fp64_launches"], 1)
        dom_launches = st["fp64_launches"]
    else:
        dom_ms_per = st["dom_ms"] / max(st["dom_launches"], 1)
        dom_flops_per = st["dom_flops"] / max(st["dom_launches"], 1)
        dom_launches = st["dom_launches"]
    achieved_tf = dom_flops_per / (dom_ms_per * 1e-3) / 1e12 if dom_ms_per > 0 else None
    if prec == B.MBE_FP64:
        kname = "k_contract_fp64"
        peak_tf = fp_peaks["fp64_tflops"]
        peak_src = "FP64 FMA, measured by mbe_measure_peaks on this GPU"
        bound = "alu"
        ksrc = "paper_1905_02786_gb300/csrc/mbe_ci.cu"
    else:
        # the sigma contraction: k_gemm_haa (one-spin part) + k_sigma_ab
        # (two-spin part), timed together with CUDA events on the library's
        # stream; algorithmic flops 2 N_det npair^2 per sigma vector
        kname = "k_gemm_haa+k_sigma_ab"
        peak_tf = pk.get("bf16_tflops_sustained", 1700.0)
        peak_src = f"bf16 dense sustained, {pk_kind}"
        bound = "tensor"
        ksrc = "paper_1905_02786_gb300/csrc/mbe_sigma_tc.cu"
    # DRAM bytes per algorithmic flop from one ncu capture of the kernels
    # (8e/12o batch of 64 tuples, bench --profile-batch 64), scaled to this
    # run's average launch; null once a kernel source has changed
    traffic = 0.0
    for kn in kname.split("+"):
        tr = TRAFFIC.get(kn)
        if not tr or tr["sha"] != src_sha(ksrc, kn):
            traffic = None
            break
        traffic += tr["bytes_per_flop"] * dom_flops_per
    roofline = {"bound": bound, "kernel": kname, "achieved": achieved_tf, "peak": peak_tf,
                "unit": "TFLOP/s", "frac": (achieved_tf / peak_tf) if achieved_tf else None,
                "traffic": traffic, "peak_source": peak_src,
                "flops_per_launch": dom_flops_per, "ms_per_launch": dom_ms_per,
                "launches": dom_launches,
                "kernel_ms_total": dom_ms_per * dom_launches, "step_ms_total": t_ms}

    # plain FP64 GPU path, one tuple at a time, vs the mixed batched path on
    # the same bounded samples: seeded tuples of orders 5 and 6 (the orders
    # that dominate the step; half of them with orbital 0, i.e. the 8-electron
    # CASCIs) and of orders 2-4
    cmp = None
    if rank == 0 and not args.no_fp64_compare:
        rest = [o for o in w["exp"] if o != 0]

        def high(k, n, seed):
            with0 = [(0,) + t for t in ms.sample_tuples(rest, k - 1, n // 2, seed)]
            return np.array(with0 + ms.sample_tuples(rest, k, n - n // 2, seed + 50),
                            dtype=np.int32)

        samples = {
            "orders_5_6": ({5: high(5, 8, 501), 6: high(6, 8, 601)},
                           "8 seeded tuples each of orders 5 and 6 (4 with orbital 0: 8e/11o "
                           "and 8e/12o CASCIs; 4 without: 6e/11o and 6e/12o) of " + args.workload),
            "orders_2_4": ({k: np.array(ms.sample_tuples(w["exp"], k, 8, 300 + k), dtype=np.int32)
                            for k in (2, 3, 4)},
                           "8 seeded random tuples each of orders 2, 3, 4 of " + args.workload)}
        cmp = {}
        for key, (sample, desc) in samples.items():
            rates = {}
            for label, opts in (("fp64_one_tuple", dict(precision=B.MBE_FP64, max_batch=1)),
                                ("mixed_batched", dict(precision=B.MBE_MIXED_BF16X3,
                                                       max_batch=args.max_batch))):
                mm = B.MBE(local, timing=1, **opts)
                mm.load(h, eri, w["nel"])
                B.mbe_set_reference(mm.ctx, w["ref"], w["exp"])
                B.mbe_reset_stats(mm.ctx)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                nt = 0
                for k, tk in sample.items():
                    B.mbe_solve_tuples(mm.ctx, tk, k)
                    nt += len(tk)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                s2 = B.mbe_get_stats(mm.ctx)
                rates[label] = {"value": nt / dt, "unit": UNIT, "tuples": nt,
                                "sigma_tflops_tensor_core": (s2["dom_flops"] / (s2["dom_ms"] * 1e-3)
                                                             / 1e12) if s2["dom_ms"] else None,
                                "sigma_tflops_fp64": (s2["fp64_flops"] / (s2["fp64_ms"] * 1e-3)
                                                      / 1e12) if s2["fp64_ms"] else None}
                mm.close()
            rates["speedup"] = rates["mixed_batched"]["value"] / rates["fp64_one_tuple"]["value"]
            rates["sample"] = desc
            cmp[key] = rates

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, dt, desc, cores, sec = oracle_sample_rate(w, h, eri)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
               "seconds": dt, "oracle_seconds_per_casci_by_order": sec}
        if args.workload == DEFAULT_WORKLOAD:
            # the CASCIs that dominate the step are too large for the oracle's
            # Davidson within the bench: one oracle sigma vector of an order-6
            # 8e/12o CASCI is timed instead, beside the GPU's sigma vectors
            sg_s, sg_ndet = oracle_sigma_seconds(w, h, eri, 6)
            cpu["oracle_sigma_vector_s"] = {"order": 6, "ndet": sg_ndet, "seconds": sg_s}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": t_ms / args.steps, "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None,
                "dtype": "f64" if prec == B.MBE_FP64 else "bf16x3(f32 acc)+f64",
                "data": "synthetic",
                "config": {"workload": args.workload, "norb": w["norb"], "nelec": w["nel"],
                           "reference": f"CAS({2 * sum(1 for r in w['ref'] if r < w['nocc'])}e,"
                                        f"{len(w['ref'])}o)",
                           "expansion_orbitals": len(w["exp"]), "max_order": max_order,
                           "screen_thr": w["thr"], "precision": args.precision,
                           "tuples_per_step": ntup // args.steps,
                           "l2": "256 MiB buffer written before each step (flushed); "
                                 "Davidson working set exceeds L2",
                           "parallelism": f"tuple-sharded x{world}" if world > 1 else "1 GPU",
                           **({"options": opts_json(args)}
                              if (args.mbe_opt or args.tune_file) else {})},
                "sigma_tflops": {
                    "tensor_core": (st["dom_flops"] / (st["dom_ms"] * 1e-3) / 1e12)
                    if st["dom_ms"] else None,
                    "fp64": (st["fp64_flops"] / (st["fp64_ms"] * 1e-3) / 1e12)
                    if st["fp64_ms"] else None,
                    "tensor_core_ms": st["dom_ms"], "fp64_ms": st["fp64_ms"],
                    "tensor_core_vectors_per_casci": st["dom_flops"] / max(st["sigma_flops"], 1)
                    * st["sigma_vectors"] / max(st["casci"], 1),
                    "fp64_vectors_per_casci": st["fp64_flops"] / max(st["sigma_flops"], 1)
                    * st["sigma_vectors"] / max(st["casci"], 1)},
                "davidson_iters_mean": st["iters_total"] / max(st["casci"], 1),
                "seconds_per_order": list(order_s),
                "backward_s_per_step": (sum(bwd_s[-args.steps:]) / args.steps) if bwd_s else None,
                "noconv": st["noconv"],
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "measured_fp_peaks": fp_peaks,
                "mixed_vs_fp64_gpu": cmp,
                "gpu_launches": int(st["launches"]),
                "host_launches": int(st["host_launches"]),
                "graph_launches": int(st["graph_launches"]), "clocks": clk,
                "total_energy": res["total"]}
        print(json.dumps(line), flush=True)
    m.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

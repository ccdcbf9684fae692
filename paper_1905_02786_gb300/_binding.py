"""Thin ctypes binding of libmbe (include/mbe.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts NumPy
arrays to pointers, checks return codes and raises ``MBEError`` with the
library's message.  The library must have been built
(``paper_1905_02786_gb300.build.build()``); a missing library raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libmbe.so")

MBE_OK, MBE_EINVAL, MBE_ENOMEM, MBE_ECUDA, MBE_ENOCONV, MBE_ELOOKUP, MBE_ESTATE, MBE_ETIMEOUT = \
    0, -1, -2, -3, -4, -5, -6, -7
MBE_FP64, MBE_MIXED_BF16X3, MBE_EMULATED_FP64 = 0, 1, 2
ERROR_NAMES = {0: "MBE_OK", -1: "MBE_EINVAL", -2: "MBE_ENOMEM", -3: "MBE_ECUDA",
               -4: "MBE_ENOCONV", -5: "MBE_ELOOKUP", -6: "MBE_ESTATE", -7: "MBE_ETIMEOUT"}

EXPORTED = ["mbe_default_options", "mbe_create", "mbe_destroy", "mbe_last_error",
            "mbe_load_integrals", "mbe_set_reference", "mbe_solve_tuples",
            "mbe_increments", "mbe_next_tuples", "mbe_energy_backward", "mbe_sigma",
            "mbe_get_stats", "mbe_reset_stats", "mbe_set_order_energies", "mbe_set_stream",
            "mbe_sigma_noalloc", "mbe_measure_peaks", "mbe_set_pruning_pairs",
            "mbe_set_spin"]


class MBEError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


class mbe_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("max_batch", ctypes.c_int),
                ("max_subspace", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("conv_tol_r", ctypes.c_double), ("conv_tol_e", ctypes.c_double),
                ("spin_shift", ctypes.c_double), ("keep_ci", ctypes.c_int),
                ("deterministic", ctypes.c_int), ("mem_cap_bytes", ctypes.c_int64),
                ("timing", ctypes.c_int), ("verbose", ctypes.c_int),
                ("backward_share", ctypes.c_int), ("warm_start", ctypes.c_int),
                ("mixed_stage_tol", ctypes.c_double), ("mixed_round_drop", ctypes.c_double),
                ("mixed_rel_tol", ctypes.c_double), ("pspace", ctypes.c_int),
                ("wait_limit", ctypes.c_int64), ("autotune", ctypes.c_int),
                ("tune_file", ctypes.c_char_p), ("graphs", ctypes.c_int)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libmbe.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"libmbe.so not found at {path}: run paper_1905_02786_gb300.build.build()")
    L = ctypes.CDLL(path)
    c_int, c_double, c_i64 = ctypes.c_int, ctypes.c_double, ctypes.c_int64
    vp = ctypes.c_void_p
    L.mbe_default_options.argtypes = [ctypes.POINTER(mbe_options)]
    L.mbe_default_options.restype = None
    L.mbe_create.argtypes = [ctypes.POINTER(vp), c_int, ctypes.POINTER(mbe_options)]
    L.mbe_destroy.argtypes = [vp]
    L.mbe_destroy.restype = None
    L.mbe_last_error.argtypes = [vp]
    L.mbe_last_error.restype = ctypes.c_char_p
    L.mbe_load_integrals.argtypes = [vp, c_int, c_int, vp, vp]
    L.mbe_set_reference.argtypes = [vp, vp, c_int, vp, c_int, vp]
    L.mbe_solve_tuples.argtypes = [vp, c_int, vp, c_i64, vp, vp]
    L.mbe_increments.argtypes = [vp, c_int, c_double, vp, vp, vp, vp]
    L.mbe_next_tuples.argtypes = [vp, c_int, vp, c_i64, vp]
    L.mbe_energy_backward.argtypes = [vp, c_double, vp, vp]
    L.mbe_sigma.argtypes = [vp, vp, c_int, vp, vp, vp]
    L.mbe_sigma_noalloc.argtypes = [vp, vp, c_int, vp, vp, ctypes.c_int64, vp]
    L.mbe_measure_peaks.argtypes = [c_int, vp, vp]
    L.mbe_set_pruning_pairs.argtypes = [vp, vp, c_int]
    L.mbe_set_spin.argtypes = [vp, c_int]
    for name in EXPORTED:
        if name not in ("mbe_default_options", "mbe_destroy", "mbe_last_error",
                        "mbe_get_stats", "mbe_reset_stats", "mbe_set_order_energies",
                        "mbe_set_stream"):
            getattr(L, name).restype = c_int
    _lib = L
    return L


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(ctx, rc, allow=()):
    if rc != MBE_OK and rc not in allow:
        msg = load_library().mbe_last_error(ctx).decode() if ctx else "no context"
        raise MBEError(rc, msg)
    return rc


def mbe_default_options(**overrides) -> mbe_options:
    """The library's defaults, with the named fields replaced."""
    o = mbe_options()
    load_library().mbe_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def mbe_create(device: int = 0, options: mbe_options | None = None):
    L = load_library()
    h = ctypes.c_void_p()
    rc = L.mbe_create(ctypes.byref(h), device, ctypes.byref(options) if options else None)
    if rc != MBE_OK:
        raise MBEError(rc, "mbe_create failed")
    return h


def mbe_destroy(ctx):
    load_library().mbe_destroy(ctx)


def mbe_last_error(ctx) -> str:
    return load_library().mbe_last_error(ctx).decode()


def mbe_load_integrals(ctx, h, eri, nelec: int):
    h = np.ascontiguousarray(h, dtype=np.float64)
    eri = np.ascontiguousarray(eri, dtype=np.float64)
    norb = h.shape[0]
    return _check(ctx, load_library().mbe_load_integrals(ctx, norb, int(nelec), _p(h), _p(eri)))


def mbe_set_reference(ctx, ref, exp) -> float:
    ref = np.ascontiguousarray(ref, dtype=np.int32)
    exp = np.ascontiguousarray(exp, dtype=np.int32)
    e = np.zeros(1)
    _check(ctx, load_library().mbe_set_reference(ctx, _p(ref), ref.size, _p(exp), exp.size, _p(e)))
    return float(e[0])


def mbe_solve_tuples(ctx, tuples, order: int | None = None, allow_noconv=False):
    t = np.ascontiguousarray(tuples, dtype=np.int32)
    if t.ndim == 1:
        t = t.reshape(-1, order or 1)
    ntup, order = t.shape[0], (order or t.shape[1])
    eps = np.zeros(ntup)
    st = np.zeros(ntup, dtype=np.int32)
    _check(ctx, load_library().mbe_solve_tuples(ctx, order, _p(t), ntup, _p(eps), _p(st)),
           allow=(MBE_ENOCONV,) if allow_noconv else ())
    return eps, st


def mbe_increments(ctx, order: int, screen_thr: float, ntup: int):
    inc = np.zeros(max(ntup, 1))
    keep = np.zeros(max(ntup, 1), dtype=np.uint8)
    eo = np.zeros(1)
    et = np.zeros(1)
    _check(ctx, load_library().mbe_increments(ctx, order, float(screen_thr), _p(inc), _p(keep),
                                              _p(eo), _p(et)))
    return inc[:ntup], keep[:ntup].astype(bool), float(eo[0]), float(et[0])


def mbe_next_tuples(ctx, order: int):
    n = np.zeros(1, dtype=np.int64)
    L = load_library()
    _check(ctx, L.mbe_next_tuples(ctx, order, None, 0, _p(n)))
    out = np.zeros((max(int(n[0]), 1), order), dtype=np.int32)
    _check(ctx, L.mbe_next_tuples(ctx, order, _p(out), int(n[0]), _p(n)))
    return out[: int(n[0])]


def mbe_energy_backward(ctx, norb: int, scale: float = 1.0):
    npair = norb * (norb + 1) // 2
    dh = np.zeros((norb, norb))
    dg = np.zeros((npair, npair))
    _check(ctx, load_library().mbe_energy_backward(ctx, float(scale), _p(dh), _p(dg)))
    return dh, dg


def mbe_sigma(ctx, act, c):
    act = np.ascontiguousarray(sorted(act), dtype=np.int32)
    c = np.ascontiguousarray(c, dtype=np.float64).ravel()
    sig = np.zeros_like(c)
    ec = np.zeros(1)
    _check(ctx, load_library().mbe_sigma(ctx, _p(act), act.size, _p(c), _p(sig), _p(ec)))
    return sig, float(ec[0])


def mbe_sigma_noalloc(ctx, act, c_dev, sigma_dev, want_core=True):
    """FP64 sigma without device allocation.  c_dev and sigma_dev are CUDA
    float64 tensors (nstr*nstr elements, contiguous) on the context's device;
    sigma_dev is overwritten.  Returns the inactive-core energy if want_core
    (the call then waits for the context stream), else None."""
    act = np.ascontiguousarray(sorted(act), dtype=np.int32)
    for t in (c_dev, sigma_dev):
        if not (t.is_cuda and t.dtype.is_floating_point and t.element_size() == 8
                and t.is_contiguous()):
            raise TypeError("c_dev and sigma_dev must be contiguous CUDA float64 tensors")
    if c_dev.numel() != sigma_dev.numel():
        raise ValueError("c_dev and sigma_dev differ in size")
    ec = np.zeros(1)
    _check(ctx, load_library().mbe_sigma_noalloc(ctx, _p(act), act.size,
                                                 ctypes.c_void_p(c_dev.data_ptr()),
                                                 ctypes.c_void_p(sigma_dev.data_ptr()),
                                                 c_dev.numel(), _p(ec) if want_core else None))
    return float(ec[0]) if want_core else None


class MBE:
    """Convenience owner of one context; runs whole expansions through the
    C ABI (host loop over orders: next tuples -> solve -> increments)."""

    def __init__(self, device=0, **opts):
        o = mbe_default_options()
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown option {k}")
            setattr(o, k, v)
        self.options = o
        self.ctx = mbe_create(device, o)

    def close(self):
        if self.ctx:
            mbe_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, h, eri, nelec, two_sz=None):
        mbe_load_integrals(self.ctx, h, eri, nelec)
        if two_sz is not None:
            mbe_set_spin(self.ctx, two_sz)
        self.norb = h.shape[0]

    def run(self, ref, exp, max_order, thr=0.0, callback=None, pairs=None):
        """Full expansion (pi-pruned over ``pairs`` if given); returns
        dict(eps_ref, orders=[...], total)."""
        e_ref = mbe_set_reference(self.ctx, ref, exp)
        if pairs:
            mbe_set_pruning_pairs(self.ctx, pairs)
        orders = []
        total = e_ref
        empty_run = 0
        for k in range(1, max_order + 1):
            tuples = mbe_next_tuples(self.ctx, k)
            if len(tuples) == 0:
                # a pair adds two orbitals: with pruning an empty order can
                # precede a non-empty one, two empty orders end the expansion
                empty_run += 1
                if empty_run >= (2 if pairs else 1):
                    break
            else:
                empty_run = 0
            eps, st = mbe_solve_tuples(self.ctx, tuples.reshape(-1, k), k)
            inc, keep, e_order, total = mbe_increments(self.ctx, k, thr, len(tuples))
            rec = dict(order=k, tuples=tuples, eps=eps, status=st, inc=inc, keep=keep,
                       E_order=e_order)
            orders.append(rec)
            if callback:
                callback(rec)
        return dict(eps_ref=e_ref, orders=orders, total=total)

    def backward(self, scale=1.0):
        """dE/dh (norb x norb) and dE/d eri_packed (npair x npair) of the
        expansion run last (needs keep_ci=1)."""
        return mbe_energy_backward(self.ctx, self.norb, scale)


class mbe_stats(ctypes.Structure):
    _fields_ = [("casci", ctypes.c_int64), ("sigma_vectors", ctypes.c_int64),
                ("sigma_flops", ctypes.c_double), ("iters_total", ctypes.c_int64),
                ("iters_max", ctypes.c_int64), ("noconv", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("dom_launches", ctypes.c_int64),
                ("dom_ms", ctypes.c_double), ("dom_flops", ctypes.c_double),
                ("fp64_launches", ctypes.c_int64), ("fp64_ms", ctypes.c_double),
                ("fp64_flops", ctypes.c_double), ("host_launches", ctypes.c_int64),
                ("graph_launches", ctypes.c_int64), ("graph_builds", ctypes.c_int64)]


def mbe_set_order_energies(ctx, tuples, eps, order: int | None = None):
    t = np.ascontiguousarray(tuples, dtype=np.int32)
    if t.ndim == 1:
        t = t.reshape(-1, order or 1)
    e = np.ascontiguousarray(eps, dtype=np.float64)
    L = load_library()
    L.mbe_set_order_energies.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                         ctypes.c_int64, ctypes.c_void_p]
    _check(ctx, L.mbe_set_order_energies(ctx, order or t.shape[1], _p(t), t.shape[0], _p(e)))


def mbe_get_stats(ctx) -> dict:
    s = mbe_stats()
    L = load_library()
    L.mbe_get_stats.argtypes = [ctypes.c_void_p, ctypes.POINTER(mbe_stats)]
    _check(ctx, L.mbe_get_stats(ctx, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in mbe_stats._fields_}


def mbe_reset_stats(ctx):
    L = load_library()
    L.mbe_reset_stats.argtypes = [ctypes.c_void_p]
    _check(ctx, L.mbe_reset_stats(ctx))


def mbe_set_stream(ctx, stream_handle):
    """Issue the context's work on a caller-owned cudaStream_t (an int handle,
    e.g. torch.cuda.Stream().cuda_stream); 0/None restores its own stream."""
    L = load_library()
    L.mbe_set_stream.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    _check(ctx, L.mbe_set_stream(ctx, ctypes.c_void_p(stream_handle or None)))


def mbe_measure_peaks(device: int = 0) -> dict:
    """FP64 and FP32 FMA peaks (TFLOP/s) of the device, measured by the
    library's probe kernels."""
    out = np.zeros(2)
    rc = load_library().mbe_measure_peaks(int(device), _p(out[:1]), _p(out[1:]))
    if rc != MBE_OK:
        raise MBEError(rc, "mbe_measure_peaks failed")
    return {"fp64_tflops": float(out[0]), "fp32_tflops": float(out[1])}


def mbe_set_spin(ctx, two_sz: int):
    """High-spin reference determinant with n_alpha - n_beta = two_sz (Fig. 2 (b))."""
    return _check(ctx, load_library().mbe_set_spin(ctx, int(two_sz)))


def mbe_set_pruning_pairs(ctx, pairs):
    """pi-pruning over pairs of degenerate expansion orbitals (Sec. 3)."""
    pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    return _check(ctx, load_library().mbe_set_pruning_pairs(ctx, _p(pr) if pr.size else None,
                                                            pr.shape[0]))

"""Oracle (test infrastructure only): CASCI of one orbital tuple.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs may import this package.  It shares no code with the
CUDA path.

What it computes (Sec. 2, the paragraphs around Eqs. 1-3 and Fig. 2): for a
tuple of expansion orbitals the active space is the reference space plus the
tuple; occupied orbitals outside it stay doubly occupied (inactive), virtual
orbitals outside it are deleted, and the CASCI energy is the lowest
eigenvalue of H in the determinant space of the active electrons.  Here the
determinants live in the FULL orbital space (core bits set, deleted bits
clear) and the matrix elements are the Slater-Condon rules of ``sc_fci.c``,
so the energy is the total electronic energy including the inactive core.

Target state, closed-shell reference (``nocc`` an int: orbitals below it
doubly occupied): the lowest singlet (S = 0).  It lies in the subspace
C[Ia, Ib] = C[Ib, Ia] (alpha <-> beta exchange symmetric, Ms = 0) of the
determinant convention a+_{alpha string} a+_{beta string}|0>, which holds
the even-S states; the synthetic integrals often put a quintet below the
lowest singlet there, so the singlet is selected explicitly.

High-spin open-shell reference (Fig. 2 case (b); ``nocc`` a pair
(n_alpha, n_beta), n_alpha > n_beta: orbitals below n_beta doubly occupied,
those from n_beta to n_alpha - 1 singly occupied by alpha electrons): the
determinant space has Ms = (n_alpha - n_beta) / 2 and the target is the
lowest state with S = Ms.  The singly occupied orbitals must be active (the
inactive core stays closed-shell); the space is the full alpha-string x
beta-string product, with no alpha <-> beta symmetry.

Solvers: dense ``numpy.linalg.eigh`` of the projected symmetric-subspace
matrix for up to 5000 determinants, taking the lowest eigenvector whose
<S^2> is below 1/2; otherwise a textbook Davidson iteration (Davidson,
J. Comput. Phys. 17, 87 (1975)) on H + SPIN_SHIFT * S^2 in the symmetric
subspace (the shift lifts every S >= 2 state by at least 6 * SPIN_SHIFT and
leaves singlet energies unchanged), FP64 throughout, stopped when
|dE| < 1e-13 and ||r|| < 1e-8; the energy returned is the unshifted
Rayleigh quotient c.Hc.
"""
from __future__ import annotations

import ctypes
import itertools

import numpy as np

from .build_oracle import build

_lib = None
DENSE_MAX = 5000
SPIN_SHIFT = 0.5


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        up = ctypes.POINTER(ctypes.c_uint64)
        i, l = ctypes.c_int, ctypes.c_long
        L.oracle_hdiag.argtypes = [i, dp, dp, l, up, l, up, dp]
        L.oracle_sigma.argtypes = [i, dp, dp, l, up, l, up, dp, dp]
        L.oracle_sigma_rows.argtypes = [i, dp, dp, l, up, l, up, dp, l,
                                        ctypes.POINTER(ctypes.c_long), dp]
        L.oracle_hdense.argtypes = [i, dp, dp, l, up, l, up, dp]
        L.oracle_rdm12.argtypes = [i, l, up, l, up, dp, dp, dp]
        L.oracle_s2.argtypes = [i, l, up, l, up, dp, dp, dp]
        for f in (L.oracle_hdiag, L.oracle_sigma, L.oracle_sigma_rows, L.oracle_hdense,
                  L.oracle_rdm12, L.oracle_s2):
            f.restype = None
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _up(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def occ_pair(nocc):
    """(n_alpha, n_beta) occupied orbitals of the reference determinant."""
    if isinstance(nocc, (tuple, list)):
        na, nb = int(nocc[0]), int(nocc[1])
        if na < nb or nb < 0:
            raise ValueError("high-spin reference needs n_alpha >= n_beta >= 0")
        return na, nb
    return int(nocc), int(nocc)


def tuple_strings(nocc: int, act):
    """Sorted full-space strings of one spin for the CASCI of ``act``.

    Returns ``(strs, nsig)``: ``strs`` is an (N, 2) uint64 array of
    (lo, hi) orbital bit masks, ``nsig`` the active electrons per spin.
    """
    act = sorted(set(int(a) for a in act))
    core = [i for i in range(nocc) if i not in act]
    nsig = sum(1 for a in act if a < nocc)
    corebits = 0
    for i in core:
        corebits |= 1 << i
    vals = []
    for comb in itertools.combinations(act, nsig):
        v = corebits
        for p in comb:
            v |= 1 << p
        vals.append(v)
    vals.sort()
    mask = (1 << 64) - 1
    strs = np.array([[v & mask, v >> 64] for v in vals], dtype=np.uint64).reshape(-1, 2)
    return np.ascontiguousarray(strs), nsig


class Space:
    """Determinant space (alpha strings x beta strings) with the integrals.

    ``nocc``: an int (closed shell) or (n_alpha, n_beta) (high spin)."""

    def __init__(self, h, eri, nocc, act):
        self.h = np.ascontiguousarray(h, dtype=np.float64)
        self.eri = np.ascontiguousarray(eri, dtype=np.float64)
        self.norb = self.h.shape[0]
        na, nb = occ_pair(nocc)
        act_set = set(int(a) for a in act)
        if any(o not in act_set for o in range(nb, na)):
            raise ValueError("singly occupied orbitals must be active")
        self.astrs, self.nsig = tuple_strings(na, act)
        self.bstrs, self.nsigb = tuple_strings(nb, act)
        self.strs = self.astrs
        self.nstr = self.astrs.shape[0]
        self.nstrb = self.bstrs.shape[0]
        self.ndet = self.nstr * self.nstrb
        # Ms of every determinant of the space
        self.ms = 0.5 * (self.nsig - self.nsigb)

    def _args(self):
        return (self.nstr, _up(self.astrs), self.nstrb, _up(self.bstrs))

    def hdiag(self):
        out = np.empty(self.ndet)
        lib().oracle_hdiag(self.norb, _dp(self.h), _dp(self.eri), *self._args(), _dp(out))
        return out

    def sigma(self, c):
        c = np.ascontiguousarray(c, dtype=np.float64).ravel()
        out = np.empty(self.ndet)
        lib().oracle_sigma(self.norb, _dp(self.h), _dp(self.eri), *self._args(), _dp(c),
                           _dp(out))
        return out

    def sigma_rows(self, c, rows):
        """(H c)_I for the determinant indices I in ``rows`` only."""
        c = np.ascontiguousarray(c, dtype=np.float64).ravel()
        rows = np.ascontiguousarray(rows, dtype=np.int64).ravel()
        if rows.size and (rows.min() < 0 or rows.max() >= self.ndet):
            raise ValueError("row index out of range")
        out = np.empty(rows.size)
        lib().oracle_sigma_rows(self.norb, _dp(self.h), _dp(self.eri), *self._args(), _dp(c),
                                rows.size, rows.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                                _dp(out))
        return out

    def hdense(self):
        H = np.empty((self.ndet, self.ndet))
        lib().oracle_hdense(self.norb, _dp(self.h), _dp(self.eri), *self._args(), _dp(H))
        return H

    def s2(self, c):
        """S^2 c = S- S+ c + Ms (Ms + 1) c."""
        c = np.ascontiguousarray(c, dtype=np.float64).ravel()
        out = np.empty(self.ndet)
        lib().oracle_s2(self.norb, *self._args(), _dp(c), _dp(out), None)
        return out + self.ms * (self.ms + 1.0) * c

    def s2diag(self):
        out = np.empty(self.ndet)
        lib().oracle_s2(self.norb, *self._args(), None, None, _dp(out))
        return out + self.ms * (self.ms + 1.0)

    def rdm12(self, c):
        c = np.ascontiguousarray(c, dtype=np.float64).ravel()
        n = self.norb
        g1 = np.empty((n, n))
        g2 = np.empty((n, n, n, n))
        lib().oracle_rdm12(n, *self._args(), _dp(c), _dp(g1), _dp(g2))
        return g1, g2

    def sym_basis(self):
        """Orthonormal basis of the C[a,b] = C[b,a] subspace (ndet x nsym)."""
        n = self.nstr
        cols = n * (n + 1) // 2
        P = np.zeros((self.ndet, cols))
        k = 0
        for a in range(n):
            for b in range(a + 1):
                if a == b:
                    P[a * n + a, k] = 1.0
                else:
                    P[a * n + b, k] = P[b * n + a, k] = np.sqrt(0.5)
                k += 1
        return P


def _symmetrize(v, n):
    m = v.reshape(n, n)
    return (0.5 * (m + m.T)).ravel()


def davidson(space: Space, tol_r=1e-8, tol_e=1e-13, max_iter=300, max_space=30,
             guess=None, spin_shift=SPIN_SHIFT):
    """Lowest root of H + spin_shift * S^2, in the symmetric subspace for a
    closed-shell space (in the whole space for a high-spin one); returns
    (E, c, iters) with E = c.Hc of the normalised root."""
    n = space.nstr
    sym = space.ms == 0
    proj = (lambda v: _symmetrize(v, n)) if sym else (lambda v: v)
    hd = space.hdiag()
    if spin_shift:
        hd = hd + spin_shift * space.s2diag()

    def op(v):
        out = space.sigma(v)
        if spin_shift:
            out += spin_shift * space.s2(v)
        return out

    if guess is None:
        i0 = int(np.argmin(hd))
        x0 = np.zeros(space.ndet)
        if sym:
            a, b = divmod(i0, n)
            x0[a * n + b] += 1.0
            x0[b * n + a] += 1.0
        else:
            x0[i0] = 1.0
    else:
        x0 = np.array(guess, dtype=np.float64).ravel()
    x0 = proj(x0)
    x0 /= np.linalg.norm(x0)
    V = [x0]
    S = [op(x0)]
    e_old = None
    for it in range(1, max_iter + 1):
        Vm = np.array(V)
        Sm = np.array(S)
        G = Vm @ Sm.T
        G = 0.5 * (G + G.T)
        w, Y = np.linalg.eigh(G)
        theta, y = w[0], Y[:, 0]
        x = y @ Vm
        ax = y @ Sm
        r = ax - theta * x
        rn = np.linalg.norm(r)
        if e_old is not None and abs(theta - e_old) < tol_e and rn < tol_r:
            x = x / np.linalg.norm(x)
            return float(x @ space.sigma(x)), x, it
        e_old = theta
        if len(V) >= max_space:
            nx = np.linalg.norm(x)
            V = [x / nx]
            S = [ax / nx]
        den = theta - hd
        den = np.where(np.abs(den) < 1e-8, np.copysign(1e-8, den), den)
        t = proj(r / den)
        for _ in range(2):
            for v in V:
                t -= (v @ t) * v
        tn = np.linalg.norm(t)
        if tn < 1e-14:
            x = x / np.linalg.norm(x)
            return float(x @ space.sigma(x)), x, it
        t /= tn
        V.append(t)
        S.append(op(t))
    raise RuntimeError("oracle Davidson did not converge")


def casci(h, eri, nocc, act, want_vector=False, dense_max=DENSE_MAX):
    """Lowest symmetric-subspace root for active orbitals ``act``.

    Returns the energy, or ``(energy, c, space)`` with ``want_vector``.
    """
    sp = Space(h, eri, nocc, act)
    if sp.ndet <= dense_max:
        H = sp.hdense()
        H = 0.5 * (H + H.T)
        # S = Ms: <S^2> = Ms(Ms+1); the next spin has Ms(Ms+1) + 2Ms + 2
        target = sp.ms * (sp.ms + 1.0)
        P = sp.sym_basis() if sp.ms == 0 else np.eye(sp.ndet)
        w, U = np.linalg.eigh(P.T @ H @ P)
        for k in range(len(w)):
            c = P @ U[:, k]
            if c @ sp.s2(c) < target + 0.5:
                e = float(w[k])
                break
        else:
            raise RuntimeError("no state with S = Ms in the space")
    else:
        e, c, _ = davidson(sp)
    if want_vector:
        return e, c, sp
    return e


def spin_square(space: Space, c) -> float:
    """<S^2> of a normalised Ms = 0 vector, by S^2 = S- S+ (pure-Python
    loop; small spaces only).  S+ = sum_p a+_{p alpha} a_{p beta}."""
    n = space.nstr
    c = np.asarray(c).reshape(n, n)
    strs = [int(s[0]) | (int(s[1]) << 64) for s in space.strs]
    out = {}
    norb = space.norb

    def sgn_below(bits, k):
        return -1 if bin(bits & ((1 << k) - 1)).count("1") % 2 else 1

    for ia, A in enumerate(strs):
        for ib, B in enumerate(strs):
            cij = c[ia, ib]
            if cij == 0.0:
                continue
            # det bits: alpha orbitals at 0..127, beta at 128..
            det = A | (B << 128)
            for p in range(norb):
                kb, ka = 128 + p, p
                if not (det >> kb) & 1 or (det >> ka) & 1:
                    continue
                s = sgn_below(det, kb)
                d1 = det & ~(1 << kb)
                s *= sgn_below(d1, ka)
                d2 = d1 | (1 << ka)
                out[d2] = out.get(d2, 0.0) + s * cij
    return float(sum(v * v for v in out.values()))

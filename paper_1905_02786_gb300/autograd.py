"""torch.autograd view of the MBE-FCI energy.

``mbe_energy(h, eri, nelec, ref, exp, max_order, thr)`` runs a whole
expansion (Eqs. 1-3) through the C ABI and returns the total energy as a
0-d tensor whose backward calls ``mbe_energy_backward``: by Hellmann-Feynman
each tuple energy is stationary in its CI coefficients, so the gradient is
the MBE-weighted sum of the tuples' reduced density matrices, built on the
GPU from the kept RDMs.  ``h`` is (norb, norb) and ``eri`` the
symmetric packed (npair, npair) matrix of (pq|rs); both float64 (any
device; the library copies them).  The screening decisions (which tuples
exist) are held fixed in the backward, as the energy is piecewise smooth in
the integrals.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _binding as B


class MBEEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, h, eri, nelec, ref, exp, max_order, thr, device, opts):
        m = B.MBE(device=device, keep_ci=1, **(opts or {}))
        m.load(h.detach().cpu().numpy().astype(np.float64),
               eri.detach().cpu().numpy().astype(np.float64), nelec)
        res = m.run(ref, exp, max_order, thr)
        ctx.mbe = m
        ctx.result = res
        return torch.tensor(res["total"], dtype=torch.float64, device=h.device)

    @staticmethod
    def backward(ctx, g):
        m = ctx.mbe
        dh, deri = m.backward(float(g.detach().cpu()))
        m.close()
        ctx.mbe = None
        dev = g.device
        return (torch.from_numpy(dh).to(dev), torch.from_numpy(deri).to(dev),
                None, None, None, None, None, None, None)


def mbe_energy(h, eri, nelec, ref, exp, max_order, thr=0.0, device=0, **opts):
    """Total MBE-FCI energy (Eh) as a differentiable function of h and eri."""
    return MBEEnergy.apply(h, eri, nelec, list(ref), list(exp), int(max_order), float(thr),
                           device, opts)

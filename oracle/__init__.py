"""Oracle for the MBE-FCI hot path: test infrastructure, not product code.

Plain, slow, obviously-correct CPU implementation (C + NumPy, FP64) that
shares no code with the CUDA path.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference legs
may import it.

* ``oracle.casci`` -- CASCI of one tuple by Slater-Condon rules on full-space
  determinants (dense eigh or Davidson); RDMs; <S^2>.
* ``oracle.mbe``   -- tuple enumeration with screening, increments by the
  recursion of Eq. 3 and by its Moebius closed form, Kahan order sums,
  MBE coefficients and the Hellmann-Feynman energy gradient.
"""

"""CPU FP64 oracle for the DMPT/TDA Bethe-Salpeter hot path -- TEST INFRASTRUCTURE.

This package is the slow, plainly written reference that the CUDA library is
checked against. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it; the library never does, and it shares no code
with the library (the two meet only in the seeded inputs of ``synth/``).

Modules
-------
basis      packing / sphere / grid helpers written for the oracle alone
dense_eh   explicit electron-hole Hamiltonian over the complete conduction
           manifold of S, diagonalised densely (Eqs. evp, d, k1e, k1d, tau, pdep)
pairs      overlap O_vw (Eq. overlap) and the threshold / pair-count rule
liouville  matrix-free Liouville operator with numpy FFTs (Eqs. evp-k1d) and the
           screened integrals tau_vw (Eqs. tau_from_tau_u, pdep)
davidson   block Davidson on any operator (Section 3: iterative diagonalisation)

Every function states the passage of the paper it follows. Readings of passages
the paper leaves open are listed in the design notes of the repository.
"""

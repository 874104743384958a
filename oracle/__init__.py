"""FP64 CPU oracle for the lattice Dirac operators, the Schwarz preconditioner and
the Krylov solvers of "Scaling Lattice QCD beyond 100 GPUs" (Babich et al., SC11).

This package is TEST INFRASTRUCTURE. It is a plain, slow, obviously correct
restatement of the paper's definitions in numpy float64/complex128. Only the test
suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it. The CUDA library never calls it and shares no
code, table or constant generator with it.

Modules
-------
lattice   geometry: site coordinates, neighbour gathers with boundary signs (Sec. 2.2, 2.3)
gamma     Euclidean gamma matrices in a chiral basis (Sec. 5, "similarity transforms")
wilson    Wilson dslash, clover field, Wilson-clover operator (Eq. 2)
staggered improved staggered (asqtad) dslash and operator (Eq. 3)
codecs    gauge 12/8-real compression and 16-bit storage (Sec. 5, strategies (a) and (c))
solvers   MR / additive Schwarz (Sec. 3.2, 8.1), CG, BiCGstab (Sec. 3.1), GCR-DD (Algorithm 1),
          multi-shift CG (Eq. 4)
ptc       gauge-equivariant parallel-transport network used as a learned preconditioner K of
          the flexible GCR (not in the paper; Algorithm 1 admits any K): forward, adjoint,
          loss and weight gradients, Adam

Pins: every function here is checked by ``tests/test_oracle_*.py`` against closed
forms (free-field plane waves, constant abelian field strength), symmetries
(gamma5-hermiticity, anti-hermiticity, gauge covariance), brute-force dense
linear algebra on tiny lattices, rounding bounds of the storage formats, values
counted by hand (boundary crossings) and finite differences (network gradients).
"""

"""FP64 CPU oracle for the DMRG superblock Davidson path (test infrastructure only).

This package is the slow, plain reference against which the CUDA library is checked.
It is test infrastructure: only the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference arm of ``bench.py`` may import it.  The CUDA library never
imports it and shares no code with it; both sides only consume the problem containers
produced by the separate ``dmrg_inputs`` package.

Contents (each function cites the passage of the paper it restates):

* ``sites``      site operators (Eqs. 3, 7, 8) and full-chain operators (Eqs. 1, 2, 4-6)
* ``ed``         exact diagonalisation of a chain inside a symmetry sector (Sec. 3)
* ``projection`` H_SB x by the plain Kronecker definition (Eq. 9) and by the
                 sector-decomposed products of Eq. 11
* ``davidson``   the Davidson iteration of Algorithm 3 (Sec. 5/6)
* ``dmrg``       the infinite-lattice DMRG of Algorithm 1 with the LR strategy (Sec. 4.1)

All arithmetic is float64.  Pins that tie these functions to facts outside the oracle
(closed forms, exact diagonalisation, Bethe ansatz, Lieb-Wu, invariants) live in
``tests/test_oracle_*.py``.
"""

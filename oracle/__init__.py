"""CPU oracle for non-zero noise extrapolation (arXiv 2501.13237).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of the method in NumPy/LAPACK (float64 / complex128).  Only the
test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The CUDA library never calls it, links it or
falls back to it, and it shares no code with the CUDA path: the only thing
the two sides have in common is the seeded input generator in
``workloads/``, which holds none of the method's arithmetic.

Modules
  channels    -- Kraus sets and 16x16 gate+channel superoperators
                 (Sec. 2.2.1 eq. U -> C o U; App. C.2.1), gate-dependent
                 Pauli channels (cat-qubit App. C.2.2, matchgate App. C.3.1)
  dense       -- exact density-matrix simulator for n <= 10
  statevector -- pure-state simulator (lambda = 0 reference)
  mps         -- vectorised-MPO (VMPO) emulator: theta formation, superoperator,
                 SVD truncation to fixed D, Frobenius normalisation, partial
                 fidelities (Sec. 2.1.1-2.1.2, eqs. for f_l and F), centre moves,
                 Pauli expectation values
  pure_mps    -- pure-state MPS (local dimension 2) for the noise-free level
                 lambda = 0, same schedule, truncation and gauge as mps
  matchgate   -- exact noisy expectation values of matchgate circuits under
                 Pauli noise (free-fermion covariance evolution; App. C.3)
  fit         -- noise extrapolation: polynomial, weighted log-linear and
                 three-parameter exponential fits with criteria 2-3
                 (Sec. 2.2.3 (B), App. B.2)

Parity status per function is stated in each module header; every function
is pinned by a CPU test under tests/ (test_oracle_*.py).
"""

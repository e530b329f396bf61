"""FP64 CPU oracle for the two-site DMRG H_eff*psi path (test infrastructure).

This package is test infrastructure only: it is imported by ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py``, never by the product package.  It shares no code with
the CUDA path.  Everything is plain numpy/scipy in float64.

Modules
-------
``fermion``  site operators, spin-orbital integrals of Eq. (1).
``fci``      O1: full-CI by the spin-summed excitation operators E_ij over
             alpha/beta determinant strings (exact definition of Eq. (1)).
``fock``     O2: Jordan-Wigner Fock-space Hamiltonian and the projected
             H_eff = P^T H P for a given MPS (no complementary operators).
``dmrg``     O3: dense-operator two-site DMRG with normal/complementary
             operators (partial summation, Sec. III.A.2), blocking and
             renormalisation, H_eff*psi (Eq. 2 summed over all terms),
             Davidson-free dense/Lanczos eigensolve and SVD truncation.
"""

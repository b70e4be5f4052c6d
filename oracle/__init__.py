"""CPU oracle for the Jacobi–Davidson path on the 3D Anderson model.

This package is TEST INFRASTRUCTURE.  It is a plain, slow, FP64 restatement
of what the GPU library computes, written from Schenk, Bollhöfer & Römer,
"On large scale diagonalization techniques for the Anderson model of
localization" (SIAM J. Sci. Comput., 2006; arXiv math/0508111).  Only the
test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The product library never calls into it and
shares no code, table or helper with it.

Modules
-------
rng        counter-based SplitMix64 stream and the box-distributed disorder
           potential (Section 3, the paragraph after Eq. (1)).
lattice    assembly of the Anderson matrix A of Eq. (1) (periodic and
           hard-wall boundaries, Section 7 / Table 6), its matrix-vector
           product and the W = 0 closed-form spectrum.
eig        dense cyclic Jacobi eigensolver and the "k eigenpairs nearest
           sigma" selection (the problem statement of Sections 3 and 7).
lanczos    shift-and-invert Lanczos with full reorthogonalisation over a
           sparse direct LU of A - sigma I (the shift-and-invert idea of
           Section 4.1), used where a dense eigensolver is too large.
inertia    Sylvester inertia count through a symmetric, pivot-free sparse
           LDL^T, used to prove that no eigenvalue nearer sigma was missed.
matching   maximum-product transversal (Eqs. (5.1)-(5.2)) by a dense
           Kuhn–Munkres with dual potentials, the cycle split into 1x1 and
           2x2 blocks (Section 5.2) and the symmetric scaling (Section 4.2).
krylov     plain restatements of the Krylov pieces of the hot path: the
           simplified QMR recurrences (Section 4.2), classical Gram–Schmidt
           with reorthogonalisation, and the Rayleigh–Ritz step.
ildl       one level of the incomplete block LDL^T (Sections 6.2-6.3):
           pivot blocks, L_F = F D_B^{-1} and the Schur complement with the
           drop rule, densely.

Every function says which passage it follows.  Pins that tie the oracle to
something other than itself live in ``tests/test_oracle_*.py``.
"""

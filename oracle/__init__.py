"""CPU oracle for the strong recursive skeletonisation H^2 solver.

TEST INFRASTRUCTURE ONLY.  Plain, slow float64 numpy/scipy code written from the
paper (Alg. 1-3, Sec. 2.1-2.2, Eq. 2.1) so that the CUDA library can be checked
against it.  Only the tests, the entry point's smoke check and the benchmark's CPU
baseline leg may import it; the library shares no code with it.

Parity pins (tests/test_oracle_pins.py): dense Gaussian elimination with zero
truncation (seven kernel families, including an indefinite oscillatory one), dense LU
in the no-admissible-block case, slogdet of the factors, backward error against the
tolerance, symmetry of the working blocks, colouring validity, brute-force layouts,
the paper's projection identities, near-linear growth of the factor memory, the
operation count and the one-thread time, and the augmentation variants and SVD driver
fallback.  Unpinned: the individual singular vectors, the
complement bases and the intermediate blocks at a positive tolerance (they are
fixed only up to orthogonal changes of basis).
"""

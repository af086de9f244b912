"""Plain, slow FP64 CPU oracle for black-box HBS compression (Levitt & Martinsson,
"Linear-Complexity Black-Box Randomized Compression of Rank-Structured Matrices").

TEST INFRASTRUCTURE ONLY. This package is imported by ``tests/``, by
``__graft_entry__.smoke()`` (to check one small GPU run) and by the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py``. The product path (the CUDA library and its Python
binding) never imports, calls or links anything here, and nothing here imports the product
path: the two share no code. Only the seeded input generators in ``hbs_inputs`` feed both.

Every function follows a passage of the paper, cited in its docstring by section, equation or
algorithm. Arithmetic is numpy float64; numpy's matmul and SVD-based pseudo-inverse serve as
library primitives. Householder reflectors are written out by hand with one fixed sign
convention (Golub & Van Loan, Matrix Computations, Alg. 5.1.1), so that bases that are unique
only up to sign agree with the GPU path to rounding.

Modules
-------
tree      index tree of Section 3.1 (integer bookkeeping)
philox    counter-based Gaussian generator for the test matrices (Philox4x32-10 + Box-Muller)
linalg    Householder QR, ``col`` and ``null`` of Section 2.4, Moore-Penrose pseudo-inverse
sample    Y = A Omega, Z = A^* Psi (Algorithm 2, first block)
compress  Algorithm 2 (level-by-level compression)
apply     Algorithm 1 (apply the telescoping factorization)
norms     20-step power-iteration operator norm of Section 5
"""

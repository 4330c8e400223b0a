"""The oracle: a plain, slow CPU implementation of HEGMM, for testing only.

This package is test infrastructure.  Only the test suite, the smoke check
of ``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import or
run it; the product library never does, and it shares no code with the CUDA
path (the only common module is ``workload``, the seeded input generators).

* ``oracle.slots`` -- the paper's transforms (Eqs. def:sigma..def:omega), the
  linear-transformation diagonals (Eq. lintrans), the U matrices
  (Eqs. Usigma..Uomgc), and both algorithms (Algorithm 1 HEGMM and
  Algorithm 2 HEGMM-Enhanced) on plaintext slot vectors.
* ``oracle.he`` -- RNS-BGV ciphertext arithmetic in plain C
  (``he_oracle.c``, 128-bit integer products, textbook NTT) driven from
  Python, and the ciphertext-level HEGMM executor.
"""

"""GB300-native (sm_103a) HEGMM: encrypted general matrix multiplication.

The compute path is ``libhegmm.so`` (CUDA kernels behind the C ABI in
``include/hegmm.h``); ``paper_2405_02238_gb300.hegmm`` is its ctypes binding.
"""
from .hegmm import (ALG_1, ALG_2, ALG_AUTO, ROLE_A, ROLE_B, Ciphertext, Context, HegmmError, Plaintext,  # noqa: F401
                    load)

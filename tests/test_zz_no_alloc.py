"""The scratch-free rotation (hegmm_rotate_noalloc) through the C ABI.

Some users of this library cannot allocate device memory while they run it:
their framework already holds the GPU's memory in its own pool, or their
serving loop must not block in cudaMalloc / cudaFree.  For them the library
offers a rotation whose intermediates all live in one fixed device array
inside the library.  These checks make sure that this variant returns the
same ciphertext as the ordinary hegmm_rotate (exact equality, as every
integer result in this suite), twice in a row into the same output, and
that parameter sets needing more scratch than the fixed array are refused.

The file name sorts last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

import workload as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_2405_02238_gb300 import build as B

    B.build()
    from paper_2405_02238_gb300 import hegmm

    return hegmm


@pytest.mark.parametrize("name", ["medium", "paper"])
def test_noalloc_rotation_equals_rotate_on_consecutive_calls(H, name):
    pre = W.PRESETS[name]
    ctx = H.Context.from_preset(pre)
    ctx.hegmm_keygen(99)
    x = np.random.default_rng(3).integers(0, pre.t, ctx.S)
    ct = ctx.hegmm_encrypt(ctx.hegmm_encode_slots(x), 5, 0)
    zs = [3, -5]
    ctx.hegmm_keygen_rotations(zs)
    out = ctx.hegmm_add(ct, ct)  # any ciphertext of the input's level serves as the output buffer
    for z in zs:
        ref = ctx.hegmm_rotate(ct, z)
        ctx.hegmm_rotate_noalloc(ct, z, out)
        assert (ctx.hegmm_ct_export(out) == ctx.hegmm_ct_export(ref)).all(), z
        assert (ctx.hegmm_decrypt_slots(out).astype(np.int64) == np.roll(x, -z)).all(), z


def test_noalloc_refuses_parameters_beyond_its_scratch(H):
    # 16 chain primes of 50 bits at N = 2^14 need about 20 MiB of scratch.
    ctx = H.Context(14, 65537, 16, 50, 2, 2)
    ctx.hegmm_keygen(1)
    ct = ctx.hegmm_encrypt(ctx.hegmm_encode_slots(np.arange(8)), 1, 0)
    out = ctx.hegmm_add(ct, ct)
    ctx.hegmm_keygen_rotations([1])
    with pytest.raises(H.HegmmError) as e:
        ctx.hegmm_rotate_noalloc(ct, 1, out)
    assert e.value.code == -1 and "bytes of scratch" in str(e.value)

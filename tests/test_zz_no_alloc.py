"""The scratch-free rotation (hegmm_rotate_noalloc) through the C ABI.

Some users of this library cannot allocate device memory while they run it:
their framework already holds the GPU's memory in its own pool, or their
serving loop must not block in cudaMalloc / cudaFree.  For them the library
offers a rotation whose intermediates all live in one fixed device array
inside the library.  These checks make sure that this variant returns the
same ciphertext as the ordinary hegmm_rotate (exact equality, as every
integer result in this suite), twice in a row into the same output, that
those calls take no device memory (the library's pool use, its high-water
mark, the pool's reservation and the device's free memory are unchanged
across each call), and that parameter sets needing more scratch than the
fixed array are refused.

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
    refs = {z: ctx.hegmm_ct_export(ctx.hegmm_rotate(ct, z)) for z in zs}
    # the first call on the device loads the library's scratch array and
    # looks up its address; from then on no call may take device memory
    ctx.hegmm_rotate_noalloc(ct, zs[0], out)
    before = ctx.hegmm_device_memory(reset_high=True)
    for z in zs:
        ctx.hegmm_rotate_noalloc(ct, z, out)
        after = ctx.hegmm_device_memory()
        # nothing was taken from the library's pool during the call (not even
        # briefly: the high-water mark stays at the use before it), and the
        # device's free memory is unchanged
        assert after["pool_used"] == before["pool_used"], (z, before, after)
        assert after["pool_used_high"] <= before["pool_used"], (z, before, after)
        assert after["pool_reserved"] == before["pool_reserved"], (z, before, after)
        assert after["device_free"] == before["device_free"], (z, before, after)
        assert (ctx.hegmm_ct_export(out) == refs[z]).all(), z
        assert (ctx.hegmm_decrypt_slots(out).astype(np.int64) == np.roll(x, -z)).all(), z
        before = ctx.hegmm_device_memory(reset_high=True)


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

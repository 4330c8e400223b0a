"""Failure detection on the GPU without a fault: a bounded device wait that
runs out is reported to the host as HEGMM_ETIMEOUT and leaves the context
usable.  The staged linear-transformation kernels get a test hook that
leaves one entry's shared-memory stage unarmed (no copy is issued, nothing
is written); its consumers' wait runs out after a short poll limit."""
import numpy as np
import pytest

import workload as W

pytestmark = pytest.mark.gpu
SEED = 99


@pytest.fixture(scope="module")
def H():
    from paper_2405_02238_gb300 import build as B

    B.build()
    from paper_2405_02238_gb300 import hegmm

    return hegmm


@pytest.mark.parametrize("variant", [6, 7, 8])
def test_bounded_wait_reports_timeout_and_context_survives(H, variant):
    ctx = H.Context.from_preset(W.MEDIUM)
    ctx.hegmm_keygen(SEED, [(6, 10, 9)], H.ALG_1)
    ctx.hegmm_set_keyswitch_mode(H.KS_DOUBLE | H.KS_LAZY_RELIN | H.KS_SHARED)
    ctx.hegmm_set_tuning(H.TUNE_LT_KERNEL, variant)
    m, l, n = 6, 10, 9
    A, B = W.matrices(m, l, n, *W.MEDIUM_RANGE)
    ca = ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_A, A, m, l, n, H.ALG_1), 3, 0)
    cb = ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_B, B, m, l, n, H.ALG_1), 3, 1)
    good, _ = ctx.hegmm_matmul(ca, cb, m, l, n, H.ALG_1)
    want = ctx.hegmm_ct_export(good)
    # a wait that runs out: short poll limit, the first staged entry left unarmed
    ctx.hegmm_set_tuning(H.TUNE_WAIT_LIMIT, 1 << 10)
    ctx.hegmm_set_tuning(H.TUNE_TEST_DROP, 0)
    ctx.hegmm_matmul(ca, cb, m, l, n, H.ALG_1)
    with pytest.raises(H.HegmmError) as e:
        ctx.hegmm_sync()
    assert e.value.code == -6  # HEGMM_ETIMEOUT
    # the flag is cleared once read, and the context computes correctly again
    ctx.hegmm_set_tuning(H.TUNE_TEST_DROP, -1)
    ctx.hegmm_set_tuning(H.TUNE_WAIT_LIMIT, 1 << 22)
    ctx.hegmm_sync()
    again, _ = ctx.hegmm_matmul(ca, cb, m, l, n, H.ALG_1)
    assert (ctx.hegmm_ct_export(again) == want).all()
    assert (ctx.hegmm_decrypt(again, m, l, n, H.ALG_1).astype(np.int64) == (A @ B) % W.MEDIUM.t).all()


def test_key_checkpoint_warm_start(H):
    # keys exported from one context and imported into a fresh one (no
    # hegmm_keygen, no secret key) evaluate the same product bit for bit
    pre = W.TINY
    src = H.Context.from_preset(pre)
    m, l, n = 4, 8, 6
    src.hegmm_set_keyswitch_mode(7)
    src.hegmm_keygen(5, [(m, l, n)], 0)
    src.hegmm_keygen_rotations([1])
    A, B = W.matrices(m, l, n, 0, 15, seed=8)
    ca = src.hegmm_encrypt(src.hegmm_encode(H.ROLE_A, A, m, l, n), 6, 0)
    cb = src.hegmm_encrypt(src.hegmm_encode(H.ROLE_B, B, m, l, n), 6, 1)
    C, _ = src.hegmm_matmul(ca, cb, m, l, n)
    dst = H.Context.from_preset(pre)
    dst.hegmm_set_keyswitch_mode(7)
    ids = src.hegmm_key_list()
    assert 0 in ids and len(ids) > 1
    for g in ids:
        dst.hegmm_key_import(g, src.hegmm_key_export(g))
    assert dst.hegmm_key_list() == ids
    da, db = dst.hegmm_ct_import(src.hegmm_ct_export(ca)), dst.hegmm_ct_import(src.hegmm_ct_export(cb))
    D, _ = dst.hegmm_matmul(da, db, m, l, n)
    assert (dst.hegmm_ct_export(D) == src.hegmm_ct_export(C)).all()
    got = src.hegmm_decrypt(src.hegmm_ct_import(dst.hegmm_ct_export(D)), m, l, n).astype(np.int64)
    assert (got == (A @ B) % pre.t).all()
    with pytest.raises(H.HegmmError) as e:  # no secret key in the warm-started context
        dst.hegmm_decrypt(D, m, l, n)
    assert e.value.code == -4
    # a transformation needing an imported rotation key runs; one needing a missing key cannot make it
    shift1 = [j + 1 for j in range(16)]
    r_src, r_dst = src.hegmm_lintrans(ca, shift1), dst.hegmm_lintrans(da, shift1)
    assert (dst.hegmm_ct_export(r_dst) == src.hegmm_ct_export(r_src)).all()
    z = next(z for z in range(2, dst.S) if pow(5, z, 2 * dst.N) not in ids)  # an offset without a key
    with pytest.raises(H.HegmmError) as e:
        dst.hegmm_lintrans(da, [j + z for j in range(16)])
    assert e.value.code == -4
    with pytest.raises(H.HegmmError) as e:  # a residue that is not below its prime
        dst.hegmm_key_import(0, np.full_like(src.hegmm_key_export(0), np.uint64(2**63)))
    assert e.value.code == -1

"""Batched HEGMM (many products of mixed shapes per call) against the
single-product path and the oracle.

Each product in a batch must give exactly the ciphertext it gives alone
(bit-exact), its decryption must equal A.B mod t, and a few are checked
against the oracle's ciphertext.  The full workload is the 512-product batch
of the medium ring (shapes m, l, n in 4..64 with ml, ln, mn <= 4096).
"""
import numpy as np
import pytest

import workload as W
from oracle import he as OH
from oracle import slots as SL

pytestmark = pytest.mark.gpu
SEED = 4321


@pytest.fixture(scope="module")
def H():
    from paper_2405_02238_gb300 import build as B

    B.build()
    from paper_2405_02238_gb300 import hegmm

    return hegmm


@pytest.fixture(scope="module")
def medium(H):
    ctx = H.Context.from_preset(W.MEDIUM)
    ctx.hegmm_keygen(SEED)
    return ctx


def encrypt_all(ctx, H, shapes, lo, hi, seed0=0, stream0=0):
    As, Bs, mats = [], [], []
    for i, (m, l, n) in enumerate(shapes):
        A, B = W.matrices(m, l, n, lo, hi, seed=seed0 + i)
        mats.append((A, B))
        As.append(ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_A, A, m, l, n), 77, stream0 + 2 * i))
        Bs.append(ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_B, B, m, l, n), 77, stream0 + 2 * i + 1))
    return As, Bs, mats


@pytest.mark.parametrize("mode", ["double+lazy+shared", "double+lazy", "double", "single"])
def test_batch_mixed_shapes_equal_single_and_oracle(H, medium, mode):
    ctx = medium
    parts = mode.split("+")
    base, lazy, shared = parts[0], "lazy" in parts, "shared" in parts
    ctx.hegmm_set_keyswitch_mode((H.KS_DOUBLE if base == "double" else H.KS_SINGLE) | (H.KS_LAZY_RELIN if lazy else 0)
                                 | (H.KS_SHARED if shared else 0))
    shapes = [(4, 8, 6), (5, 12, 7), (9, 4, 11), (7, 9, 2), (12, 3, 9), (3, 3, 3), (6, 40, 5), (20, 10, 30)]
    ctx.hegmm_keygen(SEED, shapes)
    As, Bs, mats = encrypt_all(ctx, H, shapes, *W.BATCH_RANGE)
    outs = ctx.hegmm_matmul_batch(As, Bs, shapes)
    for i, (m, l, n) in enumerate(shapes):
        single, _ = ctx.hegmm_matmul(As[i], Bs[i], m, l, n)
        assert (ctx.hegmm_ct_export(outs[i]) == ctx.hegmm_ct_export(single)).all(), shapes[i]
        A, B = mats[i]
        assert (ctx.hegmm_decrypt(outs[i], m, l, n).astype(np.int64) == (A @ B) % W.MEDIUM.t).all()
    # two products against the oracle's ciphertext
    o = OH.Oracle(W.MEDIUM)
    o.keygen(SEED)
    for i in (0, 3):
        m, l, n = shapes[i]
        plan = SL.make_plan(m, l, n, SL.choose_alg(m, l, n, o.S))
        ex = OH.HEGMM(o, mode=base, lazy_relin=lazy, giant=shared)
        ctA, ctB = ex.encrypt_inputs(plan, *mats[i], seed=77, streams=(2 * i, 2 * i + 1))
        assert (ctx.hegmm_ct_export(outs[i]) == ex.run(plan, ctA, ctB)).all()
    ctx.hegmm_set_keyswitch_mode(H.KS_SINGLE)  # the library default


def test_batch_with_repeated_shapes(H, medium):
    ctx = medium
    shapes = [(4, 8, 6)] * 4 + [(6, 2, 7)] * 3
    ctx.hegmm_keygen(SEED, shapes)
    As, Bs, mats = encrypt_all(ctx, H, shapes, *W.BATCH_RANGE, seed0=100, stream0=1000)
    outs = ctx.hegmm_matmul_batch(As, Bs, shapes)
    for i, (m, l, n) in enumerate(shapes):
        A, B = mats[i]
        assert (ctx.hegmm_decrypt(outs[i], m, l, n).astype(np.int64) == (A @ B) % W.MEDIUM.t).all()
    # a second call of the same batch (cached plan) gives the same ciphertexts
    again = ctx.hegmm_matmul_batch(As, Bs, shapes)
    for a, b in zip(outs, again):
        assert (ctx.hegmm_ct_export(a) == ctx.hegmm_ct_export(b)).all()


def test_batch_512_products(H, medium):
    ctx = medium
    shapes = W.batch_shapes(W.BATCH_COUNT, ctx.S)
    ctx.hegmm_keygen(SEED, shapes)
    As, Bs, mats = encrypt_all(ctx, H, shapes, *W.BATCH_RANGE, seed0=5000, stream0=5000)
    outs = ctx.hegmm_matmul_batch(As, Bs, shapes)
    for i, (m, l, n) in enumerate(shapes):
        A, B = mats[i]
        assert (ctx.hegmm_decrypt(outs[i], m, l, n).astype(np.int64) == (A @ B) % W.MEDIUM.t).all(), shapes[i]
    # sampled products equal the single-product path bit for bit
    for i in np.random.default_rng(0).choice(len(shapes), 6, replace=False):
        m, l, n = shapes[i]
        single, _ = ctx.hegmm_matmul(As[i], Bs[i], m, l, n)
        assert (ctx.hegmm_ct_export(outs[i]) == ctx.hegmm_ct_export(single)).all(), shapes[i]


def test_batch_with_per_product_algorithms(H, medium):
    # both algorithms in one call share the launches and change no bit
    ctx = medium
    shapes = [(4, 8, 6), (4, 8, 6), (9, 4, 11), (9, 4, 11), (3, 3, 3)]
    algs = [1, 2, 1, 2, 0]
    for a in (1, 2):
        ctx.hegmm_keygen(SEED, shapes, a)
    As, Bs, mats = [], [], []
    for i, (m, l, n) in enumerate(shapes):  # operands encoded for their product's algorithm
        A, B = W.matrices(m, l, n, *W.BATCH_RANGE, seed=300 + i)
        mats.append((A, B))
        As.append(ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_A, A, m, l, n, algs[i]), 77, 3000 + 2 * i))
        Bs.append(ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_B, B, m, l, n, algs[i]), 77, 3001 + 2 * i))
    for flags in (H.KS_SINGLE, H.KS_DOUBLE | H.KS_LAZY_RELIN, H.KS_DOUBLE | H.KS_LAZY_RELIN | H.KS_SHARED):
        ctx.hegmm_set_keyswitch_mode(flags)
        outs = ctx.hegmm_matmul_batch_algs(As, Bs, shapes, algs)
        for i, (m, l, n) in enumerate(shapes):
            single, _ = ctx.hegmm_matmul(As[i], Bs[i], m, l, n, algs[i])
            assert (ctx.hegmm_ct_export(outs[i]) == ctx.hegmm_ct_export(single)).all(), (shapes[i], algs[i])
            A, B = mats[i]
            got = ctx.hegmm_decrypt(outs[i], m, l, n, algs[i]).astype(np.int64)
            assert (got == (A @ B) % W.MEDIUM.t).all()
    ctx.hegmm_set_keyswitch_mode(H.KS_SINGLE)


def test_graph_replay_takes_each_calls_operands(H, medium):
    # the first call of a cached plan runs launch by launch, the second is
    # captured as a CUDA graph, later ones replay it: every call must use its
    # own operands and write its own results
    ctx = medium
    ctx.hegmm_set_keyswitch_mode(H.KS_DOUBLE | H.KS_LAZY_RELIN | H.KS_SHARED)
    shapes = [(6, 10, 9), (5, 12, 7)]
    ctx.hegmm_keygen(SEED, shapes)
    try:
        for call in range(4):
            As, Bs, mats = encrypt_all(ctx, H, shapes, *W.BATCH_RANGE, seed0=900 + 7 * call, stream0=9000 + 10 * call)
            outs = ctx.hegmm_matmul_batch(As, Bs, shapes)
            for i, (m, l, n) in enumerate(shapes):
                A, B = mats[i]
                assert (ctx.hegmm_decrypt(outs[i], m, l, n).astype(np.int64) == (A @ B) % W.MEDIUM.t).all(), call
                ctx.hegmm_set_tuning(H.TUNE_GRAPHS, 0)
                plain, _ = ctx.hegmm_matmul(As[i], Bs[i], m, l, n)
                ctx.hegmm_set_tuning(H.TUNE_GRAPHS, 1)
                assert (ctx.hegmm_ct_export(outs[i]) == ctx.hegmm_ct_export(plain)).all(), call
    finally:
        ctx.hegmm_set_keyswitch_mode(H.KS_SINGLE)


def test_autotune_keeps_results(H, medium):
    ctx = medium
    ctx.hegmm_set_keyswitch_mode(H.KS_DOUBLE | H.KS_LAZY_RELIN | H.KS_SHARED)
    shapes = [(6, 10, 9), (5, 12, 7), (4, 8, 6)]
    ctx.hegmm_keygen(SEED, shapes)
    try:
        As, Bs, mats = encrypt_all(ctx, H, shapes, *W.BATCH_RANGE, seed0=40, stream0=400)
        before = [ctx.hegmm_ct_export(c) for c in ctx.hegmm_matmul_batch(As, Bs, shapes)]
        chosen = ctx.hegmm_autotune(As, Bs, shapes, reps=1)
        assert chosen["lt_kernel"] in (0, 3, 6, 7) and chosen["lt_chunk"] in (16, 32, 64) and chosen["lt_one"] in (0, 1, 2, 3, 4)
        after = [ctx.hegmm_ct_export(c) for c in ctx.hegmm_matmul_batch(As, Bs, shapes)]
        for x, y in zip(before, after):
            assert (x == y).all()
    finally:
        ctx.hegmm_set_tuning(H.TUNE_LT_KERNEL, 6)
        ctx.hegmm_set_tuning(H.TUNE_LT_CHUNK, 32)
        ctx.hegmm_set_tuning(H.TUNE_LT_ONE, 4)
        ctx.hegmm_set_keyswitch_mode(H.KS_SINGLE)


@pytest.mark.parametrize("mode", ["double+lazy+shared", "single"])
def test_sub_batches_equal_one_batch(H, medium, mode):
    """HEGMM_TUNE_GROUPS 2 (two concurrent sub-batches on streams of their
    own) gives every product the bits of the one-plan batch, in batches,
    in sums of products (hegmm_matmul_sum) and on repeated calls (cached
    plans, graph replays)."""
    ctx = medium
    ctx.hegmm_set_keyswitch_mode(H.KS_DOUBLE | H.KS_LAZY_RELIN | H.KS_SHARED if mode != "single" else H.KS_SINGLE)
    shapes = [(16, 32, 24), (4, 8, 6), (9, 4, 11), (20, 10, 30), (12, 3, 9)]
    ctx.hegmm_keygen(SEED, shapes)
    As, Bs, mats = encrypt_all(ctx, H, shapes, *W.BATCH_RANGE, seed0=50, stream0=600)
    ref = [ctx.hegmm_ct_export(c) for c in ctx.hegmm_matmul_batch(As, Bs, shapes)]
    # two blocks of one product, summed, beside a third product
    A, B = W.matrices(8, 16, 6, *W.BATCH_RANGE, seed=9)
    ctx.hegmm_keygen(SEED, [(8, 8, 6)], 2)
    blk = [(ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_A, A[:, 8 * k:8 * k + 8], 8, 8, 6, 2), 78, 700 + 2 * k),
            ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_B, B[8 * k:8 * k + 8, :], 8, 8, 6, 2), 78, 701 + 2 * k))
           for k in range(2)]
    sum_args = ([blk[0][0], blk[1][0], As[0]], [blk[0][1], blk[1][1], Bs[0]], [(8, 8, 6), (8, 8, 6), shapes[0]],
                [0, 0, 1], 2, [2, 2, 0])
    sref = [ctx.hegmm_ct_export(c) for c in ctx.hegmm_matmul_sum(*sum_args)]
    ctx.hegmm_set_tuning(H.TUNE_GROUPS, 2)
    try:
        for _ in range(3):
            outs = ctx.hegmm_matmul_batch(As, Bs, shapes)
            for i, c in enumerate(outs):
                assert (ctx.hegmm_ct_export(c) == ref[i]).all(), shapes[i]
            souts = ctx.hegmm_matmul_sum(*sum_args)
            for g, c in enumerate(souts):
                assert (ctx.hegmm_ct_export(c) == sref[g]).all(), g
        for i, ((m, l, n), (Am, Bm)) in enumerate(zip(shapes, mats)):
            assert (ctx.hegmm_decrypt(outs[i], m, l, n).astype(np.int64) == (Am @ Bm) % W.MEDIUM.t).all()
        assert (ctx.hegmm_decrypt(souts[0], 8, 8, 6, 2).astype(np.int64) == (A @ B) % W.MEDIUM.t).all()
        with pytest.raises(H.HegmmError):
            ctx.hegmm_set_tuning(H.TUNE_GROUPS, 3)
    finally:
        ctx.hegmm_set_tuning(H.TUNE_GROUPS, 1)

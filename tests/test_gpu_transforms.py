"""GPU parity of ciphertext-side transformations and chained products.

hegmm_lintrans, hegmm_to_layout (sigma / tau under encryption, Section
3.2.2), hegmm_from_result and hegmm_chain_operand through the C ABI against
the oracle's ``HEGMM.lintrans`` / ``to_layout`` / ``from_result`` /
``chain_operand`` on the same seeded inputs, ciphertext for ciphertext
(exact equality), on the N = 2^13 ring; chains of larger products on the
N = 2^14 ring are checked by decryption against A B D mod t.
"""
import numpy as np
import pytest

import workload as W
from oracle import he as OH
from oracle import slots as SL

pytestmark = pytest.mark.gpu

SEED = 55


@pytest.fixture(scope="module")
def H():
    from paper_2405_02238_gb300 import build as B

    B.build()
    from paper_2405_02238_gb300 import hegmm

    return hegmm


@pytest.fixture(scope="module")
def medium_pair(H):
    ctx = H.Context.from_preset(W.MEDIUM)
    ctx.hegmm_keygen(SEED)
    o = OH.Oracle(W.MEDIUM)
    o.keygen(SEED)
    return ctx, o


def plain_vec(M, S):
    v = np.zeros(S, dtype=np.int64)
    r, c = M.shape
    for j in range(c):
        v[j * r:(j + 1) * r] = M[:, j]
    return v


def enc_both(ctx, o, x, stream):
    ct = ctx.hegmm_encrypt(ctx.hegmm_encode_slots(x % o.t), 21, stream)
    return ct, o.encrypt(o.encode(x % o.t), 21, stream)


def test_lintrans_bitexact(H, medium_pair):
    ctx, o = medium_pair
    rng = np.random.default_rng(1)
    x = rng.integers(0, o.t, o.S)
    ct, co = enc_both(ctx, o, x, 0)
    count = 333  # a ragged map: zeros inside and beyond it
    src = rng.integers(0, o.S, count)
    src[rng.random(count) < 0.2] = -1
    src[:40] = np.arange(40) + 7  # a shared offset
    got = ctx.hegmm_lintrans(ct, src)
    ref = OH.HEGMM(o).lintrans(co, [int(s) for s in src])
    assert (ctx.hegmm_ct_export(got) == ref).all()
    want = np.zeros(o.S, dtype=np.int64)
    want[:count] = np.where(src >= 0, x[np.maximum(src, 0)], 0)
    assert (ctx.hegmm_decrypt_slots(got).astype(np.int64) == want).all()


@pytest.mark.parametrize("shape,alg", [((3, 5, 4), 1), ((3, 5, 4), 2), ((5, 3, 4), 2), ((4, 7, 3), 2)])
def test_to_layout_then_product_bitexact(H, medium_pair, shape, alg):
    ctx, o = medium_pair
    ctx.hegmm_set_keyswitch_mode(0)
    m, l, n = shape
    A, B = W.matrices(m, l, n, 0, 15, seed=sum(shape))
    ga, oa = enc_both(ctx, o, plain_vec(A, o.S), 1)
    gb, ob = enc_both(ctx, o, plain_vec(B, o.S), 2)
    ex = OH.HEGMM(o)
    ta, tb = ctx.hegmm_to_layout(ga, 0, m, l, n, alg), ctx.hegmm_to_layout(gb, 1, m, l, n, alg)
    ra, rb = ex.to_layout(oa, 0, m, l, n, alg), ex.to_layout(ob, 1, m, l, n, alg)
    assert (ctx.hegmm_ct_export(ta) == ra).all() and (ctx.hegmm_ct_export(tb) == rb).all()
    ctx.hegmm_keygen(SEED, [shape], alg)
    C, _ = ctx.hegmm_matmul(ta, tb, m, l, n, alg)
    plan = SL.make_plan(m, l, n, alg)
    assert (ctx.hegmm_ct_export(C) == ex.run(plan, ra, rb)).all()
    assert (ctx.hegmm_decrypt(C, m, l, n, alg).astype(np.int64) == (A @ B) % o.t).all()


@pytest.mark.parametrize("alg1,alg2", [(1, 1), (2, 1), (1, 2), (2, 2)])
def test_chain_bitexact(H, medium_pair, alg1, alg2):
    ctx, o = medium_pair
    ctx.hegmm_set_keyswitch_mode(0)
    m, l, n, p = 2, 5, 3, 4
    A, B = W.matrices(m, l, n, 0, 15, seed=9)
    D = np.random.default_rng(10).integers(0, 16, (n, p))
    ctx.hegmm_keygen(SEED, [(m, l, n)], alg1)
    ctx.hegmm_keygen(SEED, [(m, n, p)], alg2)
    ex = OH.HEGMM(o)
    plan1, plan2 = SL.make_plan(m, l, n, alg1), SL.make_plan(m, n, p, alg2)
    ca = ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_A, A, m, l, n, alg1), 22, 0)
    cb = ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_B, B, m, l, n, alg1), 22, 1)
    oa, ob = ex.encrypt_inputs(plan1, A, B, seed=22, streams=(0, 1))
    C, _ = ctx.hegmm_matmul(ca, cb, m, l, n, alg1)
    oc = ex.run(plan1, oa, ob)
    assert (ctx.hegmm_ct_export(C) == oc).all()
    flat = ctx.hegmm_from_result(C, m, l, n, alg1)
    assert (ctx.hegmm_ct_export(flat) == ex.from_result(oc, m, l, n, alg1)).all()
    X = ctx.hegmm_chain_operand(C, m, l, n, alg1, 0, m, n, p, alg2)
    ox = ex.chain_operand(oc, m, l, n, alg1, 0, m, n, p, alg2)
    assert (ctx.hegmm_ct_export(X) == ox).all()
    cd = ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_B, D, m, n, p, alg2), 22, 2)
    _, od = ex.encrypt_inputs(plan2, np.zeros((m, n), dtype=np.int64), D, seed=22, streams=(3, 2))
    C2, _ = ctx.hegmm_matmul(X, cd, m, n, p, alg2)
    assert (ctx.hegmm_ct_export(C2) == ex.run(plan2, ox, od)).all()
    assert (ctx.hegmm_decrypt(C2, m, n, p, alg2).astype(np.int64) == (A @ B @ D) % o.t).all()


def test_transform_errors(H, medium_pair):
    ctx, o = medium_pair
    ct, _ = enc_both(ctx, o, np.arange(o.S), 3)
    for bad in ([o.S], list(range(o.S + 1))):
        with pytest.raises(H.HegmmError) as e:
            ctx.hegmm_lintrans(ct, bad)
        assert e.value.code == -1
    with pytest.raises(H.HegmmError) as e:  # the result is 2 x 3, operand A of (3, 2, 4) is 3 x 2
        ctx.hegmm_chain_operand(ct, 2, 5, 3, 1, 0, 3, 2, 4, 1)
    assert e.value.code == -1
    with pytest.raises(H.HegmmError) as e:
        ctx.hegmm_to_layout(ct, 0, 200, 200, 200, 1)
    assert e.value.code == -3


def test_chain_paper_ring(H):
    # larger chained products on the N = 2^14 ring (twice one product's noise
    # budget), products in the benchmark's evaluation order
    pre = W.PAPER
    ctx = H.Context.from_preset(pre)
    ctx.hegmm_set_keyswitch_mode(7)
    m, l, n, p = 16, 24, 12, 20
    A, B = W.matrices(m, l, n, *W.PAPER_RANGE, seed=12)
    D = np.random.default_rng(13).integers(0, 256, (n, p))
    ctx.hegmm_keygen(SEED, [(m, l, n), (m, n, p)], 1)
    ca = ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_A, A, m, l, n, 1), 23, 0)
    cb = ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_B, B, m, l, n, 1), 23, 1)
    C, _ = ctx.hegmm_matmul(ca, cb, m, l, n, 1)
    X = ctx.hegmm_chain_operand(C, m, l, n, 1, 0, m, n, p, 1)
    cd = ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_B, D, m, n, p, 1), 23, 2)
    C2, _ = ctx.hegmm_matmul(X, cd, m, n, p, 1)
    assert (ctx.hegmm_decrypt(C2, m, n, p, 1).astype(np.int64) == (A @ B @ D) % pre.t).all()

"""GPU parity of blocked products (Section 4.4, Table 4) and sums of products.

hegmm_matmul_blocked / hegmm_matmul_sum through the C ABI against the
oracle's ``HEGMM.blocked`` / ``HEGMM.sum_products`` on the same seeded
inputs, ciphertext for ciphertext (exact equality); the paper's 100 x 100
partitions P1 (50 + 50) and P2 (64 + 36) on the N = 2^14 ring are checked by
decryption against A B mod t (the oracle would take minutes per product
there).
"""
import numpy as np
import pytest

import workload as W
from oracle import he as OH
from oracle import slots as SL

pytestmark = pytest.mark.gpu

SEED = 77


@pytest.fixture(scope="module")
def H():
    from paper_2405_02238_gb300 import build as B

    B.build()
    from paper_2405_02238_gb300 import hegmm

    return hegmm


@pytest.fixture(scope="module")
def tiny_pair(H):
    ctx = H.Context.from_preset(W.TINY)
    ctx.hegmm_keygen(SEED)
    o = OH.Oracle(W.TINY)
    o.keygen(SEED)
    return ctx, o


MODES = {"single": (0, "single", False, False), "double+lazy+shared": (7, "double", True, True)}


def encrypt_blocks(H, ctx, o, rows, inner, cols, A, B):
    """Each block encrypted once, with its Algorithm 1 layout, on both sides."""
    rb, kb, cb = SL.block_bounds(rows), SL.block_bounds(inner), SL.block_bounds(cols)
    gA, gB, oA, oB = [], [], [], []
    for i, (r0, r1) in enumerate(rb):
        gA.append([]), oA.append([])
        for k, (k0, k1) in enumerate(kb):
            blk = A[r0:r1, k0:k1]
            gA[i].append(ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_A, blk, r1 - r0, k1 - k0, 1, 1), 3, 10 * i + k))
            if o is not None:
                lay = SL.make_plan(r1 - r0, k1 - k0, 1, 1).a_layout(blk) % o.t
                oA[i].append(o.encrypt(o.encode(lay), 3, 10 * i + k))
    for k, (k0, k1) in enumerate(kb):
        gB.append([]), oB.append([])
        for j, (c0, c1) in enumerate(cb):
            blk = B[k0:k1, c0:c1]
            gB[k].append(ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_B, blk, 1, k1 - k0, c1 - c0, 1), 4, 10 * k + j))
            if o is not None:
                lay = SL.make_plan(1, k1 - k0, c1 - c0, 1).b_layout(blk) % o.t
                oB[k].append(o.encrypt(o.encode(lay), 4, 10 * k + j))
    return gA, gB, oA, oB


def block_keys(ctx, rows, inner, cols):
    ctx.hegmm_keygen(SEED, [(r, q, c) for r in rows for q in inner for c in cols], 1)


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("split", [([3, 2], [2, 3], [2]), ([4], [3, 1, 2], [2, 3]), ([2, 1, 3], [5], [1, 4])])
def test_blocked_tiny_bitexact(H, tiny_pair, mode, split):
    ctx, o = tiny_pair
    flags, base, lazy, shared = MODES[mode]
    ctx.hegmm_set_keyswitch_mode(flags)
    rows, inner, cols = split
    rng = np.random.default_rng(sum(rows) * 100 + sum(inner) * 10 + sum(cols))
    A = rng.integers(0, 16, (sum(rows), sum(inner)))
    B = rng.integers(0, 16, (sum(inner), sum(cols)))
    block_keys(ctx, rows, inner, cols)
    gA, gB, oA, oB = encrypt_blocks(H, ctx, o, rows, inner, cols, A, B)
    C = ctx.hegmm_matmul_blocked(rows, inner, cols, gA, gB)
    ex = OH.HEGMM(o, mode=base, lazy_relin=lazy, giant=shared)
    ref = ex.blocked(rows, inner, cols, oA, oB)
    rb, cb = SL.block_bounds(rows), SL.block_bounds(cols)
    for i, (r0, r1) in enumerate(rb):
        for j, (c0, c1) in enumerate(cb):
            assert (ctx.hegmm_ct_export(C[i][j]) == ref[i][j]).all(), (i, j)
            got = ctx.hegmm_decrypt(C[i][j], r1 - r0, inner[0], c1 - c0, 1).astype(np.int64)
            assert (got == (A[r0:r1] @ B[:, c0:c1]) % o.t).all()
    ctx.hegmm_set_keyswitch_mode(0)


def test_matmul_sum_algorithm2_groups(H, tiny_pair):
    # two groups of Algorithm 2 products whose layouts agree within each group
    ctx, o = tiny_pair
    ctx.hegmm_set_keyswitch_mode(7)
    shapes = [(3, 5, 4), (3, 5, 4), (2, 6, 2), (2, 6, 2), (2, 6, 2)]
    group = [0, 0, 1, 1, 1]
    ctx.hegmm_keygen(SEED, shapes, 2)
    As, Bs, items = [], [], [[], []]
    ex = OH.HEGMM(o, mode="double", lazy_relin=True, giant=True)
    mats = []
    for p, (m, l, n) in enumerate(shapes):
        A, B = W.matrices(m, l, n, 0, 16, seed=50 + p)
        mats.append((A, B))
        As.append(ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_A, A, m, l, n, 2), 8, 2 * p))
        Bs.append(ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_B, B, m, l, n, 2), 8, 2 * p + 1))
        plan = SL.make_plan(m, l, n, 2)
        ca, cb = ex.encrypt_inputs(plan, A, B, seed=8, streams=(2 * p, 2 * p + 1))
        items[group[p]].append((plan, ca, cb))
    C = ctx.hegmm_matmul_sum(As, Bs, shapes, group, 2, algs=[2] * len(shapes))
    for g in range(2):
        assert (ctx.hegmm_ct_export(C[g]) == ex.sum_products(items[g])).all()
        m, l, n = shapes[group.index(g)]
        want = sum((mats[p][0] @ mats[p][1]) for p in range(len(shapes)) if group[p] == g) % o.t
        assert (ctx.hegmm_decrypt(C[g], m, l, n, 2).astype(np.int64) == want).all()
    ctx.hegmm_set_keyswitch_mode(0)


def test_matmul_sum_errors(H, tiny_pair):
    ctx, o = tiny_pair
    shapes = [(2, 3, 2), (2, 3, 2)]
    ctx.hegmm_keygen(SEED, shapes, 1)
    ctx.hegmm_keygen(SEED, shapes, 2)
    A, B = W.matrices(2, 3, 2, 0, 16, seed=1)
    a1 = ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_A, A, 2, 3, 2, 1), 9, 0)
    b1 = ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_B, B, 2, 3, 2, 1), 9, 1)
    a2 = ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_A, A, 2, 3, 2, 2), 9, 2)
    b2 = ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_B, B, 2, 3, 2, 2), 9, 3)
    # Algorithm 1 (2 x 2 result) and Algorithm 2 case A with t = 2 (4 x 2) in one group
    with pytest.raises(H.HegmmError) as e:
        ctx.hegmm_matmul_sum([a1, a2], [b1, b2], shapes, [0, 0], 1, algs=[1, 2])
    assert e.value.code == -3
    with pytest.raises(H.HegmmError) as e:  # group 1 has no product
        ctx.hegmm_matmul_sum([a1, a1], [b1, b1], shapes, [0, 0], 2, algs=[1, 1])
    assert e.value.code == -1
    with pytest.raises(H.HegmmError) as e:
        ctx.hegmm_matmul_sum([a1, a1], [b1, b1], shapes, [0, 3], 2, algs=[1, 1])
    assert e.value.code == -1
    with pytest.raises(H.HegmmError) as e:
        ctx.hegmm_matmul_blocked([2, 0], [3], [2], [[a1], [a1]], [[b1]])
    assert e.value.code == -1
    # the two separate groups are fine
    C = ctx.hegmm_matmul_sum([a1, a2], [b1, b2], shapes, [0, 1], 2, algs=[1, 2])
    assert (ctx.hegmm_decrypt(C[0], 2, 3, 2, 1).astype(np.int64) == (A @ B) % o.t).all()
    assert (ctx.hegmm_decrypt(C[1], 2, 3, 2, 2).astype(np.int64) == (A @ B) % o.t).all()


@pytest.mark.parametrize("split", [[50, 50], [64, 36]], ids=["P1", "P2"])
def test_blocked_paper_partitions(H, split):
    # Table 4's 100 x 100 product on the N = 2^14 ring, default evaluation order
    # of the benchmark (double hoisting, lazy relinearisation, shared baby steps)
    pre = W.PAPER
    ctx = H.Context.from_preset(pre)
    ctx.hegmm_set_keyswitch_mode(7)
    rng = np.random.default_rng(split[0])
    A = rng.integers(0, 256, (100, 100))
    B = rng.integers(0, 256, (100, 100))
    ctx.hegmm_keygen(SEED, [(r, q, c) for r in split for q in split for c in split], 1)
    gA, gB, _, _ = encrypt_blocks(H, ctx, None, split, split, split, A, B)
    C = ctx.hegmm_matmul_blocked(split, split, split, gA, gB)
    rb = SL.block_bounds(split)
    for i, (r0, r1) in enumerate(rb):
        for j, (c0, c1) in enumerate(rb):
            got = ctx.hegmm_decrypt(C[i][j], r1 - r0, split[0], c1 - c0, 1).astype(np.int64)
            assert (got == (A[r0:r1] @ B[:, c0:c1]) % pre.t).all(), (i, j)

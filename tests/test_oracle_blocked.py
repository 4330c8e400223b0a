"""Pins of the oracle's blocked product (Section 4.4, Table 4).

A matrix product too large for one ciphertext is split into blocks,
C_ij = sum_k A_ik B_kj.  What fixes the answer independently of the code:
the assembled C equals A B mod t (numpy's product), for the paper's two
partitions of a 100 x 100 product (P1: 50 + 50, P2: 64 + 36) and for ragged
splits; a block grid of one block is the plain product; Algorithm 2's result
layout depends on the case, so summing its products over k is only defined
where the layouts agree, and the oracle refuses the rest.
"""
import numpy as np
import pytest

import workload as W
from oracle import he
from oracle import slots as SL

T = 65537


@pytest.mark.parametrize("split", [[50, 50], [64, 36]], ids=["P1", "P2"])
def test_blocked_slots_paper_partitions(split):
    # 100 x 100 by 100 x 100 on the N = 2^14 ring's 8192 slots
    rng = np.random.default_rng(sum(split) + split[0])
    A = rng.integers(0, 256, (100, 100))
    B = rng.integers(0, 256, (100, 100))
    C = SL.run_blocked_slots(split, split, split, A, B, 8192, T)
    assert (C == (A @ B) % T).all()


@pytest.mark.parametrize("seed", range(4))
def test_blocked_slots_ragged(seed):
    rng = np.random.default_rng(100 + seed)
    rows = [int(v) for v in rng.integers(1, 9, size=int(rng.integers(1, 4)))]
    inner = [int(v) for v in rng.integers(1, 9, size=int(rng.integers(1, 4)))]
    cols = [int(v) for v in rng.integers(1, 9, size=int(rng.integers(1, 4)))]
    A = rng.integers(0, T, (sum(rows), sum(inner)))
    B = rng.integers(0, T, (sum(inner), sum(cols)))
    C = SL.run_blocked_slots(rows, inner, cols, A, B, 256, T)
    assert (C == (A @ B) % T).all()


def test_one_block_is_the_plain_product():
    rng = np.random.default_rng(7)
    A = rng.integers(0, 256, (6, 9))
    B = rng.integers(0, 256, (9, 5))
    C = SL.run_blocked_slots([6], [9], [5], A, B, 256, T)
    assert (C == SL.run_slots(SL.make_plan(6, 9, 5, 1), A, B, 256, T)).all()


def test_algorithm1_layout_ignores_the_inner_size():
    # the condition that makes the sum over k a slot-wise sum
    for m, n in [(3, 5), (7, 2)]:
        lays = {SL.result_layout(SL.make_plan(m, l, n, 1)) for l in (1, 2, 5, 9)}
        assert lays == {(m, n, "col")}


def test_algorithm2_mixed_layouts_are_refused():
    rng = np.random.default_rng(9)
    A = rng.integers(0, 256, (100, 100))
    B = rng.integers(0, 256, (100, 100))
    # P2 under Algorithm 2: (64, 64, 64) is case A with t = 1, (64, 36, 64) the l-case, (64, 64, 36) case B
    with pytest.raises(ValueError):
        SL.run_blocked_slots([64, 36], [64, 36], [64, 36], A, B, 8192, T, alg=2)
    # P1 under Algorithm 2: every product is 50 x 50 x 50 (case A, t = 1), one layout
    C = SL.run_blocked_slots([50, 50], [50, 50], [50, 50], A, B, 8192, T, alg=2)
    assert (C == (A @ B) % T).all()


@pytest.fixture(scope="module")
def tiny():
    o = he.Oracle(W.TINY)
    o.keygen(31)
    return o


def encrypt_blocks(o, rows, inner, cols, A, B):
    rb, kb, cb = SL.block_bounds(rows), SL.block_bounds(inner), SL.block_bounds(cols)
    ctA = [[o.encrypt(o.encode(SL.make_plan(r1 - r0, k1 - k0, 1, 1).a_layout(A[r0:r1, k0:k1]) % o.t), 5, 10 * i + k)
            for k, (k0, k1) in enumerate(kb)] for i, (r0, r1) in enumerate(rb)]
    ctB = [[o.encrypt(o.encode(SL.make_plan(1, k1 - k0, c1 - c0, 1).b_layout(B[k0:k1, c0:c1]) % o.t), 6, 10 * k + j)
            for j, (c0, c1) in enumerate(cb)] for k, (k0, k1) in enumerate(kb)]
    return ctA, ctB


@pytest.mark.parametrize("mode", ["single", "double"])
def test_blocked_ciphertexts_decrypt_to_the_product(tiny, mode):
    o = tiny
    rows, inner, cols = [3, 2], [2, 3], [2]
    rng = np.random.default_rng(41)
    A = rng.integers(0, 16, (sum(rows), sum(inner)))
    B = rng.integers(0, 16, (sum(inner), sum(cols)))
    ctA, ctB = encrypt_blocks(o, rows, inner, cols, A, B)
    ex = he.HEGMM(o, mode=mode, lazy_relin=mode == "double")
    Cc = ex.blocked(rows, inner, cols, ctA, ctB)
    rb, cb = SL.block_bounds(rows), SL.block_bounds(cols)
    for i, (r0, r1) in enumerate(rb):
        for j, (c0, c1) in enumerate(cb):
            got = ex.result(SL.make_plan(r1 - r0, inner[0], c1 - c0, 1), Cc[i][j])
            assert (got == (A[r0:r1] @ B[:, c0:c1]) % o.t).all()


def test_sum_products_refuses_mixed_layouts(tiny):
    ex = he.HEGMM(tiny)
    p1 = SL.make_plan(2, 3, 2, 1)
    p2 = SL.make_plan(2, 3, 2, 2)  # case A, t = 2: a 4 x 2 result layout
    assert SL.result_layout(p1) != SL.result_layout(p2)
    with pytest.raises(ValueError):
        ex.sum_products([(p1, None, None), (p2, None, None)])

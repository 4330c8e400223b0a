"""Pins of the oracle's ciphertext-side transformations (Section 3.2.2).

sigma and tau under encryption, the compaction of a product's result to a
plain matrix, and chained products.  What fixes the answers: the
definitions of sigma and tau (Eqs. def:sigma, def:tau), the diagonal bounds
of Theorems 1 and 2 (at most 2 min(m,l) - 1 and 2 min(n,l) - 1 diagonals,
whatever the flattening order), the client-side layouts the product
consumes, and A B mod t / A B D mod t after decryption.
"""
import numpy as np
import pytest

import workload as W
from oracle import he
from oracle import slots as SL

T = 65537


def plain_vec(M, S):
    """Plain column-major matrix slots: i + j rows holds M_ij."""
    v = np.zeros(S, dtype=np.int64)
    r, c = M.shape
    for j in range(c):
        v[j * r:(j + 1) * r] = M[:, j]
    return v


@pytest.mark.parametrize("m,l", [(1, 1), (3, 5), (5, 3), (4, 4), (7, 2), (2, 9)])
def test_sigma_map_is_the_definition(m, l):
    # sigma(A)_{i,j} = A_{i,[i+j]_l}, both sides column-major
    src = SL.layout_source(0, m, l, 3, 1)
    for i in range(m):
        for j in range(l):
            assert src[i + j * m] == i + ((i + j) % l) * m


@pytest.mark.parametrize("l,n", [(1, 1), (3, 5), (5, 3), (4, 4), (2, 7), (9, 2)])
def test_tau_map_is_the_definition(l, n):
    # tau(B)_{i,j} = B_{[i+j]_l,j}
    src = SL.layout_source(1, 3, l, n, 1)
    for i in range(l):
        for j in range(n):
            assert src[i + j * l] == (i + j) % l + j * l


def test_theorems_1_and_2_diagonal_bounds():
    for m in range(1, 11):
        for l in range(1, 11):
            for order in ("col", "row"):
                sm = SL.slot_map((m, l), (m, l), order, SL.sigma_src(l))
                assert len(SL.diagonals_of_map(sm)) <= 2 * min(m, l) - 1, (m, l, order)
                tm = SL.slot_map((l, m), (l, m), order, SL.tau_src(l))
                assert len(SL.diagonals_of_map(tm)) <= 2 * min(m, l) - 1, (l, m, order)
    # the bound is reached, e.g. by a square sigma
    assert len(SL.diagonals_of_map(SL.slot_map((6, 6), (6, 6), "col", SL.sigma_src(6)))) == 11


@pytest.mark.parametrize("shape,alg", [((3, 5, 4), 1), ((3, 5, 4), 2), ((2, 6, 2), 2), ((5, 3, 4), 2),
                                       ((4, 7, 3), 2), ((6, 4, 8), 2), ((6, 4, 8), 1)])
def test_layout_maps_reproduce_the_client_layouts(shape, alg):
    m, l, n = shape
    S = 256
    rng = np.random.default_rng(sum(shape) + alg)
    A = rng.integers(0, T, (m, l))
    B = rng.integers(0, T, (l, n))
    plan = SL.make_plan(m, l, n, alg)
    for role, M, want in ((0, A, plan.a_layout(A) % T), (1, B, plan.b_layout(B) % T)):
        diags = SL.diagonals_of_map({j: s for j, s in enumerate(SL.layout_source(role, m, l, n, alg)) if s >= 0})
        got = SL.apply_lt(plain_vec(M, S), diags, S, T)
        assert (got[: len(want)] == want).all() and not got[len(want):].any()


@pytest.fixture(scope="module")
def medium():
    o = he.Oracle(W.MEDIUM)
    o.keygen(12)
    return o


def enc_plain(o, M, stream):
    return o.encrypt(o.encode(plain_vec(M, o.S) % o.t), 13, stream)


@pytest.mark.parametrize("alg", [1, 2])
def test_encrypted_sigma_tau_then_product(medium, alg):
    o = medium
    ex = he.HEGMM(o)
    m, l, n = 3, 5, 4
    A, B = W.matrices(m, l, n, 0, 15, seed=3)
    ca = ex.to_layout(enc_plain(o, A, 0), 0, m, l, n, alg)
    cb = ex.to_layout(enc_plain(o, B, 1), 1, m, l, n, alg)
    plan = SL.make_plan(m, l, n, alg)
    assert (o.decrypt_slots(ca)[: plan.a_shape[0] * plan.a_shape[1]] == plan.a_layout(A) % o.t).all()
    C = ex.run(plan, ca, cb)
    assert (ex.result(plan, C) == (A @ B) % o.t).all()


def test_result_compaction_and_chain(medium):
    o = medium
    ex = he.HEGMM(o)
    m, l, n, p = 2, 5, 3, 4  # Algorithm 2 case A with t = 3: the result spans 6 x 3 slots
    A, B = W.matrices(m, l, n, 0, 15, seed=4)
    D = np.random.default_rng(5).integers(0, 16, (n, p))
    plan = SL.make_plan(m, l, n, 2)
    assert plan.res_shape == (6, 3)
    ca, cb = ex.encrypt_inputs(plan, A, B, seed=14)
    C = ex.run(plan, ca, cb)
    flat = o.decrypt_slots(ex.from_result(C, m, l, n, 2))
    assert (flat[: m * n] == plain_vec((A @ B) % o.t, o.S)[: m * n]).all() and not flat[m * n:].any()
    plan2 = SL.make_plan(m, n, p, 1)
    X = ex.chain_operand(C, m, l, n, 2, 0, m, n, p, 1)
    _, Y = ex.encrypt_inputs(plan2, np.zeros((m, n), dtype=np.int64), D, seed=15)
    C2 = ex.run(plan2, X, Y)
    assert (ex.result(plan2, C2) == (A @ B @ D) % o.t).all()

"""Pins of two-product packing in slot rows 0 and 1.

The slots of a BGV plaintext with t = 1 mod 2N form two rows of S = N/2; the
Galois element 5^z rotates both rows left by z, and a slot-wise product acts
on each row.  With every mask covering both rows, one HEGMM evaluation
computes the row-0 and the row-1 products.  What fixes the answers: np.roll
of each row, and A0 B0 / A1 B1 mod t after decryption.
"""
import numpy as np
import pytest

import workload as W
from oracle import he
from oracle import slots as SL


@pytest.fixture(scope="module")
def tiny():
    o = he.Oracle(W.TINY)
    o.keygen(17)
    return o


def test_rotation_moves_both_rows(tiny):
    o = tiny
    rng = np.random.default_rng(3)
    r0, r1 = rng.integers(0, o.t, o.S), rng.integers(0, o.t, o.S)
    ct = o.encrypt(o.encode(r0, r1), 4, 0)
    for z in (1, 5, o.S - 2):
        g0, g1 = o.decrypt_rows(o.rotate(ct, z))
        assert (g0 == np.roll(r0, -z)).all() and (g1 == np.roll(r1, -z)).all()


@pytest.mark.parametrize("mode", ["single", "double"])
@pytest.mark.parametrize("shape,alg", [((4, 8, 6), 1), ((4, 8, 6), 2), ((5, 3, 4), 2)])
def test_packed_product_computes_both_rows(tiny, mode, shape, alg):
    o = tiny
    m, l, n = shape
    A0, B0 = W.matrices(m, l, n, 0, 15, seed=1)
    A1, B1 = W.matrices(m, l, n, 0, 15, seed=2)
    ex = he.HEGMM(o, mode=mode, lazy_relin=mode == "double", giant=mode == "double")
    plan = SL.make_plan(m, l, n, alg)
    ca, cb = ex.encrypt_pair(plan, A0, B0, A1, B1, seed=5)
    C0, C1 = ex.result_pair(plan, ex.run(plan, ca, cb))
    assert (C0 == (A0 @ B0) % o.t).all() and (C1 == (A1 @ B1) % o.t).all()


def test_unpacked_product_leaves_row1_zero(tiny):
    o = tiny
    ex = he.HEGMM(o)
    m, l, n = 3, 4, 2
    A, B = W.matrices(m, l, n, 0, 15, seed=6)
    plan = SL.make_plan(m, l, n, 2)
    ca, cb = ex.encrypt_inputs(plan, A, B, seed=6)
    C0, C1 = ex.result_pair(plan, ex.run(plan, ca, cb))
    assert (C0 == (A @ B) % o.t).all() and not C1.any()
    assert not o.decrypt_rows(ex.run(plan, ca, cb))[1].any()

"""The oracle's pins catch plausible mistakes.

Each test plants one mistake in the oracle (on the CPU, through monkeypatch:
a wrong index in a transform, a transposed result slot, an off-by-one block
bound, a mask on one slot row only, ...) and checks that the check a pin
uses fails, while the unplanted oracle passes it.  The checks are the pins'
own criteria: A B mod t from numpy, the client layouts, both rows of a
packed product.
"""
import numpy as np

import workload as W
from oracle import he
from oracle import slots as SL

T = 65537
SHAPES = [(3, 5, 4), (5, 3, 4), (4, 7, 3), (2, 6, 2), (6, 4, 8)]


def products_ok(alg, shapes=SHAPES, S=256):
    for m, l, n in shapes:
        A, B = W.matrices(m, l, n, 0, 255, seed=m * 100 + l * 10 + n)
        if not (SL.run_slots(SL.make_plan(m, l, n, alg), A, B, S, T) == (A @ B) % T).all():
            return False
    return True


def test_unplanted_oracle_passes():
    assert products_ok(1) and products_ok(2)


def test_wrong_sigma_index_is_caught(monkeypatch):
    # sigma(A)_{i,j} = A_{i,[i+j]_l}; a sign slip gives A_{i,[i-j]_l}
    def sigma_bad(A):
        m, l = A.shape
        return np.array([[A[i, (i - j) % l] for j in range(l)] for i in range(m)])

    monkeypatch.setattr(SL, "sigma", sigma_bad)
    assert not products_ok(1)


def test_wrong_tau_index_is_caught(monkeypatch):
    # tau(B)_{i,j} = B_{[i+j]_l,j}; a transposed index B_{[i+j]_l, i} mod n
    def tau_bad(B):
        l, n = B.shape
        return np.array([[B[(i + j) % l, (i + j) % n] for j in range(n)] for i in range(l)])

    monkeypatch.setattr(SL, "tau", tau_bad)
    assert not products_ok(1)


def test_eps_offset_off_by_one_is_caught(monkeypatch):
    good = SL.eps_src
    monkeypatch.setattr(SL, "eps_src", lambda k, l: good(k + 1, l))
    assert not products_ok(1)


def test_wrong_algorithm2_case_is_caught(monkeypatch):
    # the l-case rule (t = 1) where p = m or p = n holds skips partial products
    monkeypatch.setattr(SL, "alg2_case", lambda m, l, n: ("L", min(m, l, n), 1))
    assert not products_ok(2, shapes=[(3, 5, 4), (4, 7, 3), (2, 6, 2)])


def test_transposed_result_slot_is_caught(monkeypatch):
    def slot_bad(self, i, j):
        return SL.flat(j, i, self.res_shape[1], self.res_shape[0], self.order)

    monkeypatch.setattr(SL.Plan, "result_slot", slot_bad)
    assert not products_ok(1)


def test_block_bound_off_by_one_is_caught(monkeypatch):
    rng = np.random.default_rng(4)
    A = rng.integers(0, 256, (12, 10))
    B = rng.integers(0, 256, (10, 9))
    split = ([7, 5], [6, 4], [5, 4])
    assert (SL.run_blocked_slots(*split, A, B, 256, T) == (A @ B) % T).all()
    good = SL.block_bounds

    def bounds_bad(sizes):  # every block after the first starts one row / column late
        return [(s + 1 if s > 0 else s, e) for s, e in good(sizes)]

    monkeypatch.setattr(SL, "block_bounds", bounds_bad)
    assert not (SL.run_blocked_slots(*split, A, B, 256, T) == (A @ B) % T).all()


def test_shifted_layout_map_is_caught(monkeypatch):
    m, l, n = 4, 7, 3
    A = np.random.default_rng(5).integers(0, T, (m, l))
    plan = SL.make_plan(m, l, n, 1)

    def reproduces():
        src = SL.layout_source(0, m, l, n, 1)
        diags = SL.diagonals_of_map({j: s for j, s in enumerate(src) if s >= 0})
        v = np.zeros(256, dtype=np.int64)
        for j in range(l):
            v[j * m:(j + 1) * m] = A[:, j]
        want = plan.a_layout(A) % T
        return (SL.apply_lt(v, diags, 256, T)[: len(want)] == want).all()

    assert reproduces()
    good = SL.layout_source
    monkeypatch.setattr(SL, "layout_source", lambda *a: [s + 1 if s >= 0 else s for s in good(*a)])
    assert not reproduces()


def test_single_row_masks_are_caught(monkeypatch):
    o = he.Oracle(W.TINY)
    o.keygen(23)
    m, l, n = 3, 4, 2
    A0, B0 = W.matrices(m, l, n, 0, 15, seed=1)
    A1, B1 = W.matrices(m, l, n, 0, 15, seed=2)
    plan = SL.make_plan(m, l, n, 1)

    def packed_ok():
        ex = he.HEGMM(o)
        ca, cb = ex.encrypt_pair(plan, A0, B0, A1, B1, seed=3)
        C0, C1 = ex.result_pair(plan, ex.run(plan, ca, cb))
        return (C0 == (A0 @ B0) % o.t).all() and (C1 == (A1 @ B1) % o.t).all()

    assert packed_ok()

    def mask_row0(self, dsts, scale, lv):
        v = np.zeros(self.o.S, dtype=np.int64)
        v[dsts] = scale
        return self.o.plaintext_eval(self.o.encode(v), lv)

    monkeypatch.setattr(he.HEGMM, "mask_eval", mask_row0)
    assert not packed_ok()

"""Pins of Algorithm 1 with the extended pre-layout (HEGMM_ALG_1X).

sigma(A) stored over l + n - 1 columns makes every eps^k one rotation.  What
fixes the answers: Eq. def:eps (eps^k(sigma A)_{i,j} = sigma(A)_{i,[j+k]_l})
read off the stored layout, A B mod t, one diagonal per eps^k at offset k m,
Algorithm 1's omega^k and result layout unchanged, and fewer rotations than
Algorithm 1 whenever Algorithm 1's eps^k wrap.
"""
import itertools

import numpy as np
import pytest

import workload as W
from oracle import he
from oracle import slots as SL

T = 65537


def test_stored_layout_is_sigma_extended():
    rng = np.random.default_rng(1)
    for m, l, n in [(3, 5, 4), (4, 2, 7), (1, 3, 1)]:
        A = rng.integers(0, T, (m, l))
        X = SL.make_plan(m, l, n, 3).a_matrix(A)
        assert X.shape == (m, l + n - 1)
        for i in range(m):
            for c in range(l + n - 1):
                assert X[i, c] == A[i, (i + c) % l]  # Eq. def:sigma at column c mod l
        # Eq. def:eps: eps^k(sigma A)_{i,j} = sigma(A)_{i,[j+k]_l} = X_{i,j+k}
        sA = SL.sigma(A)
        for k in range(l):
            assert (SL.eps(sA, k, m, n) == X[:, k:k + n]).all()


def test_every_shape_multiplies():
    for m, l, n in itertools.product(range(1, 7), repeat=3):
        rng = np.random.default_rng(m * 49 + l * 7 + n)
        A, B = rng.integers(0, T, (m, l)), rng.integers(0, T, (l, n))
        assert (SL.run_slots(SL.make_plan(m, l, n, 3), A, B, 512, T) == (A @ B) % T).all(), (m, l, n)


def test_one_rotation_per_eps_and_algorithm1_omega():
    for m, l, n in [(16, 32, 24), (32, 8, 48), (7, 5, 3)]:
        p3, p1 = SL.make_plan(m, l, n, 3), SL.make_plan(m, l, n, 1)
        for k, ((e3, o3), (_, o1)) in enumerate(zip(p3.iters, p1.iters)):
            assert list(e3) == [k * m] and sorted(e3[k * m]) == list(range(m * n))
            assert o3 == o1
        assert SL.result_layout(p3) == SL.result_layout(p1)
        r3 = sum(1 for e, _ in p3.iters for d in e if d)
        r1 = sum(1 for e, _ in p1.iters for d in e if d)
        assert r3 == l - 1 and r3 <= r1


def test_fits_needs_the_wider_layout():
    assert SL.fits(64, 64, 65, 3, 8192) and not SL.fits(64, 64, 66, 3, 8192)  # 64 x 128 = 8192 slots
    assert SL.fits(64, 64, 64, 1, 4096) and not SL.fits(64, 64, 64, 3, 4096)


@pytest.mark.parametrize("mode", ["single", "double"])
def test_ciphertext_product(mode):
    o = he.Oracle(W.TINY)
    o.keygen(29)
    ex = he.HEGMM(o, mode=mode, lazy_relin=mode == "double", giant=mode == "double")
    for m, l, n in [(4, 8, 6), (3, 2, 5)]:
        A, B = W.matrices(m, l, n, 0, 15, seed=m + l + n)
        plan = SL.make_plan(m, l, n, 3)
        ca, cb = ex.encrypt_inputs(plan, A, B, seed=30)
        assert (ex.result(plan, ex.run(plan, ca, cb)) == (A @ B) % o.t).all()

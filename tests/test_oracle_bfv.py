"""Pins of the BFV variant of the oracle (the paper's scheme, Section 4.1).

What fixes the answers: the negacyclic tensor over Z against a schoolbook
convolution of the centred lifts (tiny N); decryption of fresh ciphertexts
and the slot semantics of HE-Rot (np.roll), HE-CMult and HE-Mult (slot-wise
product mod t) from Section 2.1; the rounding of HE-Mult against the
defining property of a nearest integer (|t d / Q - z| <= 1/2, checked with
exact rationals); HEGMM products decrypting to A B mod t in every mode; and
the noise staying below the budget log2(Q / 2t).
"""
from fractions import Fraction

import numpy as np
import pytest

import workload as W
from oracle import he
from oracle import slots as SL

SMALL = W.Preset("bfv16", logN=4, t=65537, L=2, qbits=30, K=1, alpha=1, scheme=1)


def schoolbook(a, b, N):
    out = [0] * N
    for i in range(N):
        for j in range(N):
            k = i + j
            if k < N:
                out[k] += int(a[i]) * int(b[j])
            else:
                out[k - N] -= int(a[i]) * int(b[j])
    return out


def test_exact_tensor_is_the_integer_negacyclic_product():
    o = he.OracleBFV(SMALL)
    o.keygen(3)
    rng = np.random.default_rng(4)
    a = np.stack([np.stack([rng.integers(0, q, o.N, dtype=np.uint64) for q in o.primes[:o.L]]) for _ in range(2)])
    b = np.stack([np.stack([rng.integers(0, q, o.N, dtype=np.uint64) for q in o.primes[:o.L]]) for _ in range(2)])
    ac = [o._centred(a[i]) for i in range(2)]
    bc = [o._centred(b[i]) for i in range(2)]
    d = o.tensor_exact(a, b)
    assert list(d[0]) == schoolbook(ac[0], bc[0], o.N)
    assert list(d[1]) == [x + y for x, y in zip(schoolbook(ac[0], bc[1], o.N), schoolbook(ac[1], bc[0], o.N))]
    assert list(d[2]) == schoolbook(ac[1], bc[1], o.N)
    # centred lifts: every value within (-Q/2, Q/2]
    assert all(abs(int(x)) <= o.Q // 2 for x in ac[0])


def test_scale_round_is_the_nearest_integer():
    o = he.OracleBFV(SMALL)
    rng = np.random.default_rng(5)
    d = np.array([[int(x) * int(y) - o.Q ** 2 // 3 for x, y in zip(rng.integers(0, 2**62, o.N),
                                                                      rng.integers(0, 2**62, o.N))]], dtype=object)
    z = o.scale_round(d)
    for k in range(o.N):
        exact = Fraction(o.t * int(d[0, k]), o.Q)
        # the residues of z are those of an integer within 1/2 of t d / Q
        cand = round(exact)
        assert abs(exact - cand) <= Fraction(1, 2)
        assert all(int(z[0, i, k]) == cand % o.primes[i] for i in range(o.L))


@pytest.fixture(scope="module")
def tiny():
    o = he.OracleBFV(W.TINY_BFV)
    o.keygen(21)
    return o


def test_encrypt_decrypt_rotate_cmult_mult(tiny):
    o = tiny
    x = np.random.default_rng(1).integers(0, o.t, o.S)
    y = np.random.default_rng(2).integers(0, o.t, o.S)
    cx, cy = o.encrypt(o.encode(x), 1, 0), o.encrypt(o.encode(y), 1, 1)
    m, noise, budget = o.decrypt(cx)
    assert (o.decode(m)[0] == x).all() and noise < 8
    assert (o.decrypt_slots(o.rotate(cx, 5)) == np.roll(x, -5)).all()
    assert (o.decrypt_slots(o.cmult(cx, o.plaintext_eval(o.encode(y), o.L))) == (x * y) % o.t).all()
    p = o.mult_relin(cx, cy)
    m, noise, budget = o.decrypt(p)
    assert (o.decode(m)[0] == (x * y) % o.t).all() and noise < budget - 20
    # the key switching keeps Delta m exact: c0 + c1 s - Delta m is small
    assert o.decrypt(o.rotate(cx, 1))[1] < 16


@pytest.mark.parametrize("mode", ["single", "double", "double+lazy", "double+lazy+shared", "single+lazy"])
@pytest.mark.parametrize("alg", [1, 2, 3])
def test_hegmm_products(tiny, mode, alg):
    o = tiny
    parts = mode.split("+")
    ex = he.HEGMM(o, mode=parts[0], lazy_relin="lazy" in parts, giant="shared" in parts)
    for m, l, n in [(4, 8, 6), (3, 5, 2)]:
        A, B = W.matrices(m, l, n, 0, 15, seed=m + l + n)
        plan = SL.make_plan(m, l, n, alg)
        ca, cb = ex.encrypt_inputs(plan, A, B, seed=7)
        c = ex.run(plan, ca, cb)
        assert (ex.result(plan, c) == (A @ B) % o.t).all()
        _, noise, budget = o.decrypt(c)
        assert noise < budget - 4

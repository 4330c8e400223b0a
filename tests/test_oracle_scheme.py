"""Pins for the ciphertext-level oracle -- CPU only.

The paper fixes only HE-op semantics (Section 2.1: HE-Add, HE-Mult,
HE-CMult, HE-Rot) and the end result A.B; below that the pins are textbook
facts: primality, the NTT against schoolbook convolution and against its
definition, the slot encoding as a ring homomorphism, decryption within the
noise budget, the exact integer meaning of ModUp / ModDown, and
hoisted == unhoisted rotation.
"""
import json
import os

import numpy as np
import pytest
import sympy

import workload as W
from oracle import he
from oracle import slots as SL

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def small(logN, L=2, K=1, alpha=1, qbits=30):
    return W.Preset("small%d" % logN, logN=logN, t=65537, L=L, qbits=qbits, K=K, alpha=alpha)


@pytest.fixture(scope="module")
def tiny():
    o = he.Oracle(W.TINY)
    o.keygen(11)
    return o


def test_splitmix64_published_outputs():
    g = json.load(open(os.path.join(GOLD, "fig4_fig5_blocks.json")))["splitmix64_seed0_first_outputs"]
    got = [he.lib().or_draw(0, i) for i in range(3)]
    assert got == [int(v, 16) for v in g["values"]]


def test_is_prime_matches_sympy():
    rng = np.random.default_rng(0)
    for n in list(rng.integers(2, 2**62, size=300, dtype=np.int64)) + [2, 3, 4, 65537, 2**61 - 1, 3215031751]:
        assert he.is_prime(int(n)) == sympy.isprime(int(n)), n


@pytest.mark.parametrize("pre", [W.TINY, W.MEDIUM, W.PAPER])
def test_prime_chain_rule(pre):
    o = he.Oracle(pre)
    two_n = 2 * pre.N
    ps = o.primes
    assert len(ps) == pre.L + pre.K
    assert all(sympy.isprime(p) and p % two_n == 1 and p < 2**pre.qbits for p in ps)
    assert ps == sorted(ps, reverse=True)
    assert len(set(ps)) == len(ps) and pre.t not in ps
    # No skipped prime: every candidate above q_0 and between chain entries is composite.
    c = ((2**pre.qbits - 1) // two_n) * two_n + 1
    seq = []
    while len(seq) < len(ps):
        if sympy.isprime(c):
            seq.append(c)
        c -= two_n
    assert seq == ps
    assert pre.t % two_n == 1


@pytest.mark.parametrize("logN", [3, 4, 6])
def test_ntt_product_equals_schoolbook(logN):
    o = he.Oracle(small(logN))
    N = 1 << logN
    rng = np.random.default_rng(logN)
    for pi in range(len(o.primes)):
        q = o.primes[pi]
        a = rng.integers(0, q, N, dtype=np.uint64)
        b = rng.integers(0, q, N, dtype=np.uint64)
        x = np.zeros(N, dtype=np.uint64)
        y = np.zeros(N, dtype=np.uint64)
        he.lib().or_polymul(o.ctx, pi, he.P(a), he.P(b), he.P(x))
        he.lib().or_negacyclic_schoolbook(he.P(a), he.P(b), N, q, he.P(y))
        assert (x == y).all()
        # and against Python big integers
        ref = [0] * N
        for i in range(N):
            for j in range(N):
                v = int(a[i]) * int(b[j])
                if i + j < N:
                    ref[i + j] += v
                else:
                    ref[i + j - N] -= v
        assert [r % q for r in ref] == [int(v) for v in x]


@pytest.mark.parametrize("logN", [3, 5])
def test_ntt_is_evaluation_at_odd_powers(logN):
    o = he.Oracle(small(logN))
    N = 1 << logN
    for pi in [-1, 0]:
        q = o.t if pi < 0 else o.primes[pi]
        psi = int(he.lib().or_get_psi(o.ctx, pi))
        assert pow(psi, N, q) == q - 1  # primitive 2N-th root
        a = np.random.default_rng(1).integers(0, q, N, dtype=np.uint64)
        f = o.ntt(a, pi)
        for k in range(N):
            x = pow(psi, 2 * k + 1, q)
            assert int(f[k]) == sum(int(a[i]) * pow(x, i, q) for i in range(N)) % q
        assert (o.intt(f, pi) == a).all()


def test_zeta_and_slot_positions():
    o = he.Oracle(W.TINY)
    # zeta = 3^((t-1)/2N) has order exactly 2N (3 generates Z_65537^*).
    assert pow(o.zeta, o.N, o.t) == o.t - 1
    pos = set(o.slot_pos0.tolist()) | set(o.slot_pos1.tolist())
    assert len(pos) == o.N  # the 2 x S slots cover every evaluation point once


def test_encoding_by_direct_evaluation():
    o = he.Oracle(small(4))
    rng = np.random.default_rng(5)
    r0 = rng.integers(0, o.t, o.S)
    r1 = rng.integers(0, o.t, o.S)
    m = o.encode(r0, r1)
    assert (np.abs(m) <= (o.t - 1) // 2).all()
    for j in range(o.S):
        for row, want in ((1, r0[j]), (-1, r1[j])):
            x = pow(o.zeta, (row * pow(5, j, 2 * o.N)) % (2 * o.N), o.t)
            assert sum(int(m[i]) * pow(x, i, o.t) for i in range(o.N)) % o.t == want


def test_encoding_is_a_ring_homomorphism():
    o = he.Oracle(W.TINY)
    rng = np.random.default_rng(6)
    x, y = rng.integers(0, o.t, o.S), rng.integers(0, o.t, o.S)
    mx, my = o.encode(x), o.encode(y)
    assert (o.decode(mx)[0] == x).all()
    # product in R_t
    a = (mx % o.t).astype(np.uint64)
    b = (my % o.t).astype(np.uint64)
    fa, fb = o.ntt(a, -1), o.ntt(b, -1)
    prod = o.intt((fa.astype(object) * fb.astype(object) % o.t).astype(np.uint64), -1)
    assert (o.decode(prod)[0] == (x * y) % o.t).all()
    assert (o.decode(mx + my)[0] == (x + y) % o.t).all()


def test_encrypt_decrypt_and_noise(tiny):
    o = tiny
    x = np.random.default_rng(7).integers(0, o.t, o.S)
    ct = o.encrypt(o.encode(x), 3, 0)
    m, noise, budget = o.decrypt(ct)
    assert (o.decode(m)[0] == x).all()
    assert noise < 25 and budget > 85
    # deterministic given (seed, stream); a different stream differs
    assert (o.encrypt(o.encode(x), 3, 0) == ct).all()
    assert not (o.encrypt(o.encode(x), 3, 1) == ct).all()


@pytest.mark.parametrize("z", [1, 3, -5, 100, -2047])
def test_rotation_is_slot_rotation(tiny, z):
    # HE-Rot(ct, z) = Enc(x_z, x_{z+1}, ...)  (Section 2.1), within a row.
    o = tiny
    rng = np.random.default_rng(8)
    x, y = rng.integers(0, o.t, o.S), rng.integers(0, o.t, o.S)
    ct = o.encrypt(o.encode(x, y), 4, 0)
    r = o.rotate(ct, z)
    m, noise, budget = o.decrypt(r)
    r0, r1 = o.decode(m)
    assert (r0 == np.roll(x, -z)).all()
    assert (r1 == np.roll(y, -z)).all()
    assert noise < budget - 20


def test_hoisted_rotation_is_bit_identical(tiny):
    o = tiny
    ct = o.encrypt(o.encode(np.arange(o.S)), 5, 0)
    for z in (1, 7, -3):
        assert (o.rotate(ct, z) == o.rotate(ct, z, hoisted=True)).all()


def test_hoisted_rotation_bit_identical_two_prime_digits():
    o = he.Oracle(W.Preset("d2", logN=10, t=65537, L=4, qbits=50, K=2, alpha=2))
    o.keygen(2)
    ct = o.encrypt(o.encode(np.arange(o.S)), 5, 0)
    for z in (1, -9):
        r = o.rotate(ct, z)
        assert (r == o.rotate(ct, z, hoisted=True)).all()
        assert (o.decrypt_slots(r) == np.roll(np.arange(o.S) % o.t, -z)).all()


def test_cmult_add_mult_semantics(tiny):
    o = tiny
    rng = np.random.default_rng(9)
    x, y, w = (rng.integers(0, o.t, o.S) for _ in range(3))
    cx, cy = o.encrypt(o.encode(x), 6, 0), o.encrypt(o.encode(y), 6, 1)
    assert (o.decrypt_slots(o.add(cx, cy)) == (x + y) % o.t).all()
    pt = o.plaintext_eval(o.encode(w), o.L)
    assert (o.decrypt_slots(o.cmult(cx, pt)) == (x * w) % o.t).all()
    prod = o.mult_relin(cx, cy)
    assert (o.decrypt_slots(prod) == (x * y) % o.t).all()


def test_modswitch_scales_message(tiny):
    o = tiny
    x = np.random.default_rng(10).integers(0, o.t, o.S)
    ct = o.encrypt(o.encode(x), 7, 0)
    ms = o.modswitch(ct)
    assert ms.shape[1] == o.L - 1
    qinv = pow(o.primes[o.L - 1], -1, o.t)
    assert (o.decrypt_slots(ms) == (x * qinv) % o.t).all()


def test_keyswitch_switches_secret(tiny):
    # KS(x) = (k0, k1) with k0 + k1 s = x s' + noise, s' = tau_g(s).
    o = tiny
    g = o.galois(1)
    o.add_galois_key(g)
    x = np.random.default_rng(12).integers(0, o.primes[0], (o.L, o.N)).astype(np.uint64)
    x = o.residues(np.random.default_rng(12).integers(-(2**20), 2**20, o.N), o.L)
    ks = o.keyswitch(x, g)
    sg = o.sprime_galois(g)[: o.L]
    v = np.zeros((o.L, o.N), dtype=np.uint64)
    he.lib().or_decrypt_residues(o.ctx, o.L, he.PI(o.sk), he.P(np.ascontiguousarray(ks)), he.P(v))
    for i in range(o.L):
        q = o.primes[i]
        xs = np.zeros(o.N, dtype=np.uint64)
        he.lib().or_polymul(o.ctx, i, he.P(np.ascontiguousarray(x[i])), he.P(np.ascontiguousarray(sg[i])), he.P(xs))
        diff = (v[i].astype(object) - xs.astype(object)) % q
        diff = np.where(diff > q // 2, diff - q, diff)
        assert max(abs(int(d)) for d in diff) < 2**30  # noise, far below q_i
        # and the noise is a multiple of t (BGV)
        assert all(int(d) % o.t == 0 for d in diff)


def test_modup_is_centred_fast_base_conversion():
    o = he.Oracle(W.Preset("d2", logN=4, t=65537, L=4, qbits=50, K=2, alpha=2))
    rng = np.random.default_rng(13)
    lv = 4
    x = np.stack([rng.integers(0, o.primes[i], o.N, dtype=np.uint64) for i in range(lv)])
    D = o.modup(x)
    ext = list(range(lv)) + [o.L + k for k in range(o.K)]
    for j in range(2):
        dig = [2 * j, 2 * j + 1]
        Qj = o.primes[dig[0]] * o.primes[dig[1]]
        for c in range(o.N):
            # the integer the digit stands for, from the definition
            val = 0
            for i in dig:
                hat = Qj // o.primes[i]
                y = int(x[i, c]) * pow(hat, -1, o.primes[i]) % o.primes[i]
                if y > o.primes[i] // 2:
                    y -= o.primes[i]
                val += y * hat
            assert abs(val) <= Qj  # |e| <= alpha/2 overflow at most
            for e, gp in enumerate(ext):
                assert int(D[j, e, c]) == val % o.primes[gp]
            # and on its own primes it is x itself
            for i in dig:
                assert val % o.primes[i] == int(x[i, c])


def test_moddown_is_exact_division_with_t_correction():
    o = he.Oracle(W.Preset("d2", logN=4, t=65537, L=4, qbits=50, K=2, alpha=2))
    rng = np.random.default_rng(14)
    lv = 4
    ext = list(range(lv)) + [o.L + k for k in range(o.K)]
    u = np.stack([rng.integers(0, o.primes[gp], o.N, dtype=np.uint64) for gp in ext])
    out = o.moddown(u, lv)
    Pm = o.primes[o.L] * o.primes[o.L + 1]
    QP = Pm
    for i in range(lv):
        QP *= o.primes[i]
    for c in range(o.N):
        # U: the integer mod QP with these residues (exact CRT)
        U = 0
        for e, gp in enumerate(ext):
            pe = o.primes[gp]
            hat = QP // pe
            U += int(u[e, c]) * hat * pow(hat % pe, -1, pe)
        U %= QP
        # y~ from the definition: sum_k centred([u_k t^-1 (P/p_k)^-1]_{p_k}) (P/p_k)
        yt = 0
        for k in range(o.K):
            pk = o.primes[o.L + k]
            hat = Pm // pk
            z = int(u[lv + k, c]) * pow(o.t, -1, pk) * pow(hat, -1, pk) % pk
            if z > pk // 2:
                z -= pk
            yt += z * hat
        num = U - o.t * yt
        assert num % Pm == 0  # exact division
        w = num // Pm
        for i in range(lv):
            assert int(out[i, c]) == w % o.primes[i]


def test_hegmm_tiny_both_algorithms(tiny):
    o = tiny
    A, B = W.matrices(4, 8, 6, *W.TINY_RANGE)
    ref = (A @ B) % o.t
    for alg in (1, 2):
        plan = SL.make_plan(4, 8, 6, alg)
        ex = he.HEGMM(o)
        ctA, ctB = ex.encrypt_inputs(plan, A, B)
        o.counts = {}
        C = ex.run(plan, ctA, ctB)
        assert (ex.result(plan, C) == ref).all()
        c = plan.counts()
        assert o.counts["mult"] == c["mult"] == (8 if alg == 1 else 4)
        assert o.counts["rot"] == c["rot"]
        _, noise, budget = o.decrypt(C)
        assert noise < budget - 4


def test_hegmm_medium_alg2_small_shape():
    o = he.Oracle(W.MEDIUM)
    o.keygen(3)
    A, B = W.matrices(5, 12, 7, *W.MEDIUM_RANGE)
    plan = SL.make_plan(5, 12, 7, 2)
    ex = he.HEGMM(o)
    ctA, ctB = ex.encrypt_inputs(plan, A, B)
    C = ex.run(plan, ctA, ctB)
    assert (ex.result(plan, C) == (A @ B) % o.t).all()

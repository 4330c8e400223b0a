"""Pins of the oracle's extended-basis key switching ("double hoisting").

The identities checked here come from the definitions, not from the code
under test: ModDown is exact division by P with t-corrected rounding (pinned
on its own in test_oracle_scheme), so ModDown(u + P x) = ModDown(u) + x for
every u and x; multiplying by the constant polynomial 1 is the identity; a
product over the extended basis is the negacyclic schoolbook product modulo
each prime; and the double-hoisted HEGMM decrypts to A B mod t.
"""
import numpy as np
import pytest

import workload as W
from oracle import he
from oracle import slots as SL


def d2_preset():
    return W.Preset("d2", logN=10, t=65537, L=4, qbits=50, K=2, alpha=2)


@pytest.fixture(scope="module")
def tiny():
    o = he.Oracle(W.TINY)
    o.keygen(11)
    return o


@pytest.fixture(scope="module")
def d2():
    o = he.Oracle(d2_preset())
    o.keygen(2)
    return o


def rand_ext(o, lv, rng):
    return np.stack([rng.integers(0, o.primes[gp], o.N, dtype=np.uint64) for gp in o.ext_primes(lv)])


@pytest.mark.parametrize("which", ["tiny", "d2"])
def test_moddown_absorbs_p_multiples(which, tiny, d2):
    o = tiny if which == "tiny" else d2
    rng = np.random.default_rng(21)
    lv = o.L
    u = rand_ext(o, lv, rng)
    x = np.stack([rng.integers(0, o.primes[i], o.N, dtype=np.uint64) for i in range(lv)])
    lhs = o.moddown(o.pq_add(u, o.pq_lift(x)), lv)
    base = o.moddown(u, lv)
    for i in range(lv):
        q = np.uint64(o.primes[i])
        assert ((base[i] + x[i]) % q == lhs[i]).all()


def test_pq_lift_is_p_times_x():
    o = he.Oracle(d2_preset())
    rng = np.random.default_rng(22)
    x = np.stack([rng.integers(0, o.primes[i], o.N, dtype=np.uint64) for i in range(3)])
    y = o.pq_lift(x)
    Pm = o.primes[o.L] * o.primes[o.L + 1]
    for i in range(3):
        assert [int(v) for v in y[i, :16]] == [int(v) * Pm % o.primes[i] for v in x[i, :16]]
    assert (y[3:] == 0).all()


def test_pq_mac_is_schoolbook_product_per_prime():
    o = he.Oracle(W.Preset("s4", logN=4, t=65537, L=3, qbits=30, K=2, alpha=1))
    rng = np.random.default_rng(23)
    lv = 2
    m = rng.integers(-100, 100, o.N)
    a = rand_ext(o, lv, rng)
    acc0 = rand_ext(o, lv, rng)
    acc = acc0.copy()
    o.pq_mac(acc, a, o.plaintext_eval_pq(m, lv))
    for e, gp in enumerate(o.ext_primes(lv)):
        q = o.primes[gp]
        # negacyclic convolution written out: X^N = -1
        want = [int(acc0[e, k]) for k in range(o.N)]
        for i in range(o.N):
            for j in range(o.N):
                k, sgn = (i + j, 1) if i + j < o.N else (i + j - o.N, -1)
                want[k] += sgn * int(a[e, i]) * int(m[j])
        assert [int(v) for v in acc[e]] == [w % q for w in want]


@pytest.mark.parametrize("which", ["tiny", "d2"])
def test_unit_mask_double_hoisted_term_is_the_rotation(which, tiny, d2):
    # with the single mask 1, ModDown(u + P tau(c0)), ModDown(u1) is HE-Rot
    o = tiny if which == "tiny" else d2
    ct = o.encrypt(o.encode(np.arange(o.S) % o.t), 5, 0)
    lv = o.L
    one = np.zeros(o.N, dtype=np.int64)
    one[0] = 1
    m1 = o.plaintext_eval_pq(one, lv)
    D = o.modup(ct[1])
    for z in (1, -3, 17):
        g = o.galois(z)
        o.add_galois_key(g)
        u = o.ks_raw(D, g)
        acc = np.zeros((2, lv + o.K, o.N), dtype=np.uint64)
        o.pq_mac(acc[0], o.pq_add(u[0], o.pq_lift(o.automorph(ct[0], g, list(range(lv))))), m1)
        o.pq_mac(acc[1], u[1], m1)
        assert (o.moddown_pair(acc) == o.rotate(ct, z)).all()


def test_relin_raw_plus_p_d_is_mult(tiny):
    # ModDown(u + P d0, u1 + P d1) is HE-Mult exactly
    o = tiny
    rng = np.random.default_rng(24)
    x, y = rng.integers(0, o.t, o.S), rng.integers(0, o.t, o.S)
    a, b = o.encrypt(o.encode(x), 6, 0), o.encrypt(o.encode(y), 6, 1)
    d = o.tensor(a, b)
    u = o.ks_raw(o.modup(d[2]), 0)
    got = o.moddown_pair(np.stack([o.pq_add(u[0], o.pq_lift(d[0])), o.pq_add(u[1], o.pq_lift(d[1]))]))
    assert (got == o.mult_relin(a, b)).all()


def test_double_lt_decrypts_to_the_plain_transformation(tiny):
    o = tiny
    rng = np.random.default_rng(25)
    x = rng.integers(0, o.t, o.S)
    ct = o.encrypt(o.encode(x), 7, 0)
    diags = {0: [0, 5, 9], 3: [1, 2, 40], -7: list(range(100, 140)), 11: [7]}
    for d in diags:
        if d % o.S:
            o.add_galois_key(o.galois(d))
    ex = he.HEGMM(o, mode="double")
    y = ex.lt(ct, diags, 1)
    want = SL.apply_lt(x, diags, o.S, o.t)
    assert (o.decrypt_slots(y) == want).all()
    _, noise_d, _ = o.decrypt(y)
    _, noise_s, _ = o.decrypt(he.HEGMM(o).lt(ct, diags, 1))
    # the mask times the input noise dominates both; the rounding terms
    # (one per component here, one per term there) are far below it
    assert noise_d < noise_s + 1


@pytest.mark.parametrize("alg", [1, 2])
def test_hegmm_double_mode_tiny(tiny, alg):
    o = tiny
    A, B = W.matrices(4, 8, 6, *W.TINY_RANGE)
    plan = SL.make_plan(4, 8, 6, alg)
    single, double = he.HEGMM(o), he.HEGMM(o, mode="double")
    ctA, ctB = single.encrypt_inputs(plan, A, B)
    Cs = single.run(plan, ctA, ctB)
    Cd = double.run(plan, ctA, ctB)
    assert (double.result(plan, Cd) == (A @ B) % o.t).all()
    assert not (Cs == Cd).all()  # a different evaluation order of the same product
    _, ns, budget = o.decrypt(Cs)
    _, nd, _ = o.decrypt(Cd)
    assert nd < ns + 1 and ns < budget - 4


def test_hegmm_double_mode_two_prime_digits(d2):
    o = d2
    A, B = W.matrices(3, 5, 4, 0, 15)
    plan = SL.make_plan(3, 5, 4, 2)
    ex = he.HEGMM(o, mode="double")
    ctA, ctB = ex.encrypt_inputs(plan, A, B)
    assert (ex.result(plan, ex.run(plan, ctA, ctB)) == (A @ B) % o.t).all()


@pytest.mark.parametrize("mode", ["single", "double"])
def test_lazy_relin_of_one_product_is_mult(tiny, mode):
    # with a single iteration the summed tensor is the tensor itself, so the
    # lazy relinearisation must equal HE-Mult bit for bit in either mode
    o = tiny
    rng = np.random.default_rng(26)
    x, y = rng.integers(0, o.t, o.S), rng.integers(0, o.t, o.S)
    a, b = o.encrypt(o.encode(x), 8, 0), o.encrypt(o.encode(y), 8, 1)
    plan = SL.make_plan(1, 1, 1, 1)  # one iteration, one product
    ex = he.HEGMM(o, mode=mode, lazy_relin=True)
    d = o.tensor(a, b)
    if mode == "double":
        u = o.ks_raw(o.modup(d[2]), 0)
        got = o.moddown_pair(np.stack([o.pq_add(u[0], o.pq_lift(d[0])), o.pq_add(u[1], o.pq_lift(d[1]))]))
    else:
        got = o.add(np.ascontiguousarray(d[:2]), o.keyswitch(d[2], 0))
    assert (got == o.mult_relin(a, b)).all()
    # and a one-iteration product run lazily equals the eager run
    assert len(plan.iters) == 1
    A, B = np.array([[3]]), np.array([[5]])
    eager = he.HEGMM(o, mode=mode)
    ctA, ctB = eager.encrypt_inputs(plan, A, B, seed=4)
    assert (ex.run(plan, ctA, ctB) == eager.run(plan, ctA, ctB)).all()


def test_lazy_relin_sum_decrypts_to_sum_of_products(tiny):
    o = tiny
    rng = np.random.default_rng(27)
    xs = [rng.integers(0, o.t, o.S) for _ in range(6)]
    cts = [o.encrypt(o.encode(x), 9, i) for i, x in enumerate(xs)]
    dsum = None
    for k in range(3):
        d = o.tensor(cts[2 * k], cts[2 * k + 1])
        dsum = d if dsum is None else o.add(dsum, d)
    C = o.add(np.ascontiguousarray(dsum[:2]), o.keyswitch(dsum[2], 0))
    want = (xs[0] * xs[1] + xs[2] * xs[3] + xs[4] * xs[5]) % o.t
    assert (o.decrypt_slots(C) == want).all()


@pytest.mark.parametrize("mode", ["single", "double"])
@pytest.mark.parametrize("alg", [1, 2])
def test_hegmm_lazy_relin_tiny(tiny, mode, alg):
    o = tiny
    A, B = W.matrices(4, 8, 6, *W.TINY_RANGE)
    plan = SL.make_plan(4, 8, 6, alg)
    ex = he.HEGMM(o, mode=mode, lazy_relin=True)
    ctA, ctB = ex.encrypt_inputs(plan, A, B)
    o.counts = {}
    C = ex.run(plan, ctA, ctB)
    assert (ex.result(plan, C) == (A @ B) % o.t).all()
    # one relinearisation key switch per product
    assert o.counts.get("mult", 0) == 0
    _, noise, budget = o.decrypt(C)
    assert noise < budget - 4

"""Pins of the power-of-two key policy (Section 3.3's fallback to Algorithm 1
has offset sets too large to hold one Galois key each).

Under the policy only the keys of rotations by +-2^i exist and every
rotation Rot(x, z) is the chain of HE-Rot by the signed powers of two of the
non-adjacent form of z mod S (or of the same rotation written z - S, if
shorter).  What fixes the answers: the NAF's defining properties (value,
non-adjacency) and its minimal weight, checked by brute force over signed
binary representations; a chained rotation decrypts to np.roll of the
slots; products under the policy decrypt to A.B mod t in every mode; and the
key set it needs is the +-2^i set whatever the plan.
"""
import itertools

import numpy as np
import pytest

import workload as W
from oracle import he
from oracle import slots as SL


def test_naf_value_and_non_adjacency():
    for z in range(-700, 701):
        digits = SL.naf(z)
        assert sum(d * (1 << i) for d, i in digits) == z
        pos = [i for _, i in digits]
        assert pos == sorted(pos) and all(b - a >= 2 for a, b in zip(pos, pos[1:]))
        assert all(d in (-1, 1) for d, _ in digits)


def test_naf_has_minimal_weight():
    # brute force: every signed binary representation with digits in
    # {-1, 0, 1} of up to 8 positions, by value
    best = {}
    for digs in itertools.product((-1, 0, 1), repeat=8):
        v = sum(d << i for i, d in enumerate(digs))
        w = sum(1 for d in digs if d)
        best[v] = min(best.get(v, 99), w)
    for z in range(-100, 101):
        assert len(SL.naf(z)) == best[z], z


def test_pow2_steps_compose_the_rotation():
    for S in (8, 64, 2048, 8192):
        keys = set(SL.pow2_offsets(S))
        assert len(keys) <= 2 * S.bit_length()
        for z in list(range(0, min(S, 300))) + [S - 1, S // 2, S // 2 + 1, 3 * S // 4, -5]:
            steps = SL.pow2_steps(z, S)
            assert sum(steps) % S == z % S
            assert all(s % S in keys for s in steps)
            assert len(steps) <= (S.bit_length() + 1) // 2 + 1


@pytest.fixture(scope="module")
def tiny():
    o = he.Oracle(W.TINY)
    o.keygen(41)
    return o


def test_chained_rotation_decrypts_to_the_slot_rotation(tiny):
    o = tiny
    x = np.random.default_rng(3).integers(0, o.t, o.S)
    ct = o.encrypt(o.encode(x), 4, 0)
    for z in (0, 1, 5, 77, o.S // 2, o.S - 1, o.S - 100):
        r = o.rotate_pow2(ct, z)
        assert (o.decrypt_slots(r) == np.roll(x, -z)).all(), z


@pytest.mark.parametrize("mode", ["single", "double+lazy+shared", "double"])
@pytest.mark.parametrize("alg", [1, 2, 3])
def test_products_under_the_pow2_policy(tiny, mode, alg):
    o = tiny
    base = mode.split("+")[0]
    ex = he.HEGMM(o, mode=base, lazy_relin="lazy" in mode, giant="shared" in mode, key_policy="pow2")
    for m, l, n in [(4, 8, 6), (3, 5, 2)]:
        A, B = W.matrices(m, l, n, 0, 15, seed=m + l + n)
        plan = SL.make_plan(m, l, n, alg)
        ca, cb = ex.encrypt_inputs(plan, A, B, seed=42)
        assert (ex.result(plan, ex.run(plan, ca, cb)) == (A @ B) % o.t).all()


def test_pow2_needs_only_power_of_two_keys():
    # 128 x 16 x 64 under Algorithm 1 at S = 8192 (the N = 2^14 ring):
    # thousands of distinct offsets, one key each under the direct policy
    S = 8192
    plan = SL.make_plan(128, 16, 64, 1)
    direct = {d % S for e, om in plan.iters for diags in (e, om) for d in diags if d % S}
    assert len(direct) > 1000
    chained = {s % S for z in direct for s in SL.pow2_steps(z, S)}
    assert chained <= set(SL.pow2_offsets(S)) and len(SL.pow2_offsets(S)) <= 26

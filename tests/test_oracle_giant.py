"""Pins of the shared-baby-step evaluation order (``slots.giant_factor``).

The factorisation rests on an identity of cyclic rotations, checked here on
plaintext slot vectors against Eq. lintrans for every small shape; the
greedy rule is pinned on hand-made offset sets; the ciphertext executor's
mode is pinned by decryption to A.B and by bit equality where the rule
chooses no giant rotation.
"""
import numpy as np
import pytest

import workload as W
from oracle import he
from oracle import slots as SL


def operand_outputs(plan, s):
    return [it[s] for it in plan.iters]


@pytest.mark.parametrize("alg", [1, 2])
def test_factorisation_is_the_same_transformation(alg):
    S, t = 512, 65537
    rng = np.random.default_rng(40)
    for m in range(1, 7):
        for l in range(1, 7):
            for n in range(1, 7):
                if not SL.fits(m, l, n, alg, S):
                    continue
                plan = SL.make_plan(m, l, n, alg)
                for s in (0, 1):
                    outs = operand_outputs(plan, s)
                    fact = SL.giant_factor(outs, S, cost=1)  # cheap giants: exercise g != 0 often
                    x = rng.integers(0, t, S)
                    for diags, (g, terms) in zip(outs, fact):
                        want = SL.apply_lt(x, diags, S, t)
                        got = np.roll(SL.apply_terms(x, terms, S, t), -g)
                        assert (got == want).all(), (m, l, n, alg, s, g)


@pytest.mark.parametrize("alg", [1, 2])
def test_never_more_key_switches_than_plain_reuse(alg):
    S = 4096
    for m, l, n in [(16, 32, 24), (32, 8, 48), (5, 12, 7), (9, 4, 11), (8, 8, 8), (3, 7, 5)]:
        if not SL.fits(m, l, n, alg, S):
            continue
        plan = SL.make_plan(m, l, n, alg)
        for s in (0, 1):
            outs = operand_outputs(plan, s)
            plain = len({d % S for o in outs for d in o if d % S})
            fact = SL.giant_factor(outs, S)
            baby = {b for _, terms in fact for b, _ in terms if b}
            giants = sum(1 for g, _ in fact if g)
            assert len(baby) + giants <= plain


def test_greedy_rule_on_shifted_offsets():
    S = 64
    sl = [0]
    base = {d: sl for d in range(1, 11)}
    # a shift by 20 of ten offsets: one giant (cost 8) beats ten new offsets
    shifted = {d + 20: sl for d in range(1, 11)}
    f = SL.giant_factor([base, shifted], S)
    assert f[0][0] == 0 and f[1][0] == 20
    assert [b for b, _ in f[1][1]] == list(range(1, 11))
    assert f[1][1][0][1] == [20]  # destination slots move with the giant shift
    # a shift by 3: three new offsets (cost 3) beat a giant (cost 8)
    f = SL.giant_factor([base, {d + 3: sl for d in range(1, 11)}], S)
    assert f[1][0] == 0
    # ties go to the smaller g: offsets {30, 40} against baby {10, 20} are
    # covered by g = 20 (30 -> 10, 40 -> 20) and by g = 30 (30 -> the
    # identity, 40 -> 10) at the same cost
    f = SL.giant_factor([{10: sl, 20: sl}, {30: sl, 40: sl}], S, cost=1)
    assert f[1][0] == 20


@pytest.fixture(scope="module")
def tiny():
    o = he.Oracle(W.TINY)
    o.keygen(11)
    return o


@pytest.mark.parametrize("mode,lazy", [("single", False), ("double", True)])
@pytest.mark.parametrize("alg", [1, 2])
def test_hegmm_giant_mode_decrypts(tiny, mode, lazy, alg):
    o = tiny
    A, B = W.matrices(4, 8, 6, *W.TINY_RANGE)
    plan = SL.make_plan(4, 8, 6, alg)
    ex = he.HEGMM(o, mode=mode, lazy_relin=lazy, giant=True)
    ctA, ctB = ex.encrypt_inputs(plan, A, B)
    C = ex.run(plan, ctA, ctB)
    assert (ex.result(plan, C) == (A @ B) % o.t).all()
    _, noise, budget = o.decrypt(C)
    assert noise < budget - 4


def test_giant_mode_without_giants_is_the_plain_order(tiny):
    o = tiny
    m, l, n = 5, 12, 7
    A, B = W.matrices(m, l, n, *W.TINY_RANGE)
    plan = SL.make_plan(m, l, n, 2)
    fact = [SL.giant_factor(operand_outputs(plan, s), o.S) for s in (0, 1)]
    assert all(g == 0 for f in fact for g, _ in f)
    ex, plain = he.HEGMM(o, mode="double", giant=True), he.HEGMM(o, mode="double")
    ctA, ctB = ex.encrypt_inputs(plan, A, B)
    assert (ex.run(plan, ctA, ctB) == plain.run(plan, ctA, ctB)).all()


def test_hegmm_giant_mode_medium_alg1():
    # a shape where the rule picks giant rotations for omega (B)
    o = he.Oracle(W.MEDIUM)
    o.keygen(3)
    m, l, n = 6, 10, 9
    plan = SL.make_plan(m, l, n, 1)
    fb = SL.giant_factor(operand_outputs(plan, 1), o.S)
    assert any(g for g, _ in fb)
    A, B = W.matrices(m, l, n, *W.MEDIUM_RANGE)
    ex = he.HEGMM(o, mode="double", lazy_relin=True, giant=True)
    ctA, ctB = ex.encrypt_inputs(plan, A, B)
    assert (ex.result(plan, ex.run(plan, ctA, ctB)) == (A @ B) % o.t).all()

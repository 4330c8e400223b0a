"""GPU parity of the power-of-two key policy (HEGMM_KEYS_POW2) against the
oracle's key_policy "pow2", bit for bit, and the key set it keeps.

Under the policy a product's rotations are chains of HE-Rot by +-2^i (the
non-adjacent form of each offset); the library evaluates the chains of an
operand as a tree of batched rotations and the transformations as sums of
mask products over Q.  The oracle composes the same chains from single
rotations.
"""
import numpy as np
import pytest

import workload as W
from oracle import he as OH
from oracle import slots as SL

pytestmark = pytest.mark.gpu

SEED = 77
MODES = {"single": (0, "single", False, False), "double": (1, "double", False, False),
         "double+lazy": (3, "double", True, False), "double+lazy+shared": (7, "double", True, True),
         "single+shared": (4, "single", False, True)}


@pytest.fixture(scope="module")
def H():
    from paper_2405_02238_gb300 import build as B

    B.build()
    from paper_2405_02238_gb300 import hegmm

    return hegmm


_ctx = {}


def context(H, name):
    if name not in _ctx:
        pre = W.PRESETS[name]
        c = H.Context.from_preset(pre)
        c.hegmm_set_key_policy(H.KEYS_POW2)
        c.hegmm_keygen(SEED)
        o = OH.Oracle(pre)
        o.keygen(SEED)
        _ctx[name] = (pre, c, o)
    return _ctx[name]


def run_pow2(H, name, m, l, n, alg, mode, seed=0):
    pre, ctx, o = context(H, name)
    flags, base, lazy, shared = MODES[mode]
    ctx.hegmm_set_keyswitch_mode(flags)
    rng = W.MEDIUM_RANGE if name == "medium" else W.TINY_RANGE
    A, B = W.matrices(m, l, n, *rng, seed=seed)
    ctx.hegmm_keygen(SEED, [(m, l, n)], alg)
    ca = ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_A, A, m, l, n, alg), 13, 300)
    cb = ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_B, B, m, l, n, alg), 13, 301)
    cc, cnt = ctx.hegmm_matmul(ca, cb, m, l, n, alg)
    assert (ctx.hegmm_decrypt(cc, m, l, n, alg).astype(np.int64) == (A @ B) % pre.t).all()
    ralg = alg if alg else SL.choose_alg(m, l, n, o.S)
    plan = SL.make_plan(m, l, n, ralg)
    ex = OH.HEGMM(o, mode=base, lazy_relin=lazy, giant=shared, key_policy="pow2")
    ctA, ctB = ex.encrypt_inputs(plan, A, B, seed=13, streams=(300, 301))
    assert (ctx.hegmm_ct_export(cc) == ex.run(plan, ctA, ctB)).all()
    assert cnt["rot"] == plan.counts()["rot"] and cnt["mult"] == plan.counts()["mult"]
    return ctx, cnt


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("alg", [1, 2, 3])
def test_pow2_tiny_bitexact(H, alg, mode):
    for shape in [(4, 8, 6), (3, 5, 2)]:
        run_pow2(H, "tiny", *shape, alg, mode, seed=sum(shape))


@pytest.mark.parametrize("mode", ["single+shared", "double+lazy+shared"])
def test_pow2_medium_giants_bitexact(H, mode):
    # 6 x 10 x 9 under Algorithm 1: the shared order has giant rotations,
    # which become chains too
    run_pow2(H, "medium", 6, 10, 9, 1, mode)


def test_pow2_medium_extraction_bitexact(H):
    run_pow2(H, "medium", 16, 32, 24, 2, "double+lazy")


def test_pow2_context_keeps_only_power_of_two_keys(H):
    pre, ctx, o = context(H, "tiny")
    keys = ctx.hegmm_key_list()
    want = {o.galois(z) for z in SL.pow2_offsets(o.S)} | {0}
    assert set(keys) == want and len(keys) <= 2 * (o.S.bit_length() - 1) + 1

"""GPU parity of the BFV variant (HEGMM_SCHEME_BFV, the paper's own scheme)
against the oracle's OracleBFV, bit for bit: keys, encryption, rotation,
HE-CMult, HE-Mult (base extension to the auxiliary primes, tensor over
Q u B, rounding by t/Q, relinearisation) and whole HEGMM products in every
key-switch mode, each also decrypted and compared with the slot semantics
or A.B mod t."""
import numpy as np
import pytest

import workload as W
from oracle import he as OH
from oracle import slots as SL

pytestmark = pytest.mark.gpu

SEED = 31
MODES = {"single": (0, "single", False, False), "double": (1, "double", False, False),
         "single+lazy": (2, "single", True, False), "double+lazy": (3, "double", True, False),
         "double+lazy+shared": (7, "double", True, True)}


@pytest.fixture(scope="module")
def H():
    from paper_2405_02238_gb300 import build as B

    B.build()
    from paper_2405_02238_gb300 import hegmm

    return hegmm


_pairs = {}


def get_pair(H, name):
    if name not in _pairs:
        pre = W.PRESETS[name]
        ctx = H.Context.from_preset(pre)
        ctx.hegmm_keygen(SEED)
        o = OH.OracleBFV(pre)
        o.keygen(SEED)
        _pairs[name] = (pre, ctx, o)
    return _pairs[name]


@pytest.mark.parametrize("name", ["tiny_bfv", "medium_bfv", "paper_bfv"])
def test_bfv_operations_bitexact(H, name):
    pre, ctx, o = get_pair(H, name)
    assert (ctx.hegmm_key_export(0) == o.evk_coeff(0)).all()
    x = np.random.default_rng(1).integers(0, o.t, o.S)
    y = np.random.default_rng(2).integers(0, o.t, o.S)
    cx = ctx.hegmm_encrypt(ctx.hegmm_encode_slots(x), 5, 0)
    cy = ctx.hegmm_encrypt(ctx.hegmm_encode_slots(y), 5, 1)
    ox, oy = o.encrypt(o.encode(x), 5, 0), o.encrypt(o.encode(y), 5, 1)
    assert (ctx.hegmm_ct_export(cx) == ox).all()
    assert (ctx.hegmm_decrypt_slots(cx).astype(np.int64) == x).all()
    ctx.hegmm_keygen_rotations([3])
    r = ctx.hegmm_rotate(cx, 3)
    assert (ctx.hegmm_ct_export(r) == o.rotate(ox, 3)).all()
    assert (ctx.hegmm_decrypt_slots(r).astype(np.int64) == np.roll(x, -3)).all()
    cm = ctx.hegmm_cmult(cx, ctx.hegmm_encode_slots(y))
    assert (ctx.hegmm_ct_export(cm) == o.cmult(ox, o.plaintext_eval(o.encode(y), o.L))).all()
    p = ctx.hegmm_mult(cx, cy)
    assert (ctx.hegmm_ct_export(p) == o.mult_relin(ox, oy)).all()
    assert (ctx.hegmm_decrypt_slots(p).astype(np.int64) == (x * y) % o.t).all()


def run_bfv(H, name, m, l, n, alg, mode, seed=0):
    pre, ctx, o = get_pair(H, name)
    flags, base, lazy, shared = MODES[mode]
    ctx.hegmm_set_keyswitch_mode(flags)
    rng = W.MEDIUM_RANGE if name.startswith("medium") else W.TINY_RANGE
    A, B = W.matrices(m, l, n, *rng, seed=seed)
    ctx.hegmm_keygen(SEED, [(m, l, n)], alg)
    ca = ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_A, A, m, l, n, alg), 17, 400)
    cb = ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_B, B, m, l, n, alg), 17, 401)
    cc, cnt = ctx.hegmm_matmul(ca, cb, m, l, n, alg)
    assert (ctx.hegmm_decrypt(cc, m, l, n, alg).astype(np.int64) == (A @ B) % pre.t).all()
    plan = SL.make_plan(m, l, n, alg if alg else SL.choose_alg(m, l, n, o.S))
    ex = OH.HEGMM(o, mode=base, lazy_relin=lazy, giant=shared)
    ctA, ctB = ex.encrypt_inputs(plan, A, B, seed=17, streams=(400, 401))
    assert (ctx.hegmm_ct_export(cc) == ex.run(plan, ctA, ctB)).all()


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("alg", [1, 2, 3])
def test_bfv_tiny_products_bitexact(H, alg, mode):
    for shape in [(4, 8, 6), (3, 5, 2)]:
        run_bfv(H, "tiny_bfv", *shape, alg, mode, seed=sum(shape))


@pytest.mark.parametrize("mode", ["single", "double+lazy+shared"])
def test_bfv_medium_products_bitexact(H, mode):
    run_bfv(H, "medium_bfv", 16, 32, 24, 2, mode)
    run_bfv(H, "medium_bfv", 6, 10, 9, 1, mode)


def test_bfv_batch_equals_single(H):
    pre, ctx, o = get_pair(H, "tiny_bfv")
    ctx.hegmm_set_keyswitch_mode(7)
    shapes = [(4, 8, 6), (3, 5, 2), (6, 2, 7)]
    ctx.hegmm_keygen(SEED, shapes, H.ALG_AUTO)
    As, Bs, mats = [], [], []
    for i, (m, l, n) in enumerate(shapes):
        A, B = W.matrices(m, l, n, 0, 15, seed=i)
        mats.append((A, B))
        As.append(ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_A, A, m, l, n), 21, 2 * i))
        Bs.append(ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_B, B, m, l, n), 21, 2 * i + 1))
    outs = ctx.hegmm_matmul_batch(As, Bs, shapes)
    for i, (m, l, n) in enumerate(shapes):
        single, _ = ctx.hegmm_matmul(As[i], Bs[i], m, l, n)
        assert (ctx.hegmm_ct_export(outs[i]) == ctx.hegmm_ct_export(single)).all()
        A, B = mats[i]
        assert (ctx.hegmm_decrypt(outs[i], m, l, n).astype(np.int64) == (A @ B) % pre.t).all()


def test_bfv_refuses_a_modulus_switch(H):
    with pytest.raises(H.HegmmError):
        H.Context(12, 65537, 3, 30, 1, 1, ms_drop=1, scheme=1)

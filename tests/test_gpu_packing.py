"""GPU parity of two-product packing (slot rows 0 and 1).

hegmm_encode_pair / hegmm_matmul / hegmm_decrypt_pair through the C ABI
against the oracle's ``HEGMM.encrypt_pair`` / ``run`` / ``result_pair`` on
the same seeded inputs, ciphertext for ciphertext, and both rows' products
against A0 B0 and A1 B1 mod t.
"""
import numpy as np
import pytest

import workload as W
from oracle import he as OH
from oracle import slots as SL

pytestmark = pytest.mark.gpu

SEED = 91
MODES = {"single": (0, "single", False, False), "double+lazy+shared": (7, "double", True, True)}


@pytest.fixture(scope="module")
def H():
    from paper_2405_02238_gb300 import build as B

    B.build()
    from paper_2405_02238_gb300 import hegmm

    return hegmm


_pairs = {}


def pair(H, name):
    if name not in _pairs:
        pre = W.PRESETS[name]
        ctx = H.Context.from_preset(pre)
        ctx.hegmm_keygen(SEED)
        o = OH.Oracle(pre)
        o.keygen(SEED)
        _pairs[name] = (ctx, o)
    return _pairs[name]


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("name,shape,alg", [("tiny", (4, 8, 6), 1), ("tiny", (4, 8, 6), 2), ("tiny", (5, 3, 4), 2),
                                            ("medium", (16, 32, 24), 2)])
def test_packed_product_bitexact(H, mode, name, shape, alg):
    ctx, o = pair(H, name)
    flags, base, lazy, shared = MODES[mode]
    ctx.hegmm_set_keyswitch_mode(flags)
    m, l, n = shape
    A0, B0 = W.matrices(m, l, n, 0, 15, seed=1)
    A1, B1 = W.matrices(m, l, n, 0, 15, seed=2)
    ctx.hegmm_keygen(SEED, [shape], alg)
    ca = ctx.hegmm_encrypt(ctx.hegmm_encode_pair(H.ROLE_A, A0, A1, m, l, n, alg), 31, 0)
    cb = ctx.hegmm_encrypt(ctx.hegmm_encode_pair(H.ROLE_B, B0, B1, m, l, n, alg), 31, 1)
    C, _ = ctx.hegmm_matmul(ca, cb, m, l, n, alg)
    ex = OH.HEGMM(o, mode=base, lazy_relin=lazy, giant=shared)
    plan = SL.make_plan(m, l, n, alg)
    oa, ob = ex.encrypt_pair(plan, A0, B0, A1, B1, seed=31, streams=(0, 1))
    assert (ctx.hegmm_ct_export(ca) == oa).all()
    assert (ctx.hegmm_ct_export(C) == ex.run(plan, oa, ob)).all()
    c0, c1 = ctx.hegmm_decrypt_pair(C, m, l, n, alg)
    assert (c0.astype(np.int64) == (A0 @ B0) % o.t).all() and (c1.astype(np.int64) == (A1 @ B1) % o.t).all()
    ctx.hegmm_set_keyswitch_mode(0)


def test_pair_with_one_matrix_is_plain_encode(H):
    ctx, o = pair(H, "tiny")
    m, l, n = 3, 4, 5
    A, B = W.matrices(m, l, n, 0, 15, seed=3)
    for role, M in ((H.ROLE_A, A), (H.ROLE_B, B)):
        x = ctx.hegmm_encrypt(ctx.hegmm_encode(role, M, m, l, n, 1), 32, role)
        y = ctx.hegmm_encrypt(ctx.hegmm_encode_pair(role, M, None, m, l, n, 1), 32, role)
        assert (ctx.hegmm_ct_export(x) == ctx.hegmm_ct_export(y)).all()
    rows = ctx.hegmm_decrypt_rows(y)
    assert (rows[0] == ctx.hegmm_decrypt_slots(y)).all() and not rows[1].any()

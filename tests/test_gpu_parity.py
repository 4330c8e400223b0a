"""GPU parity: the CUDA path through the C ABI against the oracle, bit for bit.

Every ciphertext is compared in the coefficient domain (exported by the
library, computed by the oracle from the same seeds); decrypted products are
compared with A.B mod t in plain integers.  Integer work, so the bar is
exact equality everywhere.
"""
import numpy as np
import pytest

import workload as W
from oracle import he as OH
from oracle import slots as SL

pytestmark = pytest.mark.gpu

SEED = 1234


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
        o = OH.Oracle(pre)
        o.keygen(SEED)
        _pairs[name] = (pre, ctx, o)
    return _pairs[name]


PRESETS = ["tiny", "medium", "paper"]


def rand_slots(o, seed):
    return np.random.default_rng(seed).integers(0, o.t, o.S)


def enc_pair(ctx, o, x, seed, stream):
    ct = ctx.hegmm_encrypt(ctx.hegmm_encode_slots(x), seed, stream)
    co = o.encrypt(o.encode(x), seed, stream)
    return ct, co


@pytest.mark.parametrize("name", PRESETS)
def test_primes_and_keys(H, name):
    pre, ctx, o = get_pair(H, name)
    assert ctx.hegmm_get_primes() == o.primes
    assert (ctx.hegmm_key_export(0) == o.evk_coeff(0)).all()
    ctx.hegmm_keygen_rotations([1])
    g = o.galois(1)
    assert (ctx.hegmm_key_export(g) == o.evk_coeff(g)).all()


@pytest.mark.parametrize("name", PRESETS)
def test_encrypt_decrypt(H, name):
    pre, ctx, o = get_pair(H, name)
    x = rand_slots(o, 1)
    ct, co = enc_pair(ctx, o, x, 3, 7)
    assert (ctx.hegmm_ct_export(ct) == co).all()
    assert (ctx.hegmm_decrypt_slots(ct).astype(np.int64) == x).all()
    # import of the oracle's ciphertext decrypts the same
    ci = ctx.hegmm_ct_import(co)
    assert (ctx.hegmm_ct_export(ci) == co).all()
    assert (ctx.hegmm_decrypt_slots(ci).astype(np.int64) == x).all()


@pytest.mark.parametrize("name", PRESETS)
def test_rotations(H, name):
    pre, ctx, o = get_pair(H, name)
    x = rand_slots(o, 2)
    ct, co = enc_pair(ctx, o, x, 4, 0)
    zs = [1, -3, 17, o.S - 1]
    ctx.hegmm_keygen_rotations(zs)
    outs = ctx.hegmm_rotate_many(ct, zs)
    for z, r in zip(zs, outs):
        ref = o.rotate(co, z)
        assert (ctx.hegmm_ct_export(r) == ref).all(), z
        single = ctx.hegmm_rotate(ct, z)
        assert (ctx.hegmm_ct_export(single) == ref).all(), z
        assert (ctx.hegmm_decrypt_slots(r).astype(np.int64) == np.roll(x, -z)).all()


@pytest.mark.parametrize("name", PRESETS)
def test_cmult_add_mult(H, name):
    pre, ctx, o = get_pair(H, name)
    x, y, w = rand_slots(o, 3), rand_slots(o, 4), rand_slots(o, 5)
    cx, ox = enc_pair(ctx, o, x, 5, 0)
    cy, oy = enc_pair(ctx, o, y, 5, 1)
    cm = ctx.hegmm_cmult(cx, ctx.hegmm_encode_slots(w))
    om = o.cmult(ox, o.plaintext_eval(o.encode(w), o.L))
    assert (ctx.hegmm_ct_export(cm) == om).all()
    ca = ctx.hegmm_add(cx, cy)
    assert (ctx.hegmm_ct_export(ca) == o.add(ox, oy)).all()
    cp = ctx.hegmm_mult(cx, cy)
    assert (ctx.hegmm_ct_export(cp) == o.mult_relin(ox, oy)).all()
    assert (ctx.hegmm_decrypt_slots(cp).astype(np.int64) == (x * y) % o.t).all()


def test_modswitch_tiny(H):
    pre, ctx, o = get_pair(H, "tiny")
    x = rand_slots(o, 6)
    ct, co = enc_pair(ctx, o, x, 6, 0)
    ms = ctx.hegmm_modswitch(ct)
    assert ms.level == o.L - 1
    assert (ctx.hegmm_ct_export(ms) == o.modswitch(co)).all()
    # the relinearisation key restricted to the lower level still works
    p = ctx.hegmm_mult(ms, ms)
    assert (ctx.hegmm_ct_export(p) == o.mult_relin(o.modswitch(co), o.modswitch(co))).all()


MODES = ["single", "double", "single+lazy", "double+lazy", "single+shared", "double+lazy+shared"]


def set_mode(H, ctx, mode):
    """Sets the library's evaluation order; returns the oracle's (mode, lazy_relin, giant)."""
    parts = mode.split("+")
    base, lazy, shared = parts[0], "lazy" in parts, "shared" in parts
    flags = ((H.KS_DOUBLE if base == "double" else H.KS_SINGLE) | (H.KS_LAZY_RELIN if lazy else 0)
             | (H.KS_SHARED if shared else 0))
    ctx.hegmm_set_keyswitch_mode(flags)
    return base, lazy, shared


def run_both(H, name, m, l, n, alg, lo, hi, bitexact=True, seed=0, mode="double", giant_cost=SL.GIANT_COST):
    pre, ctx, o = get_pair(H, name)
    base, lazy, shared = set_mode(H, ctx, mode)
    ctx.hegmm_set_tuning(H.TUNE_GIANT_COST, giant_cost)
    A, B = W.matrices(m, l, n, lo, hi, seed=seed)
    ctx.hegmm_keygen(SEED, [(m, l, n)], alg)
    ca = ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_A, A, m, l, n, alg), 11, 100)
    cb = ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_B, B, m, l, n, alg), 11, 101)
    cc, cnt = ctx.hegmm_matmul(ca, cb, m, l, n, alg)
    got = ctx.hegmm_decrypt(cc, m, l, n, alg).astype(np.int64)
    assert (got == (A @ B) % pre.t).all()
    ralg = alg if alg else SL.choose_alg(m, l, n, o.S)
    plan = SL.make_plan(m, l, n, ralg)
    pc = plan.counts()
    assert cnt["rot"] == pc["rot"] and cnt["mult"] == pc["mult"] and cnt["cmult"] == pc["cmult"]
    assert cnt["relin"] == (1 if lazy else pc["mult"])
    if bitexact:
        ex = OH.HEGMM(o, mode=base, lazy_relin=lazy, giant=shared, giant_cost=giant_cost)
        ctA, ctB = ex.encrypt_inputs(plan, A, B, seed=11, streams=(100, 101))
        assert (ctx.hegmm_ct_export(ca) == ctA).all()
        oc = ex.run(plan, ctA, ctB)
        assert (ctx.hegmm_ct_export(cc) == oc).all()
    return cnt


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("alg", [1, 2])
def test_hegmm_tiny_bitexact(H, alg, mode):
    run_both(H, "tiny", 4, 8, 6, alg, *W.TINY_RANGE, mode=mode)


@pytest.mark.parametrize("chunk,variant,fused,one", [(1, 0, 1, 0), (3, 1, 1, 0), (4096, 2, 1, 0), (32, 3, 1, 0),
                                                      (5, 4, 1, 0), (32, 5, 1, 0), (32, 6, 1, 0), (3, 6, 1, 1),
                                                      (32, 7, 1, 0), (2, 7, 1, 1), (32, 7, 1, 2), (5, 0, 1, 3),
                                                      (32, 0, 0, 0), (32, 8, 1, 0), (3, 8, 1, 0), (32, 7, 1, 4),
                                                      (2, 0, 1, 4)])
def test_double_mode_executor_settings(H, chunk, variant, fused, one):
    # work-item size, fused-kernel variants and the chunked path change no bit
    pre, ctx, o = get_pair(H, "tiny")
    ctx.hegmm_set_tuning(H.TUNE_LT_CHUNK, chunk)
    ctx.hegmm_set_tuning(H.TUNE_LT_KERNEL, variant)
    ctx.hegmm_set_tuning(H.TUNE_LT_FUSED, fused)
    ctx.hegmm_set_tuning(H.TUNE_LT_ONE, one)
    try:
        run_both(H, "tiny", 4, 8, 6, 1, *W.TINY_RANGE, mode="double")
        run_both(H, "tiny", 5, 12, 7, 1, *W.TINY_RANGE, mode="double", seed=3)
        # shared baby steps make a work item's entries serve several outputs
        run_both(H, "tiny", 5, 12, 7, 1, *W.TINY_RANGE, mode="double+lazy+shared", seed=5)
    finally:
        ctx.hegmm_set_tuning(H.TUNE_LT_CHUNK, 32)
        ctx.hegmm_set_tuning(H.TUNE_LT_KERNEL, 6)
        ctx.hegmm_set_tuning(H.TUNE_LT_FUSED, 1)
        ctx.hegmm_set_tuning(H.TUNE_LT_ONE, 4)


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 7, 1), (3, 3, 3), (5, 12, 7), (9, 4, 11), (7, 9, 2), (2, 5, 7),
                                   (5, 4, 2), (12, 3, 9)])
def test_hegmm_tiny_edge_shapes(H, shape):
    for alg in (1, 2):
        for mode in MODES:
            run_both(H, "tiny", *shape, alg, *W.TINY_RANGE, seed=sum(shape), mode=mode)


@pytest.mark.parametrize("mode", ["single", "double", "double+lazy", "double+lazy+shared"])
@pytest.mark.parametrize("shape", W.MEDIUM_SHAPES)
def test_hegmm_medium_alg2_bitexact(H, shape, mode):
    run_both(H, "medium", *shape, 2, *W.MEDIUM_RANGE, mode=mode)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("shape", W.MEDIUM_SHAPES)
def test_hegmm_medium_alg1(H, shape, mode):
    run_both(H, "medium", *shape, 1, *W.MEDIUM_RANGE, bitexact=False, mode=mode)


@pytest.mark.parametrize("mode", ["single+shared", "double+lazy+shared"])
def test_hegmm_medium_alg1_shared_bitexact(H, mode):
    # 6x10x9 under Algorithm 1: the shared-baby-step rule picks giant rotations
    assert any(g for g, _ in SL.giant_factor([it[1] for it in SL.make_plan(6, 10, 9, 1).iters], 4096))
    run_both(H, "medium", 6, 10, 9, 1, *W.MEDIUM_RANGE, mode=mode)


@pytest.mark.parametrize("cost", [1, 3])
def test_shared_mode_other_giant_costs(H, cost):
    # the giant cost picks another factorisation (and new Galois keys, made on
    # first use); each cost is bit-exact with the oracle run at that cost
    try:
        run_both(H, "tiny", 5, 12, 7, 1, *W.TINY_RANGE, mode="double+lazy+shared", seed=7, giant_cost=cost)
        run_both(H, "medium", 6, 10, 9, 1, *W.MEDIUM_RANGE, mode="single+shared", giant_cost=cost)
    finally:
        for name in ("tiny", "medium"):
            get_pair(H, name)[1].hegmm_set_tuning(H.TUNE_GIANT_COST, SL.GIANT_COST)


def test_hegmm_medium_maximum_shape(H):
    # 64 x 64 x 64 fills all 4096 slots of the N=8192 ring.
    run_both(H, "medium", 64, 64, 64, 2, *W.MEDIUM_RANGE, bitexact=False)


@pytest.mark.parametrize("mode", ["single", "double", "double+lazy"])
def test_hegmm_paper_128x16x64_bitexact(H, mode):
    run_both(H, "paper", 128, 16, 64, 0, *W.PAPER_RANGE, mode=mode)


@pytest.mark.parametrize("shape", [(64, 64, 64), (32, 128, 16)])
def test_hegmm_paper_shapes(H, shape):
    run_both(H, "paper", *shape, 0, *W.PAPER_RANGE, bitexact=False)


@pytest.mark.parametrize("mode", MODES)
def test_batch_equals_single(H, mode):
    pre, ctx, o = get_pair(H, "tiny")
    set_mode(H, ctx, mode)
    shapes = [(4, 8, 6), (3, 5, 2), (6, 2, 7)]
    ctx.hegmm_keygen(SEED, shapes, H.ALG_AUTO)
    As, Bs, Cs, mats = [], [], [], []
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


def test_errors(H):
    pre, ctx, o = get_pair(H, "tiny")
    A, B = W.matrices(4, 8, 6, 0, 15)
    with pytest.raises(H.HegmmError) as e:
        ctx.hegmm_encode(H.ROLE_A, np.zeros((65, 64), dtype=np.int64), 65, 64, 64)
    assert e.value.code == -3
    ca = ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_A, A, 4, 8, 6), 1, 0)
    cb = ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_B, B, 4, 8, 6), 1, 1)
    # a shape whose keys were never generated
    fresh = H.Context.from_preset(pre)
    fresh.hegmm_keygen(SEED)
    fa = fresh.hegmm_encrypt(fresh.hegmm_encode(H.ROLE_A, A, 4, 8, 6), 1, 0)
    fb = fresh.hegmm_encrypt(fresh.hegmm_encode(H.ROLE_B, B, 4, 8, 6), 1, 1)
    with pytest.raises(H.HegmmError) as e:
        fresh.hegmm_matmul(fa, fb, 4, 8, 6)
    assert e.value.code == -4
    # operand at the wrong level
    ms = ctx.hegmm_modswitch(ca)
    ctx.hegmm_keygen(SEED, [(4, 8, 6)])
    with pytest.raises(H.HegmmError) as e:
        ctx.hegmm_matmul(ms, cb, 4, 8, 6)
    assert e.value.code == -1


def test_batched_import_export_equal_single(H):
    pre, ctx, o = get_pair(H, "medium")
    rng = np.random.default_rng(61)
    cts = [enc_pair(ctx, o, rand_slots(o, 70 + i), 31, 200 + i)[0] for i in range(5)]
    hosts = [ctx.hegmm_ct_export(ct) for ct in cts]
    back = ctx.hegmm_ct_import_batch(hosts)
    outs = [np.zeros_like(h) for h in hosts]
    ctx.hegmm_ct_export_batch(back, outs)
    for h, b, out in zip(hosts, back, outs):
        assert (out == h).all()
        assert (ctx.hegmm_ct_export(b) == h).all()
        single = ctx.hegmm_ct_import(h)
        assert (ctx.hegmm_ct_export(single) == h).all()
    assert rng is not None


@pytest.mark.parametrize("name", ["medium", "paper"])
def test_ntt_thread_counts_change_no_bit(H, name):
    # both CTA forms of the NTT-family kernels (and the launch-size rule)
    # give the same product, which is the oracle's (a rotation checks the
    # key-switch path alone)
    pre, ctx, o = get_pair(H, name)
    x = rand_slots(o, 12)
    ct, co = enc_pair(ctx, o, x, 8, 0)
    ctx.hegmm_keygen_rotations([5])
    ref = o.rotate(co, 5)
    try:
        for nt in (512, 1024, 0):
            ctx.hegmm_set_tuning(H.TUNE_NTT_THREADS, nt)
            assert (ctx.hegmm_ct_export(ctx.hegmm_rotate(ct, 5)) == ref).all(), nt
            assert (ctx.hegmm_ct_export(ctx.hegmm_mult(ct, ct)) == o.mult_relin(co, co)).all(), nt
    finally:
        ctx.hegmm_set_tuning(H.TUNE_NTT_THREADS, 0)


@pytest.mark.parametrize("name", ["medium", "paper"])
def test_moddown_split_changes_no_bit(H, name):
    # the fused ModDown as two half-limb CTAs per limb gives the oracle's
    # rotation and relinearised product, and a double-hoisted product (whose
    # outputs all go through the fused ModDown) equal to the one-CTA form's
    pre, ctx, o = get_pair(H, name)
    x = rand_slots(o, 13)
    ct, co = enc_pair(ctx, o, x, 9, 0)
    ctx.hegmm_keygen_rotations([7])
    shape = (16, 32, 24) if name == "medium" else (32, 64, 16)
    ctx.hegmm_keygen(SEED, [shape], 2)
    A, B = W.matrices(*shape, 0, 15, seed=2)
    ca = ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_A, A, *shape, 2), 9, 10)
    cb = ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_B, B, *shape, 2), 9, 11)
    ctx.hegmm_set_keyswitch_mode(H.KS_DOUBLE | H.KS_LAZY_RELIN | H.KS_SHARED)
    try:
        ctx.hegmm_set_tuning(H.TUNE_MODDOWN_SPLIT, 0)
        ref, _ = ctx.hegmm_matmul(ca, cb, *shape, 2)
        ref = ctx.hegmm_ct_export(ref)
        for split in (1, 2, 1):
            ctx.hegmm_set_tuning(H.TUNE_MODDOWN_SPLIT, split)
            assert (ctx.hegmm_ct_export(ctx.hegmm_rotate(ct, 7)) == o.rotate(co, 7)).all(), split
            assert (ctx.hegmm_ct_export(ctx.hegmm_mult(ct, ct)) == o.mult_relin(co, co)).all(), split
            c, _ = ctx.hegmm_matmul(ca, cb, *shape, 2)
            assert (ctx.hegmm_ct_export(c) == ref).all(), split
        assert (ctx.hegmm_decrypt(c, *shape, 2).astype(np.int64) == (A @ B) % pre.t).all()
    finally:
        ctx.hegmm_set_tuning(H.TUNE_MODDOWN_SPLIT, 2)
        ctx.hegmm_set_keyswitch_mode(H.KS_SINGLE)

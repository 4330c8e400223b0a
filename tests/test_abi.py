"""CPU checks of the C ABI: the library loads, exports every declared entry
point, and its host-side planner agrees with the oracle's planner.

No GPU is touched: only the host-only planner entry points are called.
"""
import itertools
import os
import re

import numpy as np
import pytest

import workload as W
from oracle import slots as SL

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def H():
    from paper_2405_02238_gb300 import build as B

    B.build()
    from paper_2405_02238_gb300 import hegmm

    hegmm.load()
    return hegmm


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hegmm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hegmm_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(H):
    lib = H.load()
    names = declared_functions()
    assert len(names) >= 30
    for n in names:
        assert hasattr(lib, n), n
    # and the binding declares each one
    assert set(names) == set(H.EXPORTS)


def test_library_is_built_for_sm_103a_only():
    out = os.path.join(ROOT, "paper_2405_02238_gb300", "build.py")
    src = open(out).read()
    assert "arch=compute_103a,code=sm_103a" in src


def oracle_describe(m, l, n, alg, S):
    p = SL.make_plan(m, l, n, alg)
    v = [alg, ord(p.case), 1 if p.order == "col" else 0, len(p.iters), len(p.extract)]
    for e, o in p.iters:
        for diags in (e, o):
            v.append(len(diags))
            for d in sorted(diags):
                v += [d, len(diags[d])] + list(diags[d])
    v += p.extract
    v += [p.result_slot(i, j) for i in range(m) for j in range(n)]
    return v


def test_host_planner_matches_oracle_small_shapes(H):
    for m, l, n in itertools.product(range(1, 8), repeat=3):
        for alg in (1, 2, 3):
            assert H.hegmm_plan_describe(m, l, n, alg, 4096) == oracle_describe(m, l, n, alg, 4096), (m, l, n, alg)


@pytest.mark.parametrize("shape", W.TINY_SHAPES + W.MEDIUM_SHAPES + [(64, 64, 64), (128, 16, 64), (2, 5, 7), (5, 4, 2)])
def test_host_planner_matches_oracle_config_shapes(H, shape):
    m, l, n = shape
    for alg in (1, 2, 3):
        S = 8192
        if not SL.fits(m, l, n, alg, S):
            continue
        assert H.hegmm_plan_describe(m, l, n, alg, S) == oracle_describe(m, l, n, alg, S)
        c = H.hegmm_plan_counts(m, l, n, alg, S)
        oc = SL.make_plan(m, l, n, alg).counts()
        for k in ("rot", "cmult", "mult", "extract"):
            assert c[k] == oc[k]


def test_host_layouts_match_oracle(H):
    rng = np.random.default_rng(0)
    for m, l, n in [(4, 8, 6), (5, 3, 9), (7, 5, 2), (3, 3, 3), (6, 2, 4)]:
        A = rng.integers(-8, 8, size=(m, l))
        B = rng.integers(-8, 8, size=(l, n))
        for alg in (1, 2, 3):
            p = SL.make_plan(m, l, n, alg)
            got_a = H.hegmm_plan_layout(m, l, n, alg, 4096, 0, A, 65537)
            got_b = H.hegmm_plan_layout(m, l, n, alg, 4096, 1, B, 65537)
            assert (got_a.astype(np.int64) == p.a_layout(A) % 65537).all()
            assert (got_b.astype(np.int64) == p.b_layout(B) % 65537).all()


def test_host_slot_maps_match_oracle(H):
    # the maps behind hegmm_to_layout / hegmm_from_result / hegmm_chain_operand
    # and the result layouts hegmm_matmul_sum groups by, for every shape <= 6^3
    for m in range(1, 7):
        for l in range(1, 7):
            for n in range(1, 7):
                for alg in (1, 2, 3):
                    for role in (0, 1):
                        assert H.hegmm_plan_slot_map(m, l, n, alg, 256, role) == SL.layout_source(role, m, l, n, alg)
                    assert H.hegmm_plan_slot_map(m, l, n, alg, 256, 2) == SL.result_source(m, l, n, alg)
                    assert H.hegmm_plan_result_layout(m, l, n, alg, 256) == SL.result_layout(SL.make_plan(m, l, n, alg))
    with pytest.raises(H.HegmmError):
        H.hegmm_plan_slot_map(3, 3, 3, 1, 256, 3)


def test_auto_algorithm_and_shape_errors(H):
    # 32x128x16 does not fit Algorithm 2 at 8192 slots: AUTO gives Algorithm 1.
    assert H.hegmm_plan_describe(32, 128, 16, H.ALG_AUTO, 8192)[0] == 1
    assert H.hegmm_plan_describe(128, 16, 64, H.ALG_AUTO, 8192)[0] == 2
    with pytest.raises(H.HegmmError) as e:
        H.hegmm_plan_describe(200, 200, 200, H.ALG_AUTO, 8192)
    assert e.value.code == -3
    with pytest.raises(H.HegmmError):
        H.hegmm_plan_counts(32, 128, 16, H.ALG_2, 8192)
    with pytest.raises(H.HegmmError):
        H.hegmm_plan_counts(0, 3, 3, H.ALG_1, 8192)


def test_ksw_counts_share_rotations_across_iterations(H):
    # Key switches executed = distinct offsets per operand + one per HE-Mult +
    # one per extraction rotation; never more than the paper's HE-Rot count
    # plus HE-Mult count.
    for m, l, n in [(16, 32, 24), (32, 8, 48), (4, 8, 6)]:
        for alg in (1, 2):
            c = H.hegmm_plan_counts(m, l, n, alg, 4096)
            p = SL.make_plan(m, l, n, alg)
            zs = [set(), set()]
            for e, o in p.iters:
                zs[0].update(d % 4096 for d in e if d % 4096)
                zs[1].update(d % 4096 for d in o if d % 4096)
            assert c["ksw"] == len(zs[0]) + len(zs[1]) + len(p.iters) + len(p.extract)
            assert c["ksw"] <= c["rot"] + c["mult"]


def oracle_giant(m, l, n, alg, S, role, cost=SL.GIANT_COST):
    plan = SL.make_plan(m, l, n, alg)
    f = SL.giant_factor([it[role] for it in plan.iters], S, cost)
    v = [len(f)]
    for g, terms in f:
        v += [g, len(terms)]
        for b, dst in terms:
            v += [b, len(dst)] + list(dst)
    return v


def test_host_shared_baby_steps_match_oracle(H):
    # the greedy factorisation is implemented twice (C++ planner, Python
    # oracle) and must agree term for term
    for m, l, n in list(itertools.product(range(1, 7), repeat=3)) + [(16, 32, 24), (32, 8, 48), (32, 128, 16),
                                                                    (64, 64, 64)]:
        for alg in (1, 2):
            S = 8192 if max(m, l, n) > 16 else 512
            if not SL.fits(m, l, n, alg, S):
                continue
            for role in (0, 1):
                assert H.hegmm_plan_giant(m, l, n, alg, S, role) == oracle_giant(m, l, n, alg, S, role), \
                    (m, l, n, alg, role)
                for cost in (1, 3, 40):
                    assert H.hegmm_plan_giant(m, l, n, alg, S, role, cost) == \
                        oracle_giant(m, l, n, alg, S, role, cost), (m, l, n, alg, role, cost)


def test_host_planner_matches_oracle_serving_shapes(H):
    # larger, uneven shapes of the serving mix (17..64 per dimension): the
    # diagonals (grouped by counting passes) and the shared-baby-step
    # factorisation (giant shifts rotate sorted slot lists) term for term
    rng = np.random.default_rng(11)
    shapes = []
    while len(shapes) < 5:
        m, l, n = (int(v) for v in rng.integers(17, 65, size=3))
        if SL.fits(m, l, n, 1, 8192):
            shapes.append((m, l, n))
    for m, l, n in shapes:
        for alg in (1, 2, 3):
            if not SL.fits(m, l, n, alg, 8192):
                continue
            assert H.hegmm_plan_describe(m, l, n, alg, 8192) == oracle_describe(m, l, n, alg, 8192), (m, l, n, alg)
            if alg != 3:
                for role in (0, 1):
                    assert H.hegmm_plan_giant(m, l, n, alg, 8192, role) == oracle_giant(m, l, n, alg, 8192, role), \
                        (m, l, n, alg, role)


def test_context_refuses_more_modup_limbs_than_a_limb_pattern_holds(H):
    # L = 12, K = 4, alpha = 1: digits(L) (L + K) - L = 180 new limbs per
    # ModUp, more than one limb pattern holds; refused before any CUDA call
    import ctypes

    lib = H.load()
    prm = H.hegmm_params(14, 65537, 12, 50, 4, 1, 21, 0)
    h = ctypes.c_void_p()
    rc = lib.hegmm_ctx_create(ctypes.byref(prm), ctypes.c_void_p(0), ctypes.byref(h))
    assert rc == -1 and not h.value


def test_host_pow2_steps_match_oracle(H):
    for S in (8, 64, 2048, 4096, 8192):
        for z in list(range(-40, 300)) + [S - 1, S // 2, 3 * S // 4 + 1, S + 5]:
            assert H.hegmm_plan_pow2_steps(z, S) == SL.pow2_steps(z, S), (S, z)

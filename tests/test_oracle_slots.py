"""Pins for the slot-level oracle (transforms, diagonals, plans) -- CPU only.

Each test checks the oracle against something the paper or mathematics fixes:
the closed form A.B, the paper's printed U formulas and worked examples,
brute-force diagonal counts against Theorems 1-4, and Theorems 5-6.
"""
import itertools
import json
import os

import numpy as np
import pytest

from oracle import slots as SL

GOLD = os.path.join(os.path.dirname(__file__), "golden")
T = 65537


def rand(m, n, seed):
    return np.random.default_rng(seed).integers(0, 100, size=(m, n))


def test_elementwise_identity_closed_form():
    # Eq. elementwise == plain A.B for every shape up to 6 (proof in Sec. 3.1).
    for m, l, n in itertools.product(range(1, 7), repeat=3):
        A, B = rand(m, l, m * 100 + l), rand(l, n, n * 7 + l)
        assert (SL.elementwise_product(A, B) == A @ B).all(), (m, l, n)


def test_transforms_on_small_example():
    # sigma rotates row i left by i; tau rotates column j up by j (Sec. 3.1 text).
    A = np.arange(12).reshape(3, 4)
    sA = SL.sigma(A)
    for i in range(3):
        assert (sA[i] == np.roll(A[i], -i)).all()
    B = np.arange(12).reshape(4, 3)
    tB = SL.tau(B)
    for j in range(3):
        assert (tB[:, j] == np.roll(B[:, j], -j)).all()
    # eps^0 duplicates / crops columns cyclically, omega^0 rows.
    assert (SL.eps(A, 0, 3, 6)[:, 4:] == A[:, :2]).all()
    assert (SL.omega(B, 0, 6, 3)[4:] == B[:2]).all()


def paper_U_sigma(m, l):
    # Eq. Usigma: U_{i+j m, h} = 1 iff h = i + [i+j]_l m.
    U = np.zeros((m * l, m * l), dtype=np.int64)
    for i in range(m):
        for j in range(l):
            U[i + j * m, i + ((i + j) % l) * m] = 1
    return U


def paper_U_tau(l, n):
    # Eq. Utau: U_{i+j l, h} = 1 iff h = [i+j]_l + j l.
    U = np.zeros((l * n, l * n), dtype=np.int64)
    for i in range(l):
        for j in range(n):
            U[i + j * l, (i + j) % l + j * l] = 1
    return U


def paper_U_eps(m, l, n, k):
    # Eq. Uepsc: U_{i,j} = 1 iff j = [k m + i]_{m l}, i < mn, j < ml.
    U = np.zeros((m * n, m * l), dtype=np.int64)
    for i in range(m * n):
        U[i, (k * m + i) % (m * l)] = 1
    return U


def paper_U_omega(m, l, n, k):
    # Eq. Uomgc: U_{i,j} = 1 iff j = [k + [i]_m]_l + floor(i/m) l.
    U = np.zeros((m * n, l * n), dtype=np.int64)
    for i in range(m * n):
        U[i, (k + i % m) % l + (i // m) * l] = 1
    return U


def test_U_matrices_match_printed_column_major_formulas():
    for m, l, n in itertools.product(range(1, 6), repeat=3):
        assert (SL.u_matrix((m, l), (m, l), "col", SL.sigma_src(l)) == paper_U_sigma(m, l)).all()
        assert (SL.u_matrix((l, n), (l, n), "col", SL.tau_src(l)) == paper_U_tau(l, n)).all()
        for k in range(l):
            assert (SL.u_matrix((m, n), (m, l), "col", SL.eps_src(k, l)) == paper_U_eps(m, l, n, k)).all()
            assert (SL.u_matrix((m, n), (l, n), "col", SL.omega_src(k, l)) == paper_U_omega(m, l, n, k)).all()


@pytest.mark.parametrize("order", ["col", "row"])
def test_lintrans_equals_matrix_vector(order):
    # Eq. lintrans: sum_z u_z (.) Rot(m; z) == U . m, with diagonals taken
    # from U itself and from the slot map (they must agree).
    rng = np.random.default_rng(3)
    S = 128
    for m, l, n in [(3, 4, 5), (5, 3, 4), (2, 7, 3), (4, 4, 4), (6, 2, 5)]:
        for k in range(l):
            for dst, src, fn in [((m, n), (m, l), SL.eps_src(k, l)), ((m, n), (l, n), SL.omega_src(k, l)),
                                 ((m, l), (m, l), SL.sigma_src(l)), ((l, n), (l, n), SL.tau_src(l))]:
                U = SL.u_matrix(dst, src, order, fn)
                dmat = SL.diagonals_of_matrix(U)
                dmap = SL.diagonals_of_map(SL.slot_map(dst, src, order, fn))
                assert set(dmat) == set(dmap)
                for z, u in dmat.items():
                    assert sorted(np.nonzero(u)[0].tolist()) == dmap[z]
                x = np.zeros(S, dtype=np.int64)
                x[: U.shape[1]] = rng.integers(0, 1000, U.shape[1])
                y = SL.apply_lt(x, dmap, S, T)
                ref = (U @ x[: U.shape[1]]) % T
                assert (y[: U.shape[0]] == ref).all()
                assert not y[U.shape[0]:].any()


def test_figure3_worked_examples():
    g = json.load(open(os.path.join(GOLD, "fig3_diagonals.json")))
    e = g["eps"]
    d = SL.diagonals_of_map(SL.slot_map((e["m"], e["n"]), (e["m"], e["l"]), e["order"], SL.eps_src(e["k"], e["l"])))
    want = {int(z): v for z, v in e["diagonals"].items()}
    assert set(d) == set(want)
    for z, v in want.items():
        assert d[z] == [i for i, x in enumerate(v) if x]
    # The caption's counts: u_5 has ten ones, u_-10 five ones.
    assert len(d[5]) == 10 and len(d[-10]) == 5
    w = g["omega"]
    d = SL.diagonals_of_map(SL.slot_map((w["m"], w["n"]), (w["l"], w["n"]), w["order"], SL.omega_src(w["k"], w["l"])))
    want = {int(z): v for z, v in w["diagonals"].items()}
    assert set(d) == set(want)
    for z, v in want.items():
        assert d[z] == [i for i, x in enumerate(v) if x]
    assert len(d[1]) == 10 and len(d[-2]) == 5


def ndiag(dst, src, order, fn):
    return SL.count_diagonals(dst, src, order, fn)


def test_theorems_1_and_2_bounds():
    for m, l, n in itertools.product(range(1, 11), repeat=3):
        for order in ("col", "row"):
            assert ndiag((m, l), (m, l), order, SL.sigma_src(l)) <= 2 * min(m, l) - 1
            assert ndiag((l, n), (l, n), order, SL.tau_src(l)) <= 2 * min(n, l) - 1


def test_theorems_3_and_4_bounds_with_errata():
    # Theorem 3 (col-major) and Theorem 4 (row-major) print floor(n/l)+1 and
    # floor(m/l)+1; brute force shows the bound is ceil(.)+1 when l does not
    # divide n (resp. m).  The other printed bounds hold as stated.
    for m, l, n in itertools.product(range(1, 11), repeat=3):
        for k in range(l):
            ec = ndiag((m, n), (m, l), "col", SL.eps_src(k, l))
            er = ndiag((m, n), (m, l), "row", SL.eps_src(k, l))
            oc = ndiag((m, n), (l, n), "col", SL.omega_src(k, l))
            orr = ndiag((m, n), (l, n), "row", SL.omega_src(k, l))
            assert ec <= -(-n // l) + 1
            assert er <= (n // l + 2) * m
            assert oc <= (m // l + 2) * n
            assert orr <= -(-m // l) + 1
            if n == l:
                assert ec <= 2 and er <= 2
            if m == l:
                assert oc <= 2 and orr <= 2
            if n % l == 0:
                assert ec <= n // l + 1
            if m % l == 0:
                assert orr <= m // l + 1


def test_theorem3_column_major_counterexample():
    # m=1, l=3, n=2, k=2: eps^2 needs two diagonals, floor(2/3)+1 = 1.
    assert ndiag((1, 2), (1, 3), "col", SL.eps_src(2, 3)) == 2


def test_figure4_and_figure5_blocks():
    g = json.load(open(os.path.join(GOLD, "fig4_fig5_blocks.json")))
    f4 = g["fig4"]
    case, p, t = SL.alg2_case(f4["m"], f4["l"], f4["n"])
    assert (case, t) == (f4["case"], f4["t"])
    assert SL.theorem5_blocks(f4["m"], f4["l"], 0, t) == f4["blocks_k0"]
    # Over k = 0..m-1 the partial product p=0 appears twice.
    allp = [q for k in range(f4["m"]) for q in SL.theorem5_blocks(f4["m"], f4["l"], k, t)]
    assert allp.count(f4["duplicated_partial_product"]) == 2
    assert sorted(set(allp)) == list(range(f4["l"]))
    f5 = g["fig5"]
    case, p, t = SL.alg2_case(f5["m"], f5["l"], f5["n"])
    assert (case, t) == (f5["case"], f5["t"])
    assert SL.theorem5_blocks(f5["n"], f5["l"], 0, t) == f5["blocks_k0"]
    assert SL.theorem5_blocks(f5["n"], f5["l"], 1, t) == f5["blocks_k1"]


def test_theorem5_6_block_contents():
    # Block h of eps^k(sigma(Abar)) (.) omega^k(tau(B)) equals the m x n
    # partial product of index [k + h p]_l (Theorems 5 and 6), checked on
    # the matrices directly.
    for m, l, n in [(2, 5, 7), (3, 7, 9), (5, 4, 2), (4, 9, 3)]:
        A, B = rand(m, l, 1), rand(l, n, 2)
        case, p, t = SL.alg2_case(m, l, n)
        sA, tB = SL.sigma(A), SL.tau(B)
        if case == "A":
            Abar = np.vstack([A] * t)
            for k in range(p):
                prod = SL.eps(SL.sigma(Abar), k, t * m, n) * SL.omega(tB, k, t * m, n)
                for h in range(t):
                    q = (k + h * m) % l
                    ref = SL.eps(sA, q, m, n) * SL.omega(tB, q, m, n)
                    assert (prod[h * m:(h + 1) * m] == ref).all()
        else:
            Bbar = np.hstack([B] * t)
            for k in range(p):
                prod = SL.eps(sA, k, m, t * n) * SL.omega(SL.tau(Bbar), k, m, t * n)
                for h in range(t):
                    q = (k + h * n) % l
                    ref = SL.eps(sA, q, m, n) * SL.omega(tB, q, m, n)
                    assert (prod[:, h * n:(h + 1) * n] == ref).all()


def test_plans_compute_the_product():
    S = 512
    for m, l, n in itertools.product(range(1, 9), repeat=3):
        A, B = rand(m, l, 11), rand(l, n, 12)
        ref = (A @ B) % T
        for alg in (1, 2):
            plan = SL.make_plan(m, l, n, alg)
            assert plan.length <= S
            assert (SL.run_slots(plan, A, B, S, T) == ref).all(), (m, l, n, alg)
    # row-major Algorithm 1 as well
    for m, l, n in [(3, 5, 4), (6, 2, 7)]:
        A, B = rand(m, l, 5), rand(l, n, 6)
        plan = SL.make_plan(m, l, n, 1, order="row")
        assert (SL.run_slots(plan, A, B, S, T) == (A @ B) % T).all()


def test_operation_counts_follow_the_paper():
    for m, l, n in itertools.product(range(1, 10), repeat=3):
        p1 = SL.plan_alg1(m, l, n)
        p2 = SL.plan_alg2(m, l, n)
        # HE-Mult count: l for Algorithm 1 (Sec. 3.2.2), p = min(m,l,n) for
        # Algorithm 2 (Sec. 3.3), and t-1 extraction rotations.
        assert p1.counts()["mult"] == l
        assert p2.counts()["mult"] == min(m, l, n)
        assert p2.counts()["extract"] == p2.t - 1
        # Each transform of Algorithm 1 stays within Theorems 3-4 (corrected).
        for e, o in p1.iters:
            assert len(e) <= -(-n // l) + 1
            assert len(o) <= (m // l + 2) * n
        # Algorithm 2 with the case's preferred order needs at most two
        # diagonals for the transform of the duplicated operand (Sec. 3.3).
        for e, o in p2.iters:
            if p2.case == "A":
                assert len(o) <= 2
            if p2.case == "B":
                assert len(e) <= 2


def test_slot_capacity_and_auto_choice():
    # 32x128x16 needs 16384 slots under Algorithm 2 (128 columns duplicated
    # for n=16, t=8), more than the 8192 of N=2^14: AUTO falls back to
    # Algorithm 1 (Sec. 3.3: "we can always resort to Algorithm 1").
    assert SL.alg2_length(32, 128, 16) == 16384
    assert SL.choose_alg(32, 128, 16, 8192) == 1
    assert SL.choose_alg(128, 16, 64, 8192) == 2
    assert SL.choose_alg(64, 64, 64, 8192) == 2
    assert SL.choose_alg(200, 200, 200, 8192) == 0

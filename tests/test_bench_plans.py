"""The benchmark's plan choice per shape (host planner only, no GPU): the
fewest executed key switches among Algorithm 2, the extended pre-layout and
Algorithm 1, and for a shape Algorithm 2 does not fit, Algorithm 2 on the
fewest equal l-blocks that fit.  The blocks of one product share their
result layout (so their sum is the block sum of Section 4.4), and the oracle
planner agrees that the chosen plans compute A.B."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import workload as W  # noqa: E402
from oracle import slots as SL  # noqa: E402


@pytest.fixture(scope="module")
def env():
    from paper_2405_02238_gb300 import build as B

    B.build()
    from paper_2405_02238_gb300 import hegmm as H

    import bench

    return H, bench


def test_paper_plans(env):
    H, bench = env
    S = W.PAPER.slots
    got = bench.workload_products("paper", H, S)
    assert got == [(64, 64, 64, 3, 1), (32, 128, 16, 2, 2), (128, 16, 64, 2, 1)]
    # unblocked: Algorithm 2 does not fit 32x128x16 at S = 8192
    with pytest.raises(H.HegmmError):
        H.hegmm_plan_counts(32, 128, 16, 2, S)
    assert bench.workload_products("paper", H, S, blocks=False)[1] == (32, 128, 16, 3, 1)
    # the blocked plan executes fewer key switches than the best unblocked one
    k2 = 2 * bench.shared_keyswitches(H, 32, 64, 16, 2, S)
    k3 = bench.shared_keyswitches(H, 32, 128, 16, 3, S)
    assert k2 < k3


def test_blocks_share_a_result_layout_and_sum_to_the_product():
    """The chosen blocked plan on plaintext slot vectors: Algorithm 2 on two
    l-blocks of 32x128x16, block results added slot by slot (the HE-Add of
    hegmm_matmul_sum), equals A.B mod t; both blocks have one result layout."""
    m, l, n, nb = 32, 128, 16, 2
    lb = l // nb
    plans = [SL.make_plan(m, lb, n, 2) for _ in range(nb)]
    assert len({SL.result_layout(p) for p in plans}) == 1
    A, B = W.matrices(m, l, n, *W.PAPER_RANGE)
    t, S = W.PAPER.t, W.PAPER.slots
    C = SL.run_blocked_slots([m], [lb] * nb, [n], A, B, S, t, alg=2)
    assert (C == (A @ B) % t).all()

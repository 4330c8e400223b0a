"""Serving (continuous batching) through the C ABI.

Requests arrive while earlier batches are on the GPU; each one's result must
be bit-identical to the same product computed alone, and decrypt to A.B mod t.
"""
import time

import numpy as np
import pytest

import workload as W

pytestmark = pytest.mark.gpu
SEED = 999


@pytest.fixture(scope="module")
def H():
    from paper_2405_02238_gb300 import build as B

    B.build()
    from paper_2405_02238_gb300 import hegmm

    return hegmm


def make_requests(ctx, H, pre, shapes, lo, hi, stream0):
    reqs = []
    for i, (m, l, n) in enumerate(shapes):
        A, B = W.matrices(m, l, n, lo, hi, seed=stream0 + i)
        ca = ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_A, A, m, l, n), 31, stream0 + 2 * i)
        cb = ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_B, B, m, l, n), 31, stream0 + 2 * i + 1)
        reqs.append(((m, l, n), A, B, ca, cb))
    return reqs


def test_serving_mix_equals_alone(H):
    pre = W.TINY
    ctx = H.Context.from_preset(pre)
    rng = np.random.default_rng(1)
    shapes = []
    while len(shapes) < 24:
        m, l, n = (int(v) for v in rng.integers(1, 17, size=3))
        shapes.append((m, l, n))
    ctx.hegmm_keygen(SEED, shapes)
    reqs = make_requests(ctx, H, pre, shapes, 0, 15, 0)
    alone = []
    for (m, l, n), _, _, ca, cb in reqs:
        c, _ = ctx.hegmm_matmul(ca, cb, m, l, n)
        alone.append(ctx.hegmm_ct_export(c))
    srv = H.Server(ctx, max_batch=4, streams=2)
    tickets = []
    for i, ((m, l, n), _, _, ca, cb) in enumerate(reqs):
        tickets.append(srv.hegmm_server_submit(ca, cb, m, l, n))
        if i % 3 == 2:
            srv.hegmm_server_poll()  # later requests arrive while these batches run
    srv.hegmm_server_poll(wait=True)
    st = srv.hegmm_server_stats_get()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["batches"] >= 6 and st["max_batch"] <= 4
    assert st["p99_ms"] >= st["p50_ms"] > 0
    for t, ((m, l, n), A, B, _, _), ref in zip(tickets, reqs, alone):
        got = srv.hegmm_server_result(t)
        assert got is not None
        c, lat = got
        assert lat > 0
        assert (ctx.hegmm_ct_export(c) == ref).all(), (m, l, n)
        assert (ctx.hegmm_decrypt(c, m, l, n).astype(np.int64) == (A @ B) % pre.t).all()
    srv.close()


def test_serving_batches_overlap_on_the_device(H):
    """Two streams, batches of two medium products: with the plans cached by
    a first pass, the second stream's batch is launched while the first
    one's products still run, so their device intervals intersect."""
    pre = W.MEDIUM
    ctx = H.Context.from_preset(pre)
    shapes = [(16, 32, 24)] * 8
    ctx.hegmm_keygen(SEED, shapes[:1])
    reqs = make_requests(ctx, H, pre, shapes, -8, 7, 700)
    for rnd in range(2):  # the first round builds and caches the batch plans
        srv = H.Server(ctx, max_batch=2, streams=2)
        tickets = [srv.hegmm_server_submit(ca, cb, m, l, n) for (m, l, n), _, _, ca, cb in reqs]
        srv.hegmm_server_poll(wait=True)
        st = srv.hegmm_server_stats_get()
        assert st["completed"] == len(reqs) and st["batches"] == 4
        outs = [srv.hegmm_server_result(t)[0] for t in tickets]
        srv.close()
    assert st["max_batches_in_flight"] == 2
    assert st["overlapped_batches"] >= 2, st
    ref, _ = ctx.hegmm_matmul(reqs[0][3], reqs[0][4], 16, 32, 24)
    for ((m, l, n), A, B, ca, cb), c in zip(reqs, outs):
        assert (ctx.hegmm_decrypt(c, m, l, n).astype(np.int64) == (A @ B) % pre.t).all()
    assert (ctx.hegmm_ct_export(outs[0]) == ctx.hegmm_ct_export(ref)).all()


def test_serving_paper_ring(H):
    """The serving mix at N = 2^14 (small, medium and 128x16x64 requests):
    every result decrypts to A.B mod t and equals the product alone."""
    pre = W.PAPER
    ctx = H.Context.from_preset(pre)
    arrivals = W.serving_requests(24, 200.0, ctx.S, seed=5)
    shapes = [s for _, s in arrivals]
    if (128, 16, 64) not in shapes:
        shapes[-1] = (128, 16, 64)
    ctx.hegmm_keygen(SEED, shapes)
    reqs = make_requests(ctx, H, pre, shapes, *W.PAPER_RANGE, 800)
    srv = H.Server(ctx, max_batch=8, streams=2)
    t0 = time.perf_counter()
    tickets = []
    for (at, _), ((m, l, n), _, _, ca, cb) in zip(arrivals, reqs):
        while time.perf_counter() - t0 < at:
            srv.hegmm_server_poll()
        tickets.append(srv.hegmm_server_submit(ca, cb, m, l, n))
        srv.hegmm_server_poll()
    srv.hegmm_server_poll(wait=True)
    st = srv.hegmm_server_stats_get()
    assert st["completed"] == len(reqs) and st["failed"] == 0 and st["batches"] >= 2
    assert st["p99_ms"] >= st["p50_ms"] > 0
    for i, (t, ((m, l, n), A, B, ca, cb)) in enumerate(zip(tickets, reqs)):
        c, _ = srv.hegmm_server_result(t)
        assert (ctx.hegmm_decrypt(c, m, l, n).astype(np.int64) == (A @ B) % pre.t).all(), (m, l, n)
        if i % 4 == 0 or (m, l, n) == (128, 16, 64):
            alone, _ = ctx.hegmm_matmul(ca, cb, m, l, n)
            assert (ctx.hegmm_ct_export(c) == ctx.hegmm_ct_export(alone)).all(), (m, l, n)
    srv.close()


def test_serving_poisson_medium(H):
    pre = W.MEDIUM
    ctx = H.Context.from_preset(pre)
    arrivals = W.serving_requests(40, 400.0, ctx.S, seed=3)
    shapes = [s if s != (128, 16, 64) else (32, 16, 32) for _, s in arrivals]  # N=8192 ring holds 4096 slots
    ctx.hegmm_keygen(SEED, shapes)
    reqs = make_requests(ctx, H, pre, shapes, 0, 15, 500)
    srv = H.Server(ctx, max_batch=16, streams=2)
    t0 = time.perf_counter()
    tickets = []
    for (at, _), ((m, l, n), _, _, ca, cb) in zip(arrivals, reqs):
        while time.perf_counter() - t0 < at:
            srv.hegmm_server_poll()
        tickets.append(srv.hegmm_server_submit(ca, cb, m, l, n))
        srv.hegmm_server_poll()
    srv.hegmm_server_poll(wait=True)
    st = srv.hegmm_server_stats_get()
    assert st["completed"] == len(reqs) and st["batches"] >= 2
    for i, (t, ((m, l, n), A, B, ca, cb)) in enumerate(zip(tickets, reqs)):
        c, _ = srv.hegmm_server_result(t)
        assert (ctx.hegmm_decrypt(c, m, l, n).astype(np.int64) == (A @ B) % pre.t).all(), (m, l, n)
        if i % 8 == 0:
            alone, _ = ctx.hegmm_matmul(ca, cb, m, l, n)
            assert (ctx.hegmm_ct_export(c) == ctx.hegmm_ct_export(alone)).all()
    srv.close()


def test_serving_reports_a_failed_request(H):
    ctx = H.Context.from_preset(W.TINY)
    ctx.hegmm_keygen(SEED, [(3, 4, 5)])
    (_, _, _, ca, cb), = make_requests(ctx, H, W.TINY, [(5, 6, 7)], 0, 15, 900)  # no keys for this shape
    (_, A2, B2, ca2, cb2), = make_requests(ctx, H, W.TINY, [(3, 4, 5)], 0, 15, 950)
    srv = H.Server(ctx, max_batch=1, streams=1)
    bad = srv.hegmm_server_submit(ca, cb, 5, 6, 7)
    good = srv.hegmm_server_submit(ca2, cb2, 3, 4, 5)
    srv.hegmm_server_poll(wait=True)
    with pytest.raises(H.HegmmError) as e:
        srv.hegmm_server_result(bad)
    assert e.value.code == -4
    c, _ = srv.hegmm_server_result(good)
    assert (ctx.hegmm_decrypt(c, 3, 4, 5).astype(np.int64) == (A2 @ B2) % W.TINY.t).all()
    assert srv.hegmm_server_stats_get()["failed"] == 1
    srv.close()

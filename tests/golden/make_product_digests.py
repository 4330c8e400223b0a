"""Writes tests/golden/product_digests.json: the oracle's ciphertexts of the
products the benchmark times, in its evaluation order, as SHA-256 digests of
their bytes plus sampled coefficients.

The oracle (oracle/) is the only thing this script runs.  Each case is one
HEGMM product (Algorithm 1 / 2 of the paper, or Algorithm 1 with the
extended pre-layout) computed by ``oracle.he.HEGMM`` in the double-hoisting
+ lazy-relinearisation + shared-baby-step order (giant cost 8) from the
seeds the GPU test uses: keys from seed 1234, matrices from
``workload.matrices(m, l, n, lo, hi, seed=0)``, operands encrypted with seed
11 on streams 100 (A) and 101 (B).  The digest is taken over the
ciphertext's coefficient-domain residues, little-endian uint64 in
[2][level][N] order (the library's export layout); the samples are 64
(index, value) pairs at positions drawn from numpy's default_rng(case
number), so a mismatch can be located.

Run:  python tests/golden/make_product_digests.py  (about 15 minutes on 8
cores; the cases run in parallel processes).
"""
from __future__ import annotations

import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

KEY_SEED = 1234
ENC_SEED = 11
STREAMS = (100, 101)
GIANT_COST = 8

# (preset, m, l, n, alg[, blocks]): alg 0 = AUTO (Algorithm 2 when it fits), 3 = the extended
# pre-layout; blocks b > 1: the sum of the b products A_k B_k over equal l-blocks (A's column
# blocks, B's row blocks; block k encrypted on streams 100 + 2k, 101 + 2k), in k order
CASES = [
    ("medium", 16, 32, 24, 1),
    ("medium", 32, 8, 48, 1),
    ("medium", 16, 32, 24, 3),
    ("medium", 32, 8, 48, 3),
    ("paper", 64, 64, 64, 0),
    ("paper", 128, 16, 64, 0),
    ("paper", 32, 128, 16, 0),
    ("paper", 64, 64, 64, 3),
    ("paper", 32, 128, 16, 3),
    ("paper", 32, 128, 16, 2, 2),
]


def case_key(pre, m, l, n, alg, blocks=1):
    if blocks > 1:
        return "%s %dx%dx%d alg %d on %d l-blocks double+lazy+shared" % (pre, m, l, n, alg, blocks)
    return "%s %dx%dx%d alg %d double+lazy+shared" % (pre, m, l, n, alg)


def one(args):
    idx, case = args
    pname, m, l, n, alg = case[:5]
    nb = case[5] if len(case) > 5 else 1
    import workload as W
    from oracle import he as OH
    from oracle import slots as SL

    t0 = time.time()
    pre = W.PRESETS[pname]
    o = OH.Oracle(pre)
    o.keygen(KEY_SEED)
    rng_lo_hi = W.PAPER_RANGE if pname == "paper" else W.MEDIUM_RANGE
    A, B = W.matrices(m, l, n, *rng_lo_hi, seed=0)
    lb = l // nb
    ralg = alg if alg else SL.choose_alg(m, lb, n, o.S)
    plan = SL.make_plan(m, lb, n, ralg)
    ex = OH.HEGMM(o, mode="double", lazy_relin=True, giant=True, giant_cost=GIANT_COST)
    items = []
    for k in range(nb):
        ctA, ctB = ex.encrypt_inputs(plan, A[:, k * lb:(k + 1) * lb], B[k * lb:(k + 1) * lb, :], seed=ENC_SEED,
                                     streams=(STREAMS[0] + 2 * k, STREAMS[1] + 2 * k))
        items.append((plan, ctA, ctB))
    ct = ex.run(plan, items[0][1], items[0][2]) if nb == 1 else ex.sum_products(items)
    ct = np.ascontiguousarray(ct, dtype="<u8")
    assert (ex.result(plan, ct) == (A @ B) % o.t).all()
    flat = ct.reshape(-1)
    pos = np.sort(np.random.default_rng(idx).choice(flat.size, 64, replace=False))
    return case_key(*case), {
        "preset": pname, "m": m, "l": l, "n": n, "alg": alg, "blocks": nb, "resolved_alg": ralg,
        "shape": list(ct.shape),
        "sha256": hashlib.sha256(ct.tobytes()).hexdigest(),
        "samples": [[int(i), int(flat[i])] for i in pos], "oracle_s": round(time.time() - t0, 1)}


def main():
    from oracle import he as OH

    OH.build()
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "product_digests.json")
    part = path + ".partial"
    res = json.load(open(part)) if os.path.exists(part) else {}  # cases finished by an earlier run
    todo = [(i, c) for i, c in enumerate(CASES) if case_key(*c) not in res]
    ctx = mp.get_context("spawn")
    with ctx.Pool(max(1, min(len(todo), os.cpu_count() or 1))) as pool:
        for k, v in pool.imap_unordered(one, todo):
            res[k] = v
            with open(part, "w") as f:
                json.dump(res, f)
    res = {case_key(*c): res[case_key(*c)] for c in CASES}
    out = {"how": "oracle.he.HEGMM(mode=double, lazy_relin=True, giant=True, giant_cost=%d); keys seed %d; "
                  "operands encrypted with seed %d, streams %s; matrices workload.matrices(m, l, n, lo, hi, seed=0); "
                  "digest of the [2][level][N] little-endian uint64 coefficient-domain residues"
                  % (GIANT_COST, KEY_SEED, ENC_SEED, list(STREAMS)),
           "cases": res}
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    if os.path.exists(part):
        os.remove(part)
    print("wrote", path, {k: v["oracle_s"] for k, v in res.items()})


if __name__ == "__main__":
    main()

"""Benchmark: encrypted HEGMM products per second on one GB300 (or N replicas).

Default workload (the paper-scale configuration): ring N=16384, t=65537,
eight chain primes below 2^50 plus two special primes (hybrid key switching,
dnum=4); products A 64x64 . B 64x64, A 32x128 . B 128x16 (Algorithm 1:
Algorithm 2 would need 16384 > 8192 slots) and A 128x16 . B 16x64
(Algorithm 2), entries uniform in [0, 255], seed 0.  One step = these three
encrypted products in one batched call.  Operands are encrypted before the
timed region and stay resident in HBM; the per-step working set (Galois keys,
masks) is far larger than L2, and L2 is also flushed between timed steps
(outside the per-step CUDA events).  The one-product-per-launch path is timed
beside it (``per_product_path``), and the medium configuration (N=8192,
16x32x24 and 32x8x48 under both algorithms) under ``medium_workload``.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload paper|medium|batch|serve|blocked|product]

Prints one JSON line.  --impl reference times the plain CPU oracle
(oracle/) on this host's cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workload as W  # noqa: E402

METRIC = "HEGMM encrypted matmuls/s (N=8192 ring, 16x32x24 + 32x8x48, Alg 1 + Alg 2)"
METRIC_BATCH = "HEGMM encrypted matmuls/s (batch of 512 mixed shapes, N=8192 ring)"
METRIC_PAPER = "HEGMM encrypted matmuls/s (N=16384 ring, 64x64x64 + 32x128x16 + 128x16x64)"
UNIT = "matmul/s"
KEY_SEED = 7
SERVE_ARENA_GIB = 16  # server workspace, split over its streams
SERVE_PLAN_GIB = 8  # workspace the plain path's cached plans may keep
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
HBM_FALLBACK = 6800.0
COUNTERS = os.path.join(ROOT, "profiles", "ncu_traffic.json")
# hegmm_set_keyswitch_mode flags per --ks-mode (KS_DOUBLE = 1, KS_LAZY_RELIN = 2, KS_SHARED = 4)
KS_MODES = {"double+lazy+shared": 7, "double+lazy": 3, "double": 1, "single": 0, "single+lazy": 2,
            "single+shared": 4}


def shared_keyswitches(H, m, l, n, alg, slots):
    """Key switches one product executes in the shared-baby-step order
    (distinct baby offsets and giant rotations of both operands, one
    relinearisation, the extraction rotations), from the host planner."""
    ksw = 1 + H.hegmm_plan_counts(m, l, n, alg, slots)["extract"]
    for role in (0, 1):
        v = H.hegmm_plan_giant(m, l, n, alg, slots, role)
        pos, babies, giants = 1, set(), 0
        for _ in range(v[0]):
            g, nt = v[pos], v[pos + 1]
            pos += 2
            giants += g != 0
            for _ in range(nt):
                b, c = v[pos], v[pos + 1]
                pos += 2 + c
                if b:
                    babies.add(b)
        ksw += len(babies) + giants
    return ksw


def fewest_keyswitch_plan(H, m, l, n, slots):
    """(alg, blocks) of a product: of Algorithm 2, Algorithm 1 with the
    extended pre-layout and Algorithm 1 (in that order of preference), the
    one that fits and executes the fewest key switches in the
    shared-baby-step order; and where Algorithm 2 does not fit the slots,
    also Algorithm 2 on the fewest equal l-blocks that fit, summed
    (C = sum_k A_k B_k, Section 4.4's split; the client encodes each block
    pair for Algorithm 2)."""
    cands = []
    for order, alg in enumerate((2, 3, 1)):
        try:
            cands.append((shared_keyswitches(H, m, l, n, alg, slots), order, alg, 1))
        except Exception:
            continue  # does not fit
    if not any(c[2] == 2 for c in cands):
        for b in range(2, l + 1):
            if l % b:
                continue
            try:
                cands.append((b * shared_keyswitches(H, m, l // b, n, 2, slots), 3, 2, b))
                break
            except Exception:
                continue
    best = min(cands)
    return best[2], best[3]


def fewest_keyswitch_alg(H, m, l, n, slots):
    """The algorithm of fewest_keyswitch_plan among unblocked plans."""
    best = None
    for alg in (2, 3, 1):
        try:
            k = shared_keyswitches(H, m, l, n, alg, slots)
        except Exception:
            continue
        if best is None or k < best[1]:
            best = (alg, k)
    return best[0]


def workload_products(kind, H=None, slots=None, blocks=True):
    """[(m, l, n, alg, blocks)] of a throughput workload (alg 0 = AUTO).  The
    paper-scale products take, per shape, the plan with the fewest executed
    key switches (fewest_keyswitch_plan; blocks=False: unblocked plans only)
    when the library is at hand (H), else AUTO."""
    if kind == "paper":
        if H is None:
            return [(m, l, n, 0, 1) for (m, l, n) in W.PAPER_SHAPES]
        if not blocks:
            return [(m, l, n, fewest_keyswitch_alg(H, m, l, n, slots), 1) for (m, l, n) in W.PAPER_SHAPES]
        return [(m, l, n) + fewest_keyswitch_plan(H, m, l, n, slots) for (m, l, n) in W.PAPER_SHAPES]
    if kind == "medium":
        return [(m, l, n, a, 1) for (m, l, n) in W.MEDIUM_SHAPES for a in (1, 2)]
    raise ValueError(kind)


def workload_preset(kind):
    return {"paper": W.PAPER, "medium": W.MEDIUM, "batch": W.MEDIUM}[kind]


def workload_config(extra=None):
    cfg = {
        "workload": "medium: N=8192, t=65537, 5x40-bit + 1 special prime, dnum=5; "
                    "A16x32.B32x24 and A32x8.B8x48, Algorithm 1 and Algorithm 2 each; entries U[-8,7] seed 0",
        "products_per_step": len(workload_products("medium")),
        "l2": "flushed between timed steps (256 MiB write) and per-step key working set > L2",
        "launch": "each cached product plan replayed as one CUDA graph; per-kernel times from a second pass of the "
                  "same steps launched kernel by kernel with CUDA events on the library stream",
    }
    if extra:
        cfg.update(extra)
    return cfg


def paper_config(extra=None):
    cfg = {
        "workload": "paper: N=16384, t=65537, 8x50-bit + 2 special primes, dnum=4; A64x64.B64x64, A32x128.B128x16 "
                    "(Algorithm 2 would need 16384 > 8192 slots), A128x16.B16x64; per shape the plan with the fewest "
                    "executed key switches (see algorithms): Algorithm 2, 1 with the extended pre-layout (3) or 1, "
                    "or, where Algorithm 2 does not fit, Algorithm 2 on the fewest equal l-blocks that fit, summed "
                    "(Section 4.4's split; the client encrypts each block pair); entries U[0,255] seed 0; one "
                    "hegmm_matmul_sum (or hegmm_matmul_batch_algs when nothing is blocked) call per step; "
                    "per_product_path = the plain one-product-per-launch path (hegmm_matmul per block, hegmm_add); "
                    "unblocked_plans = the same products with one ciphertext per matrix",
        "products_per_step": len(W.PAPER_SHAPES),
        "l2": "flushed between timed steps (256 MiB write); per-step key working set (key_bytes) >> L2",
        "launch": "the cached plan replayed as one CUDA graph; per-kernel times from a second pass of the same "
                  "steps launched kernel by kernel with CUDA events on the library stream",
    }
    if extra:
        cfg.update(extra)
    return cfg


def batch_config(extra=None):
    cfg = {
        "workload": "batch: N=8192, t=65537, 5x40-bit + 1 special prime; 512 products with m,l,n uniform in "
                    "4..64 (ml, ln, mn <= 4096), AUTO algorithm, entries U[0,15], seed 0; one "
                    "hegmm_matmul_batch_algs call per step",
        "products_per_step": W.BATCH_COUNT,
        "l2": "flushed between timed steps (256 MiB write); per-step working set (keys 15 GB, masks) >> L2",
        "launch": "the cached plan replayed as one CUDA graph; per-kernel times from a second pass of the same "
                  "steps launched kernel by kernel with CUDA events on the library stream",
    }
    if extra:
        cfg.update(extra)
    return cfg


# ----------------------------------------------------------------------------- clocks


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if not self.rows:
            return None
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) < 9:
                continue
            for i, nm in enumerate(names):
                if r[5 + i].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


# ----------------------------------------------------------------------------- oracle (CPU) timing


_oracle_cache = {}
SAMPLE_KEYS = 4  # distinct rotation offsets of the sample (a rotation's cost does not depend on it)


def oracle_sample(prods, preset, nrot=6, ncm=6, nmul=2):
    """Times the oracle on a bounded sample of a workload.

    The oracle executes a product as a fixed sequence of HE-Rot, HE-CMult,
    HE-Add and HE-Mult calls (no reuse between iterations: the paper's cost
    model), so its time per workload step is the plans' op counts times the
    measured time of each op.  The sample runs ``nrot`` rotations (cycling
    over SAMPLE_KEYS offsets), ``ncm`` mask products and additions and
    ``nmul`` relinearised products at the workload's parameters; key
    generation is excluded.  prods: [(m, l, n, alg[, blocks])], alg 0 =
    AUTO; a product of b blocks runs b products of l / b and b - 1 adds.
    Returns (extrapolated seconds per workload step, description, seconds
    the sample itself took).
    """
    from oracle import he as OH
    from oracle import slots as SL

    pre = preset
    if pre.name not in _oracle_cache:
        o = OH.Oracle(pre)
        o.keygen(KEY_SEED)
        for z in range(1, SAMPLE_KEYS + 1):
            o.add_galois_key(o.galois(z))
        _oracle_cache[pre.name] = o
    o = _oracle_cache[pre.name]
    x = np.arange(o.S) % o.t
    ct = o.encrypt(o.encode(x), 1, 0)
    pt = o.plaintext_eval(o.encode((x * 3) % o.t), o.L)
    s0 = time.perf_counter()
    t0 = time.perf_counter()
    for i in range(nrot):
        o.rotate(ct, 1 + i % SAMPLE_KEYS)
    t_rot = (time.perf_counter() - t0) / nrot
    t0 = time.perf_counter()
    for _ in range(ncm):
        r = o.cmult(ct, pt)
    t_cm = (time.perf_counter() - t0) / ncm
    t0 = time.perf_counter()
    for _ in range(ncm):
        o.add(ct, r)
    t_add = (time.perf_counter() - t0) / ncm
    t0 = time.perf_counter()
    for _ in range(nmul):
        o.mult_relin(ct, r)
    t_mul = (time.perf_counter() - t0) / nmul
    sample_s = time.perf_counter() - s0
    total = 0.0
    for pr in prods:
        m, l, n, alg = pr[:4]
        nb = pr[4] if len(pr) > 4 else 1
        a = alg if alg else SL.choose_alg(m, l // nb, n, o.S)
        c = SL.make_plan(m, l // nb, n, a).counts()
        total += nb * (c["rot"] * t_rot + c["cmult"] * (t_cm + t_add) + c["mult"] * (t_mul + t_add))
        total += (nb - 1) * t_add  # the block sum
    desc = ("%d rotations, %d mask products + adds, %d relinearised products at N=%d/L=%d timed (%.1f s); "
            "per-step time = op counts of the %d plans (the oracle's single-mode op sequence) x measured op times "
            "(%.1f/%.2f/%.2f/%.1f ms rot/cmult/add/mult); keygen excluded"
            % (nrot, ncm, nmul, o.N, o.L, sample_s, len(prods), t_rot * 1e3, t_cm * 1e3, t_add * 1e3, t_mul * 1e3))
    return total, desc, sample_s


def _oracle_worker(args):
    """One all-cores worker (spawned process): set-up, then the sample once
    the parent releases every worker together."""
    prods, preset_name, nrot, ncm, nmul, ready, go = args
    pre = W.PRESETS[preset_name]
    oracle_sample(prods, pre, 1, 1, 1)  # keys and tables, untimed
    ready.put(1)
    go.wait()
    sec, _, sample_s = oracle_sample(prods, pre, nrot, ncm, nmul)
    return sec, sample_s


def cpu_baseline(prods, preset, single=(40, 40, 12), each=(16, 16, 4)):
    """The oracle on this host's cores: the single-core sample (about 10 s
    of CPU work at N=2^14), then every core running the smaller sample at
    once (spawned processes, released together).  Both are extrapolated from
    timed op samples to the workload step (see oracle_sample)."""
    sec, desc, sample_s = oracle_sample(prods, preset, *single)
    one = len(prods) / sec
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    out = {"value": one, "unit": UNIT, "cores": 1, "kind": "oracle", "method": "extrapolated",
           "sample": desc, "sample_s": sample_s}
    if cores > 1:
        ctx = mp.get_context("spawn")
        with ctx.Manager() as man:
            go, ready = man.Event(), man.Queue()
            with ctx.Pool(cores) as pool:
                res = pool.map_async(_oracle_worker, [(prods, preset.name, *each, ready, go)] * cores)
                for _ in range(cores):  # every worker has finished its set-up
                    ready.get(timeout=600)
                w0 = time.perf_counter()
                go.set()
                got = res.get(timeout=600)
                wall = time.perf_counter() - w0
        allv = sum(len(prods) / sec_i for sec_i, _ in got)
        out = {"value": allv, "unit": UNIT, "cores": cores, "kind": "oracle", "method": "extrapolated",
               "sample": "every core at once (spawned processes released together, %.1f s wall): %d rotations, "
                         "%d mask products + adds, %d relinearised products each, extrapolated per core as the "
                         "single-core figure and summed" % (wall, *each),
               "single_core": out}
    return out


def run_reference(args):
    """The reference arm: the plain CPU oracle (there is no other
    implementation of the paper's method; its own code is not published) on
    this host's cores, on the bench's workload.  Each step is a bounded
    sample of the workload's operations, timed; the line's ms_per_step is
    that sample's measured time and its value the throughput the sample
    extrapolates to for the whole workload step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    kind = args.workload if args.workload in ("paper", "medium") else "paper"
    prods = workload_products(kind)
    if kind == "paper" and not args.paper_auto:
        # the algorithms the GPU arm picks (host planner queries only; no GPU)
        try:
            from paper_2405_02238_gb300 import build as B

            B.build()
            from paper_2405_02238_gb300 import hegmm as H

            prods = workload_products(kind, H, W.PAPER.slots)
        except Exception:
            pass
    pre = workload_preset(kind)
    for _ in range(args.warmup):
        oracle_sample(prods, pre)
    secs, samples = [], []
    desc = ""
    for _ in range(args.steps):
        sec, desc, sample_s = oracle_sample(prods, pre)
        secs.append(sec)
        samples.append(sample_s)
    sec = statistics.mean(secs)
    value = len(prods) / sec
    cfg = (paper_config if kind == "paper" else workload_config)()
    line = {
        "impl": "reference", "metric": METRIC_PAPER if kind == "paper" else METRIC, "value": value, "unit": UNIT,
        "n_gpus": 0, "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(samples) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": cfg,
        "value_method": "extrapolated: each step times an op sample of the workload (ms_per_step) and scales it by "
                        "the plans' op counts to a whole workload step (%.1f s per step on one core)" % sec,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "method": "extrapolated",
                         "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def max_over_ranks(ms: float, world: int, dist=None, device="cpu") -> float:
    """The step time of the job: the slowest rank's (all_reduce MAX)."""
    if world <= 1:
        return ms
    import torch

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(products_per_rank: int, world: int, ms: float) -> float:
    """Matmuls per second over all ranks (replicas: each rank runs its own products)."""
    return products_per_rank * world / (ms / 1e3)


# ----------------------------------------------------------------------------- serving


def run_serve(args):
    """Poisson arrivals on the paper ring (N=16384), swept over rates.

    For each rate, min(max_requests, rate * serve_seconds) requests arrive
    (70% m,l,n in 1..16, 25% in 17..64 fitting 8192 slots, 5% 128x16x64;
    entries U[0,255]); the server (continuous batching) is compared with the
    plain path that runs each request alone, in arrival order, as soon as the
    previous one is done.  Keys and masks of every shape are prepared first.
    """
    import torch

    from paper_2405_02238_gb300 import build as B

    B.build()
    from paper_2405_02238_gb300 import hegmm as H

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    pre = W.PAPER
    ctx = H.Context.from_preset(pre, stream=stream.cuda_stream)
    ctx.hegmm_set_keyswitch_mode(KS_MODES[args.ks_mode])
    rates = [float(r) for r in args.rates.split(",")]
    per_rate = {}
    for r in rates:
        cnt = int(max(20, min(args.max_requests, r * args.serve_seconds)))
        per_rate[r] = W.serving_requests(cnt, r, ctx.S, seed=int(r))
    shapes = sorted({s for v in per_rate.values() for _, s in v})
    t0 = time.perf_counter()
    ctx.hegmm_keygen(KEY_SEED, shapes, H.ALG_AUTO)
    torch.cuda.synchronize()
    # masks take what the keys leave, less the server's arenas, the cached
    # plans of the plain path, the largest rate's operands and results (three
    # ciphertexts a request) and a margin
    free_b, _ = torch.cuda.mem_get_info(dev)
    ct_b = 2 * pre.L * (1 << pre.logN) * 8
    keep = (SERVE_ARENA_GIB + SERVE_PLAN_GIB + 8 << 30) + 3 * ct_b * max(len(v) for v in per_rate.values())
    mask_b = min(args.mask_gib << 30, max(1 << 30, free_b - keep))
    ctx.hegmm_set_budgets(mask_bytes=mask_b, plan_bytes=SERVE_PLAN_GIB << 30)
    print("serve: %d shapes, %.1f GiB free after keys, mask budget %.1f GiB"
          % (len(shapes), free_b / 2**30, mask_b / 2**30), file=sys.stderr)
    ctx.hegmm_prepare(shapes, H.ALG_AUTO)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    results = []
    for r in rates:
        arr = per_rate[r]
        ops = []
        for i, (_, (m, l, n)) in enumerate(arr):
            A, Bm = W.matrices(m, l, n, *W.PAPER_RANGE, seed=i)
            ca = ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_A, A, m, l, n), 5, 2 * i)
            cb = ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_B, Bm, m, l, n), 5, 2 * i + 1)
            ops.append((m, l, n, A, Bm, ca, cb))
        torch.cuda.synchronize()
        # continuous batching
        srv = H.Server(ctx, max_batch=args.max_batch, streams=2, mem_budget=SERVE_ARENA_GIB << 30)
        tickets, late = [], []
        s0 = time.perf_counter()
        for (at, _), (m, l, n, _, _, ca, cb) in zip(arr, ops):
            while time.perf_counter() - s0 < at:
                srv.hegmm_server_poll()
            tickets.append(srv.hegmm_server_submit(ca, cb, m, l, n))
            late.append((time.perf_counter() - s0 - at) * 1e3)  # host delay before the request was queued
            srv.hegmm_server_poll()
        srv.hegmm_server_poll(wait=True)
        span = time.perf_counter() - s0
        st = srv.hegmm_server_stats_get()
        ok = True
        slat = []
        for j, (t, (m, l, n, A, Bm, _, _)) in enumerate(zip(tickets, ops)):
            c, lm = srv.hegmm_server_result(t)
            slat.append(lm + late[j])  # from the scheduled arrival to completion
            if j % 16 == 0:
                ok &= bool((ctx.hegmm_decrypt(c, m, l, n).astype(np.int64) == (A @ Bm) % pre.t).all())
        srv.close()
        slat.sort()
        # plain path: each request alone, in arrival order
        lat = []
        s0 = time.perf_counter()
        for (at, _), (m, l, n, _, _, ca, cb) in zip(arr, ops):
            while time.perf_counter() - s0 < at:
                pass
            c, _ = ctx.hegmm_matmul(ca, cb, m, l, n)
            torch.cuda.current_stream().synchronize()
            stream.synchronize()
            lat.append((time.perf_counter() - s0 - at) * 1e3)
        pspan = time.perf_counter() - s0
        lat.sort()
        results.append({
            "rate_req_per_s": r, "requests": len(arr),
            "served": {"throughput_req_per_s": len(arr) / span, "p50_ms": slat[len(slat) // 2],
                       "p99_ms": slat[min(len(slat) - 1, int(0.99 * len(slat)))],
                       "server_p50_ms": st["p50_ms"], "server_p99_ms": st["p99_ms"],
                       "batches": st["batches"], "max_batch": st["max_batch"]},
            "plain": {"throughput_req_per_s": len(arr) / pspan, "p50_ms": lat[len(lat) // 2],
                      "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))]},
            "decrypt_checked_ok": ok,
        })
        del ops
    line = {
        "metric": "HEGMM serving: throughput and p50/p99 latency vs Poisson arrival rate (N=16384 ring)",
        "value": max(x["served"]["throughput_req_per_s"] for x in results), "unit": "req/s", "n_gpus": 1,
        "higher_is_better": True, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "serving: N=16384, t=65537, 8x50-bit + 2 special primes, dnum=4; Poisson arrivals; "
                               "70% small (1..16), 25% medium (17..64, fitting), 5% 128x16x64; entries U[0,255]",
                   "distinct_shapes": len(shapes), "setup_s_keys_and_masks": setup_s,
                   "max_batch": args.max_batch, "streams": 2, "keyswitch_mode": args.ks_mode,
                   "free_gib_after_keys": free_b / 2**30, "mask_budget_gib": mask_b / 2**30},
        "rates": results,
    }
    print(json.dumps(line))


BLOCK_PARTITIONS = {"P1": [50, 50], "P2": [64, 36]}  # Section 4.4: 100 x 100 split two ways


def run_blocked(args):
    """Table 4's blocked 100 x 100 products on the N=16384 ring: one step is a
    P1 (50 + 50) and a P2 (64 + 36) product, each one hegmm_matmul_blocked
    call (the eight block products in one batch, then the block sums); every
    block is encrypted once under Algorithm 1.  The plain path (one
    hegmm_matmul per block product, hegmm_add for the sums) is timed beside
    it.  Entries U[0,255]."""
    import torch

    from paper_2405_02238_gb300 import build as B

    B.build()
    from paper_2405_02238_gb300 import hegmm as H

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    pre = W.PAPER
    ctx = H.Context.from_preset(pre, stream=stream.cuda_stream)
    ctx.hegmm_set_keyswitch_mode(KS_MODES[args.ks_mode])
    parts = {}
    for name, split in BLOCK_PARTITIONS.items():
        A, Bm = W.matrices(100, 100, 100, *W.PAPER_RANGE, seed=split[0])
        shapes = [(r, q, c) for r in split for q in split for c in split]
        ctx.hegmm_keygen(KEY_SEED, shapes, H.ALG_1)
        bb = np.cumsum([0] + split)
        gA = [[ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_A, A[bb[i]:bb[i + 1], bb[k]:bb[k + 1]], split[i], split[k], 1,
                                                  H.ALG_1), 1, 10 * i + k) for k in range(2)] for i in range(2)]
        gB = [[ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_B, Bm[bb[k]:bb[k + 1], bb[j]:bb[j + 1]], 1, split[k], split[j],
                                                  H.ALG_1), 2, 10 * k + j) for j in range(2)] for k in range(2)]
        parts[name] = (split, A, Bm, gA, gB, bb)

    def blocked(name):
        split, _, _, gA, gB, _ = parts[name]
        return ctx.hegmm_matmul_blocked(split, split, split, gA, gB)

    def plain(name):
        split, _, _, gA, gB, _ = parts[name]
        out = []
        for i in range(2):
            for j in range(2):
                acc = None
                for k in range(2):
                    c, _ = ctx.hegmm_matmul(gA[i][k], gB[k][j], split[i], split[k], split[j], H.ALG_1)
                    acc = c if acc is None else ctx.hegmm_add(acc, c)
                out.append(acc)
        return out

    def check(name, C):
        split, A, Bm, _, _, bb = parts[name]
        for i in range(2):
            for j in range(2):
                got = ctx.hegmm_decrypt(C[i][j], split[i], split[0], split[j], H.ALG_1).astype(np.int64)
                want = (A[bb[i]:bb[i + 1]] @ Bm[:, bb[j]:bb[j + 1]]) % pre.t
                assert (got == want).all(), "wrong blocked product %s block (%d, %d)" % (name, i, j)

    tuning = None
    if not args.no_autotune:
        # the knobs on the block products of both partitions, batched as the blocked calls batch them
        As, Bs, shp = [], [], []
        for split, _, _, gA, gB, _ in parts.values():
            for i in range(2):
                for j in range(2):
                    for k in range(2):
                        As.append(gA[i][k]), Bs.append(gB[k][j]), shp.append((split[i], split[k], split[j]))
        tuning = ctx.hegmm_autotune(As, Bs, shp, [H.ALG_1] * len(shp), reps=2)
    for _ in range(max(3, args.warmup)):
        outs = {name: blocked(name) for name in parts}
    for name, C in outs.items():
        check(name, C)
    del outs

    def timed(fn, steps):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            ev[k][0].record(stream)
            r = fn()
            ev[k][1].record(stream)
            del r
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / steps

    clk = ClockSampler(0)
    torch.cuda.synchronize()
    clk.start()
    time.sleep(0.3)
    ms = timed(lambda: [blocked(name) for name in parts], args.steps)
    clocks = clk.stop()
    per_part = {name: timed(lambda name=name: blocked(name), args.steps) for name in parts}
    plain_outs = {name: plain(name) for name in parts}
    for name, flat in plain_outs.items():
        check(name, [flat[0:2], flat[2:4]])
    del plain_outs
    plain_part = {name: timed(lambda name=name: plain(name), max(1, args.steps // 2)) for name in parts}
    line = {
        "metric": "blocked 100x100 encrypted matmuls/s (N=16384 ring, Section 4.4 partitions P1 50+50 and P2 64+36)",
        "value": len(parts) / (ms / 1e3), "unit": "matmul/s", "n_gpus": 1, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "blocked: N=16384, t=65537, 8x50-bit + 2 special primes, dnum=4; A, B 100x100 "
                               "U[0,255]; P1 and P2 of one step each one hegmm_matmul_blocked call (8 Algorithm 1 "
                               "block products + 4 block sums); keys and masks resident, larger than L2",
                   "keyswitch_mode": args.ks_mode, "tuning": tuning or "defaults"},
        "per_partition_ms": per_part,
        "plain_path_ms": plain_part,
        "paper_table4_s": {"P1": 39.12, "P2": 26.17},
        "clocks": clocks,
    }
    print(json.dumps(line))


def kernel_source_sha():
    """Hash of the sources the stored ncu traffic ratio was taken on (the
    kernels and their device arithmetic)."""
    h = hashlib.sha256()
    for f in ("kernels.cu", "device.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2405_02238_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:12]


# The library's kernel buckets (hegmm_kernel_stats) of the CUDA kernels an
# ncu log names, first match wins.
NCU_BUCKETS = [("k_ntt<", lambda n: "ntt_inv" if n.split("<")[1].split(",")[1].strip() in ("1", "true") else "ntt_fwd"),
               ("k_modup_", "modup"), ("k_divround_", "divround_ntt"), ("k_ksw_ip", "ksw_inner_product"),
               ("k_lt_grp", "lt_keyswitch"), ("k_lt_one", "lt_keyswitch"), ("k_lt_acc", "lt_accumulate"),
               ("k_tensor", "tensor"),
               ("k_sum", "sum")]
NCU_UNITS = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "inst": 1, "Kinst": 1e3, "Minst": 1e6,
             "Ginst": 1e9, "": 1}


def ncu_bucket(kernel_name):
    name = kernel_name.split("(")[0].replace("void ", "").replace("hg::", "").strip()
    for prefix, b in NCU_BUCKETS:
        if name.startswith(prefix):
            return b(name) if callable(b) else b
    return None


def ingest_ncu(pairs):
    """Per kernel bucket, summed over the given product runs: DRAM bytes
    (read + write) over the library's algorithmic bytes, and warp-
    instructions over butterflies; written with the hash of the kernel
    sources to profiles/ncu_traffic.json, which the roofline entries read."""
    import csv
    import io

    sums = {}
    for pair in pairs:
        csv_path, json_path = pair.split(":")
        txt = open(csv_path).read()
        rows = list(csv.DictReader(io.StringIO(txt[txt.index('"ID"'):])))
        for r in rows:
            b = ncu_bucket(r["Kernel Name"])
            if b is None:
                continue
            if r["Metric Name"] not in ("dram__bytes_read.sum", "dram__bytes_write.sum", "smsp__inst_executed.sum"):
                continue
            v = float(r["Metric Value"].replace(",", "")) * NCU_UNITS[r["Metric Unit"]]
            d = sums.setdefault(b, {"dram": 0.0, "inst": 0.0, "bytes": 0.0, "bfly": 0.0})
            if r["Metric Name"] in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
                d["dram"] += v
            elif r["Metric Name"] == "smsp__inst_executed.sum":
                d["inst"] += v
        line = [ln for ln in open(json_path).read().splitlines() if ln.startswith("{")][-1]
        for b, k in json.loads(line)["kernels"].items():
            if b in sums:
                sums[b]["bytes"] += k["algorithmic_bytes"]
                sums[b]["bfly"] += k["butterflies"]
    out = {"kernels_sha": kernel_source_sha(),
           "traffic_per_algorithmic_byte": {b: round(d["dram"] / d["bytes"], 4) for b, d in sorted(sums.items())
                                            if d["bytes"] > 0 and d["dram"] > 0},
           "warp_inst_per_butterfly": {b: round(d["inst"] / d["bfly"], 4) for b, d in sorted(sums.items())
                                       if d["bfly"] > 0 and d["inst"] > 0},
           "source": "ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,smsp__inst_executed.sum of the timed "
                     "launches of: " + "; ".join(os.path.basename(p.split(":")[1]) for p in pairs) +
                     " (bench.py --workload product runs); sha over csrc/kernels.cu and csrc/device.cuh"}
    with open(COUNTERS, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out))


def run_product(args):
    """One product of --shape on the --ring preset (medium by default), run
    once and then --reps times; prints the per-kernel times of the repeated
    runs (the small case of the ncu captures: with --reps 1 the second
    product's launches are the captured ones, a few GB on the device)."""
    import torch

    from paper_2405_02238_gb300 import build as B

    B.build()
    from paper_2405_02238_gb300 import hegmm as H

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    pre = W.PRESETS[args.ring]
    ctx = H.Context.from_preset(pre, stream=stream.cuda_stream)
    ctx.hegmm_set_keyswitch_mode(KS_MODES[args.ks_mode])
    if args.lt_kernel >= 0:
        ctx.hegmm_set_tuning(H.TUNE_LT_KERNEL, args.lt_kernel)
    if args.lt_one >= 0:
        ctx.hegmm_set_tuning(H.TUNE_LT_ONE, args.lt_one)
    if args.lt_chunk >= 0:
        ctx.hegmm_set_tuning(H.TUNE_LT_CHUNK, args.lt_chunk)
    if args.ntt_threads >= 0:
        ctx.hegmm_set_tuning(H.TUNE_NTT_THREADS, args.ntt_threads)
    if args.moddown_split >= 0:
        ctx.hegmm_set_tuning(H.TUNE_MODDOWN_SPLIT, args.moddown_split)
    m, l, n = (int(v) for v in args.shape.lower().split("x"))
    A, Bm = W.matrices(m, l, n, *(W.PAPER_RANGE if args.ring == "paper" else W.MEDIUM_RANGE))
    ctx.hegmm_keygen(KEY_SEED, [(m, l, n)], args.alg)
    ca = ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_A, A, m, l, n, args.alg), 1, 0)
    cb = ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_B, Bm, m, l, n, args.alg), 1, 1)
    ctx.hegmm_matmul(ca, cb, m, l, n, args.alg)
    torch.cuda.synchronize()
    ctx.hegmm_kernel_reset()
    ctx.hegmm_set_timing(True)
    torch.cuda.profiler.start()  # a profiler started with capture off records these products only
    for _ in range(max(1, args.reps)):
        c, _ = ctx.hegmm_matmul(ca, cb, m, l, n, args.alg)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    ctx.hegmm_set_timing(False)
    if not (ctx.hegmm_decrypt(c, m, l, n, args.alg).astype(np.int64) == (A @ Bm) % pre.t).all():
        raise SystemExit("product: decrypted result differs from A @ B mod t")
    ks = {k: {"ms": v[0], "launches": v[1], "algorithmic_bytes": v[2], "butterflies": v[3]}
          for k, v in ctx.hegmm_kernel_stats().items() if v[1]}
    print(json.dumps({"workload": "product %dx%dx%d, algorithm %d, %s ring" % (m, l, n, args.alg, args.ring),
                      "keyswitch_mode": args.ks_mode, "lt_kernel": args.lt_kernel, "lt_one": args.lt_one, "reps": args.reps,
                      "kernels": ks}))


# ----------------------------------------------------------------------------- GPU arm


def load_counters():
    """ncu counters of the current kernel sources (profiles/ncu_traffic.json):
    DRAM traffic per algorithmic byte and warp-instructions per butterfly,
    per kernel; empty when the sources changed since they were taken."""
    if not os.path.exists(COUNTERS):
        return {}
    try:
        tj = json.load(open(COUNTERS))
    except Exception:
        return {}
    return tj if tj.get("kernels_sha") == kernel_source_sha() else {}


def roofline(name, stats, hbm_peak, bfly_peak, issue_peak, counters):
    """Roofline entry of one kernel bucket from the per-kernel pass: HBM
    kernels against the measured copy rate; NTT-family kernels (integer
    pipes) against the chip's warp-instruction issue rate (SMs x 4 schedulers
    x 1 instruction per cycle x the sampled SM clock) divided by the
    kernel's warp-instructions per butterfly from ncu, with the in-library
    register-only butterfly probe beside it."""
    kms, kn, kbytes, kwork = stats[name]
    r = {"kernel": name, "launches": kn, "avg_launch_us": kms * 1e3 / max(kn, 1),
         "share_of_kernel_time": kms / max(sum(v[0] for v in stats.values()), 1e-9)}
    if kwork > 0:
        bps = kwork / (kms / 1e3)
        ipb = counters.get("warp_inst_per_butterfly", {}).get(name)
        r.update({"bound": "alu", "unit": "Gbutterfly/s", "achieved": bps / 1e9,
                  "butterflies_per_launch": kwork / max(kn, 1),
                  "butterfly_probe_peak": bfly_peak / 1e9, "frac_of_butterfly_probe": bps / bfly_peak})
        if ipb:
            r.update({"peak": issue_peak["warp_inst_per_s"] / ipb / 1e9, "warp_inst_per_butterfly": ipb,
                      "peak_source": "derived: %d SMs x 4 schedulers x 1 warp-instruction/cycle x %.0f MHz (median "
                                     "SM clock in the timed region) / %.2f warp-instructions per butterfly (ncu, "
                                     "these kernel sources)" % (issue_peak["sms"], issue_peak["mhz"], ipb)})
        else:
            r.update({"peak": bfly_peak / 1e9, "peak_source": "measured: hegmm_peak_butterflies (register-only "
                                                               "lazy Shoup butterflies on every SM)"})
    else:
        r.update({"bound": "hbm", "unit": "GB/s", "achieved": kbytes / (kms / 1e3) / 1e9,
                  "peak": hbm_peak or HBM_FALLBACK,
                  "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if hbm_peak else "fallback"})
    r["frac"] = r["achieved"] / r["peak"]
    r["algorithmic_bytes_per_launch"] = kbytes / max(kn, 1)
    tr = counters.get("traffic_per_algorithmic_byte", {}).get(name)
    r["traffic"] = tr * r["algorithmic_bytes_per_launch"] if tr else None
    return r


def measure_throughput(kind, args, H, dev, stream, world, rank, full=True, profile=True):
    """Times one throughput workload (paper, medium or batch): autotune,
    warm-up with a decryption check of every product, the timed steps (CUDA
    events on the library stream around graph replays, L2 flushed between
    steps), a per-kernel pass, the plain per-product path, e2e through host
    buffers; with full, the other key-switch order and two-row packing too.
    Returns the JSON line's fields."""
    import torch

    pre = workload_preset(kind)
    ctx = H.Context.from_preset(pre, stream=stream.cuda_stream)
    ks_code = KS_MODES
    ctx.hegmm_set_keyswitch_mode(ks_code[args.ks_mode])
    if args.giant_cost:
        ctx.hegmm_set_tuning(H.TUNE_GIANT_COST, args.giant_cost)
    prods = []  # (m, l, n, alg, blocks, A, B)
    if kind == "batch":
        for i, (m, l, n) in enumerate(W.batch_shapes(W.BATCH_COUNT, ctx.S)):
            A, Bm = W.matrices(m, l, n, *W.BATCH_RANGE, seed=i)
            prods.append((m, l, n, H.ALG_AUTO, 1, A, Bm))
        rng = W.BATCH_RANGE
    else:
        rng = W.PAPER_RANGE if kind == "paper" else W.MEDIUM_RANGE
        for (m, l, n, alg, nb) in workload_products(kind, None if args.paper_auto else H, ctx.S,
                                                    blocks=not args.no_blocks):
            A, Bm = W.matrices(m, l, n, *rng)
            prods.append((m, l, n, alg, nb, A, Bm))
    # the products the library runs: a product of b blocks is b products of
    # l / b (A's column blocks times B's row blocks), summed
    units, group = [], []  # (m, l / b, n, alg, A_k, B_k), the product each belongs to
    for i, (m, l, n, alg, nb, A, Bm) in enumerate(prods):
        lb = l // nb
        for k in range(nb):
            units.append((m, lb, n, alg, A[:, k * lb:(k + 1) * lb], Bm[k * lb:(k + 1) * lb, :]))
            group.append(i)
    blocked = any(p[4] > 1 for p in prods)
    for alg in sorted({u[3] for u in units}):
        ctx.hegmm_keygen(KEY_SEED, [u[:3] for u in units if u[3] == alg], alg)
    ops = []
    for i, (m, l, n, alg, A, Bm) in enumerate(units):
        ca = ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_A, A, m, l, n, alg), 1 + rank, 2 * i)
        cb = ctx.hegmm_encrypt(ctx.hegmm_encode(H.ROLE_B, Bm, m, l, n, alg), 1 + rank, 2 * i + 1)
        ops.append((ca, cb))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    algs = [u[3] for u in units]
    ushapes = [u[:3] for u in units]
    first_unit = [group.index(i) for i in range(len(prods))]

    def run(A_cts, B_cts):
        """Every product of the workload in one call: hegmm_matmul_batch_algs,
        or hegmm_matmul_sum when a product is blocked (one result each)."""
        if blocked:
            return ctx.hegmm_matmul_sum(A_cts, B_cts, ushapes, group, len(prods), algs)
        return ctx.hegmm_matmul_batch_algs(A_cts, B_cts, ushapes, algs)

    def step():  # one step = every product of the workload in one call
        return run([a for a, _ in ops], [b for _, b in ops])

    def single_path(sample):
        """The plain path: one hegmm_matmul call per product (per block, and
        hegmm_add for the block sums)."""
        outs = []
        for i in sample:
            c = None
            for u in (j for j in range(len(units)) if group[j] == i):
                m, l, n, alg = units[u][:4]
                r = ctx.hegmm_matmul(ops[u][0], ops[u][1], m, l, n, alg)[0]
                c = r if c is None else ctx.hegmm_add(c, r)
            outs.append(c)
        return outs

    def decrypt(i, c, pair=False):
        m, l, n, alg = units[first_unit[i]][:4]
        return (ctx.hegmm_decrypt_pair if pair else ctx.hegmm_decrypt)(c, m, l, n, alg)

    def timed(fn, steps):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            with torch.cuda.stream(stream):
                flush.fill_(k & 0xFF)
            ev[k][0].record(stream)
            r = fn()
            ev[k][1].record(stream)
            del r
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev]

    def check(outs, what):
        for i, ((m, l, n, alg, nb, A, Bm), c) in enumerate(zip(prods, outs)):
            got = decrypt(i, c).astype(np.int64)
            assert (got == (A @ Bm) % pre.t).all(), "wrong product %dx%dx%d alg %d (%s)" % (m, l, n, alg, what)

    # the library's autotuner picks the bit-neutral kernel knobs on this
    # workload, unless they are given (a profiler's serialised launches would
    # mislead the autotuner: profiling runs pass the plain run's choice)
    tuning = None
    fixed = {k: v for k, v in (("lt_kernel", args.lt_kernel), ("lt_chunk", args.lt_chunk), ("lt_one", args.lt_one),
                               ("ntt_threads", args.ntt_threads), ("groups", args.groups),
                               ("moddown_split", args.moddown_split)) if v >= 0}
    if fixed:
        knob = {"lt_kernel": H.TUNE_LT_KERNEL, "lt_chunk": H.TUNE_LT_CHUNK, "lt_one": H.TUNE_LT_ONE,
                "ntt_threads": H.TUNE_NTT_THREADS, "groups": H.TUNE_GROUPS, "moddown_split": H.TUNE_MODDOWN_SPLIT}
        for k, v in fixed.items():
            ctx.hegmm_set_tuning(knob[k], v)
        tuning = dict(fixed, given=True)
    elif not args.no_autotune:
        tuning = ctx.hegmm_autotune([a for a, _ in ops], [b for _, b in ops], ushapes, algs,
                                    reps=3 if len(units) <= 64 else 1)
    for _ in range(max(args.warmup, 1)):  # builds plans and masks, captures graphs
        outs = step()
    check(outs, args.ks_mode)
    del outs
    sample = list(range(len(prods))) if len(prods) <= 8 else list(range(0, len(prods), len(prods) // 32))
    check_sample = single_path(sample)
    for i, c in zip(sample, check_sample):
        A, Bm = prods[i][5:]
        assert (decrypt(i, c).astype(np.int64) == (A @ Bm) % pre.t).all()
    del check_sample
    sc = [H.hegmm_plan_counts(m, l, n, alg if alg else 0, ctx.S) for (m, l, n, alg, _, _) in units]
    for _ in range(2):
        single_path(sample)
    single_ms = sum(timed(lambda: single_path(sample), 3)) / 3
    single_value = len(sample) / (single_ms / 1e3)

    clk = ClockSampler(dev.index or 0)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    time.sleep(0.3)
    t_wall0 = time.perf_counter()
    if profile:  # profilers started with capture off record the headline's timed steps only
        torch.cuda.profiler.start()
    step_ms = timed(step, args.steps)
    if world > 1:
        dist.barrier()
    if profile:
        torch.cuda.profiler.stop()
    wall = time.perf_counter() - t_wall0
    clocks = clk.stop()
    ms = max_over_ranks(sum(step_ms) / len(step_ms), world, dist if world > 1 else None, dev)
    per_step = len(prods)
    value = whole_job_value(per_step, world, ms)
    # per-kernel device time: the same steps once more, launched kernel by
    # kernel with CUDA events on the library's stream (the timed steps above
    # replay each plan as one CUDA graph)
    ctx.hegmm_kernel_reset()
    ctx.hegmm_set_timing(True)
    timed(step, args.steps)
    ctx.hegmm_set_timing(False)
    stats = ctx.hegmm_kernel_stats()

    out = {"value": value, "ms_per_step": ms, "products_per_step": per_step, "tuning": tuning or "defaults",
           "clocks": clocks, "wall_s_timed": wall,
           "keyswitches_per_step": sum(c["ksw"] for c in sc), "paper_rotations_per_step": sum(c["rot"] for c in sc),
           "per_product_path": {"value": single_value * world, "unit": UNIT, "ms_per_product": single_ms / len(sample),
                                "how": "one hegmm_matmul call per product, %d of the %d products, warm"
                                       % (len(sample), len(prods))},
           "batch_over_per_product": value / (single_value * world)}
    out["keyswitches_per_s"] = out["keyswitches_per_step"] * world / (ms / 1e3)

    if full:
        # the other key-switch evaluation order on the same products
        other = "single" if args.ks_mode != "single" else "double+lazy+shared"
        ctx.hegmm_set_keyswitch_mode(ks_code[other])
        outs = step()
        check(outs, other)
        del outs
        other_ms = sum(timed(step, args.steps)) / args.steps
        ctx.hegmm_set_keyswitch_mode(ks_code[args.ks_mode])
        out["other_keyswitch_mode"] = {"mode": other, "value": per_step * world / (other_ms / 1e3), "unit": UNIT,
                                       "ms_per_step": other_ms}
        # two products per ciphertext pair (slot rows 0 and 1): every product of
        # the workload with a second one of its shape, the same launches per step
        pk_ops, pk_mats = [], []
        for i, (m, l, n, alg, nb, A, Bm) in enumerate(prods):
            pk_mats.append(W.matrices(m, l, n, *rng, seed=1000 + i))
        for u, (m, lb, n, alg, A, Bm) in enumerate(units):
            i, k = group[u], u - first_unit[group[u]]
            A2 = pk_mats[i][0][:, k * lb:(k + 1) * lb]
            B2 = pk_mats[i][1][k * lb:(k + 1) * lb, :]
            pa = ctx.hegmm_encrypt(ctx.hegmm_encode_pair(H.ROLE_A, A, A2, m, lb, n, alg), 1 + rank, 2 * u)
            pb = ctx.hegmm_encrypt(ctx.hegmm_encode_pair(H.ROLE_B, Bm, B2, m, lb, n, alg), 1 + rank, 2 * u + 1)
            pk_ops.append((pa, pb))

        def packed_step():
            return run([a for a, _ in pk_ops], [b for _, b in pk_ops])

        outs = packed_step()
        for i, ((m, l, n, alg, nb, A, Bm), (A2, B2), c) in enumerate(zip(prods, pk_mats, outs)):
            r0, r1 = decrypt(i, c, pair=True)
            assert (r0.astype(np.int64) == (A @ Bm) % pre.t).all() and (r1.astype(np.int64) == (A2 @ B2) % pre.t).all()
        del outs
        packed_ms = sum(timed(packed_step, args.steps)) / args.steps
        out["two_row_packing"] = {"value": 2 * per_step * world / (packed_ms / 1e3), "unit": UNIT,
                                  "ms_per_step": packed_ms, "products_per_step": 2 * per_step,
                                  "how": "each ciphertext pair carries a second product of the same shape in slot "
                                         "row 1 (hegmm_encode_pair); same calls, both rows checked by "
                                         "hegmm_decrypt_pair"}
        del pk_ops

    # e2e: host ciphertexts (coefficient domain, pinned) -> import -> product -> export
    host_in = []
    for ca, cb in ops:
        host_in.append((torch.from_numpy(ctx.hegmm_ct_export(ca)).pin_memory(),
                        torch.from_numpy(ctx.hegmm_ct_export(cb)).pin_memory()))
    lv1 = ctx.level_after_product
    host_out = [torch.empty((2, lv1, ctx.N), dtype=torch.uint64).pin_memory() for _ in prods]
    h2d = sum(a.numel() * 8 + b.numel() * 8 for a, b in host_in)
    d2h = sum(o.numel() * 8 for o in host_out)
    host_flat = [t.numpy() for ab in host_in for t in ab]
    host_out_np = [o.numpy() for o in host_out]

    def e2e_step():
        cts = ctx.hegmm_ct_import_batch(host_flat)
        res = run(cts[0::2], cts[1::2])
        ctx.hegmm_ct_export_batch(res, host_out_np)

    e2e_step()
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - e0) * 1e3 / args.steps
    out["e2e"] = {"value": per_step * world / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                  "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms}

    # roofline of the dominant kernel, of the key inner product (the HBM
    # part of key switching) and of the linear-transformation kernel
    peaks = json.load(open(PEAKS)) if os.path.exists(PEAKS) else {}
    hbm_peak = peaks.get("hbm_gbs")
    bfly_peak = ctx.hegmm_peak_butterflies()
    props = torch.cuda.get_device_properties(dev)
    mhz = (clocks or {}).get("sm_mhz") or peaks.get("sm_max_mhz") or 2070.0
    issue = {"sms": props.multi_processor_count, "mhz": mhz,
             "warp_inst_per_s": props.multi_processor_count * 4 * mhz * 1e6}
    counters = load_counters()
    name = max(stats.items(), key=lambda kv: kv[1][0])[0]
    out["roofline"] = roofline(name, stats, hbm_peak, bfly_peak, issue, counters)
    for extra, key in (("ksw_inner_product", "roofline_key_inner_product"), ("lt_keyswitch", "roofline_lt_keyswitch"),
                       ("divround_ntt", "roofline_moddown"), ("modup", "roofline_modup"), ("ntt_inv", "roofline_ntt_inv")):
        if extra != name and stats.get(extra, (0, 0))[1]:
            out[key] = roofline(extra, stats, hbm_peak, bfly_peak, issue, counters)
    out["kernels"] = {k: {"ms": v[0], "launches": v[1]} for k, v in stats.items() if v[1]}
    out["gpu_launches"] = int(sum(v[1] for v in stats.values()) / max(args.steps, 1)) * args.steps
    out["prods"] = [p[:5] for p in prods]
    dnum = -(-pre.L // pre.alpha)
    out["key_bytes"] = (len(ctx.hegmm_key_list())) * dnum * 2 * (pre.L + pre.K) * ctx.N * 8
    out["preset"] = pre
    del ops
    ctx.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-medium", action="store_true", help="skip the medium workload's extra key")
    ap.add_argument("--paper-auto", action="store_true",
                    help="paper workload: AUTO algorithm per shape instead of the fewest-key-switch choice")
    ap.add_argument("--no-blocks", action="store_true",
                    help="paper workload: unblocked plans only (one ciphertext per matrix for every product)")
    ap.add_argument("--workload", default="paper", choices=["paper", "medium", "batch", "serve", "product", "blocked"],
                    help="paper: the three N=16384 products (default); medium: the four N=8192 products; batch: 512 "
                         "mixed shapes; serve: Poisson arrivals on the N=16384 ring; product: one product of --shape "
                         "on --ring, run twice (the small case the ncu captures use); blocked: the 100x100 products "
                         "of Section 4.4 split as P1 and P2 (N=16384 ring)")
    ap.add_argument("--shape", default="16x32x24", help="m x l x n of --workload product")
    ap.add_argument("--ring", default="medium", choices=list(W.PRESETS), help="ring preset of --workload product")
    ap.add_argument("--alg", type=int, default=1, help="algorithm of --workload product (1, 2, 3; 0 = auto)")
    ap.add_argument("--lt-kernel", type=int, default=-1,
                    help="HEGMM_TUNE_LT_KERNEL variant (-1: autotuned, or the default for --workload product); "
                         "--lt-kernel / --lt-chunk / --lt-one given replace the autotuner")
    ap.add_argument("--lt-chunk", type=int, default=-1, help="HEGMM_TUNE_LT_CHUNK entries per item (-1: autotuned)")
    ap.add_argument("--reps", type=int, default=1, help="--workload product: timed products after the first")
    ap.add_argument("--lt-one", type=int, default=-1,
                    help="HEGMM_TUNE_LT_ONE one-output kernel (-1: autotuned, or the default for --workload product)")
    ap.add_argument("--ntt-threads", type=int, default=-1,
                    help="HEGMM_TUNE_NTT_THREADS (0 by launch size, 512, 1024; -1: autotuned, or the library's choice "
                         "for --workload product)")
    ap.add_argument("--moddown-split", type=int, default=-1,
                    help="HEGMM_TUNE_MODDOWN_SPLIT (0 or 1; -1: autotuned, or the library default for --workload product)")
    ap.add_argument("--groups", type=int, default=-1,
                    help="HEGMM_TUNE_GROUPS concurrent sub-batches (1 or 2; -1: autotuned)")
    ap.add_argument("--ingest-ncu", nargs="+", metavar="CSV:JSON",
                    help="write profiles/ncu_traffic.json for the current kernel sources from ncu CSV logs "
                         "(dram__bytes_read.sum, dram__bytes_write.sum, smsp__inst_executed.sum of the timed "
                         "launches of --workload product runs) and the JSON lines those runs printed")
    ap.add_argument("--rates", default="10,30,100,300,1000,2000")
    ap.add_argument("--serve-seconds", type=float, default=8.0)
    ap.add_argument("--max-requests", type=int, default=1000)
    ap.add_argument("--mask-gib", type=int, default=190, help="resident mask budget for the serve workload")
    ap.add_argument("--max-batch", type=int, default=64)
    ap.add_argument("--no-autotune", action="store_true", help="keep the default tuning instead of hegmm_autotune")
    ap.add_argument("--giant-cost", type=int, default=0,
                    help="HEGMM_TUNE_GIANT_COST of the shared-baby-step order (0: the library default, 8); it selects "
                         "the factorisation, so it changes the ciphertext bits")
    ap.add_argument("--ks-mode", default="double+lazy+shared", choices=list(KS_MODES),
                    help="evaluation order of the key switches in a product (hegmm_set_keyswitch_mode)")
    args = ap.parse_args()
    if args.ingest_ncu:
        return ingest_ncu(args.ingest_ncu)
    if args.impl == "reference":
        return run_reference(args)
    single_gpu = {"serve": run_serve, "product": run_product, "blocked": run_blocked}
    if args.workload in single_gpu:
        if int(os.environ.get("RANK", "0")) != 0:
            return None  # these workloads run on one GPU: other ranks exit without work
        return single_gpu[args.workload](args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2405_02238_gb300 import build as B

    B.build()
    from paper_2405_02238_gb300 import hegmm as H

    stream = torch.cuda.Stream(device=dev)
    kind = args.workload
    r = measure_throughput(kind, args, H, dev, stream, world, rank, full=True)
    cfg = {"paper": paper_config, "medium": workload_config, "batch": batch_config}[kind]
    line = {
        "metric": {"paper": METRIC_PAPER, "medium": METRIC, "batch": METRIC_BATCH}[kind], "value": r["value"],
        "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": cfg({"parallelism": "replicas" if world > 1 else "single-gpu", "keyswitch_mode": args.ks_mode,
                       "giant_cost": args.giant_cost or 8,
                       "tuning": r["tuning"],
                       "algorithms": ({"%dx%dx%d" % p[:3]: (p[3] if p[4] == 1 else "%d on %d l-blocks" % (p[3], p[4]))
                                       for p in r["prods"]} if kind != "batch" else "AUTO"),
                       "key_bytes": r["key_bytes"]}),
    }
    for k in ("per_product_path", "batch_over_per_product", "other_keyswitch_mode", "two_row_packing",
              "keyswitches_per_s", "keyswitches_per_step", "paper_rotations_per_step", "wall_s_timed", "e2e",
              "gpu_launches", "roofline", "roofline_key_inner_product", "roofline_lt_keyswitch", "roofline_moddown",
              "roofline_modup", "roofline_ntt_inv", "kernels", "clocks"):
        if k in r:
            line[k] = r[k]
    if kind == "paper" and not args.no_blocks and any(p[4] > 1 for p in r["prods"]):
        # the same products with one ciphertext per matrix (no blocked plan)
        args.no_blocks = True
        u = measure_throughput("paper", args, H, dev, stream, world, rank, full=False, profile=False)
        args.no_blocks = False
        line["unblocked_plans"] = {
            "value": u["value"], "unit": UNIT, "ms_per_step": u["ms_per_step"],
            "algorithms": {"%dx%dx%d" % p[:3]: p[3] for p in u["prods"]}, "tuning": u["tuning"],
            "per_product_path": u["per_product_path"], "e2e": u["e2e"], "keyswitches_per_step": u["keyswitches_per_step"],
            "key_bytes": u["key_bytes"], "roofline": u["roofline"], "kernels": u["kernels"], "clocks": u["clocks"]}
    if kind == "paper" and not args.no_medium:
        # the medium configuration, measured the same way (fewer extras)
        m = measure_throughput("medium", args, H, dev, stream, world, rank, full=False, profile=False)
        line["medium_workload"] = {
            "workload": workload_config()["workload"], "metric": METRIC, "value": m["value"], "unit": UNIT,
            "ms_per_step": m["ms_per_step"], "products_per_step": m["products_per_step"], "tuning": m["tuning"],
            "per_product_path": m["per_product_path"], "e2e": m["e2e"], "keyswitches_per_step": m["keyswitches_per_step"],
            "roofline": m["roofline"], "roofline_key_inner_product": m.get("roofline_key_inner_product"),
            "kernels": m["kernels"], "clocks": m["clocks"]}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(r["prods"], r["preset"])
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

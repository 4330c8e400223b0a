"""ctypes binding of libhegmm.so (include/hegmm.h), argument marshalling only.

Every function here has the name of the C entry point it calls and only
converts arguments and results; all work runs in the library's CUDA
kernels.  If the library cannot be loaded the import fails loudly: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhegmm.so")

HEGMM_OK = 0
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ESHAPE", -4: "ENOKEY", -5: "ECUDA", -6: "ETIMEOUT"}
ALG_AUTO, ALG_1, ALG_2 = 0, 1, 2
KS_SINGLE, KS_DOUBLE, KS_LAZY_RELIN, KS_SHARED = 0, 1, 2, 4  # hegmm_set_keyswitch_mode (flags combine)
ALG_1X = 3  # Algorithm 1 with the extended pre-layout (not in the paper; AUTO never picks it)
TUNE_LT_CHUNK, TUNE_LT_FUSED, TUNE_LT_KERNEL, TUNE_GIANT_COST, TUNE_GRAPHS, TUNE_LT_ONE = 1, 2, 3, 4, 5, 6
TUNE_WAIT_LIMIT, TUNE_TEST_DROP, TUNE_NTT_THREADS, TUNE_GROUPS, TUNE_MODDOWN_SPLIT = 7, 8, 9, 10, 11
ROLE_A, ROLE_B = 0, 1
KEYS_DIRECT, KEYS_POW2 = 0, 1  # hegmm_set_key_policy


class HegmmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


class hegmm_params(ctypes.Structure):
    _fields_ = [
        ("logN", ctypes.c_int),
        ("t", ctypes.c_uint64),
        ("L", ctypes.c_int),
        ("qbits", ctypes.c_int),
        ("K", ctypes.c_int),
        ("alpha", ctypes.c_int),
        ("eta", ctypes.c_int),
        ("ms_drop", ctypes.c_int),
        ("scheme", ctypes.c_int),
    ]


class hegmm_opcount(ctypes.Structure):
    _fields_ = [(n, ctypes.c_longlong) for n in
                ("rot", "cmult", "add", "mult", "relin", "extract", "ksw", "modup", "modswitch")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class hegmm_server_opts(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_int), ("streams", ctypes.c_int), ("mem_budget", ctypes.c_uint64)]


class hegmm_server_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_longlong) for n in
                ("submitted", "completed", "failed", "batches", "queued", "in_flight", "max_batch")] + \
               [(n, ctypes.c_double) for n in ("p50_ms", "p99_ms", "mean_ms", "max_ms")] + \
               [(n, ctypes.c_longlong) for n in ("max_batches_in_flight", "overlapped_batches")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


u64p = ctypes.POINTER(ctypes.c_uint64)
i64p = ctypes.POINTER(ctypes.c_int64)
intp = ctypes.POINTER(ctypes.c_int)
vp = ctypes.c_void_p

_SIGS = {
    "hegmm_ctx_create": (ctypes.c_int, [ctypes.POINTER(hegmm_params), vp, ctypes.POINTER(vp)]),
    "hegmm_ctx_destroy": (None, [vp]),
    "hegmm_last_error": (ctypes.c_char_p, [vp]),
    "hegmm_get_primes": (ctypes.c_int, [vp, u64p]),
    "hegmm_keygen": (ctypes.c_int, [vp, ctypes.c_uint64, intp, ctypes.c_int, ctypes.c_int]),
    "hegmm_keygen_rotations": (ctypes.c_int, [vp, intp, ctypes.c_int]),
    "hegmm_key_export": (ctypes.c_int, [vp, ctypes.c_uint64, u64p]),
    "hegmm_key_import": (ctypes.c_int, [vp, ctypes.c_uint64, u64p]),
    "hegmm_key_list": (ctypes.c_int, [vp, u64p, ctypes.c_int, intp]),
    "hegmm_encode": (ctypes.c_int, [vp, ctypes.c_int, i64p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(vp)]),
    "hegmm_encode_slots": (ctypes.c_int, [vp, u64p, ctypes.c_int, ctypes.POINTER(vp)]),
    "hegmm_encode_pair": (ctypes.c_int, [vp, ctypes.c_int, i64p, i64p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.POINTER(vp)]),
    "hegmm_decrypt_rows": (ctypes.c_int, [vp, vp, u64p]),
    "hegmm_decrypt_pair": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, u64p, u64p]),
    "hegmm_encrypt": (ctypes.c_int, [vp, vp, ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(vp)]),
    "hegmm_matmul": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(vp), ctypes.POINTER(hegmm_opcount)]),
    "hegmm_matmul_batch_algs": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(vp), intp, intp,
                                               ctypes.POINTER(vp)]),
    "hegmm_matmul_batch": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(vp), intp,
                                          ctypes.c_int, ctypes.POINTER(vp)]),
    "hegmm_lintrans": (ctypes.c_int, [vp, vp, intp, ctypes.c_int, ctypes.POINTER(vp)]),
    "hegmm_to_layout": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(vp)]),
    "hegmm_from_result": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(vp)]),
    "hegmm_chain_operand": (ctypes.c_int, [vp, vp] + [ctypes.c_int] * 9 + [ctypes.POINTER(vp)]),
    "hegmm_matmul_sum": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(vp), intp, intp, intp,
                                        ctypes.c_int, ctypes.POINTER(vp)]),
    "hegmm_matmul_blocked": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, intp, intp, intp,
                                            ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp)]),
    "hegmm_decrypt": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, u64p]),
    "hegmm_decrypt_slots": (ctypes.c_int, [vp, vp, u64p]),
    "hegmm_rotate": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.POINTER(vp)]),
    "hegmm_rotate_many": (ctypes.c_int, [vp, vp, intp, ctypes.c_int, ctypes.POINTER(vp)]),
    "hegmm_rotate_noalloc": (ctypes.c_int, [vp, vp, ctypes.c_int, vp]),
    "hegmm_device_memory": (ctypes.c_int, [vp, ctypes.c_int, u64p]),
    "hegmm_set_key_policy": (ctypes.c_int, [vp, ctypes.c_int]),
    "hegmm_plan_pow2_steps": (ctypes.c_int, [ctypes.c_longlong, ctypes.c_int, intp, ctypes.c_int]),
    "hegmm_cmult": (ctypes.c_int, [vp, vp, vp, ctypes.POINTER(vp)]),
    "hegmm_add": (ctypes.c_int, [vp, vp, vp, ctypes.POINTER(vp)]),
    "hegmm_mult": (ctypes.c_int, [vp, vp, vp, ctypes.POINTER(vp)]),
    "hegmm_modswitch": (ctypes.c_int, [vp, vp, ctypes.POINTER(vp)]),
    "hegmm_ct_level": (ctypes.c_int, [vp]),
    "hegmm_ct_export": (ctypes.c_int, [vp, vp, u64p]),
    "hegmm_ct_import": (ctypes.c_int, [vp, u64p, ctypes.c_int, ctypes.POINTER(vp)]),
    "hegmm_ct_import_batch": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(u64p), ctypes.c_int, ctypes.POINTER(vp)]),
    "hegmm_ct_export_batch": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(u64p)]),
    "hegmm_sync": (ctypes.c_int, [vp]),
    "hegmm_pt_destroy": (None, [vp]),
    "hegmm_ct_destroy": (None, [vp]),
    "hegmm_set_timing": (ctypes.c_int, [vp, ctypes.c_int]),
    "hegmm_kernel_kinds": (ctypes.c_int, []),
    "hegmm_kernel_name": (ctypes.c_char_p, [ctypes.c_int]),
    "hegmm_kernel_stats": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double)]),
    "hegmm_peak_butterflies": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_double)]),
    "hegmm_prepare": (ctypes.c_int, [vp, intp, ctypes.c_int, ctypes.c_int]),
    "hegmm_set_keyswitch_mode": (ctypes.c_int, [vp, ctypes.c_int]),
    "hegmm_set_tuning": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_longlong]),
    "hegmm_autotune": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(vp), intp, intp,
                                      ctypes.c_int, intp]),
    "hegmm_set_budgets": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]),
    "hegmm_server_create": (ctypes.c_int, [vp, ctypes.POINTER(hegmm_server_opts), ctypes.POINTER(vp)]),
    "hegmm_server_submit": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_uint64)]),
    "hegmm_server_poll": (ctypes.c_int, [vp, ctypes.c_int]),
    "hegmm_server_result": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_double)]),
    "hegmm_server_stats_get": (ctypes.c_int, [vp, ctypes.POINTER(hegmm_server_stats)]),
    "hegmm_server_destroy": (None, [vp]),
    "hegmm_kernel_reset": (ctypes.c_int, [vp]),
    "hegmm_plan_counts": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(hegmm_opcount)]),
    "hegmm_plan_describe": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           intp, ctypes.c_int]),
    "hegmm_plan_giant": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, intp, ctypes.c_int]),
    "hegmm_plan_layout": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, i64p, ctypes.c_uint64, u64p, ctypes.c_int]),
    "hegmm_plan_slot_map": (ctypes.c_int, [ctypes.c_int] * 6 + [intp, ctypes.c_int]),
    "hegmm_plan_result_layout": (ctypes.c_int, [ctypes.c_int] * 5 + [intp]),
}

EXPORTS = tuple(_SIGS)

_lib = None


def load(path: str = LIB_PATH):
    """Loads libhegmm.so and declares every entry point of include/hegmm.h."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError("libhegmm.so not built (%s); run __graft_entry__.build()" % path)
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def hegmm_plan_counts(m: int, l: int, n: int, alg: int, slots: int) -> dict:
    cnt = hegmm_opcount()
    rc = load().hegmm_plan_counts(m, l, n, alg, slots, ctypes.byref(cnt))
    if rc != HEGMM_OK:
        raise HegmmError(rc, "plan_counts")
    return cnt.as_dict()


def hegmm_plan_describe(m: int, l: int, n: int, alg: int, slots: int) -> List[int]:
    lib = load()
    need = lib.hegmm_plan_describe(m, l, n, alg, slots, None, 0)
    if need < 0:
        raise HegmmError(need, "plan_describe")
    buf = (ctypes.c_int * need)()
    lib.hegmm_plan_describe(m, l, n, alg, slots, buf, need)
    return list(buf)


def hegmm_plan_pow2_steps(z: int, slots: int) -> List[int]:
    lib = load()
    need = lib.hegmm_plan_pow2_steps(z, slots, None, 0)
    if need < 0:
        raise HegmmError(need, "plan_pow2_steps")
    buf = (ctypes.c_int * max(need, 1))()
    lib.hegmm_plan_pow2_steps(z, slots, buf, need)
    return list(buf)[:need]


def hegmm_plan_giant(m: int, l: int, n: int, alg: int, slots: int, role: int, cost: int = 0) -> List[int]:
    lib = load()
    need = lib.hegmm_plan_giant(m, l, n, alg, slots, role, cost, None, 0)
    if need < 0:
        raise HegmmError(need, "plan_giant")
    buf = (ctypes.c_int * need)()
    lib.hegmm_plan_giant(m, l, n, alg, slots, role, cost, buf, need)
    return list(buf)


def hegmm_plan_layout(m: int, l: int, n: int, alg: int, slots: int, role: int, mat, t: int) -> np.ndarray:
    lib = load()
    a = np.ascontiguousarray(mat, dtype=np.int64)
    need = lib.hegmm_plan_layout(m, l, n, alg, slots, role, a.ctypes.data_as(i64p), t, None, 0)
    if need < 0:
        raise HegmmError(need, "plan_layout")
    out = np.zeros(need, dtype=np.uint64)
    lib.hegmm_plan_layout(m, l, n, alg, slots, role, a.ctypes.data_as(i64p), t, out.ctypes.data_as(u64p), need)
    return out


def hegmm_plan_slot_map(m: int, l: int, n: int, alg: int, slots: int, role: int) -> List[int]:
    lib = load()
    need = lib.hegmm_plan_slot_map(m, l, n, alg, slots, role, None, 0)
    if need < 0:
        raise HegmmError(need, "plan_slot_map")
    buf = (ctypes.c_int * max(1, need))()
    lib.hegmm_plan_slot_map(m, l, n, alg, slots, role, buf, need)
    return list(buf)[:need]


def hegmm_plan_result_layout(m: int, l: int, n: int, alg: int, slots: int):
    out = (ctypes.c_int * 3)()
    rc = load().hegmm_plan_result_layout(m, l, n, alg, slots, out)
    if rc != HEGMM_OK:
        raise HegmmError(rc, "plan_result_layout")
    return out[0], out[1], "col" if out[2] else "row"


def _u64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint64)


def _ptr(a: np.ndarray, t=u64p):
    return a.ctypes.data_as(t)


class Context:
    """Owns one hegmm_ctx; methods are thin wrappers of the C entry points."""

    def __init__(self, logN, t, L, qbits, K, alpha, eta=21, ms_drop=0, stream=None, scheme=0):
        self.lib = load()
        self.params = hegmm_params(logN, t, L, qbits, K, alpha, eta, ms_drop, scheme)
        if stream is None:
            import torch

            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        h = vp()
        rc = self.lib.hegmm_ctx_create(ctypes.byref(self.params), vp(stream), ctypes.byref(h))
        if rc != HEGMM_OK:
            raise HegmmError(rc, "hegmm_ctx_create")
        self.h = h
        self.N = 1 << logN
        self.S = self.N // 2
        self.L = L
        self.K = K
        self.t = t
        self.level_after_product = L - ms_drop

    @classmethod
    def from_preset(cls, p, stream=None):
        return cls(p.logN, p.t, p.L, p.qbits, p.K, p.alpha, p.eta, p.ms_drop, stream, getattr(p, "scheme", 0))

    def close(self):
        if getattr(self, "h", None):
            self.lib.hegmm_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int, what: str):
        if rc != HEGMM_OK:
            msg = self.lib.hegmm_last_error(self.h)
            raise HegmmError(rc, "%s: %s" % (what, msg.decode() if msg else ""))

    # ------------------------------------------------------------ wrappers
    def hegmm_get_primes(self) -> List[int]:
        out = np.zeros(self.L + self.K, dtype=np.uint64)
        self._check(self.lib.hegmm_get_primes(self.h, _ptr(out)), "get_primes")
        return [int(x) for x in out]

    def hegmm_keygen(self, seed: int, shapes: Sequence[Tuple[int, int, int]] = (), alg: int = ALG_AUTO):
        arr = np.ascontiguousarray(np.array(shapes, dtype=np.int32).reshape(-1))
        self._check(self.lib.hegmm_keygen(self.h, seed, arr.ctypes.data_as(intp), len(shapes), alg), "keygen")

    def hegmm_prepare(self, shapes: Sequence[Tuple[int, int, int]], alg: int = ALG_AUTO):
        arr = np.ascontiguousarray(np.array(shapes, dtype=np.int32).reshape(-1))
        self._check(self.lib.hegmm_prepare(self.h, arr.ctypes.data_as(intp), len(shapes), alg), "prepare")

    def hegmm_set_keyswitch_mode(self, mode: int):
        """KS_SINGLE: one ModDown per key switch; KS_DOUBLE: sums kept over PQ;
        | KS_LAZY_RELIN: one relinearisation per product."""
        self._check(self.lib.hegmm_set_keyswitch_mode(self.h, int(mode)), "set_keyswitch_mode")

    def hegmm_autotune(self, As, Bs, shapes, algs=None, reps: int = 3) -> dict:
        """Times the bit-neutral tuning candidates on these products and keeps the fastest."""
        n = len(As)
        pa = (vp * n)(*[a.h for a in As])
        pb = (vp * n)(*[b.h for b in Bs])
        mln = np.ascontiguousarray(np.array(shapes, dtype=np.int32).reshape(-1))
        al = None if algs is None else np.ascontiguousarray(np.array(algs, dtype=np.int32))
        chosen = np.zeros(6, dtype=np.int32)
        self._check(self.lib.hegmm_autotune(self.h, n, pa, pb, mln.ctypes.data_as(intp),
                                            None if al is None else al.ctypes.data_as(intp), int(reps),
                                            chosen.ctypes.data_as(intp)), "autotune")
        return {"lt_kernel": int(chosen[0]), "lt_chunk": int(chosen[1]), "lt_one": int(chosen[2]),
                "ntt_threads": int(chosen[3]), "groups": int(chosen[4]), "moddown_split": int(chosen[5])}

    def hegmm_set_tuning(self, knob: int, value: int):
        self._check(self.lib.hegmm_set_tuning(self.h, int(knob), int(value)), "set_tuning")

    def hegmm_set_budgets(self, mask_bytes: int = 0, plan_bytes: int = 0, chunk_bytes: int = 0):
        self._check(self.lib.hegmm_set_budgets(self.h, mask_bytes, plan_bytes, chunk_bytes), "set_budgets")

    def hegmm_keygen_rotations(self, zs: Sequence[int]):
        arr = np.ascontiguousarray(np.array(zs, dtype=np.int32))
        self._check(self.lib.hegmm_keygen_rotations(self.h, arr.ctypes.data_as(intp), len(zs)), "keygen_rotations")

    def hegmm_key_export(self, which: int) -> np.ndarray:
        dnum = self.params.L // self.params.alpha
        out = np.zeros((dnum, 2, self.L + self.K, self.N), dtype=np.uint64)
        self._check(self.lib.hegmm_key_export(self.h, which, _ptr(out)), "key_export")
        return out

    def hegmm_key_import(self, which: int, key: np.ndarray):
        a = np.ascontiguousarray(key, dtype=np.uint64)
        self._check(self.lib.hegmm_key_import(self.h, which, _ptr(a)), "key_import")

    def hegmm_key_list(self):
        n = ctypes.c_int()
        self._check(self.lib.hegmm_key_list(self.h, None, 0, ctypes.byref(n)), "key_list")
        out = np.zeros(max(1, n.value), dtype=np.uint64)
        self._check(self.lib.hegmm_key_list(self.h, _ptr(out), n.value, ctypes.byref(n)), "key_list")
        return [int(x) for x in out[: n.value]]

    def hegmm_encode(self, role: int, mat: np.ndarray, m: int, l: int, n: int, alg: int = ALG_AUTO) -> "Plaintext":
        a = np.ascontiguousarray(mat, dtype=np.int64)
        out = vp()
        self._check(self.lib.hegmm_encode(self.h, role, _ptr(a, i64p), m, l, n, alg, ctypes.byref(out)), "encode")
        return Plaintext(self, out)

    def hegmm_encode_pair(self, role: int, mat0: np.ndarray, mat1, m: int, l: int, n: int,
                          alg: int = ALG_AUTO) -> "Plaintext":
        """hegmm_encode_pair: mat0 in slot row 0, mat1 (None: zeros) in row 1."""
        a = np.ascontiguousarray(mat0, dtype=np.int64)
        b = None if mat1 is None else np.ascontiguousarray(mat1, dtype=np.int64)
        out = vp()
        self._check(self.lib.hegmm_encode_pair(self.h, role, _ptr(a, i64p), None if b is None else _ptr(b, i64p), m, l,
                                               n, alg, ctypes.byref(out)), "encode_pair")
        return Plaintext(self, out)

    def hegmm_encode_slots(self, slots) -> "Plaintext":
        a = _u64(slots)
        out = vp()
        self._check(self.lib.hegmm_encode_slots(self.h, _ptr(a), len(a), ctypes.byref(out)), "encode_slots")
        return Plaintext(self, out)

    def hegmm_encrypt(self, pt: "Plaintext", seed: int, stream_id: int) -> "Ciphertext":
        out = vp()
        self._check(self.lib.hegmm_encrypt(self.h, pt.h, seed, stream_id, ctypes.byref(out)), "encrypt")
        return Ciphertext(self, out)

    def hegmm_matmul(self, A: "Ciphertext", B: "Ciphertext", m: int, l: int, n: int, alg: int = ALG_AUTO):
        out = vp()
        cnt = hegmm_opcount()
        self._check(self.lib.hegmm_matmul(self.h, A.h, B.h, m, l, n, alg, ctypes.byref(out), ctypes.byref(cnt)),
                    "matmul")
        return Ciphertext(self, out), cnt.as_dict()

    def hegmm_matmul_batch(self, As, Bs, shapes, alg: int = ALG_AUTO):
        n = len(As)
        pa = (vp * n)(*[a.h for a in As])
        pb = (vp * n)(*[b.h for b in Bs])
        mln = np.ascontiguousarray(np.array(shapes, dtype=np.int32).reshape(-1))
        outs = (vp * n)()
        self._check(self.lib.hegmm_matmul_batch(self.h, n, pa, pb, mln.ctypes.data_as(intp), alg, outs),
                    "matmul_batch")
        return [Ciphertext(self, vp(outs[i])) for i in range(n)]

    def hegmm_matmul_batch_algs(self, As, Bs, shapes, algs=None):
        """One batch with one algorithm per product (None: AUTO for all)."""
        n = len(As)
        pa = (vp * n)(*[a.h for a in As])
        pb = (vp * n)(*[b.h for b in Bs])
        mln = np.ascontiguousarray(np.array(shapes, dtype=np.int32).reshape(-1))
        al = None if algs is None else np.ascontiguousarray(np.array(algs, dtype=np.int32))
        outs = (vp * n)()
        self._check(self.lib.hegmm_matmul_batch_algs(self.h, n, pa, pb, mln.ctypes.data_as(intp),
                                                     None if al is None else al.ctypes.data_as(intp), outs),
                    "matmul_batch_algs")
        return [Ciphertext(self, vp(outs[i])) for i in range(n)]

    def hegmm_lintrans(self, ct: "Ciphertext", src) -> "Ciphertext":
        """hegmm_lintrans: slot j of the result takes slot src[j] (< 0: zero)."""
        s = np.ascontiguousarray(np.array(src, dtype=np.int32))
        out = vp()
        self._check(self.lib.hegmm_lintrans(self.h, ct.h, s.ctypes.data_as(intp), len(s), ctypes.byref(out)),
                    "lintrans")
        return Ciphertext(self, out)

    def hegmm_to_layout(self, ct: "Ciphertext", role: int, m: int, l: int, n: int, alg: int = ALG_AUTO):
        out = vp()
        self._check(self.lib.hegmm_to_layout(self.h, ct.h, role, m, l, n, alg, ctypes.byref(out)), "to_layout")
        return Ciphertext(self, out)

    def hegmm_from_result(self, ct: "Ciphertext", m: int, l: int, n: int, alg: int = ALG_AUTO):
        out = vp()
        self._check(self.lib.hegmm_from_result(self.h, ct.h, m, l, n, alg, ctypes.byref(out)), "from_result")
        return Ciphertext(self, out)

    def hegmm_chain_operand(self, ct: "Ciphertext", m: int, l: int, n: int, alg: int, role: int, m2: int, l2: int,
                            n2: int, alg2: int):
        out = vp()
        self._check(self.lib.hegmm_chain_operand(self.h, ct.h, m, l, n, alg, role, m2, l2, n2, alg2,
                                                 ctypes.byref(out)), "chain_operand")
        return Ciphertext(self, out)

    def hegmm_matmul_sum(self, As, Bs, shapes, group, ngroups: int, algs=None):
        """hegmm_matmul_sum: C[g] = sum of the products p with group[p] == g."""
        n = len(As)
        pa = (vp * n)(*[a.h for a in As])
        pb = (vp * n)(*[b.h for b in Bs])
        mln = np.ascontiguousarray(np.array(shapes, dtype=np.int32).reshape(-1))
        al = None if algs is None else np.ascontiguousarray(np.array(algs, dtype=np.int32))
        gr = np.ascontiguousarray(np.array(group, dtype=np.int32))
        outs = (vp * max(1, ngroups))()
        self._check(self.lib.hegmm_matmul_sum(self.h, n, pa, pb, mln.ctypes.data_as(intp),
                                              None if al is None else al.ctypes.data_as(intp),
                                              gr.ctypes.data_as(intp), int(ngroups), outs), "matmul_sum")
        return [Ciphertext(self, vp(outs[g])) for g in range(ngroups)]

    def hegmm_matmul_blocked(self, rows, inner, cols, A_blocks, B_blocks):
        """hegmm_matmul_blocked: A_blocks[i][k], B_blocks[k][j] (Algorithm 1
        encodings); returns C[i][j] = sum_k A_ik B_kj."""
        nr, nk, nc = len(rows), len(inner), len(cols)
        pa = (vp * (nr * nk))(*[A_blocks[i][k].h for i in range(nr) for k in range(nk)])
        pb = (vp * (nk * nc))(*[B_blocks[k][j].h for k in range(nk) for j in range(nc)])
        r = np.ascontiguousarray(np.array(rows, dtype=np.int32))
        q = np.ascontiguousarray(np.array(inner, dtype=np.int32))
        s = np.ascontiguousarray(np.array(cols, dtype=np.int32))
        outs = (vp * (nr * nc))()
        self._check(self.lib.hegmm_matmul_blocked(self.h, nr, nk, nc, r.ctypes.data_as(intp), q.ctypes.data_as(intp),
                                                  s.ctypes.data_as(intp), pa, pb, outs), "matmul_blocked")
        return [[Ciphertext(self, vp(outs[i * nc + j])) for j in range(nc)] for i in range(nr)]

    def hegmm_decrypt(self, ct: "Ciphertext", m: int, l: int, n: int, alg: int = ALG_AUTO) -> np.ndarray:
        out = np.zeros((m, n), dtype=np.uint64)
        self._check(self.lib.hegmm_decrypt(self.h, ct.h, m, l, n, alg, _ptr(out)), "decrypt")
        return out

    def hegmm_decrypt_slots(self, ct: "Ciphertext") -> np.ndarray:
        out = np.zeros(self.S, dtype=np.uint64)
        self._check(self.lib.hegmm_decrypt_slots(self.h, ct.h, _ptr(out)), "decrypt_slots")
        return out

    def hegmm_decrypt_rows(self, ct: "Ciphertext") -> np.ndarray:
        """Both slot rows: [2][S]."""
        out = np.zeros(2 * self.S, dtype=np.uint64)
        self._check(self.lib.hegmm_decrypt_rows(self.h, ct.h, _ptr(out)), "decrypt_rows")
        return out.reshape(2, self.S)

    def hegmm_decrypt_pair(self, ct: "Ciphertext", m: int, l: int, n: int, alg: int = ALG_AUTO):
        o0 = np.zeros((m, n), dtype=np.uint64)
        o1 = np.zeros((m, n), dtype=np.uint64)
        self._check(self.lib.hegmm_decrypt_pair(self.h, ct.h, m, l, n, alg, _ptr(o0), _ptr(o1)), "decrypt_pair")
        return o0, o1

    def hegmm_rotate(self, ct: "Ciphertext", z: int) -> "Ciphertext":
        out = vp()
        self._check(self.lib.hegmm_rotate(self.h, ct.h, z, ctypes.byref(out)), "rotate")
        return Ciphertext(self, out)

    def hegmm_rotate_many(self, ct: "Ciphertext", zs: Sequence[int]) -> List["Ciphertext"]:
        arr = np.ascontiguousarray(np.array(zs, dtype=np.int32))
        outs = (vp * len(zs))()
        self._check(self.lib.hegmm_rotate_many(self.h, ct.h, arr.ctypes.data_as(intp), len(zs), outs), "rotate_many")
        return [Ciphertext(self, vp(outs[i])) for i in range(len(zs))]

    def hegmm_rotate_noalloc(self, ct: "Ciphertext", z: int, out: "Ciphertext") -> "Ciphertext":
        """Rotation into an existing ciphertext, with no device allocation
        inside the library (for callers that cannot allocate while running;
        see include/hegmm.h)."""
        self._check(self.lib.hegmm_rotate_noalloc(self.h, ct.h, z, out.h), "rotate_noalloc")
        return out

    def hegmm_cmult(self, ct: "Ciphertext", pt: "Plaintext") -> "Ciphertext":
        out = vp()
        self._check(self.lib.hegmm_cmult(self.h, ct.h, pt.h, ctypes.byref(out)), "cmult")
        return Ciphertext(self, out)

    def hegmm_add(self, a: "Ciphertext", b: "Ciphertext") -> "Ciphertext":
        out = vp()
        self._check(self.lib.hegmm_add(self.h, a.h, b.h, ctypes.byref(out)), "add")
        return Ciphertext(self, out)

    def hegmm_mult(self, a: "Ciphertext", b: "Ciphertext") -> "Ciphertext":
        out = vp()
        self._check(self.lib.hegmm_mult(self.h, a.h, b.h, ctypes.byref(out)), "mult")
        return Ciphertext(self, out)

    def hegmm_modswitch(self, ct: "Ciphertext") -> "Ciphertext":
        out = vp()
        self._check(self.lib.hegmm_modswitch(self.h, ct.h, ctypes.byref(out)), "modswitch")
        return Ciphertext(self, out)

    def hegmm_ct_export(self, ct: "Ciphertext", out: Optional[np.ndarray] = None) -> np.ndarray:
        lv = self.lib.hegmm_ct_level(ct.h)
        if out is None:
            out = np.zeros((2, lv, self.N), dtype=np.uint64)
        self._check(self.lib.hegmm_ct_export(self.h, ct.h, _ptr(out)), "ct_export")
        return out

    def hegmm_ct_import(self, host: np.ndarray) -> "Ciphertext":
        a = _u64(host)
        lv = a.shape[1]
        out = vp()
        self._check(self.lib.hegmm_ct_import(self.h, _ptr(a), lv, ctypes.byref(out)), "ct_import")
        return Ciphertext(self, out)

    def hegmm_ct_import_batch(self, hosts) -> List["Ciphertext"]:
        """hosts: [2][level][N] uint64 arrays (the same level); one transform launch."""
        arrs = [_u64(h) for h in hosts]
        n = len(arrs)
        if n == 0:
            return []
        lv = arrs[0].shape[1]
        ptrs = (u64p * n)(*[_ptr(a) for a in arrs])
        outs = (vp * n)()
        self._check(self.lib.hegmm_ct_import_batch(self.h, n, ptrs, lv, outs), "ct_import_batch")
        return [Ciphertext(self, vp(outs[i])) for i in range(n)]

    def hegmm_ct_export_batch(self, cts, outs) -> None:
        """Writes each ciphertext into the matching [2][level][N] uint64 array; one synchronisation."""
        n = len(cts)
        if n == 0:
            return
        for o in outs:
            assert o.dtype == np.uint64 and o.flags["C_CONTIGUOUS"]
        pc = (vp * n)(*[c.h for c in cts])
        po = (u64p * n)(*[_ptr(o) for o in outs])
        self._check(self.lib.hegmm_ct_export_batch(self.h, n, pc, po), "ct_export_batch")

    def hegmm_sync(self):
        self._check(self.lib.hegmm_sync(self.h), "sync")

    def hegmm_set_timing(self, enable: bool):
        self._check(self.lib.hegmm_set_timing(self.h, int(bool(enable))), "set_timing")

    def hegmm_kernel_stats(self):
        """{kernel name: (total ms, launches, algorithmic bytes, butterflies)}."""
        out = {}
        for k in range(self.lib.hegmm_kernel_kinds()):
            ms, n, b, w = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double()
            self._check(self.lib.hegmm_kernel_stats(self.h, k, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(b),
                                                    ctypes.byref(w)), "kernel_stats")
            out[self.lib.hegmm_kernel_name(k).decode()] = (ms.value, n.value, b.value, w.value)
        return out

    def hegmm_kernel_reset(self):
        self._check(self.lib.hegmm_kernel_reset(self.h), "kernel_reset")

    def hegmm_set_key_policy(self, policy: int):
        self._check(self.lib.hegmm_set_key_policy(self.h, policy), "set_key_policy")

    def hegmm_device_memory(self, reset_high: bool = False) -> dict:
        """{pool_used, pool_used_high, pool_reserved, device_free} in bytes."""
        out = np.zeros(4, dtype=np.uint64)
        self._check(self.lib.hegmm_device_memory(self.h, int(bool(reset_high)), out.ctypes.data_as(u64p)),
                    "device_memory")
        return dict(zip(("pool_used", "pool_used_high", "pool_reserved", "device_free"), (int(v) for v in out)))

    def hegmm_peak_butterflies(self) -> float:
        v = ctypes.c_double()
        self._check(self.lib.hegmm_peak_butterflies(self.h, ctypes.byref(v)), "peak_butterflies")
        return v.value


class Plaintext:
    def __init__(self, ctx: Context, h):
        self.ctx = ctx
        self.h = h

    def __del__(self):
        try:
            if self.h and self.ctx.h:
                self.ctx.lib.hegmm_pt_destroy(self.h)
        except Exception:
            pass


class Ciphertext:
    def __init__(self, ctx: Context, h):
        self.ctx = ctx
        self.h = h

    @property
    def level(self) -> int:
        return self.ctx.lib.hegmm_ct_level(self.h)

    def __del__(self):
        try:
            if self.h and self.ctx.h:
                self.ctx.lib.hegmm_ct_destroy(self.h)
        except Exception:
            pass


class Server:
    """Continuous-batching request loop (hegmm_server_*); driven by poll()."""

    def __init__(self, ctx: Context, max_batch: int = 0, streams: int = 0, mem_budget: int = 0):
        self.ctx = ctx
        self.lib = ctx.lib
        opts = hegmm_server_opts(max_batch, streams, mem_budget)
        h = vp()
        ctx._check(self.lib.hegmm_server_create(ctx.h, ctypes.byref(opts), ctypes.byref(h)), "server_create")
        self.h = h
        self._keep = {}

    def hegmm_server_submit(self, A: "Ciphertext", B: "Ciphertext", m: int, l: int, n: int,
                            alg: int = ALG_AUTO) -> int:
        t = ctypes.c_uint64()
        self.ctx._check(self.lib.hegmm_server_submit(self.h, A.h, B.h, m, l, n, alg, ctypes.byref(t)), "server_submit")
        self._keep[t.value] = (A, B)  # operands must outlive the request
        return t.value

    def hegmm_server_poll(self, wait: bool = False):
        self.ctx._check(self.lib.hegmm_server_poll(self.h, int(bool(wait))), "server_poll")

    def hegmm_server_result(self, ticket: int):
        """(Ciphertext, latency_ms) once the request has completed, else None."""
        out = vp()
        lat = ctypes.c_double()
        self.ctx._check(self.lib.hegmm_server_result(self.h, ticket, ctypes.byref(out), ctypes.byref(lat)),
                        "server_result")
        if not out.value:
            return None
        self._keep.pop(ticket, None)
        return Ciphertext(self.ctx, out), lat.value

    def hegmm_server_stats_get(self) -> dict:
        st = hegmm_server_stats()
        self.ctx._check(self.lib.hegmm_server_stats_get(self.h, ctypes.byref(st)), "server_stats")
        return st.as_dict()

    def close(self):
        if getattr(self, "h", None):
            self.lib.hegmm_server_destroy(self.h)
            self.h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""Ciphertext-level oracle: BGV operations (plain C) and the HEGMM executor.

Test infrastructure (see ``oracle/__init__.py``).  The ring and scheme
arithmetic lives in ``he_oracle.c``; this module loads it through ctypes,
adds slot encoding (Python + the C NTT mod t), decryption with an exact
big-integer CRT, and runs Algorithms 1 and 2 of the paper on ciphertexts,
using the plans of ``oracle.slots``.

Slot layout (BGV with t = 1 mod 2N): the slot vector is one row of S = N/2
slots; slot j of row 0 is the evaluation of the plaintext at
zeta^(5^j mod 2N), slot j of row 1 the evaluation at zeta^(-5^j), with
zeta = 3^((t-1)/2N) mod t.  HE-Rot by z (Section 2.1) is the automorphism
X -> X^g, g = 5^(z mod S) mod 2N: it rotates both rows left by z.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from typing import Dict, List, Optional, Tuple

import numpy as np

from . import slots as SL

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "he_oracle.c")
_LIB = os.path.join(_HERE, "libhe_oracle.so")

u64p = ctypes.POINTER(ctypes.c_uint64)
i64p = ctypes.POINTER(ctypes.c_int64)
intp = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile he_oracle.c into libhe_oracle.so with gcc (plain C, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.or_new.restype = ctypes.c_void_p
        L.or_new.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.or_free.argtypes = [ctypes.c_void_p]
        L.or_get_primes.argtypes = [ctypes.c_void_p, u64p]
        L.or_get_psi.restype = ctypes.c_uint64
        L.or_get_psi.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.or_is_prime.restype = ctypes.c_int
        L.or_is_prime.argtypes = [ctypes.c_uint64]
        L.or_find_primes.restype = ctypes.c_int
        L.or_find_primes.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, u64p]
        for name in ("or_mix64",):
            getattr(L, name).restype = ctypes.c_uint64
            getattr(L, name).argtypes = [ctypes.c_uint64]
        L.or_stream.restype = ctypes.c_uint64
        L.or_stream.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        L.or_draw.restype = ctypes.c_uint64
        L.or_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.or_ntt.argtypes = [ctypes.c_void_p, ctypes.c_int, u64p]
        L.or_intt.argtypes = [ctypes.c_void_p, ctypes.c_int, u64p]
        L.or_negacyclic_schoolbook.argtypes = [u64p, u64p, ctypes.c_int, ctypes.c_uint64, u64p]
        L.or_polymul.argtypes = [ctypes.c_void_p, ctypes.c_int, u64p, u64p, u64p]
        L.or_sample_secret.argtypes = [ctypes.c_void_p, ctypes.c_uint64, i64p]
        L.or_gen_evk.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, i64p, u64p, u64p]
        L.or_encrypt.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, i64p, i64p, u64p]
        L.or_decrypt_residues.argtypes = [ctypes.c_void_p, ctypes.c_int, i64p, u64p, u64p]
        L.or_encrypt_scaled.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, i64p, i64p, u64p, u64p]
        L.or_set_error_factor.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
        L.or_automorph.argtypes = [ctypes.c_void_p, ctypes.c_int, intp, u64p, ctypes.c_uint64, u64p]
        L.or_automorph_int.argtypes = [ctypes.c_void_p, i64p, ctypes.c_uint64, i64p]
        L.or_modup.argtypes = [ctypes.c_void_p, ctypes.c_int, u64p, u64p]
        L.or_ks_inner.argtypes = [ctypes.c_void_p, ctypes.c_int, u64p, u64p, u64p]
        L.or_moddown.argtypes = [ctypes.c_void_p, ctypes.c_int, u64p, u64p]
        L.or_keyswitch.argtypes = [ctypes.c_void_p, ctypes.c_int, u64p, u64p, u64p]
        L.or_rotate.argtypes = [ctypes.c_void_p, ctypes.c_int, u64p, ctypes.c_uint64, u64p, u64p]
        L.or_rotate_hoisted.argtypes = [ctypes.c_void_p, ctypes.c_int, u64p, ctypes.c_uint64, u64p, u64p]
        L.or_add.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, u64p, u64p, u64p]
        L.or_cmult.argtypes = [ctypes.c_void_p, ctypes.c_int, u64p, u64p, u64p]
        L.or_tensor.argtypes = [ctypes.c_void_p, ctypes.c_int, u64p, u64p, u64p]
        L.or_mult_relin.argtypes = [ctypes.c_void_p, ctypes.c_int, u64p, u64p, u64p, u64p]
        L.or_modswitch.argtypes = [ctypes.c_void_p, ctypes.c_int, u64p, u64p]
        L.or_ks_raw.argtypes = [ctypes.c_void_p, ctypes.c_int, u64p, ctypes.c_uint64, u64p, u64p]
        L.or_pq_lift.argtypes = [ctypes.c_void_p, ctypes.c_int, u64p, u64p]
        L.or_pq_mac.argtypes = [ctypes.c_void_p, ctypes.c_int, u64p, u64p, u64p]
        L.or_to_eval.argtypes = [ctypes.c_void_p, ctypes.c_int, intp, u64p]
        L.or_to_coeff.argtypes = [ctypes.c_void_p, ctypes.c_int, intp, u64p]
        _lib = L
    return _lib


def P(a: np.ndarray):
    """ctypes pointer to a contiguous uint64 array."""
    assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(u64p)


def PI(a: np.ndarray):
    assert a.dtype == np.int64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(i64p)


def PINT(idx: List[int]):
    arr = (ctypes.c_int * len(idx))(*idx)
    return arr


def mix64(z: int) -> int:
    return lib().or_mix64(z)


def is_prime(n: int) -> bool:
    return bool(lib().or_is_prime(n))


class Oracle:
    """BGV over R_Q, Q = q_0 ... q_{L-1}, with K special primes, for one preset."""

    def __init__(self, preset):
        self.pre = preset
        self.N = preset.N
        self.S = preset.N // 2
        self.L = preset.L
        self.K = preset.K
        self.alpha = preset.alpha
        self.t = preset.t
        self.ctx = lib().or_new(preset.logN, preset.t, preset.L, preset.qbits, preset.K, preset.alpha, preset.eta)
        if not self.ctx:
            raise RuntimeError("oracle: parameter set not available")
        pr = np.zeros(self.L + self.K, dtype=np.uint64)
        lib().or_get_primes(self.ctx, P(pr))
        self.primes = [int(x) for x in pr]
        self.zeta = int(lib().or_get_psi(self.ctx, -1))
        # slot j of row 0 <-> NTT index (5^j mod 2N - 1)/2 of the oracle's
        # natural-order negacyclic NTT mod t; row 1 <-> (-5^j mod 2N - 1)/2.
        two_n = 2 * self.N
        self.slot_pos0 = np.array([((pow(5, j, two_n)) - 1) // 2 for j in range(self.S)], dtype=np.int64)
        self.slot_pos1 = np.array([((-pow(5, j, two_n)) % two_n - 1) // 2 for j in range(self.S)], dtype=np.int64)
        self.sk: Optional[np.ndarray] = None
        self.keys: Dict[int, np.ndarray] = {}   # galois element (0 = relin) -> evk in NTT form
        self.key_seed = None
        self.counts = {}

    def __del__(self):
        try:
            if self.ctx:
                lib().or_free(self.ctx)
        except Exception:
            pass

    # ---------------------------------------------------------------- NTT
    def ntt(self, a: np.ndarray, pi: int) -> np.ndarray:
        a = np.ascontiguousarray(a, dtype=np.uint64).copy()
        lib().or_ntt(self.ctx, pi, P(a))
        return a

    def intt(self, a: np.ndarray, pi: int) -> np.ndarray:
        a = np.ascontiguousarray(a, dtype=np.uint64).copy()
        lib().or_intt(self.ctx, pi, P(a))
        return a

    # ------------------------------------------------------------ encoding
    def encode(self, row0, row1=None) -> np.ndarray:
        """Slot vectors (values mod t) -> centred plaintext coefficients (int64)."""
        ev = np.zeros(self.N, dtype=np.uint64)
        r0 = np.zeros(self.S, dtype=np.int64)
        r0[: len(row0)] = np.asarray(row0, dtype=np.int64) % self.t
        ev[self.slot_pos0] = r0.astype(np.uint64)
        if row1 is not None:
            r1 = np.zeros(self.S, dtype=np.int64)
            r1[: len(row1)] = np.asarray(row1, dtype=np.int64) % self.t
            ev[self.slot_pos1] = r1.astype(np.uint64)
        m = self.intt(ev, -1).astype(np.int64)
        m[m > (self.t - 1) // 2] -= self.t
        return m

    def decode(self, coeffs) -> Tuple[np.ndarray, np.ndarray]:
        """Plaintext coefficients (any integers) -> (row 0, row 1) slot values mod t."""
        c = (np.asarray(coeffs, dtype=np.int64) % self.t).astype(np.uint64)
        ev = self.ntt(c, -1).astype(np.int64)
        return ev[self.slot_pos0], ev[self.slot_pos1]

    def residues(self, m: np.ndarray, lv: int) -> np.ndarray:
        """Signed coefficients -> residues over q_0..q_{lv-1}, [lv][N] uint64."""
        out = np.empty((lv, self.N), dtype=np.uint64)
        for i in range(lv):
            out[i] = (np.asarray(m, dtype=object) % self.primes[i]).astype(np.uint64)
        return out

    def plaintext_eval(self, m: np.ndarray, lv: int) -> np.ndarray:
        """Plaintext in the form or_cmult expects (NTT of residues)."""
        r = self.residues(m, lv)
        lib().or_to_eval(self.ctx, lv, PINT(list(range(lv))), P(r))
        return r

    # ------------------------------------------------------------- keys
    def galois(self, z: int) -> int:
        """Galois element of a left rotation by z (negative z: S + z)."""
        return pow(5, z % self.S, 2 * self.N)

    def secret(self, seed: int) -> np.ndarray:
        s = np.zeros(self.N, dtype=np.int64)
        lib().or_sample_secret(self.ctx, seed, PI(s))
        return s

    def _evk(self, seed: int, gtag: int, sprime_res: np.ndarray, eval_form: bool = True) -> np.ndarray:
        nk = self.L + self.K
        dnum = -(-self.L // self.alpha)
        evk = np.zeros((dnum, 2, nk, self.N), dtype=np.uint64)
        lib().or_gen_evk(self.ctx, seed, gtag, PI(self.sk), P(np.ascontiguousarray(sprime_res)), P(evk))
        if eval_form:
            flat = evk.reshape(-1, self.N)
            lib().or_to_eval(self.ctx, flat.shape[0], PINT([r % nk for r in range(flat.shape[0])]), P(flat))
        return evk

    def sprime_galois(self, g: int) -> np.ndarray:
        sg = np.zeros(self.N, dtype=np.int64)
        lib().or_automorph_int(self.ctx, PI(self.sk), g, PI(sg))
        nk = self.L + self.K
        out = np.empty((nk, self.N), dtype=np.uint64)
        for i in range(nk):
            out[i] = (sg % self.primes[i]).astype(np.uint64)
        return out

    def sprime_square(self) -> np.ndarray:
        nk = self.L + self.K
        out = np.empty((nk, self.N), dtype=np.uint64)
        for i in range(nk):
            sr = (self.sk % self.primes[i]).astype(np.uint64)
            o = np.zeros(self.N, dtype=np.uint64)
            lib().or_polymul(self.ctx, i, P(sr), P(sr), P(o))
            out[i] = o
        return out

    def keygen(self, seed: int, galois_elements=()):
        """Secret key, relinearisation key and the listed Galois keys."""
        self.key_seed = seed
        self.sk = self.secret(seed)
        self.keys = {0: self._evk(seed, 0, self.sprime_square())}
        for g in galois_elements:
            self.add_galois_key(g)

    def add_galois_key(self, g: int):
        if g not in self.keys:
            self.keys[g] = self._evk(self.key_seed, g, self.sprime_galois(g))

    def evk_coeff(self, g: int) -> np.ndarray:
        """A key in coefficient form (for comparison with exported keys)."""
        sp = self.sprime_square() if g == 0 else self.sprime_galois(g)
        return self._evk(self.key_seed, g, sp, eval_form=False)

    # ------------------------------------------------------- encryption
    def encrypt(self, m: np.ndarray, seed: int, stream: int) -> np.ndarray:
        ct = np.zeros((2, self.L, self.N), dtype=np.uint64)
        mm = np.ascontiguousarray(m, dtype=np.int64)
        lib().or_encrypt(self.ctx, seed, stream, PI(self.sk), PI(mm), P(ct))
        return ct

    def decrypt(self, ct: np.ndarray, lv: Optional[int] = None):
        """Returns (plaintext coefficients mod t, noise bits, budget bits).

        v = [c0 + c1 s]_Q with an exact CRT, centred; the plaintext is v mod t;
        noise bits = log2 max |v|, budget = log2(Q/2).
        """
        lv = ct.shape[1] if lv is None else lv
        v = np.zeros((lv, self.N), dtype=np.uint64)
        lib().or_decrypt_residues(self.ctx, lv, PI(self.sk), P(np.ascontiguousarray(ct)), P(v))
        Q = 1
        for i in range(lv):
            Q *= self.primes[i]
        acc = np.zeros(self.N, dtype=object)
        for i in range(lv):
            qi = self.primes[i]
            Qi = Q // qi
            coef = Qi * pow(Qi % qi, -1, qi)
            acc = acc + v[i].astype(object) * coef
        acc = acc % Q
        half = Q // 2
        acc = np.where(acc > half, acc - Q, acc)
        mx = max(abs(int(x)) for x in acc)
        noise = math.log2(mx) if mx > 0 else 0.0
        m = np.array([int(x) % self.t for x in acc], dtype=np.int64)
        return m, noise, math.log2(Q / 2)

    def decrypt_slots(self, ct: np.ndarray) -> np.ndarray:
        m, _, _ = self.decrypt(ct)
        return self.decode(m)[0]

    def decrypt_rows(self, ct: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
        m, _, _ = self.decrypt(ct)
        return self.decode(m)

    # -------------------------------------------------------- operations
    def rotate(self, ct: np.ndarray, z: int, hoisted: bool = False) -> np.ndarray:
        lv = ct.shape[1]
        if z % self.S == 0:
            return ct.copy()
        g = self.galois(z)
        self.add_galois_key(g)
        out = np.zeros_like(ct)
        fn = lib().or_rotate_hoisted if hoisted else lib().or_rotate
        fn(self.ctx, lv, P(np.ascontiguousarray(ct)), g, P(self.keys[g]), P(out))
        self.counts["rot"] = self.counts.get("rot", 0) + 1
        return out

    def rotate_pow2(self, ct: np.ndarray, z: int) -> np.ndarray:
        """Rotation under the power-of-two key policy: the chain of HE-Rot by
        the steps of slots.pow2_steps(z, S), least significant first; only
        keys of +-2^i rotations are used."""
        out = ct.copy()
        for step in SL.pow2_steps(z, self.S):
            out = self.rotate(out, step)
        return out

    def cmult(self, ct: np.ndarray, pt_eval: np.ndarray) -> np.ndarray:
        lv = ct.shape[1]
        out = np.zeros_like(ct)
        lib().or_cmult(self.ctx, lv, P(np.ascontiguousarray(ct)), P(np.ascontiguousarray(pt_eval[:lv])), P(out))
        self.counts["cmult"] = self.counts.get("cmult", 0) + 1
        return out

    def add(self, a: np.ndarray, b: np.ndarray) -> np.ndarray:
        lv = a.shape[1]
        out = np.zeros_like(a)
        lib().or_add(self.ctx, lv, a.shape[0], P(np.ascontiguousarray(a)), P(np.ascontiguousarray(b)), P(out))
        return out

    def mult_relin(self, a: np.ndarray, b: np.ndarray) -> np.ndarray:
        lv = a.shape[1]
        out = np.zeros_like(a)
        lib().or_mult_relin(self.ctx, lv, P(np.ascontiguousarray(a)), P(np.ascontiguousarray(b)), P(self.keys[0]), P(out))
        self.counts["mult"] = self.counts.get("mult", 0) + 1
        return out

    def tensor(self, a: np.ndarray, b: np.ndarray) -> np.ndarray:
        lv = a.shape[1]
        d = np.zeros((3, lv, self.N), dtype=np.uint64)
        lib().or_tensor(self.ctx, lv, P(np.ascontiguousarray(a)), P(np.ascontiguousarray(b)), P(d))
        return d

    def keyswitch(self, x: np.ndarray, g: int) -> np.ndarray:
        lv = x.shape[0]
        out = np.zeros((2, lv, self.N), dtype=np.uint64)
        lib().or_keyswitch(self.ctx, lv, P(np.ascontiguousarray(x)), P(self.keys[g]), P(out))
        return out

    def modswitch(self, ct: np.ndarray) -> np.ndarray:
        lv = ct.shape[1]
        out = np.zeros((2, lv - 1, self.N), dtype=np.uint64)
        lib().or_modswitch(self.ctx, lv, P(np.ascontiguousarray(ct)), P(out))
        self.counts["modswitch"] = self.counts.get("modswitch", 0) + 1
        return out

    def modup(self, x: np.ndarray) -> np.ndarray:
        lv = x.shape[0]
        nd = -(-lv // self.alpha)
        D = np.zeros((nd, lv + self.K, self.N), dtype=np.uint64)
        lib().or_modup(self.ctx, lv, P(np.ascontiguousarray(x)), P(D))
        return D

    def moddown(self, u: np.ndarray, lv: int) -> np.ndarray:
        out = np.zeros((lv, self.N), dtype=np.uint64)
        lib().or_moddown(self.ctx, lv, P(np.ascontiguousarray(u)), P(out))
        return out

    def automorph(self, a: np.ndarray, g: int, prime_idx: List[int]) -> np.ndarray:
        out = np.zeros_like(a)
        lib().or_automorph(self.ctx, len(prime_idx), PINT(prime_idx), P(np.ascontiguousarray(a)), g, P(out))
        return out

    # ------------------------------------- key switching kept in the basis PQ
    # The inner product of a key switch produces u over the extended basis
    # (q_0..q_{lv-1}, p_0..p_{K-1}); ModDown divides by P = prod p_k with
    # t-corrected rounding.  Because ModDown(u + P x) = ModDown(u) + x holds
    # exactly, sums of key-switched terms (with plaintext factors) can be
    # formed over PQ and divided once ("double hoisting").

    def ext_primes(self, lv: int) -> List[int]:
        return list(range(lv)) + [self.L + k for k in range(self.K)]

    def ks_raw(self, D: np.ndarray, tag: int) -> np.ndarray:
        """u = <tau_g(D), evk_g> before ModDown, [2][lv+K][N] coefficient form.

        D is the ModUp of c1 at its level; tag is the Galois element, or 0
        for the relinearisation key (no automorphism)."""
        nd, ne, _ = D.shape
        lv = ne - self.K
        u = np.zeros((2, ne, self.N), dtype=np.uint64)
        g = 1 if tag == 0 else tag
        lib().or_ks_raw(self.ctx, lv, P(np.ascontiguousarray(D)), g, P(self.keys[tag]), P(u))
        self.counts["ksw_raw"] = self.counts.get("ksw_raw", 0) + 1
        return u

    def pq_lift(self, x: np.ndarray) -> np.ndarray:
        """P x on the chain primes, 0 on the special primes: [lv+K][N]."""
        lv = x.shape[0]
        out = np.zeros((lv + self.K, self.N), dtype=np.uint64)
        lib().or_pq_lift(self.ctx, lv, P(np.ascontiguousarray(x)), P(out))
        return out

    def pq_add(self, a: np.ndarray, b: np.ndarray) -> np.ndarray:
        ne = a.shape[0]
        out = np.empty_like(a)
        for e, gp in enumerate(self.ext_primes(ne - self.K)):
            out[e] = (a[e] + b[e]) % np.uint64(self.primes[gp])
        return out

    def pq_mac(self, acc: np.ndarray, a: np.ndarray, m_eval: np.ndarray) -> None:
        """acc += m a over the extended basis (m_eval from plaintext_eval_pq)."""
        lv = a.shape[0] - self.K
        lib().or_pq_mac(self.ctx, lv, P(np.ascontiguousarray(a)), P(np.ascontiguousarray(m_eval)), P(acc))

    def plaintext_eval_pq(self, m: np.ndarray, lv: int) -> np.ndarray:
        """Plaintext residues over the extended basis of level lv, NTT form."""
        ext = self.ext_primes(lv)
        r = np.empty((len(ext), self.N), dtype=np.uint64)
        for e, gp in enumerate(ext):
            r[e] = (np.asarray(m, dtype=object) % self.primes[gp]).astype(np.uint64)
        lib().or_to_eval(self.ctx, len(ext), PINT(ext), P(r))
        return r

    def moddown_pair(self, acc: np.ndarray) -> np.ndarray:
        lv = acc.shape[1] - self.K
        return np.stack([self.moddown(acc[0], lv), self.moddown(acc[1], lv)])


# --------------------------------------------------------------------------
# HEGMM on ciphertexts (Algorithms 1 and 2)
# --------------------------------------------------------------------------


class OracleBFV(Oracle):
    """The BFV variant (the paper's own scheme, Section 4.1: Pyfhel's BFV):
    the same ring, keys, key switching and slot encoding, with the message
    scaled instead of the noise:

    * encryption c0 = -a s + e + Delta m, c1 = a, Delta = floor(Q / t);
      decryption m = round(t [c0 + c1 s]_Q / Q) mod t (exact, big integers);
    * switching keys b_j = -a_j s + e_j + [P]_{q_i} s' (no factor t) and a
      ModDown with plain centred rounding: the BGV operations of the C
      oracle with its error factor set to 1;
    * HE-Mult: the tensor of the centred lifts of both operands over Z,
      (d0, d1, d2) = (a0 b0, a0 b1 + a1 b0, a1 b1), scaled by t / Q and
      rounded to the nearest integer (never a tie: Q is odd), reduced mod
      Q, then d2 relinearised with the relinearisation key.  The exact
      tensor is computed modulo enough auxiliary NTT primes and put together
      by the Chinese remainder theorem (an exact product by multi-modular
      arithmetic).
    """

    bfv = True

    def __init__(self, preset):
        super().__init__(preset)
        if preset.ms_drop:
            raise ValueError("the BFV variant has no modulus switch")
        lib().or_set_error_factor(self.ctx, 1)
        self.Q = 1
        for q in self.primes[: self.L]:
            self.Q *= q
        self.delta = self.Q // self.t
        self.delta_res = np.array([self.delta % q for q in self.primes[: self.L]], dtype=np.uint64)
        # auxiliary primes for exact products: their product exceeds
        # 2 (N Q^2 / 2) + margin, the bound of a lazy sum of up to 2^12 tensors
        need = self.pre.logN + 2 * self.Q.bit_length() + 16
        naux = -(-need // 59)
        self.aux = lib().or_new(self.pre.logN, self.t, naux, 60, 1, 1, self.pre.eta)
        if not self.aux:
            raise RuntimeError("oracle: no auxiliary primes")
        pr = np.zeros(naux + 1, dtype=np.uint64)
        lib().or_get_primes(self.aux, P(pr))
        self.aux_primes = [int(x) for x in pr[:naux]]
        self.aux_M = 1
        for p in self.aux_primes:
            self.aux_M *= p

    def __del__(self):
        try:
            if getattr(self, "aux", None):
                lib().or_free(self.aux)
        except Exception:
            pass
        super().__del__()

    def encrypt(self, m: np.ndarray, seed: int, stream: int) -> np.ndarray:
        ct = np.zeros((2, self.L, self.N), dtype=np.uint64)
        mm = np.ascontiguousarray(m, dtype=np.int64)
        lib().or_encrypt_scaled(self.ctx, seed, stream, PI(self.sk), PI(mm), P(self.delta_res), P(ct))
        return ct

    def _centred(self, res: np.ndarray) -> np.ndarray:
        """Residues [lv][N] over q_0..q_{lv-1} -> centred integers (object)."""
        lv = res.shape[0]
        Q = 1
        for i in range(lv):
            Q *= self.primes[i]
        acc = np.zeros(self.N, dtype=object)
        for i in range(lv):
            qi = self.primes[i]
            Qi = Q // qi
            acc = acc + res[i].astype(object) * (Qi * pow(Qi % qi, -1, qi))
        acc = acc % Q
        return np.where(acc > Q // 2, acc - Q, acc)

    def decrypt(self, ct: np.ndarray, lv: Optional[int] = None):
        """Returns (plaintext coefficients mod t, noise bits, budget bits):
        m = round(t v / Q) mod t for v = [c0 + c1 s]_Q centred; the noise is
        v - Delta m' (m' = round(t v / Q)), the budget log2(Q / (2 t))."""
        lv = ct.shape[1] if lv is None else lv
        v = np.zeros((lv, self.N), dtype=np.uint64)
        lib().or_decrypt_residues(self.ctx, lv, PI(self.sk), P(np.ascontiguousarray(ct)), P(v))
        vc = self._centred(v)
        Q = self.Q
        mr = [(2 * self.t * int(x) + Q) // (2 * Q) for x in vc]
        noise = max(abs(int(x) - self.delta * r) for x, r in zip(vc, mr))
        m = np.array([r % self.t for r in mr], dtype=np.int64)
        return m, (math.log2(noise) if noise > 0 else 0.0), math.log2(Q / (2 * self.t))

    def tensor_exact(self, a: np.ndarray, b: np.ndarray) -> np.ndarray:
        """(a0 b0, a0 b1 + a1 b0, a1 b1) over Z of the centred lifts of two
        ciphertexts, exact: computed modulo the auxiliary primes (negacyclic
        NTT products) and recombined by CRT; object array [3][N]."""
        ac = [self._centred(np.ascontiguousarray(a[i])) for i in range(2)]
        bc = [self._centred(np.ascontiguousarray(b[i])) for i in range(2)]
        res = np.zeros((3, len(self.aux_primes), self.N), dtype=np.uint64)
        for j, p in enumerate(self.aux_primes):
            ar = [(x % p).astype(np.uint64) for x in ac]
            br = [(x % p).astype(np.uint64) for x in bc]
            prod = {}
            for (u, v) in ((0, 0), (0, 1), (1, 0), (1, 1)):
                o = np.zeros(self.N, dtype=np.uint64)
                lib().or_polymul(self.aux, j, P(ar[u]), P(br[v]), P(o))
                prod[(u, v)] = o.astype(object)
            res[0, j] = (prod[(0, 0)] % p).astype(np.uint64)
            res[1, j] = ((prod[(0, 1)] + prod[(1, 0)]) % p).astype(np.uint64)
            res[2, j] = (prod[(1, 1)] % p).astype(np.uint64)
        M = self.aux_M
        out = np.zeros((3, self.N), dtype=object)
        for k in range(3):
            acc = np.zeros(self.N, dtype=object)
            for j, p in enumerate(self.aux_primes):
                Mj = M // p
                acc = acc + res[k, j].astype(object) * (Mj * pow(Mj % p, -1, p))
            acc = acc % M
            out[k] = np.where(acc > M // 2, acc - M, acc)
        return out

    def scale_round(self, d: np.ndarray) -> np.ndarray:
        """round(t d / Q) of exact integers d [3][N], as residues [3][L][N]."""
        Q, t = self.Q, self.t
        out = np.zeros((d.shape[0], self.L, self.N), dtype=np.uint64)
        for k in range(d.shape[0]):
            z = np.array([(2 * t * int(x) + Q) // (2 * Q) for x in d[k]], dtype=object)
            for i in range(self.L):
                out[k, i] = (z % self.primes[i]).astype(np.uint64)
        return out

    def tensor(self, a: np.ndarray, b: np.ndarray) -> np.ndarray:
        """HE-Mult before relinearisation: the scaled, rounded tensor."""
        return self.scale_round(self.tensor_exact(a, b))

    def mult_relin(self, a: np.ndarray, b: np.ndarray) -> np.ndarray:
        d = self.tensor(a, b)
        ks = self.keyswitch(d[2], 0)
        self.counts["mult"] = self.counts.get("mult", 0) + 1
        return self.add(np.ascontiguousarray(d[:2]), ks)

    def modswitch(self, ct: np.ndarray) -> np.ndarray:
        raise ValueError("the BFV variant has no modulus switch")


def make_oracle(preset) -> Oracle:
    """The oracle of a preset's scheme (BGV, or the BFV variant)."""
    return OracleBFV(preset) if getattr(preset, "scheme", 0) == 1 else Oracle(preset)


def mask_scale(o: Oracle) -> int:
    """Mask entry value: 1, or [q_drop]_t when the product level drops primes.

    A modulus switch multiplies the message by q_drop^-1 mod t; encoding the
    eps/omega masks with q_drop cancels that factor on both operands.
    """
    s = 1
    for i in range(o.pre.ms_drop):
        s = s * o.primes[o.L - 1 - i] % o.t
    return s


class HEGMM:
    """Runs a plan of ``oracle.slots`` on ciphertexts, op by op."""

    MODES = ("single", "double")

    def __init__(self, o: Oracle, mode: str = "single", lazy_relin: bool = False, giant: bool = False,
                 giant_cost: int = SL.GIANT_COST, key_policy: str = "direct"):
        """mode "single": every key switch ends in its own ModDown, as the
        HE operations Rot, CMult, Mult and Add compose (the paper's cost
        model).  mode "double": the sums of key-switched terms (each linear
        transformation, the HE-Add of the per-iteration products, the
        extraction sum) are formed over the extended basis PQ and take one
        ModDown each; decrypts to the same product, with lower noise.
        lazy_relin: the per-iteration tensors (d0, d1, d2) are summed first
        and the sum is relinearised once (one key switch per product instead
        of one per HE-Mult); in double mode that key switch keeps P (d0, d1)
        in its sum over PQ.
        giant: every linear transformation of an operand is evaluated as
        Rot(sum_d u'_d (.) Rot(ct, b_d), g) with the offsets b_d shared by all
        iterations (``slots.giant_factor``); the inner sum is evaluated in the
        chosen mode, the outer rotation is one HE-Rot.
        key_policy "direct": one Galois key per rotation offset; "pow2": only
        keys of rotations by +-2^i, every rotation is Oracle.rotate_pow2 (a
        chain of HE-Rot).  Under pow2 a linear transformation is the sum of
        the mask products of its chained rotations in either mode (the
        double mode's sum over PQ of lifted ciphertexts P x is divided back
        exactly, ModDown(P x) = x), and so is the extraction sum."""
        if mode not in self.MODES:
            raise ValueError(mode)
        if key_policy not in ("direct", "pow2"):
            raise ValueError(key_policy)
        self.pow2 = key_policy == "pow2"
        self.o = o
        self.mode = mode
        self.lazy_relin = lazy_relin
        self.giant = giant
        self.giant_cost = giant_cost
        self._mask_cache: Dict[Tuple, np.ndarray] = {}

    def mask_eval(self, dsts: List[int], scale: int, lv: int) -> np.ndarray:
        """The mask u_d of Eq. lintrans: ``scale`` on the destination slots of
        both slot rows (a rotation moves both rows alike, so a second
        product in row 1 is transformed the same way), 0 elsewhere."""
        key = (tuple(dsts), scale, lv)
        if key not in self._mask_cache:
            v = np.zeros(self.o.S, dtype=np.int64)
            v[dsts] = scale
            self._mask_cache[key] = self.o.plaintext_eval(self.o.encode(v, v), lv)
        return self._mask_cache[key]

    def galois_needed(self, plan: SL.Plan) -> List[int]:
        """Galois elements of every rotation the run key-switches: the plan's
        diagonals and extraction offsets, and in the shared-baby-step order
        the baby offsets and giant rotations of its factorisation."""
        if self.pow2:
            return sorted({self.o.galois(z) for z in SL.pow2_offsets(self.o.S)})
        zs = set()
        for e, om in plan.iters:
            zs.update(d for d in e if d % self.o.S)
            zs.update(d for d in om if d % self.o.S)
        zs.update(z for z in plan.extract if z % self.o.S)
        if self.giant:
            for s in (0, 1):
                for g, terms in SL.giant_factor([it[s] for it in plan.iters], self.o.S, self.giant_cost):
                    zs.update(z for z in [g] + [b for b, _ in terms] if z % self.o.S)
        return sorted({self.o.galois(z) for z in zs})

    def encrypt_inputs(self, plan: SL.Plan, A, B, seed: int = 1, streams=(0, 1)):
        o = self.o
        ctA = o.encrypt(o.encode(plan.a_layout(A) % o.t), seed, streams[0])
        ctB = o.encrypt(o.encode(plan.b_layout(B) % o.t), seed, streams[1])
        return ctA, ctB

    def encrypt_pair(self, plan: SL.Plan, A0, B0, A1, B1, seed: int = 1, streams=(0, 1)):
        """Two products of one plan in one ciphertext pair: the first in
        slot row 0, the second in slot row 1."""
        o = self.o
        ctA = o.encrypt(o.encode(plan.a_layout(A0) % o.t, plan.a_layout(A1) % o.t), seed, streams[0])
        ctB = o.encrypt(o.encode(plan.b_layout(B0) % o.t, plan.b_layout(B1) % o.t), seed, streams[1])
        return ctA, ctB

    def mask_eval_pq(self, dsts: List[int], scale: int, lv: int) -> np.ndarray:
        key = ("pq", tuple(dsts), scale, lv)
        if key not in self._mask_cache:
            v = np.zeros(self.o.S, dtype=np.int64)
            v[dsts] = scale
            self._mask_cache[key] = self.o.plaintext_eval_pq(self.o.encode(v, v), lv)
        return self._mask_cache[key]

    def lt_double(self, ct: np.ndarray, terms: List[Tuple[int, List[int]]], scale: int) -> np.ndarray:
        """Eq. lintrans with one ModUp of c1 and one ModDown per component:
        y = ModDown(sum_d m_d (.) v_d) over PQ, v_0 = P ct and, for d != 0,
        v_d = (u0_d + P tau_d(c0), u1_d) with u_d the inner product of the
        hoisted key switch of tau_d(c1).  terms: [(d, destination slots)]."""
        o = self.o
        lv = ct.shape[1]
        acc = np.zeros((2, lv + o.K, o.N), dtype=np.uint64)
        D = o.modup(ct[1])
        for d, dst in terms:
            m = self.mask_eval_pq(dst, scale, lv)
            if d % o.S == 0:
                v = [o.pq_lift(ct[0]), o.pq_lift(ct[1])]
            else:
                g = o.galois(d)
                u = o.ks_raw(D, g)
                v = [o.pq_add(u[0], o.pq_lift(o.automorph(ct[0], g, list(range(lv))))), u[1]]
            for comp in range(2):
                o.pq_mac(acc[comp], v[comp], m)
        return o.moddown_pair(acc)

    def rot(self, ct: np.ndarray, z: int) -> np.ndarray:
        """HE-Rot under the executor's key policy."""
        return self.o.rotate_pow2(ct, z) if self.pow2 else self.o.rotate(ct, z)

    def lt_terms(self, ct: np.ndarray, terms: List[Tuple[int, List[int]]], scale: int) -> np.ndarray:
        """sum over terms (d, slots) of u (.) Rot(ct, d), in the given order."""
        if self.mode == "double" and not self.pow2:
            return self.lt_double(ct, terms, scale)
        lv = ct.shape[1]
        acc = None
        for d, dst in terms:
            r = self.rot(ct, d)
            term = self.o.cmult(r, self.mask_eval(dst, scale, lv))
            acc = term if acc is None else self.o.add(acc, term)
        return acc

    def lt(self, ct: np.ndarray, diags: Dict[int, List[int]], scale: int) -> np.ndarray:
        """sum_d u_d (.) Rot(ct, d), diagonals in ascending d (Eq. lintrans)."""
        return self.lt_terms(ct, [(d, diags[d]) for d in sorted(diags)], scale)

    def lt_giant(self, ct: np.ndarray, fact: Tuple[int, List[Tuple[int, List[int]]]], scale: int) -> np.ndarray:
        """Rot(sum_b u'_b (.) Rot(ct, b), g) for one factored transformation."""
        g, terms = fact
        inner = self.lt_terms(ct, terms, scale)
        return self.rot(inner, g) if g % self.o.S else inner

    def run(self, plan: SL.Plan, ctA: np.ndarray, ctB: np.ndarray) -> np.ndarray:
        o = self.o
        for g in self.galois_needed(plan):
            o.add_galois_key(g)
        scale = mask_scale(o)
        C = None
        acc = None
        dsum = None
        if self.giant:
            fa = SL.giant_factor([e for e, _ in plan.iters], o.S, self.giant_cost)
            fb = SL.giant_factor([om for _, om in plan.iters], o.S, self.giant_cost)
        for k, (e, om) in enumerate(plan.iters):
            if self.giant:
                a = self.lt_giant(ctA, fa[k], scale)
                b = self.lt_giant(ctB, fb[k], scale)
            else:
                a = self.lt(ctA, e, scale)
                b = self.lt(ctB, om, scale)
            for _ in range(o.pre.ms_drop):
                a = o.modswitch(a)
                b = o.modswitch(b)
            if self.lazy_relin:
                if getattr(o, "bfv", False):
                    # BFV: the exact tensors are summed and scaled once
                    d = o.tensor_exact(a, b)
                    dsum = d if dsum is None else dsum + d
                    continue
                d = o.tensor(a, b)
                dsum = d if dsum is None else o.add(dsum, d)
                continue
            if self.mode == "double":
                # HE-Mult without its ModDown, summed over PQ (Eq. of C)
                d = o.tensor(a, b)
                u = o.ks_raw(o.modup(d[2]), 0)
                v = np.stack([o.pq_add(u[0], o.pq_lift(d[0])), o.pq_add(u[1], o.pq_lift(d[1]))])
                acc = v if acc is None else np.stack([o.pq_add(acc[0], v[0]), o.pq_add(acc[1], v[1])])
                continue
            prod = o.mult_relin(a, b)
            C = prod if C is None else o.add(C, prod)
        if self.lazy_relin:
            if getattr(o, "bfv", False):
                dsum = o.scale_round(dsum)
            # one relinearisation of the summed tensor (Eq. elementwise's
            # sum taken before the key switch)
            if self.mode == "double":
                u = o.ks_raw(o.modup(dsum[2]), 0)
                acc = np.stack([o.pq_add(u[0], o.pq_lift(dsum[0])), o.pq_add(u[1], o.pq_lift(dsum[1]))])
            else:
                C = o.add(np.ascontiguousarray(dsum[:2]), o.keyswitch(dsum[2], 0))
        if self.mode == "double":
            C = o.moddown_pair(acc)
            if not plan.extract:
                return C
            if self.pow2:
                out = C
                for z in plan.extract:
                    out = o.add(out, self.rot(C, z))
                return out
            lv = C.shape[1]
            D = o.modup(C[1])
            ex = None
            for z in plan.extract:
                if z % o.S == 0:
                    v = np.stack([o.pq_lift(C[0]), o.pq_lift(C[1])])
                else:
                    g = o.galois(z)
                    u = o.ks_raw(D, g)
                    v = np.stack([o.pq_add(u[0], o.pq_lift(o.automorph(C[0], g, list(range(lv))))), u[1]])
                ex = v if ex is None else np.stack([o.pq_add(ex[0], v[0]), o.pq_add(ex[1], v[1])])
            return o.add(C, o.moddown_pair(ex))
        out = C
        for z in plan.extract:
            out = o.add(out, self.rot(C, z))
        return out

    def lintrans(self, ct: np.ndarray, src: List[int]) -> np.ndarray:
        """Eq. lintrans on a ciphertext, composed of the HE operations of
        Section 2.1 whatever the mode: the sum over diagonals d (ascending)
        of HE-CMult(HE-Rot(ct, d), u_d); slot j of the result takes slot
        src[j] of ct (negative: zero)."""
        diags = SL.diagonals_of_map({j: s for j, s in enumerate(src) if s >= 0})
        acc = np.zeros_like(ct)
        for d in sorted(diags):
            term = self.o.cmult(self.o.rotate(ct, d), self.mask_eval(diags[d], 1, ct.shape[1]))
            acc = self.o.add(acc, term)
        return acc

    def to_layout(self, ct: np.ndarray, role: int, m: int, l: int, n: int, alg: int) -> np.ndarray:
        """sigma(A) / tau(B) (and Algorithm 2's operand layout) under
        encryption, from a plain column-major matrix ciphertext (Section
        3.2.2 counts these transformations' HE operations)."""
        return self.lintrans(ct, SL.layout_source(role, m, l, n, alg))

    def from_result(self, ct: np.ndarray, m: int, l: int, n: int, alg: int) -> np.ndarray:
        """A product's result as a plain column-major m x n matrix ciphertext."""
        return self.lintrans(ct, SL.result_source(m, l, n, alg))

    def chain_operand(self, ct: np.ndarray, m: int, l: int, n: int, alg: int, role: int, m2: int, l2: int, n2: int,
                      alg2: int) -> np.ndarray:
        """The result of product (m, l, n, alg) as operand ``role`` of product
        (m2, l2, n2, alg2), in one transformation: the operand layout's map
        from the plain matrix composed with the result's map into it."""
        assert (m2, l2) == (m, n) if role == 0 else (l2, n2) == (m, n)
        res = SL.result_source(m, l, n, alg)
        return self.lintrans(ct, [res[s] if s >= 0 else -1 for s in SL.layout_source(role, m2, l2, n2, alg2)])

    def sum_products(self, items: List[Tuple[SL.Plan, np.ndarray, np.ndarray]]) -> np.ndarray:
        """The HE-Add (Section 2.1) of the results of products that share a
        result layout, in list order: the block sum C_ij = sum_k A_ik B_kj of
        Section 4.4.  items: [(plan, ctA, ctB)]."""
        if len({SL.result_layout(p) for p, _, _ in items}) != 1:
            raise ValueError("products of one sum have different result layouts")
        acc = None
        for plan, a, b in items:
            c = self.run(plan, a, b)
            acc = c if acc is None else self.o.add(acc, c)
        return acc

    def blocked(self, rows: List[int], inner: List[int], cols: List[int], ctA, ctB):
        """Blocked product of Section 4.4 under Algorithm 1: ctA[i][k] and
        ctB[k][j] encrypt the Algorithm 1 layouts of blocks A_ik and B_kj;
        returns C[i][j] = sum over k (ascending) of the products A_ik B_kj."""
        return [[self.sum_products([(SL.make_plan(rows[i], inner[k], cols[j], 1), ctA[i][k], ctB[k][j])
                                    for k in range(len(inner))])
                 for j in range(len(cols))] for i in range(len(rows))]

    def result_pair(self, plan: SL.Plan, ct: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
        """The products of slot rows 0 and 1."""
        rows = self.o.decrypt_rows(ct)
        out = []
        for r in rows:
            Cm = np.zeros((plan.m, plan.n), dtype=np.int64)
            for i in range(plan.m):
                for j in range(plan.n):
                    Cm[i, j] = r[plan.result_slot(i, j)]
            out.append(Cm)
        return out[0], out[1]

    def result(self, plan: SL.Plan, ct: np.ndarray) -> np.ndarray:
        slots = self.o.decrypt_slots(ct)
        Cm = np.zeros((plan.m, plan.n), dtype=np.int64)
        for i in range(plan.m):
            for j in range(plan.n):
                Cm[i, j] = slots[plan.result_slot(i, j)]
        return Cm

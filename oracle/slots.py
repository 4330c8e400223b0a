"""Slot-level model of HEGMM: transforms, diagonals and both algorithms.

Test infrastructure (see ``oracle/__init__.py``): nothing in the product
imports this module.

Everything here works on plaintext integer vectors; a ciphertext rotation is
modelled as a cyclic left shift of the slot vector (``Rot(x, z)_i =
x_{i+z}``, Section 2.1).  The ciphertext-level executor in ``oracle.he``
consumes the plans built here.

Paper references (arXiv 2405.02238):
* Eqs. def:sigma, def:tau, def:eps, def:omega (Section 3.1) -- the four
  matrix transforms.
* Eq. elementwise (Section 3.1) -- A.B = sum_k eps^k(sigma A) (.) omega^k(tau B).
* Eq. lintrans and the diagonal vectors u_z (Section 3.2.1).
* Eqs. Usigma, Utau, Uepsc, Uomgc (Section 3.2.1) -- column-major U matrices.
* Theorems 1-4 (Section 3.2.1) -- diagonal-count bounds.
* Algorithm 1 (HEGMM) and Algorithm 2 (HEGMM-Enhanced), Theorems 5-6
  (Section 3.3).
* Section 4.4 and Table 4 -- blocking: a product too large for one
  ciphertext is split into blocks, C_ij = sum_k A_ik B_kj, each block
  product one HEGMM product and the sum over k one HE-Add per term.

Readings of points the paper leaves open (each also listed in the design
notes):
* Rotations are cyclic within one row of S = N/2 slots; the zero-padded
  diagonals of Eq. lintrans make the wrap point irrelevant while every vector
  fits in S slots.  A negative offset z is a left rotation by S + z.
* Algorithm 1 flattens column-major by default (the order the paper's U
  matrices are printed for); row-major is an option.
* Algorithm 2 checks p = m first, then p = n, else the l-case (t = 1).
* Algorithm 2's initial ``C <- sA (.) tB`` is read as ``C <- 0``: the loop
  starts at k = 0, so a literal reading counts the k = 0 term twice.
* Algorithm 2's eps^k_{MxN}(ct.sA) reads destination column j from the stored
  (column-duplicated) layout at the column c = j + k - l*r with the smallest
  r >= 0 that keeps c inside the stored width; omega^k likewise on rows.
* Algorithm 2's "if not yet accumulated" is a first-occurrence keep mask over
  (k ascending, block h ascending), folded into the eps^k diagonal masks; the
  t copies are then summed by rotations of h*p slots after the loop.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Dict, List, Optional, Tuple

import numpy as np

# --------------------------------------------------------------------------
# The four transforms, as written in Eqs. def:sigma .. def:omega.
# --------------------------------------------------------------------------


def sigma(A: np.ndarray) -> np.ndarray:
    """sigma(A)_{i,j} = A_{i,[i+j]_l}  (Eq. def:sigma): row i rotated left by i."""
    m, l = A.shape
    out = np.empty_like(A)
    for i in range(m):
        for j in range(l):
            out[i, j] = A[i, (i + j) % l]
    return out


def tau(B: np.ndarray) -> np.ndarray:
    """tau(B)_{i,j} = B_{[i+j]_l,j}  (Eq. def:tau): column j rotated up by j."""
    l, n = B.shape
    out = np.empty_like(B)
    for i in range(l):
        for j in range(n):
            out[i, j] = B[(i + j) % l, j]
    return out


def eps(A: np.ndarray, k: int, rows: int, cols: int) -> np.ndarray:
    """eps^k_{rows x cols}(A)_{i,j} = A_{i,[j+k]_l}  (Eq. def:eps), l = A's width."""
    l = A.shape[1]
    out = np.empty((rows, cols), dtype=A.dtype)
    for i in range(rows):
        for j in range(cols):
            out[i, j] = A[i, (j + k) % l]
    return out


def omega(B: np.ndarray, k: int, rows: int, cols: int) -> np.ndarray:
    """omega^k_{rows x cols}(B)_{i,j} = B_{[i+k]_l,j}  (Eq. def:omega), l = B's height."""
    l = B.shape[0]
    out = np.empty((rows, cols), dtype=B.dtype)
    for i in range(rows):
        for j in range(cols):
            out[i, j] = B[(i + k) % l, j]
    return out


def elementwise_product(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Right-hand side of Eq. elementwise: sum_k eps^k(sigma A) (.) omega^k(tau B)."""
    m, l = A.shape
    n = B.shape[1]
    sA, tB = sigma(A), tau(B)
    C = np.zeros((m, n), dtype=np.int64)
    for k in range(l):
        C += eps(sA, k, m, n) * omega(tB, k, m, n)
    return C


# --------------------------------------------------------------------------
# Flattening, slot maps and diagonals (Eq. lintrans).
# --------------------------------------------------------------------------


def flat(i: int, j: int, rows: int, cols: int, order: str) -> int:
    """Slot of entry (i, j) of a rows x cols matrix flattened in ``order``."""
    if order == "col":
        return i + j * rows
    if order == "row":
        return i * cols + j
    raise ValueError(order)


def flatten(M: np.ndarray, order: str) -> np.ndarray:
    rows, cols = M.shape
    v = np.zeros(rows * cols, dtype=M.dtype)
    for i in range(rows):
        for j in range(cols):
            v[flat(i, j, rows, cols, order)] = M[i, j]
    return v


SrcFn = Callable[[int, int], Optional[Tuple[int, int]]]


def slot_map(dst_shape, src_shape, order: str, src_of: SrcFn) -> Dict[int, int]:
    """dst slot -> src slot for a transform Y[i,j] = X[src_of(i,j)].

    ``src_of`` returning None leaves that destination at zero.
    """
    rd, cd = dst_shape
    rs, cs = src_shape
    out = {}
    for i in range(rd):
        for j in range(cd):
            s = src_of(i, j)
            if s is None:
                continue
            out[flat(i, j, rd, cd, order)] = flat(s[0], s[1], rs, cs, order)
    return out


def u_matrix(dst_shape, src_shape, order: str, src_of: SrcFn) -> np.ndarray:
    """Dense 0/1 transformation matrix U with U . flatten(X) = flatten(Y)."""
    y = dst_shape[0] * dst_shape[1]
    x = src_shape[0] * src_shape[1]
    U = np.zeros((y, x), dtype=np.int64)
    for dst, src in slot_map(dst_shape, src_shape, order, src_of).items():
        U[dst, src] = 1
    return U


def diagonals_of_matrix(U: np.ndarray) -> Dict[int, np.ndarray]:
    """Non-zero diagonal vectors u_z of U (Eq. lintrans), -y <= z < x.

    u_z[i] = U[i, i+z] where 0 <= i+z < x, and 0 elsewhere; only diagonals
    with a non-zero entry are returned.
    """
    y, x = U.shape
    out = {}
    for z in range(-y, x):
        u = np.zeros(y, dtype=np.int64)
        for i in range(y):
            if 0 <= i + z < x:
                u[i] = U[i, i + z]
        if u.any():
            out[z] = u
    return out


def diagonals_of_map(smap: Dict[int, int]) -> Dict[int, List[int]]:
    """Group a slot map by offset d = src - dst: {d: [dst slots]}."""
    out: Dict[int, List[int]] = {}
    for dst, src in smap.items():
        out.setdefault(src - dst, []).append(dst)
    for d in out:
        out[d].sort()
    return out


def apply_lt(x: np.ndarray, diags: Dict[int, List[int]], S: int, mod: int, scale: int = 1) -> np.ndarray:
    """sum_d u_d (.) Rot(x, d) on an S-slot vector (Eq. lintrans), mod ``mod``.

    Rot(x, d)_i = x_{(i+d) mod S}; u_d is ``scale`` on the listed slots.
    """
    y = np.zeros(S, dtype=np.int64)
    for d in sorted(diags):
        mask = np.zeros(S, dtype=np.int64)
        mask[diags[d]] = scale
        y = (y + mask * np.roll(x, -d)) % mod
    return y


# Source maps of the four transforms, used both for the U matrices and for
# the algorithms' linear transformations.


def sigma_src(l: int) -> SrcFn:
    return lambda i, j: (i, (i + j) % l)


def tau_src(l: int) -> SrcFn:
    return lambda i, j: ((i + j) % l, j)


def eps_src(k: int, l: int) -> SrcFn:
    return lambda i, j: (i, (j + k) % l)


def omega_src(k: int, l: int) -> SrcFn:
    return lambda i, j: ((i + k) % l, j)


def count_diagonals(dst_shape, src_shape, order, src_of) -> int:
    return len(diagonals_of_map(slot_map(dst_shape, src_shape, order, src_of)))


# --------------------------------------------------------------------------
# Plans: the sequence of linear transformations of Algorithms 1 and 2.
# --------------------------------------------------------------------------


@dataclasses.dataclass
class Plan:
    """A slot-level program for one product A (m x l) . B (l x n).

    * ``a_layout(A)`` / ``b_layout(B)``: client-side plaintext slot vectors
      (sigma/tau and, for Algorithm 2, duplication and eps^0/omega^0).
    * ``iters[k] = (eps_diags, omg_diags)``: diagonals {d: dst slots} of the
      two linear transformations of iteration k.
    * ``extract``: rotation offsets h*p (h = 1..t-1) summed onto the
      accumulator after the loop (Algorithm 2 only).
    * ``result_slot(i, j)``: slot of C_{i,j} in the decrypted result.
    """

    m: int
    l: int
    n: int
    alg: int
    case: str
    order: str
    p: int
    t: int
    M: int
    Np: int
    a_shape: Tuple[int, int]
    b_shape: Tuple[int, int]
    a_matrix: Callable[[np.ndarray], np.ndarray]
    b_matrix: Callable[[np.ndarray], np.ndarray]
    iters: List[Tuple[Dict[int, List[int]], Dict[int, List[int]]]]
    extract: List[int]
    res_shape: Tuple[int, int]
    length: int

    def a_layout(self, A: np.ndarray) -> np.ndarray:
        return flatten(self.a_matrix(A), self.order)

    def b_layout(self, B: np.ndarray) -> np.ndarray:
        return flatten(self.b_matrix(B), self.order)

    def result_slot(self, i: int, j: int) -> int:
        return flat(i, j, self.res_shape[0], self.res_shape[1], self.order)

    # Operation counts in the paper's terms: every non-zero offset of every
    # linear transformation is one HE-Rot, every diagonal one HE-CMult.
    def counts(self) -> Dict[str, int]:
        rot = sum(sum(1 for d in e if d != 0) + sum(1 for d in o if d != 0) for e, o in self.iters)
        cm = sum(len(e) + len(o) for e, o in self.iters)
        rot += len(self.extract)
        return {
            "rot": rot,
            "cmult": cm,
            "mult": len(self.iters),
            "relin": len(self.iters),
            "ksw": rot + len(self.iters),
            "extract": len(self.extract),
        }


# --------------------------------------------------------------------------
# Shared baby steps: an evaluation order of Eq. lintrans across iterations.
# --------------------------------------------------------------------------

# Cost of one giant rotation (its own ModUp, key switch and ModDowns) in units
# of one baby key switch (a key read); a constant of the evaluation mode.
GIANT_COST = 8


def giant_factor(outputs: List[Dict[int, List[int]]], S: int,
                 cost: int = GIANT_COST) -> List[Tuple[int, List[Tuple[int, List[int]]]]]:
    """Rewrites each linear transformation of one operand (Eq. lintrans),
    in execution order, as a rotation of a sum over shared offsets:

        sum_d u_d (.) Rot(x, d) = Rot( sum_d u'_d (.) Rot(x, b_d), g ),
        b_d = (d - g) mod S,  u'_d = Rot(u_d, -g)  (destination slots + g),

    which holds for cyclic rotations of an S-slot row.  The rotations
    Rot(x, b) are shared by every transformation of the operand, so a
    transformation whose offsets are a shift of offsets already used costs
    one giant rotation instead of its own key switches.

    Greedy rule, per transformation in order, with B the non-zero offsets
    key-switched so far: over g = 0 and every (z - b) mod S (z an offset of
    the transformation mod S, b in B or 0), minimise
        cost(g) = #{distinct (z - g) mod S not in B and != 0} + (cost if g != 0),
    ties to the smaller g in [0, S); then B gains the new offsets.

    Returns per transformation (g, terms) with terms [(b_d, destination
    slots of u'_d)] in the order of the original diagonals (ascending d).
    """
    baby: set = set()
    out = []
    for diags in outputs:
        Z = sorted({d % S for d in diags})
        hits: Dict[int, int] = {}
        for z in Z:
            for b in [0] + sorted(baby):
                g = (z - b) % S
                hits[g] = hits.get(g, 0) + 1
        best_g, best_c = 0, len(Z) - hits.get(0, 0)
        for g in sorted(hits):
            if g == 0:
                continue
            c = len(Z) - hits[g] + cost
            if c < best_c:
                best_g, best_c = g, c
        g = best_g
        terms = []
        for d in sorted(diags):
            b = (d - g) % S
            terms.append((b, sorted((t + g) % S for t in diags[d])))
            if b:
                baby.add(b)
        out.append((g, terms))
    return out


def naf(z: int) -> List[Tuple[int, int]]:
    """Non-adjacent form of an integer z: [(sign, i)] with z = sum sign 2^i,
    signs +-1, no two consecutive positions i, ascending i (least
    significant first).  The standard recoding: while z != 0, an odd z takes
    the digit 2 - (z mod 4), which leaves z - digit divisible by 4."""
    out = []
    i = 0
    while z:
        if z & 1:
            d = 2 - (z % 4)
            out.append((d, i))
            z -= d
        z //= 2
        i += 1
    return out


def pow2_steps(z: int, S: int) -> List[int]:
    """The power-of-two key policy's decomposition of a left rotation by z
    over S slots: the signed powers of two d 2^i of the NAF of z mod S or of
    (z mod S) - S (the same rotation), whichever has fewer digits (ties: the
    non-negative one), in ascending i.  Rot(x, z) is the chain of HE-Rot by
    these steps."""
    a = z % S
    fa, fb = naf(a), naf(a - S)
    best = fb if len(fb) < len(fa) else fa
    return [d * (1 << i) for d, i in best]


def pow2_offsets(S: int) -> List[int]:
    """Every rotation step the power-of-two policy can use (its keys):
    +-2^i for 2^i < S, as left-rotation offsets mod S."""
    out = set()
    i = 0
    while (1 << i) < S:
        out.add((1 << i) % S)
        out.add((-(1 << i)) % S)
        i += 1
    return sorted(out)


def apply_terms(x: np.ndarray, terms: List[Tuple[int, List[int]]], S: int, mod: int, scale: int = 1) -> np.ndarray:
    """sum over (b, slots) of u (.) Rot(x, b), u = scale on the slots."""
    y = np.zeros(S, dtype=np.int64)
    for b, dst in terms:
        mask = np.zeros(S, dtype=np.int64)
        mask[dst] = scale
        y = (y + mask * np.roll(x, -b)) % mod
    return y


def plan_alg1(m: int, l: int, n: int, order: str = "col") -> Plan:
    """Algorithm 1: sigma/tau on the client, then l iterations of eps^k, omega^k."""
    iters = []
    for k in range(l):
        e = diagonals_of_map(slot_map((m, n), (m, l), order, eps_src(k, l)))
        o = diagonals_of_map(slot_map((m, n), (l, n), order, omega_src(k, l)))
        iters.append((e, o))
    return Plan(
        m=m, l=l, n=n, alg=1, case="1", order=order, p=l, t=1, M=m, Np=n,
        a_shape=(m, l), b_shape=(l, n), a_matrix=sigma, b_matrix=tau,
        iters=iters, extract=[], res_shape=(m, n), length=max(m * l, l * n, m * n),
    )


def plan_alg1x(m: int, l: int, n: int) -> Plan:
    """Algorithm 1 with an extended pre-layout (a cost-reducing mode, not in
    the paper): sigma(A) is stored over W = l + n - 1 columns, column c
    holding sigma(A)'s column c mod l.  eps^k_{m x n}(sigma(A))_{i,j} =
    sigma(A)_{i,[j+k]_l} (Eq. def:eps) is then the stored entry (i, j + k),
    so in column-major order every eps^k is one rotation by k m under one
    mask; omega^k, the loop and the result layout are Algorithm 1's."""
    W = l + n - 1

    def a_matrix(A):
        return sigma(A)[:, [c % l for c in range(W)]]

    iters = []
    for k in range(l):
        e = diagonals_of_map(slot_map((m, n), (m, W), "col", lambda i, j, k=k: (i, j + k)))
        o = diagonals_of_map(slot_map((m, n), (l, n), "col", omega_src(k, l)))
        iters.append((e, o))
    return Plan(
        m=m, l=l, n=n, alg=3, case="X", order="col", p=l, t=1, M=m, Np=n,
        a_shape=(m, W), b_shape=(l, n), a_matrix=a_matrix, b_matrix=tau,
        iters=iters, extract=[], res_shape=(m, n), length=max(m * W, l * n),
    )


def alg2_case(m: int, l: int, n: int) -> Tuple[str, int, int]:
    """(case, p, t) of Algorithm 2; p = m is checked first, then p = n."""
    p = min(m, l, n)
    if p == m:
        return "A", p, -(-l // p)
    if p == n:
        return "B", p, -(-l // p)
    return "L", p, 1


def alg2_dims(m: int, l: int, n: int):
    case, p, t = alg2_case(m, l, n)
    M = t * m if case == "A" else m
    Np = t * n if case == "B" else n
    WA = max(l, Np)  # stored width of eps^0_{M x max(l,N)}(sigma(Abar))
    HB = max(l, M)   # stored height of omega^0_{max(l,M) x N}(tau(Bbar))
    return case, p, t, M, Np, WA, HB


def alg2_length(m: int, l: int, n: int) -> int:
    _, _, _, M, Np, WA, HB = alg2_dims(m, l, n)
    return max(M * WA, HB * Np, M * Np)


def plan_alg2(m: int, l: int, n: int) -> Plan:
    """Algorithm 2 (HEGMM-Enhanced) with the readings listed in the module doc."""
    case, p, t, M, Np, WA, HB = alg2_dims(m, l, n)
    order = "row" if case == "B" else "col"

    def a_matrix(A):
        Abar = np.vstack([A] * t) if case == "A" else A
        return eps(sigma(Abar), 0, M, WA)

    def b_matrix(B):
        Bbar = np.hstack([B] * t) if case == "B" else B
        return omega(tau(Bbar), 0, HB, Np)

    seen = set()
    iters = []
    for k in range(p):
        keep = []
        for h in range(t):
            ph = (k + h * p) % l
            keep.append(ph not in seen)
            seen.add(ph)

        def kept(i, j, keep=keep):
            if case == "A":
                return keep[i // m]
            if case == "B":
                return keep[j // n]
            return True

        def e_src(i, j, k=k, kept=kept):
            if not kept(i, j):
                return None
            c = j + k
            while c >= WA:
                c -= l
            return (i, c)

        def o_src(i, j, k=k):
            r = i + k
            while r >= HB:
                r -= l
            return (r, j)

        e = diagonals_of_map(slot_map((M, Np), (M, WA), order, e_src))
        o = diagonals_of_map(slot_map((M, Np), (HB, Np), order, o_src))
        iters.append((e, o))
    extract = [h * p for h in range(1, t)]
    return Plan(
        m=m, l=l, n=n, alg=2, case=case, order=order, p=p, t=t, M=M, Np=Np,
        a_shape=(M, WA), b_shape=(HB, Np), a_matrix=a_matrix, b_matrix=b_matrix,
        iters=iters, extract=extract, res_shape=(M, Np),
        length=max(M * WA, HB * Np, M * Np),
    )


def fits(m: int, l: int, n: int, alg: int, S: int) -> bool:
    if alg == 1:
        return max(m * l, l * n, m * n) <= S
    if alg == 3:
        return max(m * (l + n - 1), l * n) <= S
    return alg2_length(m, l, n) <= S


def choose_alg(m: int, l: int, n: int, S: int) -> int:
    """AUTO: Algorithm 2 when it fits S slots, else Algorithm 1 (Section 3.3), else 0."""
    if fits(m, l, n, 2, S):
        return 2
    if fits(m, l, n, 1, S):
        return 1
    return 0


def make_plan(m: int, l: int, n: int, alg: int, order: str = "col") -> Plan:
    if alg == 3:
        return plan_alg1x(m, l, n)
    return plan_alg1(m, l, n, order) if alg == 1 else plan_alg2(m, l, n)


def run_slots(plan: Plan, A: np.ndarray, B: np.ndarray, S: int, t: int) -> np.ndarray:
    """Execute a plan on plaintext slot vectors (rotation = cyclic shift).

    Returns the m x n result read from the result slots, mod t.
    """
    a = np.zeros(S, dtype=np.int64)
    b = np.zeros(S, dtype=np.int64)
    va, vb = plan.a_layout(A) % t, plan.b_layout(B) % t
    a[: len(va)] = va
    b[: len(vb)] = vb
    acc = np.zeros(S, dtype=np.int64)
    for e, o in plan.iters:
        x = apply_lt(a, e, S, t)
        y = apply_lt(b, o, S, t)
        acc = (acc + x * y) % t
    out = acc.copy()
    for z in plan.extract:
        out = (out + np.roll(acc, -z)) % t
    C = np.zeros((plan.m, plan.n), dtype=np.int64)
    for i in range(plan.m):
        for j in range(plan.n):
            C[i, j] = out[plan.result_slot(i, j)]
    return C


def layout_source(role: int, m: int, l: int, n: int, alg: int) -> List[int]:
    """The operand layout of a product (m, l, n, alg) as a slot map from the
    plain column-major matrix (A: m x l for role 0, B: l x n for role 1; slot
    i + j rows holds M_ij): for every destination slot the plain slot it
    copies, -1 for zero.  sigma / tau (Section 3.1) and, for Algorithm 2, the
    duplication and eps^0 / omega^0 only move entries, so an index matrix
    (entry = its plain slot + 1) carried through the layout names them."""
    plan = make_plan(m, l, n, alg)
    rows, cols = (m, l) if role == 0 else (l, n)
    idx = 1 + (np.arange(rows)[:, None] + np.arange(cols)[None, :] * rows)
    v = plan.a_layout(idx) if role == 0 else plan.b_layout(idx)
    return [int(x) - 1 for x in v]


def result_source(m: int, l: int, n: int, alg: int) -> List[int]:
    """The result of a product as a slot map into the plain column-major
    m x n matrix: destination i + j m takes the result slot of C_ij."""
    plan = make_plan(m, l, n, alg)
    src = [-1] * (m * n)
    for i in range(m):
        for j in range(n):
            src[i + j * m] = plan.result_slot(i, j)
    return src


def block_bounds(sizes: List[int]) -> List[Tuple[int, int]]:
    """[start, stop) of consecutive blocks of the given sizes (Section 4.4)."""
    out, s = [], 0
    for b in sizes:
        out.append((s, s + b))
        s += b
    return out


def result_layout(plan: Plan) -> Tuple[int, int, str]:
    """What decides where C_ij sits: the result shape and the flattening order."""
    return plan.res_shape[0], plan.res_shape[1], plan.order


def run_blocked_slots(rows: List[int], inner: List[int], cols: List[int], A: np.ndarray, B: np.ndarray,
                      S: int, t: int, alg: int = 1) -> np.ndarray:
    """The blocked product of Section 4.4 on slot vectors: for every output
    block (i, j) the slot vectors of the products A_ik B_kj (k ascending) are
    added slot by slot, then C_ij is read from the common result slots.
    Every product of a block must share the result layout (checked)."""
    rb, kb, cb = block_bounds(rows), block_bounds(inner), block_bounds(cols)
    assert A.shape == (rb[-1][1], kb[-1][1]) and B.shape == (kb[-1][1], cb[-1][1])
    C = np.zeros((rb[-1][1], cb[-1][1]), dtype=np.int64)
    for (r0, r1) in rb:
        for (c0, c1) in cb:
            acc, lay, ref = np.zeros(S, dtype=np.int64), None, None
            for (k0, k1) in kb:
                plan = make_plan(r1 - r0, k1 - k0, c1 - c0, alg)
                if lay is None:
                    lay, ref = result_layout(plan), plan
                elif result_layout(plan) != lay:
                    raise ValueError("block products of one output block have different result layouts")
                acc = (acc + slot_vector(plan, A[r0:r1, k0:k1], B[k0:k1, c0:c1], S, t)) % t
            for i in range(r1 - r0):
                for j in range(c1 - c0):
                    C[r0 + i, c0 + j] = acc[ref.result_slot(i, j)]
    return C


def slot_vector(plan: Plan, A: np.ndarray, B: np.ndarray, S: int, t: int) -> np.ndarray:
    """The whole result slot vector of ``run_slots`` (before reading C)."""
    a = np.zeros(S, dtype=np.int64)
    b = np.zeros(S, dtype=np.int64)
    va, vb = plan.a_layout(A) % t, plan.b_layout(B) % t
    a[: len(va)] = va
    b[: len(vb)] = vb
    acc = np.zeros(S, dtype=np.int64)
    for e, o in plan.iters:
        acc = (acc + apply_lt(a, e, S, t) * apply_lt(b, o, S, t)) % t
    out = acc.copy()
    for z in plan.extract:
        out = (out + np.roll(acc, -z)) % t
    return out


def theorem5_blocks(m: int, l: int, k: int, t: int) -> List[int]:
    """Partial-product indices p_h = [k + h m]_l held by block h (Theorem 5)."""
    return [(k + h * m) % l for h in range(t)]

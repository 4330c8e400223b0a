/*
 * hegmm.h -- C ABI of the GB300 (sm_103a) HEGMM library.
 *
 * HEGMM (arXiv 2405.02238) multiplies an encrypted m x l matrix A by an
 * encrypted l x n matrix B.  Each matrix is packed into the slots of one
 * ciphertext; the cloud computes
 *     A.B = sum_k eps^k(sigma(A)) (.) omega^k(tau(B))        (Eq. elementwise)
 * where each transform is a linear transformation evaluated by rotations and
 * plaintext-mask products, sum_z u_z (.) Rot(x; z)            (Eq. lintrans),
 * sequenced as Algorithm 1 (HEGMM, l iterations) or Algorithm 2
 * (HEGMM-Enhanced, min(m,l,n) iterations plus t-1 extraction rotations).
 * The HE operations of Section 2.1 (HE-Add, HE-Mult, HE-CMult, HE-Rot) are
 * realised as RNS-BGV over Z_Q[X]/(X^N+1): negacyclic NTTs, Galois
 * automorphisms with hybrid key switching (ModUp, key inner product,
 * ModDown), mask products and tensoring with relinearisation.
 *
 * Conventions shared by every entry point:
 *  - Return value: 0 (HEGMM_OK) or a negative HEGMM_E* code; after an error
 *    hegmm_last_error(ctx) returns a message.  No entry point aborts the
 *    process; a CUDA error is reported as HEGMM_ECUDA.
 *  - Every call is ordered on the context's CUDA stream (the stream handle
 *    given to hegmm_ctx_create, e.g. a PyTorch stream).  Calls that return
 *    host data (decrypt, export) synchronise that stream.
 *  - Handles (hegmm_ctx, hegmm_pt, hegmm_ct) and their device memory are
 *    owned by the library and released by the matching *_destroy call.
 *    Host arrays passed in are owned by the caller and only read during the
 *    call; host output arrays are owned by the caller and must be large
 *    enough for the sizes stated at each function.
 *  - Slots: a ciphertext holds two rows of S = N/2 slots; rotations are
 *    cyclic within a row.  Matrices use row 0.  Plaintext values are
 *    integers mod t (the plaintext modulus, a prime with t = 1 mod 2N).
 *  - Ciphertexts on the device are [2][level][N] uint64 residues in the
 *    NTT domain.  Exported / imported host ciphertexts are [2][level][N]
 *    uint64 in the coefficient domain, component 0 then 1, chain prime i
 *    at index i, residues in [0, q_i).
 */
#ifndef HEGMM_H
#define HEGMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HEGMM_OK 0
#define HEGMM_EINVAL (-1)   /* bad argument or parameter set */
#define HEGMM_ENOMEM (-2)   /* device or host allocation failed */
#define HEGMM_ESHAPE (-3)   /* the product does not fit one slot row */
#define HEGMM_ENOKEY (-4)   /* a rotation has no Galois key */
#define HEGMM_ECUDA (-5)    /* a CUDA call failed */
#define HEGMM_ETIMEOUT (-6) /* a bounded device wait ran out */

#define HEGMM_ALG_AUTO 0 /* Algorithm 2 if it fits S slots, else Algorithm 1 */
#define HEGMM_ALG_1 1    /* Algorithm 1 (HEGMM) */
#define HEGMM_ALG_2 2    /* Algorithm 2 (HEGMM-Enhanced) */
/* Algorithm 1 with an extended pre-layout (not in the paper): sigma(A) is
 * stored over l + n - 1 columns, column c holding sigma(A)'s column c mod l,
 * so every eps^k is one rotation by k m under one mask (Algorithm 1 needs up
 * to two diagonals per eps^k); needs m (l + n - 1) <= S.  omega^k, the loop
 * and the result layout are Algorithm 1's.  Accepted wherever an algorithm
 * is (planner, encoding, keys, products, sums, the server, decryption,
 * transformations); AUTO never picks it. */
#define HEGMM_ALG_1X 3

#define HEGMM_ROLE_A 0
#define HEGMM_ROLE_B 1

typedef struct hegmm_ctx hegmm_ctx; /* parameters, tables, keys, plans, stream */
typedef struct hegmm_pt hegmm_pt;   /* device plaintext, NTT domain */
typedef struct hegmm_ct hegmm_ct;   /* device ciphertext [2][level][N], NTT domain */

/* Ring and modulus-chain parameters.  Chain primes q_0 > ... > q_{L-1} are
 * the L largest primes below 2^qbits with q = 1 mod 2N; the K special
 * primes are the next K such primes.  A key-switching digit is alpha
 * consecutive chain primes (dnum = L / alpha digits).  Errors are centred
 * binomial with parameter eta; the secret is ternary.  ms_drop chain primes
 * are removed by a modulus switch before every ciphertext product (0 or 1).
 * Limits: 10 <= logN <= 14, 2 <= L, 1 <= K, L + K <= 24, 20 <= qbits <= 56
 * (the NTTs reduce their values only when they leave a transform, which
 * needs 128 q < 2^63), alpha divides L, K >= alpha (so P >= every digit
 * modulus up to a bit), K <= 4, digits (L + K) - L <= 128.
 * scheme: HEGMM_SCHEME_BGV (0) or HEGMM_SCHEME_BFV (1), the paper's own
 * scheme (Section 4.1).  Under BFV the message is scaled instead of the
 * noise: c0 + c1 s = Delta m + e with Delta = floor(Q / t); switching keys
 * carry plain errors and ModDown rounds plainly; decryption is
 * round(t [c0 + c1 s]_Q / Q) mod t; HE-Mult extends both operands from Q to
 * an auxiliary base B of L + 2 more primes (the next ones below the special
 * primes), forms the tensor over Q u B and returns round(t/Q x tensor) (an
 * RNS computation of the nearest integer: a floating-point sum of at most L
 * fractions decides it, so it can differ from the exact nearest integer
 * only when t x tensor / Q lies within about L 2^-52 of a half-integer) before
 * relinearising; a lazy sum of tensors is formed over Q u B and rounded
 * once.  BFV needs ms_drop = 0 and 2 L + K + 3 <= 25. */
#define HEGMM_SCHEME_BGV 0
#define HEGMM_SCHEME_BFV 1
typedef struct {
    int logN;
    uint64_t t;
    int L;
    int qbits;
    int K;
    int alpha;
    int eta;
    int ms_drop;
    int scheme;
} hegmm_params;

/* Operation counts of one product.  rot/cmult/mult follow the paper's
 * counting (one HE-Rot per non-zero diagonal of every transform, one
 * HE-CMult per diagonal, one HE-Mult per iteration); ksw is the number of
 * key switches actually executed (rotations shared between iterations of
 * the same source ciphertext are computed once), modup the number of hoisted
 * ModUps. */
typedef struct {
    long long rot, cmult, add, mult, relin, extract, ksw, modup, modswitch;
} hegmm_opcount;

/* Creates a context: finds the primes, builds NTT and base-conversion
 * tables on the device.  cuda_stream is a cudaStream_t (NULL = legacy
 * default stream) on which every later call is ordered; the caller keeps it
 * alive until hegmm_ctx_destroy.  Errors: HEGMM_EINVAL for parameters
 * outside the limits, HEGMM_ENOMEM, HEGMM_ECUDA. */
int hegmm_ctx_create(const hegmm_params *params, void *cuda_stream, hegmm_ctx **out);
void hegmm_ctx_destroy(hegmm_ctx *ctx);
const char *hegmm_last_error(const hegmm_ctx *ctx);

/* Copies the L + K primes (chain then special) into out[L + K]. */
int hegmm_get_primes(const hegmm_ctx *ctx, uint64_t *out);

/* Key generation from one seed: ternary secret s, the relinearisation key
 * (s^2 -> s) and the Galois keys of every rotation that the plans of the
 * listed products need.  shapes_mln holds n_shapes triples (m, l, n); alg is
 * HEGMM_ALG_* and is resolved per shape.  A later call with the same seed
 * adds keys; a different seed replaces all keys.  Keys stay resident in
 * device memory.  Errors: HEGMM_ESHAPE if a shape fits no algorithm. */
int hegmm_keygen(hegmm_ctx *ctx, uint64_t seed, const int *shapes_mln, int n_shapes, int alg);

/* Key policy of products (the fallback to Algorithm 1 of Section 3.3 can
 * need thousands of distinct rotation offsets, one Galois key each: about
 * 7300 for 128 x 16 x 64 at N = 2^14, 10 MiB per key).
 *   HEGMM_KEYS_DIRECT (default): one key per rotation offset a plan uses.
 *   HEGMM_KEYS_POW2: only the keys of rotations by +-2^i (2^i < S, at most
 *     2 log2 S keys); every rotation of a product (the diagonals of each
 *     linear transformation, giant and extraction rotations) is the chain of
 *     HE-Rot by the signed powers of two of the non-adjacent form of its
 *     offset z mod S, or of the same rotation written z - S when that has
 *     fewer digits, least significant first (hegmm_plan_pow2_steps).  The
 *     chains of one operand share their common prefixes; a linear
 *     transformation is then the sum over its diagonals of the mask product
 *     of the chained rotation, in every key-switch mode (the double mode's
 *     lifted sum over PQ would divide back to the same value), and Algorithm
 *     2's extraction adds the chained rotations of C_acc.  Bit-exact with the
 *     oracle's key_policy "pow2".
 * Applies to hegmm_keygen and to products started after the call; with a
 * secret key the power-of-two keys are made at once.  The ciphertext-side
 * transformations (hegmm_lintrans ...) keep using direct keys.  Errors:
 * HEGMM_EINVAL. */
#define HEGMM_KEYS_DIRECT 0
#define HEGMM_KEYS_POW2 1
int hegmm_set_key_policy(hegmm_ctx *ctx, int policy);

/* Adds Galois keys for left rotations by z[0..count) (negative z rotates
 * right); requires a previous hegmm_keygen. */
int hegmm_keygen_rotations(hegmm_ctx *ctx, const int *z, int count);

/* Copies a key to the host in the coefficient domain, layout
 * [dnum][2][L+K][N] (component 0 = b_j, 1 = a_j).  which = 0 selects the
 * relinearisation key, otherwise which is a Galois element g (odd, < 2N).
 * Errors: HEGMM_ENOKEY. */
int hegmm_key_export(hegmm_ctx *ctx, uint64_t which, uint64_t *host);

/* Checkpoint / warm start of an evaluation context: hegmm_key_import loads a
 * key in hegmm_key_export's layout and domain (residues below their primes,
 * else HEGMM_EINVAL) under `which` (0: relinearisation, else an odd Galois
 * element < 2N); an existing key of that element is overwritten in place.
 * A context that only imports keys (no hegmm_keygen) evaluates products of
 * imported ciphertexts (hegmm_ct_import) but has no secret key: it cannot
 * encrypt, decrypt or make missing keys (HEGMM_ENOKEY).  hegmm_key_list
 * writes up to cap of the key elements held (ascending) and their number to
 * *count.  Synchronise the stream. */
int hegmm_key_import(hegmm_ctx *ctx, uint64_t which, const uint64_t *host);
int hegmm_key_list(hegmm_ctx *ctx, uint64_t *which, int cap, int *count);

/* Client-side preprocessing of a plaintext matrix (Algorithm 1 step 1,
 * Algorithm 2 lines 1-18): sigma (role A) or tau (role B), the duplication
 * and eps^0 / omega^0 of Algorithm 2, flattening in the plan's order, and
 * slot encoding.  mat is row-major (m x l for role A, l x n for role B),
 * entries taken mod t (negative values wrap).  *out is a new plaintext.
 * Errors: HEGMM_ESHAPE. */
int hegmm_encode(hegmm_ctx *ctx, int role, const int64_t *mat, int m, int l, int n, int alg, hegmm_pt **out);

/* Two products in one ciphertext pair.  The slots form two rows of S = N/2;
 * a rotation moves both rows alike and every mask of a product covers both
 * rows, so a product computes the row-0 and the row-1 products of its
 * operands at the cost of one.  hegmm_encode_pair lays mat0 out in row 0
 * and mat1 (NULL: zeros, the same plaintext as hegmm_encode) in row 1, as
 * hegmm_encode does for one matrix. */
int hegmm_encode_pair(hegmm_ctx *ctx, int role, const int64_t *mat0, const int64_t *mat1, int m, int l, int n, int alg,
                      hegmm_pt **out);

/* Encodes count <= N slot values (slots 0..S-1 of row 0, then row 1; the
 * rest zero) into a plaintext. */
int hegmm_encode_slots(hegmm_ctx *ctx, const uint64_t *slots, int count, hegmm_pt **out);

/* Secret-key encryption: c1 = a, c0 = -a s + t e + m, with a and e drawn
 * from the counter-mode SplitMix64 streams of (seed, stream_id). */
int hegmm_encrypt(hegmm_ctx *ctx, const hegmm_pt *pt, uint64_t seed, uint64_t stream_id, hegmm_ct **out);

/* The encrypted product C = A.B of an m x l and an l x n matrix (Algorithm 1
 * or 2 of the paper), on ciphertexts made by hegmm_encode + hegmm_encrypt
 * (or imported) for the same (m, l, n, alg).  *C is a new ciphertext; cnt
 * (may be NULL) receives the operation counts.  Errors: HEGMM_ESHAPE,
 * HEGMM_ENOKEY (keygen did not cover this shape), HEGMM_EINVAL (operand
 * level does not match). */
int hegmm_matmul(hegmm_ctx *ctx, const hegmm_ct *A, const hegmm_ct *B, int m, int l, int n, int alg,
                 hegmm_ct **C, hegmm_opcount *cnt);

/* count independent products in one call; mln holds count triples, A[i],
 * B[i] the operands, C[i] receives new ciphertexts.  Products are batched
 * into shared kernel launches.  On error no C[i] is returned. */
int hegmm_matmul_batch(hegmm_ctx *ctx, int count, const hegmm_ct *const *A, const hegmm_ct *const *B,
                       const int *mln, int alg, hegmm_ct **C);

/* How products (hegmm_matmul, hegmm_matmul_batch, the server) evaluate their
 * sums of key switches.  The results decrypt to the same matrix product.
 *   HEGMM_KS_SINGLE (default): every rotation and relinearisation ends in its own
 *     ModDown, as composing the paper's HE-Rot, HE-CMult, HE-Mult and HE-Add
 *     (Algorithms 1 and 2, Section 2.1) does; bit-identical to those
 *     operations called one by one.
 *   HEGMM_KS_DOUBLE: each linear transformation (Eq. lintrans),
 *     the HE-Add over the iterations' products and the extraction sum are
 *     formed over the extended basis PQ from the key-switch inner products
 *     (with P tau(c0), P d0, P d1 folded in) and divided by P once
 *     ("double hoisting"; ModDown(u + P x) = ModDown(u) + x).  Fewer
 *     ModDowns, lower noise.
 *   | HEGMM_KS_LAZY_RELIN (with either): the tensors (d0, d1, d2) of all
 *     iterations of a product are summed and the sum is relinearised once
 *     (one key switch per product instead of one per HE-Mult; the sum of
 *     Eq. elementwise taken before the key switch).
 * Each mode is bit-exact with the oracle's mode of the same name.  Applies
 * to products started after the call.  Errors: HEGMM_EINVAL. */
#define HEGMM_KS_SINGLE 0
#define HEGMM_KS_DOUBLE 1
#define HEGMM_KS_LAZY_RELIN 2
/*   | HEGMM_KS_SHARED (with any of the above): every linear transformation
 *     of an operand is evaluated as Rot(sum_d u'_d (.) Rot(ct, b_d), g):
 *     the offsets b_d are shared by all iterations of the product (and
 *     key-switched once per product), g is one HE-Rot per transformation
 *     that needs it (hegmm_plan_giant gives the factorisation; its keys are
 *     made by hegmm_keygen). */
#define HEGMM_KS_SHARED 4
int hegmm_set_keyswitch_mode(hegmm_ctx *ctx, int mode);

/* Tuning knobs of the product executor (no effect on results; plans built
 * before the call keep their values).
 *   HEGMM_TUNE_LT_CHUNK: in HEGMM_KS_DOUBLE mode, the most terms of one
 *     linear-transformation entries (shared rotations) handled by one work
 *     item of the fused key-switch kernel (1..4096, default 32); longer
 *     entry lists are split into partial sums.
 * Errors: HEGMM_EINVAL (unknown knob or value out of range). */
#define HEGMM_TUNE_LT_CHUNK 1
/*   HEGMM_TUNE_LT_FUSED: in HEGMM_KS_DOUBLE mode, 1 (default) evaluates each
 *     linear transformation in the fused kernel; 0 key-switches every
 *     distinct rotation once into a workspace chunk (chunk size set by
 *     hegmm_set_budgets' chunk_bytes) and applies the masks after each chunk. */
#define HEGMM_TUNE_LT_FUSED 2
/*   HEGMM_TUNE_LT_KERNEL: variant of the fused kernel for items of several
 *     outputs, by resident CTAs per SM (its register cap) and the form of
 *     its per-output sums (lazy 128-bit, or reduced after every use):
 *     0 = 4 lazy, 1 = 2 lazy, 2 = 3 lazy, 3 = 4 reduced, 4 = 5 reduced,
 *     5 = 6 reduced; 6 (default) = key rows and masks staged in shared
 *     memory by bulk asynchronous copies (TMA engine, double-buffered with
 *     mbarriers), 2 CTAs per SM, for dnum <= 8 (else variant 0); 7 = the
 *     same with a producer warp and full / empty mbarriers over 3 stages
 *     instead of a block barrier per entry; 8 = the form of 7 as one
 *     persistent launch (two CTAs per SM) that walks the flattened queue of
 *     every (work item, limb, 256-coefficient slice) unit, items of one
 *     output included (HEGMM_TUNE_LT_ONE then has no effect).
 *   HEGMM_TUNE_LT_ONE: kernel of the items of one output: 0 plain
 *     loads, 6 CTAs per SM (40 registers); 1 = key rows and masks staged by
 *     bulk asynchronous copies, 3 CTAs per SM (only with variants 6 and 7,
 *     else as 0); 2 = plain loads, 5 CTAs per SM (48 registers);
 *     3 = plain loads, 4 CTAs per SM (64 registers); 4 (default) = every
 *     operand of an entry fetched by per-thread asynchronous copies into
 *     shared memory, 6 CTAs per SM (at most 8 digits, else as 0). */
#define HEGMM_TUNE_LT_KERNEL 3
/*   HEGMM_TUNE_GIANT_COST: the cost of one giant rotation, in baby key
 *     switches, in the greedy rule of HEGMM_KS_SHARED (1..65536, default 8).
 *     It selects which factorisation is used, so it changes the ciphertext
 *     bits (each value matches the oracle run with the same cost); Galois
 *     keys the new factorisation needs are made from the context's secret
 *     key when a plan first needs them. */
#define HEGMM_TUNE_GIANT_COST 4
/*   HEGMM_TUNE_GRAPHS: 1 (default) replays the launch sequence of a cached
 *     product plan (hegmm_matmul, hegmm_matmul_batch*) as a CUDA graph from
 *     its second call on; 0 launches kernel by kernel.  While per-kernel
 *     timing is on (hegmm_set_timing) plans always run kernel by kernel. */
#define HEGMM_TUNE_GRAPHS 5
#define HEGMM_TUNE_LT_ONE 6
/*   HEGMM_TUNE_WAIT_LIMIT: polls of every bounded mbarrier wait of the staged
 *     kernels (default 2^22, about a second); when one runs out the kernel
 *     stops, drains its copies and the next synchronising call reports
 *     HEGMM_ETIMEOUT.
 *   HEGMM_TUNE_TEST_DROP: a test hook of that path: the staged kernels leave
 *     entry number `value` of every work item unarmed, so its bounded wait
 *     runs out (-1, the default: none).  No copy is issued for it and no memory is
 *     touched; the GPU and the context stay usable. */
#define HEGMM_TUNE_WAIT_LIMIT 7
#define HEGMM_TUNE_TEST_DROP 8
/*   HEGMM_TUNE_NTT_THREADS: threads of each CTA of the NTT-family kernels
 *     (one CTA per limb): 0 (default) picks by launch size (1024 at
 *     N = 2^14; at N = 2^13 512, or 1024 when a launch has no more CTAs than
 *     SMs), 512 or 1024 force that form where the ring has it (N / 8 of at
 *     least that many); at N = 2^14 the 512-thread form has 128 registers a
 *     thread instead of 64. */
#define HEGMM_TUNE_NTT_THREADS 9
/*   HEGMM_TUNE_GROUPS: 1 (default) runs a batch of products as one plan,
 *     every stage one launch over all of them; 2 splits a batch of at least
 *     two products into two sub-batches (by estimated workspace, largest
 *     first to the lighter group), each with its own cached plan on a
 *     stream of its own, forked from and joined back into the context
 *     stream, so that one group's small launches run beside the other's
 *     large ones.  Results are the same bits.  Not used while the context
 *     stream is being captured, nor by the server. */
#define HEGMM_TUNE_GROUPS 10
/*   HEGMM_TUNE_MODDOWN_SPLIT: 0 runs the fused ModDown with one CTA per
 *     output limb; 1 splits every limb between two CTAs of 512 threads, one
 *     per half (rings with N >= 2^13; smaller rings ignore it): each
 *     converts the whole limb for the transform's first stage and finishes
 *     its half, so that two CTAs share an SM; 2 (default) splits only
 *     launches of fewer limbs than twice the SMs.  Same bits. */
#define HEGMM_TUNE_MODDOWN_SPLIT 11
int hegmm_set_tuning(hegmm_ctx *ctx, int knob, long long value);

/* As hegmm_matmul_batch, with one algorithm per product: algs[i] in
 * {HEGMM_ALG_AUTO, 1, 2, 3} (algs may be NULL: AUTO for all).  Products of
 * both algorithms share each stage's launches. */
int hegmm_matmul_batch_algs(hegmm_ctx *ctx, int count, const hegmm_ct *const *A, const hegmm_ct *const *B,
                            const int *mln, const int *algs, hegmm_ct **C);

/* Linear transformations of ciphertexts (Eq. lintrans, Section 3.2.1),
 * evaluated as the paper composes them: out = sum over the diagonals d
 * (ascending) of HE-CMult(HE-Rot(ct, d), u_d), with the rotations of up to
 * 64 diagonals sharing one hoisted ModUp; the result keeps ct's level.
 * Galois keys that are missing are made from the context's secret key.
 *
 * hegmm_lintrans: slot j of *out takes slot src[j] of ct for j < count
 * (src[j] < 0 and slots from count on: 0); 0 <= src[j] < S, count <= S
 * (HEGMM_EINVAL otherwise); d = src[j] - j mod S.  The masks cover both
 * slot rows, so row 1 is transformed by the same map.
 *
 * A plain matrix ciphertext holds M (rows x cols) column-major: slot
 * i + j rows = M_ij.
 * hegmm_to_layout: ct holds A (m x l, role HEGMM_ROLE_A) or B (l x n, role
 * HEGMM_ROLE_B) as a plain matrix ciphertext; *out holds the operand layout
 * hegmm_encode would give for (m, l, n, alg): sigma(A) / tau(B) under
 * encryption (Section 3.2.2: at most 2 min(m,l) - 1 / 2 min(n,l) - 1
 * diagonals, Theorems 1-2), and for Algorithm 2 the duplication and
 * eps^0 / omega^0 as well.
 * hegmm_from_result: ct is the result of a product (m, l, n, alg); *out
 * holds C (m x n) as a plain matrix ciphertext, so a product can feed the
 * next one through hegmm_to_layout (for Algorithm 1 the result already has
 * this layout and the transformation only clears the other slots).
 * hegmm_chain_operand: ct is the result of a product (m, l, n, alg); *out
 * holds that m x n matrix in the layout of operand `role` of the next
 * product (m2, l2, n2, alg2): (m2, l2) = (m, n) for role A, (l2, n2) =
 * (m, n) for role B, else HEGMM_EINVAL.  One transformation (the
 * composition of hegmm_from_result and hegmm_to_layout), so one mask
 * product's noise: a chain of two products needs about twice the noise
 * budget of one (the N = 2^14, 8 x 50-bit ring has it).
 * Errors: HEGMM_EINVAL, HEGMM_ESHAPE (a shape that does not fit),
 * HEGMM_ENOMEM; *out is NULL on error. */
int hegmm_lintrans(hegmm_ctx *ctx, const hegmm_ct *ct, const int *src, int count, hegmm_ct **out);
int hegmm_to_layout(hegmm_ctx *ctx, const hegmm_ct *ct, int role, int m, int l, int n, int alg, hegmm_ct **out);
int hegmm_from_result(hegmm_ctx *ctx, const hegmm_ct *ct, int m, int l, int n, int alg, hegmm_ct **out);
int hegmm_chain_operand(hegmm_ctx *ctx, const hegmm_ct *ct, int m, int l, int n, int alg, int role, int m2, int l2,
                        int n2, int alg2, hegmm_ct **out);

/* Sums of products, the building block of blocked products (Section 4.4,
 * Table 4: a matrix larger than one ciphertext is split into blocks and
 * C_ij = sum_k A_ik B_kj).  Products are given as for hegmm_matmul_batch_algs
 * (algs may be NULL: AUTO); group[p] in [0, ngroups) names the sum product p
 * joins, and C[g] (ngroups new ciphertexts, owned by the caller) receives
 * the HE-Add of the results of group g's products.  Every group needs at
 * least one product, and all products of a group the same result layout
 * (hegmm_decrypt decodes C[g] with any member's m, l, n, alg); Algorithm 1
 * places C_ij at slot i + j m for every l.  Errors: HEGMM_EINVAL (bad
 * group index, empty group, bad algorithm), HEGMM_ESHAPE (a shape that does
 * not fit, or layouts that differ within a group), HEGMM_ENOKEY, HEGMM_ENOMEM;
 * on error every C[g] is NULL.  All products run in one batched call, the
 * sums in one more launch. */
int hegmm_matmul_sum(hegmm_ctx *ctx, int count, const hegmm_ct *const *A, const hegmm_ct *const *B,
                     const int *mln, const int *algs, const int *group, int ngroups, hegmm_ct **C);

/* Blocked product under Algorithm 1 (Section 4.4): an (sum rows) x
 * (sum inner) matrix times an (sum inner) x (sum cols) matrix, split into
 * nr x nk and nk x nc blocks.  A[i nk + k] encrypts block A_ik (rows[i] x
 * inner[k]) and B[k nc + j] block B_kj (inner[k] x cols[j]), each encoded
 * for Algorithm 1 with its own shape (hegmm_encode role A with m = rows[i],
 * l = inner[k]; role B with l = inner[k], n = cols[j]; the other dimension
 * does not change these layouts).  C[i nc + j] receives sum_k A_ik B_kj;
 * decrypt it with hegmm_decrypt(ctx, C, rows[i], inner[0], cols[j], 1).
 * Keys: those of every (rows[i], inner[k], cols[j]) under Algorithm 1.
 * Block sizes must be positive; errors as hegmm_matmul_sum. */
int hegmm_matmul_blocked(hegmm_ctx *ctx, int nr, int nk, int nc, const int *rows, const int *inner, const int *cols,
                         const hegmm_ct *const *A, const hegmm_ct *const *B, hegmm_ct **C);

/* Autotuner of the bit-neutral tuning knobs: runs the given products (as
 * hegmm_matmul_batch_algs would) under every candidate (kernel variant 0, 3,
 * 6, 7, 8; entries per item 16, 32, 64; one-output kernel 4, and 1 with
 * variants 6 / 7), then, from the fastest, the one-output kernels 0, 2 and
 * 3;
 * each candidate is timed over reps calls with CUDA events on the context
 * stream after a plan-building and a graph-capturing call, and the fastest
 * is kept in the context; then, with the fastest of those, the NTT-family
 * thread counts (HEGMM_TUNE_NTT_THREADS 0, 512, 1024, on rings where both
 * forms exist), then the half-limb ModDown always or never
 * (HEGMM_TUNE_MODDOWN_SPLIT 1, 0; rings with N >= 2^13), then two sub-batches (HEGMM_TUNE_GROUPS 2) for two or
 * more products, kept only when at least 2% faster.  chosen (may be NULL,
 * else 6 ints) receives {kernel variant, entries per item, one-output
 * kernel, NTT threads, sub-batches, ModDown split}.  Results stay
 * bit for bit the same (every candidate is an execution order of the same
 * sums).  The linear-transformation knobs only steer the HEGMM_KS_DOUBLE
 * kernels; in single mode only the NTT threads are tuned.  Cached product
 * plans are released (they are rebuilt on the next call). */
int hegmm_autotune(hegmm_ctx *ctx, int count, const hegmm_ct *const *A, const hegmm_ct *const *B, const int *mln,
                   const int *algs, int reps, int *chosen);

/* Builds and caches the per-shape plan data of the listed products (the
 * encoded diagonal masks of every linear transformation, Eq. lintrans), so
 * that the first product of each shape does not pay for it.  Needs the
 * shapes' keys.  Cached masks are released least recently used first when
 * they exceed the context's mask budget (96 GiB). */
int hegmm_prepare(hegmm_ctx *ctx, const int *shapes_mln, int n_shapes, int alg);

/* Memory budgets of a context (0 leaves a value unchanged): mask_bytes caps
 * the resident per-shape masks (default 96 GiB, least recently used shapes
 * are released first), plan_bytes the workspace kept by cached batch plans
 * (default 48 GiB), chunk_bytes the scratch of one chunked stage of a batch
 * (default 1 GiB; smaller chunks mean more launches). */
int hegmm_set_budgets(hegmm_ctx *ctx, uint64_t mask_bytes, uint64_t plan_bytes, uint64_t chunk_bytes);

/* ---- Serving: continuous batching of product requests ------------------
 * A server queues requests (two operand ciphertexts and a shape) and runs
 * them through the batch executor of hegmm_matmul_batch.  The caller's
 * event loop drives it: hegmm_server_poll retires finished batches (their
 * results become available to hegmm_server_result) and admits queued
 * requests into a new batch whenever one of the server's device streams is
 * free and the batch's estimated workspace fits in the memory budget minus
 * what in-flight batches hold -- so requests that arrive while others run
 * join the next batch, and batches on different streams overlap on the GPU.
 * Each result is bit-identical to the same product computed alone.
 * Operands must stay alive until their request completes.  While a server
 * exists, the context must be used from the thread that polls it. */
typedef struct hegmm_server hegmm_server;

typedef struct {
    int max_batch;       /* products per batch (0 = 64) */
    int streams;         /* device streams that batches rotate over (0 = 2, at most 8) */
    uint64_t mem_budget; /* device workspace the server preallocates, split evenly over its
                            streams (0 = 16 GiB); a batch admits requests while their estimated
                            workspace fits one stream's share */
} hegmm_server_opts;

typedef struct {
    long long submitted, completed, failed, batches, queued, in_flight, max_batch;
    double p50_ms, p99_ms, mean_ms, max_ms; /* submit-to-completion latency */
    long long max_batches_in_flight;        /* most batches launched and not yet retired at once */
    long long overlapped_batches;           /* retired batches whose device interval (from a timed event
                                               before its first launch to one after its last, on its
                                               stream) intersected that of a batch on another stream;
                                               each is compared with the 64 batches retired before it */
} hegmm_server_stats;

int hegmm_server_create(hegmm_ctx *ctx, const hegmm_server_opts *opts, hegmm_server **out);
/* Queues C = A.B; *ticket identifies the request.  Errors: HEGMM_ESHAPE,
 * HEGMM_EINVAL (operand level). */
int hegmm_server_submit(hegmm_server *srv, const hegmm_ct *A, const hegmm_ct *B, int m, int l, int n, int alg,
                        uint64_t *ticket);
/* Retires finished batches and launches new ones; with wait != 0 returns
 * only when every submitted request has completed. */
int hegmm_server_poll(hegmm_server *srv, int wait);
/* If the request has completed, *C receives its result (owned by the caller)
 * and latency_ms its submit-to-completion time; otherwise *C = NULL.
 * Returns the request's error code if its batch failed. */
int hegmm_server_result(hegmm_server *srv, uint64_t ticket, hegmm_ct **C, double *latency_ms);
int hegmm_server_stats_get(hegmm_server *srv, hegmm_server_stats *out);
/* Waits for every request, frees uncollected results and the server. */
void hegmm_server_destroy(hegmm_server *srv);

/* Decrypts a product of hegmm_matmul and reads C (m x n, row-major, values
 * in [0, t)) from the plan's result slots.  Synchronises the stream. */
int hegmm_decrypt(hegmm_ctx *ctx, const hegmm_ct *ct, int m, int l, int n, int alg, uint64_t *out);

/* Decrypts all S row-0 slots into out[S].  Synchronises the stream. */
int hegmm_decrypt_slots(hegmm_ctx *ctx, const hegmm_ct *ct, uint64_t *out);
/* Decrypts both slot rows into out[N] (row 0, then row 1). */
int hegmm_decrypt_rows(hegmm_ctx *ctx, const hegmm_ct *ct, uint64_t *out);
/* hegmm_decrypt of both rows of a product of hegmm_encode_pair operands:
 * the row-0 product into out0, the row-1 product into out1 (m x n each). */
int hegmm_decrypt_pair(hegmm_ctx *ctx, const hegmm_ct *ct, int m, int l, int n, int alg, uint64_t *out0,
                       uint64_t *out1);

/* Single HE operations (Section 2.1), each returning a new ciphertext. */
int hegmm_rotate(hegmm_ctx *ctx, const hegmm_ct *ct, int z, hegmm_ct **out);
/* Hoisted rotations: one ModUp of ct shared by count rotations. */
int hegmm_rotate_many(hegmm_ctx *ctx, const hegmm_ct *ct, const int *z, int count, hegmm_ct **outs);
int hegmm_cmult(hegmm_ctx *ctx, const hegmm_ct *ct, const hegmm_pt *pt, hegmm_ct **out);
int hegmm_add(hegmm_ctx *ctx, const hegmm_ct *a, const hegmm_ct *b, hegmm_ct **out);
int hegmm_mult(hegmm_ctx *ctx, const hegmm_ct *a, const hegmm_ct *b, hegmm_ct **out); /* tensor + relin */
int hegmm_modswitch(hegmm_ctx *ctx, const hegmm_ct *ct, hegmm_ct **out);          /* drop last prime */

/* HE-Rot of `in` by z into the caller's existing ciphertext `out` (same
 * level, not the same handle), allocating no device memory.  The paper has
 * no counterpart: it is a variant of hegmm_rotate for callers that cannot
 * allocate while they run this library -- for example an application whose
 * framework already holds the GPU's memory in its own pool, or a serving
 * loop that must not block in cudaMalloc / cudaFree (cudaFree synchronises
 * the device).  All intermediates live in one fixed 12 MiB device array
 * inside the library, which every GPU that loads the library keeps until the
 * process exits; parameter sets whose rotation needs more scratch than that
 * are rejected with HEGMM_EINVAL and a message.  The first call on a device
 * looks up that array's device address (with that device current); a call
 * while the context's stream is capturing is refused with HEGMM_EINVAL, as
 * is a device ordinal beyond the library's table.  Every call reuses the same
 * array and leaves its contents behind (nothing in it needs clearing: each
 * call writes every word it reads), so calls whose GPU work overlaps -- on
 * different streams, contexts or threads -- race and give wrong results.
 * The result is bit-identical to hegmm_rotate.  Errors: HEGMM_EINVAL,
 * HEGMM_ENOKEY, HEGMM_ECUDA. */
int hegmm_rotate_noalloc(hegmm_ctx *ctx, const hegmm_ct *in, int z, hegmm_ct *out);

/* Device memory seen by the library, after synchronising its stream:
 * out[0] bytes in use from the device's default stream-ordered pool (the
 * pool every allocation of this library comes from), out[1] the pool's
 * high-water mark of that use since the last reset, out[2] bytes the pool
 * holds from the device, out[3] free device memory (cudaMemGetInfo).  With
 * reset_high != 0 the high-water mark restarts from the current use after
 * it is read, so a later call shows whether anything in between allocated
 * from the pool.  out is caller-owned, 4 entries.  Errors: HEGMM_EINVAL,
 * HEGMM_ECUDA. */
int hegmm_device_memory(hegmm_ctx *ctx, int reset_high, uint64_t *out);

/* Level (number of chain primes) of a ciphertext. */
int hegmm_ct_level(const hegmm_ct *ct);

/* Host <-> device ciphertext transfer in the coefficient domain,
 * host layout [2][level][N].  Export synchronises the stream. */
int hegmm_ct_export(hegmm_ctx *ctx, const hegmm_ct *ct, uint64_t *host);
int hegmm_ct_import(hegmm_ctx *ctx, const uint64_t *host, int level, hegmm_ct **out);
/* The same for count ciphertexts at once: one transform launch for all of
 * them (and, for export, one synchronisation).  host[i] is a caller-owned
 * [2][level][N] buffer (pinned host memory makes the copies asynchronous
 * DMA); export needs every ciphertext at the same level.  Import returns
 * new ciphertexts in out[i] (all NULL on error). */
int hegmm_ct_import_batch(hegmm_ctx *ctx, int count, const uint64_t *const *host, int level, hegmm_ct **out);
int hegmm_ct_export_batch(hegmm_ctx *ctx, int count, const hegmm_ct *const *cts, uint64_t *const *host);

/* Waits for all work queued on the context's stream.  Returns
 * HEGMM_ETIMEOUT if, since the last check, a kernel's bounded wait for its
 * staged copies ran out (its products are then invalid; the context stays
 * usable).  hegmm_decrypt*, hegmm_ct_export and hegmm_ct_export_batch make
 * the same check. */
int hegmm_sync(hegmm_ctx *ctx);

void hegmm_pt_destroy(hegmm_pt *pt);
void hegmm_ct_destroy(hegmm_ct *ct);

/* Host-only planner queries (no context, no GPU).  slots = S = N/2.
 * hegmm_plan_counts fills the operation counts of hegmm_matmul for the
 * shape (ksw counts each distinct rotation offset of an operand once, plus
 * one key switch per HE-Mult and per extraction rotation).
 * hegmm_plan_describe writes the plan as ints into buf[cap] and returns the
 * number of ints it needs (call with cap = 0 to size the buffer), or a
 * negative HEGMM_E* code:
 *   alg, case ('1','A','B','L'), column_major, iterations, extractions,
 *   then per iteration, for eps then omega: number of diagonals, and per
 *   diagonal its offset d, its slot count c and the c destination slots;
 *   then the extraction offsets; then the m*n result slots (row-major).
 * hegmm_plan_layout writes the client-side slot vector of role A or B for
 * the plan (values mod t) into out[cap] and returns its length. */
/* hegmm_plan_giant writes the shared-baby-step factorisation of role A (0,
 * the eps^k) or B (1, the omega^k) used by HEGMM_KS_SHARED, for the giant
 * cost `cost` (0: the default 8; see HEGMM_TUNE_GIANT_COST), as ints into
 * buf[cap] and returns the number it needs: iterations, then per iteration
 * its giant rotation g (0: none) and term count, and per term its baby
 * offset b in [0, S), slot count c and the c destination slots. */
int hegmm_plan_giant(int m, int l, int n, int alg, int slots, int role, int cost, int *buf, int cap);
int hegmm_plan_counts(int m, int l, int n, int alg, int slots, hegmm_opcount *out);
int hegmm_plan_describe(int m, int l, int n, int alg, int slots, int *buf, int cap);
int hegmm_plan_layout(int m, int l, int n, int alg, int slots, int role, const int64_t *mat, uint64_t t,
                      uint64_t *out, int cap);
/* hegmm_plan_slot_map writes the slot map hegmm_to_layout (role 0: A,
 * 1: B) or hegmm_from_result (role 2) applies for the plan: for every
 * destination slot the source slot it copies, -1 for zero (plain matrices
 * column-major, slot i + j rows = M_ij), into buf[cap]; returns its length.
 * hegmm_plan_result_layout writes {result rows, result columns,
 * column-major} of the plan (where C_ij sits; hegmm_matmul_sum groups
 * products with equal triples). */
int hegmm_plan_slot_map(int m, int l, int n, int alg, int slots, int role, int *buf, int cap);
int hegmm_plan_result_layout(int m, int l, int n, int alg, int slots, int *rows_cols_col);
/* hegmm_plan_pow2_steps writes the chain of signed power-of-two rotation
 * offsets that HEGMM_KEYS_POW2 applies for a left rotation by z over `slots`
 * slots into buf[cap] and returns its length (0 for z = 0 mod slots). */
int hegmm_plan_pow2_steps(long long z, int slots, int *buf, int cap);

/* Per-kernel device timing: while enabled, every launch of the library's
 * kernels is bracketed by CUDA events on the context stream and its
 * duration added to the kernel's bucket.  kind indexes the table named by
 * hegmm_kernel_name (0 .. hegmm_kernel_kinds()-1).  Reading the stats
 * synchronises the stream; hegmm_kernel_reset zeroes them.  bytes is the
 * launches' algorithmic HBM traffic (inputs read once, outputs written
 * once); butterflies counts (N/2) log2 N per limb NTT the launches ran. */
int hegmm_set_timing(hegmm_ctx *ctx, int enable);
int hegmm_kernel_kinds(void);
const char *hegmm_kernel_name(int kind);
int hegmm_kernel_stats(hegmm_ctx *ctx, int kind, double *total_ms, long long *launches, double *bytes,
                       double *butterflies);
int hegmm_kernel_reset(hegmm_ctx *ctx);

/* Measures the integer-pipe ceiling of the NTT butterfly on this device: the
 * lazy Shoup butterfly of the NTT kernels repeated on registers by every SM,
 * no memory traffic.  *per_s receives butterflies per second.  Synchronous. */
int hegmm_peak_butterflies(hegmm_ctx *ctx, double *per_s);

#ifdef __cplusplus
}
#endif

#endif /* HEGMM_H */

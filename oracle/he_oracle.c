/*
 * he_oracle.c -- plain C reference of the RNS-BGV arithmetic under HEGMM.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this library; the product never
 * does, and it shares no code with the CUDA path.
 *
 * The paper (arXiv 2405.02238, Section 2.1) uses HE-Add, HE-Mult, HE-CMult
 * and HE-Rot as library calls and fixes nothing below them.  This file is
 * the written-out definition of those operations for a BGV scheme over
 * R_q = Z_q[X]/(X^N + 1) in RNS form, following the conventions the CUDA
 * path must reproduce bit for bit:
 *
 *  - every polynomial is held in the coefficient domain, residues in [0, q);
 *  - ring products are computed as inverse-NTT(NTT(a) * NTT(b)) with a
 *    textbook negacyclic NTT (checked against schoolbook convolution);
 *  - modular products are (unsigned __int128)a * b % q -- slow and plain;
 *  - every lift between primes is centred: v in [0, q) stands for v when
 *    v <= (q-1)/2 and for v - q otherwise;
 *  - key switching is hybrid: ModUp of each digit by a centred fast base
 *    conversion, inner product with the switching key over Q*P, and a
 *    ModDown that converts y = [t^-1 u]_P (not t*y) so that the rounding
 *    error is a multiple of the plaintext modulus t;
 *  - the BGV modulus switch drops the last chain prime the same way.
 *
 * Random numbers: SplitMix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) read in counter mode:
 * draw(stream, i) = mix64(stream + (i + 1) * GAMMA), the i-th output of the
 * generator seeded with ``stream``; stream = mix64(seed ^ mix64(domain << 48
 * | obj)).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef uint64_t u64;
typedef int64_t i64;
typedef unsigned __int128 u128;

#define MAXP 32

/* ------------------------------------------------------------------ */
/* Modular arithmetic                                                  */
/* ------------------------------------------------------------------ */

static u64 mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
static u64 addmod(u64 a, u64 b, u64 q) { u64 r = a + b; return r >= q ? r - q : r; }
static u64 submod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }

static u64 powmod(u64 a, u64 e, u64 q) {
    u64 r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mulmod(r, a, q);
        a = mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}

static u64 invmod(u64 a, u64 q) { return powmod(a, q - 2, q); } /* q prime */

/* A signed integer reduced into [0, q). */
static u64 smod(i64 v, u64 q) {
    if (v >= 0) return (u64)v % q;
    u64 r = (u64)(-(v + 1)) % q; /* avoids overflow at INT64_MIN */
    return q - 1 - r;
}

/* Centred lift of v in [0, p), reduced into [0, r). */
static u64 centred_to(u64 v, u64 p, u64 r) {
    if (v <= (p - 1) / 2) return v % r;
    u64 mag = (p - v) % r; /* v stands for -(p - v) */
    return mag == 0 ? 0 : r - mag;
}

/* Deterministic Miller-Rabin for n < 2^64 with the first 12 prime bases. */
int or_is_prime(u64 n) {
    static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    u64 d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; s++; }
    for (int i = 0; i < 12; i++) {
        u64 x = powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int comp = 1;
        for (int r = 1; r < s; r++) {
            x = mulmod(x, x, n);
            if (x == n - 1) { comp = 0; break; }
        }
        if (comp) return 0;
    }
    return 1;
}

/* The ``count`` largest primes below 2^bits that are 1 mod 2N, descending. */
int or_find_primes(int logN, int bits, int count, u64 *out) {
    u64 two_n = (u64)2 << logN;
    u64 c = ((((u64)1 << bits) - 1) / two_n) * two_n + 1;
    if (c >= ((u64)1 << bits)) c -= two_n;
    int got = 0;
    while (got < count && c > two_n) {
        if (or_is_prime(c)) out[got++] = c;
        c -= two_n;
    }
    return got;
}

/* ------------------------------------------------------------------ */
/* SplitMix64 in counter mode                                          */
/* ------------------------------------------------------------------ */

#define GAMMA 0x9E3779B97F4A7C15ULL

u64 or_mix64(u64 z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

u64 or_stream(u64 seed, u64 domain, u64 obj) {
    return or_mix64(seed ^ or_mix64((domain << 48) | obj));
}

u64 or_draw(u64 stream, u64 idx) { return or_mix64(stream + (idx + 1) * GAMMA); }

static i64 cbd(u64 r, int eta) {
    u64 msk = ((u64)1 << eta) - 1;
    return (i64)__builtin_popcountll(r & msk) - (i64)__builtin_popcountll((r >> eta) & msk);
}

/* Domains of the random streams. */
enum { DOM_SK = 1, DOM_KEY_A = 2, DOM_KEY_E = 3, DOM_ENC_A = 4, DOM_ENC_E = 5 };

/* ------------------------------------------------------------------ */
/* Context                                                             */
/* ------------------------------------------------------------------ */

typedef struct {
    int logN, N, L, K, alpha, eta;
    u64 t;
    u64 te;          /* factor of every error term and of the rounding correction: t (BGV), 1 (BFV) */
    u64 prime[MAXP]; /* q_0 .. q_{L-1}, p_0 .. p_{K-1} */
    u64 psi[MAXP];   /* a primitive 2N-th root of unity mod each prime */
    u64 psi_t;       /* zeta = 3^((t-1)/2N) mod t */
} or_ctx;

/* Smallest-base primitive 2N-th root: g^((q-1)/2N) for the first g whose
 * power has order exactly 2N (i.e. its N-th power is -1). */
static u64 find_psi(u64 q, int N) {
    for (u64 g = 2; g < q; g++) {
        u64 w = powmod(g, (q - 1) / (2 * (u64)N), q);
        if (powmod(w, (u64)N, q) == q - 1) return w;
    }
    return 0;
}

or_ctx *or_new(int logN, u64 t, int L, int qbits, int K, int alpha, int eta) {
    if (L + K > MAXP) return 0;
    or_ctx *c = (or_ctx *)calloc(1, sizeof(or_ctx));
    c->logN = logN;
    c->N = 1 << logN;
    c->L = L;
    c->K = K;
    c->alpha = alpha;
    c->eta = eta;
    c->t = t;
    c->te = t;
    if (or_find_primes(logN, qbits, L + K, c->prime) != L + K) { free(c); return 0; }
    for (int i = 0; i < L + K; i++) c->psi[i] = find_psi(c->prime[i], c->N);
    c->psi_t = powmod(3, (t - 1) / (2 * (u64)c->N), t);
    return c;
}

void or_free(or_ctx *c) { free(c); }

/* The scheme's error factor: t for BGV (errors t e, ModDown and modulus
 * switch rounding corrected by t), 1 for BFV (errors e, plain rounding). */
void or_set_error_factor(or_ctx *c, u64 te) { c->te = te; }
void or_get_primes(const or_ctx *c, u64 *out) { memcpy(out, c->prime, sizeof(u64) * (c->L + c->K)); }
u64 or_get_psi(const or_ctx *c, int pi) { return pi < 0 ? c->psi_t : c->psi[pi]; }

static u64 modulus_of(const or_ctx *c, int pi) { return pi < 0 ? c->t : c->prime[pi]; }

/* ------------------------------------------------------------------ */
/* Negacyclic NTT: a_hat[k] = sum_i a[i] psi^(i (2k+1)), k in natural order */
/* ------------------------------------------------------------------ */

static void bitrev_permute(u64 *a, int N) {
    for (int i = 1, j = 0; i < N; i++) {
        int bit = N >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { u64 x = a[i]; a[i] = a[j]; a[j] = x; }
    }
}

/* In-place cyclic DFT of size N with root w (textbook iterative radix-2). */
static void dft(u64 *a, int N, u64 w, u64 q) {
    bitrev_permute(a, N);
    for (int len = 2; len <= N; len <<= 1) {
        u64 wl = powmod(w, (u64)(N / len), q);
        for (int i = 0; i < N; i += len) {
            u64 x = 1;
            for (int j = 0; j < len / 2; j++) {
                u64 u = a[i + j], v = mulmod(a[i + j + len / 2], x, q);
                a[i + j] = addmod(u, v, q);
                a[i + j + len / 2] = submod(u, v, q);
                x = mulmod(x, wl, q);
            }
        }
    }
}

void or_ntt(const or_ctx *c, int pi, u64 *a) {
    u64 q = modulus_of(c, pi), psi = or_get_psi(c, pi), x = 1;
    for (int i = 0; i < c->N; i++) { a[i] = mulmod(a[i], x, q); x = mulmod(x, psi, q); }
    dft(a, c->N, mulmod(psi, psi, q), q);
}

void or_intt(const or_ctx *c, int pi, u64 *a) {
    u64 q = modulus_of(c, pi), psi_inv = invmod(or_get_psi(c, pi), q);
    dft(a, c->N, mulmod(psi_inv, psi_inv, q), q);
    u64 ninv = invmod((u64)c->N, q), x = ninv;
    for (int i = 0; i < c->N; i++) { a[i] = mulmod(a[i], x, q); x = mulmod(x, psi_inv, q); }
}

/* Schoolbook product in Z_q[X]/(X^N+1): X^N = -1. */
void or_negacyclic_schoolbook(const u64 *a, const u64 *b, int N, u64 q, u64 *out) {
    for (int k = 0; k < N; k++) out[k] = 0;
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) {
            u64 p = mulmod(a[i], b[j], q);
            int k = i + j;
            if (k < N) out[k] = addmod(out[k], p, q);
            else out[k - N] = submod(out[k - N], p, q);
        }
}

void or_polymul(const or_ctx *c, int pi, const u64 *a, const u64 *b, u64 *out) {
    int N = c->N;
    u64 q = modulus_of(c, pi);
    u64 *fa = (u64 *)malloc(sizeof(u64) * N), *fb = (u64 *)malloc(sizeof(u64) * N);
    memcpy(fa, a, sizeof(u64) * N);
    memcpy(fb, b, sizeof(u64) * N);
    or_ntt(c, pi, fa);
    or_ntt(c, pi, fb);
    for (int i = 0; i < N; i++) out[i] = mulmod(fa[i], fb[i], q);
    or_intt(c, pi, out);
    free(fa);
    free(fb);
}

/* ------------------------------------------------------------------ */
/* Prime sets of a level                                               */
/* ------------------------------------------------------------------ */

/* At level lv a ciphertext lives over q_0..q_{lv-1}; the key-switching
 * basis is those primes followed by the K special primes.  Extended index
 * e maps to the global prime index below. */
static int ext_prime(const or_ctx *c, int lv, int e) { return e < lv ? e : c->L + (e - lv); }
static int digits_at(const or_ctx *c, int lv) { return (lv + c->alpha - 1) / c->alpha; }

/* ------------------------------------------------------------------ */
/* Sampling, keys, encryption, decryption                              */
/* ------------------------------------------------------------------ */

/* Ternary secret s_i = (draw % 3) - 1. */
void or_sample_secret(const or_ctx *c, u64 seed, i64 *s) {
    u64 st = or_stream(seed, DOM_SK, 0);
    for (int i = 0; i < c->N; i++) s[i] = (i64)(or_draw(st, (u64)i) % 3) - 1;
}

/* Switching key from s to s', over all L+K primes, coefficient form.
 * evk layout [dnum][2][L+K][N]; component 0 is b_j, component 1 is a_j:
 *   a_j uniform per residue, e_j centred binomial (eta),
 *   b_j = -a_j s + t e_j + [P]_{q_i} s'   on the primes q_i of digit j,
 *   b_j = -a_j s + t e_j                  on every other prime.
 * sprime: residues of s' over the L+K primes, [L+K][N]. */
void or_gen_evk(const or_ctx *c, u64 seed, u64 gtag, const i64 *s, const u64 *sprime, u64 *evk) {
    int N = c->N, L = c->L, K = c->K, np = L + K, dnum = digits_at(c, L);
    u64 *sres = (u64 *)malloc(sizeof(u64) * N), *as = (u64 *)malloc(sizeof(u64) * N);
    i64 *e = (i64 *)malloc(sizeof(i64) * N);
    for (int j = 0; j < dnum; j++) {
        u64 sta = or_stream(seed, DOM_KEY_A, gtag * 256 + (u64)j);
        u64 ste = or_stream(seed, DOM_KEY_E, gtag * 256 + (u64)j);
        for (int i = 0; i < N; i++) e[i] = cbd(or_draw(ste, (u64)i), c->eta);
        for (int pi = 0; pi < np; pi++) {
            u64 q = c->prime[pi];
            u64 *b = evk + (((size_t)j * 2 + 0) * np + pi) * N;
            u64 *a = evk + (((size_t)j * 2 + 1) * np + pi) * N;
            for (int i = 0; i < N; i++) a[i] = or_draw(sta, (u64)pi * N + i) % q;
            for (int i = 0; i < N; i++) sres[i] = smod(s[i], q);
            or_polymul(c, pi, a, sres, as);
            u64 Pmod = 1;
            for (int k = 0; k < K; k++) Pmod = mulmod(Pmod, c->prime[L + k] % q, q);
            int in_digit = pi < L && pi / c->alpha == j;
            for (int i = 0; i < N; i++) {
                u64 v = submod(mulmod(c->te % q, smod(e[i], q), q), as[i], q);
                if (in_digit) v = addmod(v, mulmod(Pmod, sprime[(size_t)pi * N + i], q), q);
                b[i] = v;
            }
        }
    }
    free(sres);
    free(as);
    free(e);
}

/* Secret-key encryption of plaintext m (centred coefficients):
 * c1 = a (uniform), c0 = -a s + t e + m over the L chain primes. */
void or_encrypt(const or_ctx *c, u64 seed, u64 stream_id, const i64 *s, const i64 *m, u64 *ct) {
    int N = c->N, L = c->L;
    u64 sta = or_stream(seed, DOM_ENC_A, stream_id), ste = or_stream(seed, DOM_ENC_E, stream_id);
    i64 *e = (i64 *)malloc(sizeof(i64) * N);
    u64 *sres = (u64 *)malloc(sizeof(u64) * N), *as = (u64 *)malloc(sizeof(u64) * N);
    for (int i = 0; i < N; i++) e[i] = cbd(or_draw(ste, (u64)i), c->eta);
    for (int pi = 0; pi < L; pi++) {
        u64 q = c->prime[pi];
        u64 *c0 = ct + (size_t)pi * N, *c1 = ct + ((size_t)L + pi) * N;
        for (int i = 0; i < N; i++) c1[i] = or_draw(sta, (u64)pi * N + i) % q;
        for (int i = 0; i < N; i++) sres[i] = smod(s[i], q);
        or_polymul(c, pi, c1, sres, as);
        for (int i = 0; i < N; i++) {
            u64 v = addmod(mulmod(c->te % q, smod(e[i], q), q), smod(m[i], q), q);
            c0[i] = submod(v, as[i], q);
        }
    }
    free(e);
    free(sres);
    free(as);
}

/* BFV secret-key encryption: c1 = a, c0 = -a s + e + Delta m over the L
 * chain primes, Delta = floor(Q / t) given by its residues delta[L]; m holds
 * the centred coefficients of the plaintext. */
void or_encrypt_scaled(const or_ctx *c, u64 seed, u64 stream_id, const i64 *s, const i64 *m, const u64 *delta,
                       u64 *ct) {
    int N = c->N, L = c->L;
    u64 sta = or_stream(seed, DOM_ENC_A, stream_id), ste = or_stream(seed, DOM_ENC_E, stream_id);
    i64 *e = (i64 *)malloc(sizeof(i64) * N);
    u64 *sres = (u64 *)malloc(sizeof(u64) * N), *as = (u64 *)malloc(sizeof(u64) * N);
    for (int i = 0; i < N; i++) e[i] = cbd(or_draw(ste, (u64)i), c->eta);
    for (int pi = 0; pi < L; pi++) {
        u64 q = c->prime[pi];
        u64 *c0 = ct + (size_t)pi * N, *c1 = ct + ((size_t)L + pi) * N;
        for (int i = 0; i < N; i++) c1[i] = or_draw(sta, (u64)pi * N + i) % q;
        for (int i = 0; i < N; i++) sres[i] = smod(s[i], q);
        or_polymul(c, pi, c1, sres, as);
        for (int i = 0; i < N; i++) {
            u64 v = addmod(mulmod(c->te % q, smod(e[i], q), q), mulmod(delta[pi] % q, smod(m[i], q), q), q);
            c0[i] = submod(v, as[i], q);
        }
    }
    free(e);
    free(sres);
    free(as);
}

/* v = c0 + c1 s over the lv chain primes (residues; CRT is done by the caller). */
void or_decrypt_residues(const or_ctx *c, int lv, const i64 *s, const u64 *ct, u64 *v) {
    int N = c->N;
    u64 *sres = (u64 *)malloc(sizeof(u64) * N);
    for (int pi = 0; pi < lv; pi++) {
        u64 q = c->prime[pi];
        for (int i = 0; i < N; i++) sres[i] = smod(s[i], q);
        or_polymul(c, pi, ct + ((size_t)lv + pi) * N, sres, v + (size_t)pi * N);
        for (int i = 0; i < N; i++) v[(size_t)pi * N + i] = addmod(v[(size_t)pi * N + i], ct[(size_t)pi * N + i], q);
    }
    free(sres);
}

/* ------------------------------------------------------------------ */
/* Automorphism X -> X^g                                               */
/* ------------------------------------------------------------------ */

/* a: np residue polynomials, primes given by global indices pidx[]. */
void or_automorph(const or_ctx *c, int np, const int *pidx, const u64 *a, u64 g, u64 *out) {
    int N = c->N;
    u64 two_n = 2 * (u64)N;
    for (int r = 0; r < np; r++) {
        u64 q = c->prime[pidx[r]];
        const u64 *src = a + (size_t)r * N;
        u64 *dst = out + (size_t)r * N;
        for (int i = 0; i < N; i++) {
            u64 e = ((u64)i * g) % two_n;
            if (e < (u64)N) dst[e] = src[i];
            else dst[e - N] = src[i] == 0 ? 0 : q - src[i];
        }
    }
}

/* Same on a signed integer polynomial (used for the secret key). */
void or_automorph_int(const or_ctx *c, const i64 *a, u64 g, i64 *out) {
    int N = c->N;
    u64 two_n = 2 * (u64)N;
    for (int i = 0; i < N; i++) {
        u64 e = ((u64)i * g) % two_n;
        if (e < (u64)N) out[e] = a[i];
        else out[e - N] = -a[i];
    }
}

/* ------------------------------------------------------------------ */
/* Key switching                                                       */
/* ------------------------------------------------------------------ */

/* ModUp of x (residues over q_0..q_{lv-1}, coefficient form).
 * D layout [digits][lv+K][N] over the extended basis of level lv.
 * On the primes of digit j, D_j = x; on every other prime r,
 *   D_j = sum_{i in j} centred([x_i (Q_j/q_i)^-1]_{q_i}) (Q_j/q_i)  mod r. */
void or_modup(const or_ctx *c, int lv, const u64 *x, u64 *D) {
    int N = c->N, ne = lv + c->K, nd = digits_at(c, lv);
    for (int j = 0; j < nd; j++) {
        int lo = j * c->alpha, hi = lo + c->alpha < lv ? lo + c->alpha : lv;
        for (int e = 0; e < ne; e++) {
            int gp = ext_prime(c, lv, e);
            u64 r = c->prime[gp];
            u64 *dst = D + ((size_t)j * ne + e) * N;
            if (e >= lo && e < hi) { memcpy(dst, x + (size_t)e * N, sizeof(u64) * N); continue; }
            for (int k = 0; k < N; k++) dst[k] = 0;
            for (int i = lo; i < hi; i++) {
                u64 qi = c->prime[i];
                u64 hat_qi = 1, hat_r = 1; /* Q_j / q_i mod q_i and mod r */
                for (int i2 = lo; i2 < hi; i2++)
                    if (i2 != i) { hat_qi = mulmod(hat_qi, c->prime[i2] % qi, qi); hat_r = mulmod(hat_r, c->prime[i2] % r, r); }
                u64 hat_inv = invmod(hat_qi, qi);
                for (int k = 0; k < N; k++) {
                    u64 y = mulmod(x[(size_t)i * N + k], hat_inv, qi);
                    dst[k] = addmod(dst[k], mulmod(centred_to(y, qi, r), hat_r, r), r);
                }
            }
        }
    }
}

/* Inner product u_c = sum_j D_j * evk[j][c] over the extended basis of level
 * lv.  evk_eval holds the full-level key [dnum][2][L+K][N] in this file's
 * NTT form (or_ntt of each residue polynomial); D is in coefficient form;
 * u is returned in coefficient form, layout [2][lv+K][N]. */
void or_ks_inner(const or_ctx *c, int lv, const u64 *D, const u64 *evk_eval, u64 *u) {
    int N = c->N, ne = lv + c->K, nd = digits_at(c, lv), npk = c->L + c->K;
    u64 *f = (u64 *)malloc(sizeof(u64) * N);
    for (int e = 0; e < ne; e++) {
        int gp = ext_prime(c, lv, e);
        u64 q = c->prime[gp];
        u64 *u0 = u + (size_t)e * N, *u1 = u + ((size_t)ne + e) * N;
        for (int k = 0; k < N; k++) { u0[k] = 0; u1[k] = 0; }
        for (int j = 0; j < nd; j++) {
            memcpy(f, D + ((size_t)j * ne + e) * N, sizeof(u64) * N);
            or_ntt(c, gp, f);
            const u64 *k0 = evk_eval + (((size_t)j * 2 + 0) * npk + gp) * N;
            const u64 *k1 = evk_eval + (((size_t)j * 2 + 1) * npk + gp) * N;
            for (int k = 0; k < N; k++) {
                u0[k] = addmod(u0[k], mulmod(f[k], k0[k], q), q);
                u1[k] = addmod(u1[k], mulmod(f[k], k1[k], q), q);
            }
        }
        or_intt(c, gp, u0);
        or_intt(c, gp, u1);
    }
    free(f);
}

/* Divide by the product D of the primes with extended indices [first, ne)
 * (the special primes for ModDown, the last chain prime for the modulus
 * switch), keeping the message mod t:
 *   z_k   = centred([u_{d_k} t^-1 (D/d_k)^-1]_{d_k})
 *   y~_i  = sum_k z_k (D/d_k)            mod q_i
 *   out_i = (u_i - t y~_i) D^-1          mod q_i,   i < first.
 * in/out use the basis primes pidx[0..ne). */
static void divide_round_t(const or_ctx *c, int ne, int first, const int *pidx, const u64 *in, u64 *out) {
    int N = c->N, nd = ne - first;
    for (int i = 0; i < first; i++) {
        u64 q = c->prime[pidx[i]];
        u64 Dmod = 1;
        for (int k = 0; k < nd; k++) Dmod = mulmod(Dmod, c->prime[pidx[first + k]] % q, q);
        u64 Dinv = invmod(Dmod, q), tq = c->te % q;
        u64 *o = out + (size_t)i * N;
        for (int x = 0; x < N; x++) o[x] = 0;
        for (int k = 0; k < nd; k++) {
            u64 dk = c->prime[pidx[first + k]];
            u64 hat_dk = 1, hat_q = 1; /* (D/d_k) mod d_k and mod q */
            for (int k2 = 0; k2 < nd; k2++)
                if (k2 != k) {
                    u64 d2 = c->prime[pidx[first + k2]];
                    hat_dk = mulmod(hat_dk, d2 % dk, dk);
                    hat_q = mulmod(hat_q, d2 % q, q);
                }
            u64 coef = mulmod(invmod(c->te % dk, dk), invmod(hat_dk, dk), dk);
            const u64 *ud = in + (size_t)(first + k) * N;
            for (int x = 0; x < N; x++) {
                u64 z = mulmod(ud[x], coef, dk);
                o[x] = addmod(o[x], mulmod(centred_to(z, dk, q), hat_q, q), q);
            }
        }
        const u64 *ui = in + (size_t)i * N;
        for (int x = 0; x < N; x++) o[x] = mulmod(submod(ui[x], mulmod(tq, o[x], q), q), Dinv, q);
    }
}

/* ModDown of one polynomial from the extended basis of level lv to q_0..q_{lv-1}. */
void or_moddown(const or_ctx *c, int lv, const u64 *u, u64 *out) {
    int pidx[MAXP], ne = lv + c->K;
    for (int e = 0; e < ne; e++) pidx[e] = ext_prime(c, lv, e);
    divide_round_t(c, ne, lv, pidx, u, out);
}

/* Full key switch of x at level lv: (k0, k1) with k0 + k1 s ~ x s'. out [2][lv][N]. */
void or_keyswitch(const or_ctx *c, int lv, const u64 *x, const u64 *evk_eval, u64 *out) {
    int N = c->N, ne = lv + c->K, nd = digits_at(c, lv);
    u64 *D = (u64 *)malloc(sizeof(u64) * (size_t)nd * ne * N);
    u64 *u = (u64 *)malloc(sizeof(u64) * (size_t)2 * ne * N);
    or_modup(c, lv, x, D);
    or_ks_inner(c, lv, D, evk_eval, u);
    or_moddown(c, lv, u, out);
    or_moddown(c, lv, u + (size_t)ne * N, out + (size_t)lv * N);
    free(D);
    free(u);
}

/* HE-Rot: ct -> (tau_g(c0) + KS(tau_g(c1))_0, KS(tau_g(c1))_1), keyed by the
 * switching key from tau_g(s) to s. */
void or_rotate(const or_ctx *c, int lv, const u64 *ct, u64 g, const u64 *evk_eval, u64 *out) {
    int N = c->N, pidx[MAXP];
    for (int i = 0; i < lv; i++) pidx[i] = i;
    u64 *r = (u64 *)malloc(sizeof(u64) * (size_t)2 * lv * N);
    u64 *k = (u64 *)malloc(sizeof(u64) * (size_t)2 * lv * N);
    or_automorph(c, lv, pidx, ct, g, r);
    or_automorph(c, lv, pidx, ct + (size_t)lv * N, g, r + (size_t)lv * N);
    or_keyswitch(c, lv, r + (size_t)lv * N, evk_eval, k);
    for (int i = 0; i < lv; i++) {
        u64 q = c->prime[i];
        for (int x = 0; x < N; x++) {
            out[(size_t)i * N + x] = addmod(r[(size_t)i * N + x], k[(size_t)i * N + x], q);
            out[((size_t)lv + i) * N + x] = k[((size_t)lv + i) * N + x];
        }
    }
    free(r);
    free(k);
}

/* Hoisted form of the same rotation: ModUp of c1 first, then the
 * automorphism on every digit.  Bit-identical to or_rotate because the
 * centred lift commutes with negation. */
void or_rotate_hoisted(const or_ctx *c, int lv, const u64 *ct, u64 g, const u64 *evk_eval, u64 *out) {
    int N = c->N, ne = lv + c->K, nd = digits_at(c, lv), pidx[MAXP];
    for (int e = 0; e < ne; e++) pidx[e] = ext_prime(c, lv, e);
    u64 *D = (u64 *)malloc(sizeof(u64) * (size_t)nd * ne * N);
    u64 *Dg = (u64 *)malloc(sizeof(u64) * (size_t)nd * ne * N);
    u64 *u = (u64 *)malloc(sizeof(u64) * (size_t)2 * ne * N);
    u64 *c0 = (u64 *)malloc(sizeof(u64) * (size_t)lv * N);
    or_modup(c, lv, ct + (size_t)lv * N, D);
    for (int j = 0; j < nd; j++) or_automorph(c, ne, pidx, D + (size_t)j * ne * N, g, Dg + (size_t)j * ne * N);
    or_ks_inner(c, lv, Dg, evk_eval, u);
    or_moddown(c, lv, u, out);
    or_moddown(c, lv, u + (size_t)ne * N, out + (size_t)lv * N);
    or_automorph(c, lv, pidx, ct, g, c0);
    for (int i = 0; i < lv; i++) {
        u64 q = c->prime[i];
        for (int x = 0; x < N; x++) out[(size_t)i * N + x] = addmod(out[(size_t)i * N + x], c0[(size_t)i * N + x], q);
    }
    free(D);
    free(Dg);
    free(u);
    free(c0);
}

/* ------------------------------------------------------------------ */
/* HE-Add, HE-CMult, HE-Mult (tensor + relinearisation), modulus switch */
/* ------------------------------------------------------------------ */

void or_add(const or_ctx *c, int lv, int npoly, const u64 *a, const u64 *b, u64 *out) {
    int N = c->N;
    for (int p = 0; p < npoly; p++)
        for (int i = 0; i < lv; i++) {
            u64 q = c->prime[i];
            size_t o = ((size_t)p * lv + i) * N;
            for (int x = 0; x < N; x++) out[o + x] = addmod(a[o + x], b[o + x], q);
        }
}

/* ct (.) pt; pt_eval = or_ntt of the plaintext's residues over q_0..q_{lv-1}. */
void or_cmult(const or_ctx *c, int lv, const u64 *ct, const u64 *pt_eval, u64 *out) {
    int N = c->N;
    u64 *f = (u64 *)malloc(sizeof(u64) * N);
    for (int p = 0; p < 2; p++)
        for (int i = 0; i < lv; i++) {
            u64 q = c->prime[i];
            size_t o = ((size_t)p * lv + i) * N;
            memcpy(f, ct + o, sizeof(u64) * N);
            or_ntt(c, i, f);
            for (int x = 0; x < N; x++) out[o + x] = mulmod(f[x], pt_eval[(size_t)i * N + x], q);
            or_intt(c, i, out + o);
        }
    free(f);
}

/* Tensor: d0 = a0 b0, d1 = a0 b1 + a1 b0, d2 = a1 b1.  d layout [3][lv][N]. */
void or_tensor(const or_ctx *c, int lv, const u64 *a, const u64 *b, u64 *d) {
    int N = c->N;
    u64 *t0 = (u64 *)malloc(sizeof(u64) * N);
    for (int i = 0; i < lv; i++) {
        u64 q = c->prime[i];
        const u64 *a0 = a + (size_t)i * N, *a1 = a + ((size_t)lv + i) * N;
        const u64 *b0 = b + (size_t)i * N, *b1 = b + ((size_t)lv + i) * N;
        u64 *d0 = d + (size_t)i * N, *d1 = d + ((size_t)lv + i) * N, *d2 = d + ((size_t)2 * lv + i) * N;
        or_polymul(c, i, a0, b0, d0);
        or_polymul(c, i, a0, b1, d1);
        or_polymul(c, i, a1, b0, t0);
        for (int x = 0; x < N; x++) d1[x] = addmod(d1[x], t0[x], q);
        or_polymul(c, i, a1, b1, d2);
    }
    free(t0);
}

/* HE-Mult: tensor, then key switch of d2 with the relinearisation key
 * (s^2 -> s): out = (d0 + k0, d1 + k1). */
void or_mult_relin(const or_ctx *c, int lv, const u64 *a, const u64 *b, const u64 *rlk_eval, u64 *out) {
    int N = c->N;
    u64 *d = (u64 *)malloc(sizeof(u64) * (size_t)3 * lv * N);
    u64 *k = (u64 *)malloc(sizeof(u64) * (size_t)2 * lv * N);
    or_tensor(c, lv, a, b, d);
    or_keyswitch(c, lv, d + (size_t)2 * lv * N, rlk_eval, k);
    or_add(c, lv, 2, d, k, out);
    free(d);
    free(k);
}

/* BGV modulus switch from level lv to lv-1 (drops q_{lv-1}); the message is
 * multiplied by q_{lv-1}^-1 mod t.  out [2][lv-1][N]. */
void or_modswitch(const or_ctx *c, int lv, const u64 *ct, u64 *out) {
    int pidx[MAXP], N = c->N;
    for (int i = 0; i < lv; i++) pidx[i] = i;
    divide_round_t(c, lv, lv - 1, pidx, ct, out);
    divide_round_t(c, lv, lv - 1, pidx, ct + (size_t)lv * N, out + (size_t)(lv - 1) * N);
}

/* ------------------------------------------------------------------ */
/* Double-hoisted linear transformation (an evaluation order of         */
/* Eq. lintrans that defers ModDown to the sum):                        */
/*   y = ( ModDown( sum_d m_d (u0_d + P tau_d(c0)) ),                   */
/*         ModDown( sum_d m_d u1_d ) )                                  */
/* with u_d the inner product of the rotation by d before ModDown, and  */
/* the d = 0 term m_0 P c.  Everything below is over the extended basis */
/* of level lv (q_0..q_{lv-1}, p_0..p_{K-1}).                           */
/* ------------------------------------------------------------------ */

/* Hoisted key switch without its ModDown: D is the ModUp of c1 (or_modup
 * layout, coefficient form); the automorphism tau_g is applied to every
 * digit (skipped for g = 1, the relinearisation key), then the inner
 * product with evk.  u [2][lv+K][N] (coefficient form). */
void or_ks_raw(const or_ctx *c, int lv, const u64 *D, u64 g, const u64 *evk_eval, u64 *u) {
    int N = c->N, ne = lv + c->K, nd = digits_at(c, lv), pidx[MAXP];
    for (int e = 0; e < ne; e++) pidx[e] = ext_prime(c, lv, e);
    if (g == 1) { or_ks_inner(c, lv, D, evk_eval, u); return; }
    u64 *Dg = (u64 *)malloc(sizeof(u64) * (size_t)nd * ne * N);
    for (int j = 0; j < nd; j++) or_automorph(c, ne, pidx, D + (size_t)j * ne * N, g, Dg + (size_t)j * ne * N);
    or_ks_inner(c, lv, Dg, evk_eval, u);
    free(Dg);
}

/* P x on the chain primes, 0 on the special primes: out [lv+K][N]. */
void or_pq_lift(const or_ctx *c, int lv, const u64 *x, u64 *out) {
    int N = c->N, ne = lv + c->K;
    for (int e = 0; e < ne; e++) {
        u64 *o = out + (size_t)e * N;
        if (e >= lv) {
            for (int k = 0; k < N; k++) o[k] = 0;
            continue;
        }
        u64 q = c->prime[e], Pm = 1;
        for (int k = 0; k < c->K; k++) Pm = mulmod(Pm, c->prime[c->L + k] % q, q);
        for (int k = 0; k < N; k++) o[k] = mulmod(x[(size_t)e * N + k], Pm, q);
    }
}

/* acc += m * a over the extended basis; m_eval is or_ntt of the mask
 * residues over the extended primes (coefficient-form a and acc). */
void or_pq_mac(const or_ctx *c, int lv, const u64 *a, const u64 *m_eval, u64 *acc) {
    int N = c->N, ne = lv + c->K;
    u64 *f = (u64 *)malloc(sizeof(u64) * N);
    for (int e = 0; e < ne; e++) {
        int gp = ext_prime(c, lv, e);
        u64 q = c->prime[gp];
        memcpy(f, a + (size_t)e * N, sizeof(u64) * N);
        or_ntt(c, gp, f);
        for (int k = 0; k < N; k++) f[k] = mulmod(f[k], m_eval[(size_t)e * N + k], q);
        or_intt(c, gp, f);
        for (int k = 0; k < N; k++) acc[(size_t)e * N + k] = addmod(acc[(size_t)e * N + k], f[k], q);
    }
    free(f);
}

/* In-place forward / inverse NTT of np residue polynomials (global prime indices). */
void or_to_eval(const or_ctx *c, int np, const int *pidx, u64 *a) {
    for (int r = 0; r < np; r++) or_ntt(c, pidx[r], a + (size_t)r * c->N);
}

void or_to_coeff(const or_ctx *c, int np, const int *pidx, u64 *a) {
    for (int r = 0; r < np; r++) or_intt(c, pidx[r], a + (size_t)r * c->N);
}

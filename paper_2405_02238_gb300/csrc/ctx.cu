// ctx.cu -- context, tables, keys, encoding, encryption and decryption.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <set>

#include "device.cuh"
#include "internal.h"
#include "plan.h"

namespace hg {

typedef unsigned __int128 u128;

static u64 hmul(u64 a, u64 b, u64 q) { return (u64)((u128)a * b % q); }
static u64 hpow(u64 a, u64 e, u64 q) {
    u64 r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = hmul(r, a, q);
        a = hmul(a, a, q);
        e >>= 1;
    }
    return r;
}
static u64 hinv(u64 a, u64 q) { return hpow(a, q - 2, q); }
static u64 shoup(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

// Miller-Rabin, deterministic below 2^64 with these bases.
static bool is_prime(u64 n) {
    static const u64 B[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (u64 b : B) {
        if (n == b) return true;
        if (n % b == 0) return false;
    }
    u64 d = n - 1;
    int s = 0;
    while (!(d & 1)) {
        d >>= 1;
        s++;
    }
    for (u64 b : B) {
        u64 x = hpow(b, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int r = 1; r < s && comp; r++) {
            x = hmul(x, x, n);
            if (x == n - 1) comp = false;
        }
        if (comp) return false;
    }
    return true;
}

int set_err(Ctx *c, int code, const std::string &msg) {
    c->err = msg;
    return code;
}

int cuda_check(Ctx *c, const char *where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_err(c, HEGMM_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
    return HEGMM_OK;
}

u64 *dalloc(Ctx *c, size_t words) {
    return (u64 *)dalloc_evicting(c, std::max<size_t>(words, 1) * 8);
}

void dfree(Ctx *c, void *p) {
    if (p) cudaFreeAsync(p, c->st);
}

LimbPat pat_ct(Ctx *c, u64 *base, int npoly, int lv, long long poly_stride) {
    LimbPat p{};
    p.base = base;
    p.outer_ptrs = nullptr;
    p.outer_stride = poly_stride >= 0 ? poly_stride : (long long)lv * c->N;
    p.inner = lv;
    p.count = npoly * lv;
    for (int i = 0; i < lv; i++) {
        p.off[i] = (unsigned short)i;
        p.mod[i] = (unsigned char)i;
    }
    return p;
}

static LimbPat pat_mods(u64 *base, int n, const int *mods, int count_outer, long long stride) {
    LimbPat p{};
    p.base = base;
    p.outer_stride = stride;
    p.inner = n;
    p.count = n * count_outer;
    for (int i = 0; i < n; i++) {
        p.off[i] = (unsigned short)i;
        p.mod[i] = (unsigned char)mods[i];
    }
    return p;
}

// ---------------------------------------------------------------- tables

// ModUp conversion table of level lv (host copy): [nd][alpha] x {hinv,
// hinv_sh}, then [nd][alpha][ne] x {hat mod r, shoup, q_i mod r}, where
// hinv = (Q_j / q_i)^-1 mod q_i and hat = Q_j / q_i mod r for prime q_i of
// digit j and prime r of the extended basis.
std::vector<u64> modup_table_host(const Ctx *c, int lv) {
    const int ne = lv + c->K, nd = c->digits(lv), a = c->alpha;
    std::vector<u64> h((size_t)nd * a * 2 + (size_t)nd * a * ne * 3, 0);
    for (int j = 0; j < nd; j++) {
        const int lo = j * a, hi = std::min(lo + a, lv);
        for (int ii = 0; ii < hi - lo; ii++) {
            const int i = lo + ii;
            const u64 qi = c->q[i];
            u64 hat_qi = 1;
            for (int i2 = lo; i2 < hi; i2++)
                if (i2 != i) hat_qi = hmul(hat_qi, c->q[i2] % qi, qi);
            const u64 hi_inv = hinv(hat_qi, qi);
            h[((size_t)j * a + ii) * 2] = hi_inv;
            h[((size_t)j * a + ii) * 2 + 1] = shoup(hi_inv, qi);
            for (int e = 0; e < ne; e++) {
                const u64 r = c->q[c->gidx(lv, e)];
                u64 hat_r = 1;
                for (int i2 = lo; i2 < hi; i2++)
                    if (i2 != i) hat_r = hmul(hat_r, c->q[i2] % r, r);
                u64 *dst = &h[(size_t)nd * a * 2 + (((size_t)j * a + ii) * ne + e) * 3];
                dst[0] = hat_r;
                dst[1] = shoup(hat_r, r);
                dst[2] = qi % r;
            }
        }
    }
    // then [nd][alpha][ne] x {r - q_i mod 2^64}: the centred lift of a value
    // below q_i into [0, r) when q_i < 2 r (centred_narrow)
    for (int j = 0; j < nd; j++)
        for (int ii = 0; ii < a; ii++)
            for (int e = 0; e < ne; e++) {
                const int i = j * a + ii;
                h.push_back(i < lv ? c->q[c->gidx(lv, e)] - c->q[i] : 0);
            }
    return h;
}

// Exact-division table (host copy) and its modulus lists.  kind 0: ModDown
// at level lv (keep q_0..q_{lv-1}, drop the K special primes); kind 1:
// modulus switch from lv (keep q_0..q_{lv-2}, drop q_{lv-1}); kind 2: the
// ModDown of kind 0 with plain rounding (correction factor 1, BFV).  Layout:
// [ndrop] x {coef, coef_sh}; [nkeep][ndrop] x {hat, hat_sh, d_k mod q_i};
// [nkeep] x {Dinv, Dinv_sh, t mod q_i, shoup}; then keep[nkeep], drop[ndrop].
std::vector<u64> div_table_host(const Ctx *c, int lv, int kind, std::vector<int> &keep, std::vector<int> &drop) {
    keep.clear();
    drop.clear();
    const u64 tt = kind == 2 ? 1 : c->t;  // the rounding correction: t, or 1 for BFV's plain ModDown
    if (kind == 0 || kind == 2) {
        for (int i = 0; i < lv; i++) keep.push_back(i);
        for (int k = 0; k < c->K; k++) drop.push_back(c->L + k);
    } else {
        for (int i = 0; i < lv - 1; i++) keep.push_back(i);
        drop.push_back(lv - 1);
    }
    const int nkeep = (int)keep.size(), ndrop = (int)drop.size();
    std::vector<u64> h;
    for (int k = 0; k < ndrop; k++) {
        const u64 dk = c->q[drop[k]];
        u64 hat = 1;
        for (int k2 = 0; k2 < ndrop; k2++)
            if (k2 != k) hat = hmul(hat, c->q[drop[k2]] % dk, dk);
        const u64 coef = hmul(hinv(tt % dk, dk), hinv(hat, dk), dk);
        h.push_back(coef);
        h.push_back(shoup(coef, dk));
    }
    for (int i = 0; i < nkeep; i++) {
        const u64 qi = c->q[keep[i]];
        for (int k = 0; k < ndrop; k++) {
            u64 hat = 1;
            for (int k2 = 0; k2 < ndrop; k2++)
                if (k2 != k) hat = hmul(hat, c->q[drop[k2]] % qi, qi);
            h.push_back(hat);
            h.push_back(shoup(hat, qi));
            h.push_back(c->q[drop[k]] % qi);
        }
    }
    for (int i = 0; i < nkeep; i++) {
        const u64 qi = c->q[keep[i]];
        u64 D = 1;
        for (int k = 0; k < ndrop; k++) D = hmul(D, c->q[drop[k]] % qi, qi);
        const u64 Di = hinv(D, qi);
        h.push_back(Di);
        h.push_back(shoup(Di, qi));
        h.push_back(tt % qi);
        h.push_back(shoup(tt % qi, qi));
    }
    for (int i = 0; i < nkeep; i++) h.push_back((u64)keep[i]);
    for (int k = 0; k < ndrop; k++) h.push_back((u64)drop[k]);
    // then the fused kernel's [nkeep][ndrop] x {t (D/d_k) mod q_i, shoup,
    // q_i - d_k mod 2^64} (its conversion yields t y~ directly; the last
    // word lifts a value below d_k centred into [0, q_i) when d_k < 2 q_i)
    for (int i = 0; i < nkeep; i++) {
        const u64 qi = c->q[keep[i]];
        for (int k = 0; k < ndrop; k++) {
            u64 hat = 1;
            for (int k2 = 0; k2 < ndrop; k2++)
                if (k2 != k) hat = hmul(hat, c->q[drop[k2]] % qi, qi);
            const u64 ht = hmul(hat, tt % qi, qi);
            h.push_back(ht);
            h.push_back(shoup(ht, qi));
            h.push_back(qi - c->q[drop[k]]);
        }
    }
    return h;
}

int build_modup_tab(Ctx *c, int lv) {
    ModUpTab tb;
    tb.lv = lv;
    tb.ne = lv + c->K;
    tb.nd = c->digits(lv);
    const std::vector<u64> h = modup_table_host(c, lv);
    tb.ext = (size_t)tb.nd * c->alpha * 2 + (size_t)tb.nd * c->alpha * tb.ne * 3;
    tb.narrow = 1;
    for (int i = 0; i < lv; i++)
        for (int e = 0; e < tb.ne; e++)
            if (c->q[i] >= 2 * c->q[c->gidx(lv, e)]) tb.narrow = 0;
    tb.d = dalloc(c, h.size());
    if (!tb.d) return set_err(c, HEGMM_ENOMEM, "modup table");
    cudaMemcpyAsync(tb.d, h.data(), h.size() * 8, cudaMemcpyHostToDevice, c->st);
    cudaStreamSynchronize(c->st);
    c->modup[lv] = tb;
    return cuda_check(c, "modup table");
}

int build_div_tab(Ctx *c, int lv, int kind) {
    DivTab tb;
    const std::vector<u64> h = div_table_host(c, lv, kind, tb.keep, tb.drop);
    tb.nkeep = (int)tb.keep.size();
    tb.ndrop = (int)tb.drop.size();
    if (tb.ndrop > 4) return set_err(c, HEGMM_EINVAL, "at most 4 special primes");
    tb.ext = (size_t)2 * tb.ndrop + (size_t)3 * tb.nkeep * tb.ndrop + (size_t)5 * tb.nkeep + tb.ndrop;
    tb.narrow = 1;
    for (int k : tb.drop)
        for (int i : tb.keep)
            if (c->q[k] >= 2 * c->q[i]) tb.narrow = 0;
    tb.d = dalloc(c, h.size());
    if (!tb.d) return set_err(c, HEGMM_ENOMEM, "div table");
    cudaMemcpyAsync(tb.d, h.data(), h.size() * 8, cudaMemcpyHostToDevice, c->st);
    cudaStreamSynchronize(c->st);
    c->divs[{lv, kind}] = tb;
    return cuda_check(c, "div table");
}

// BFV constants (layout: BfvTab in internal.h).
static int build_bfv_tab(Ctx *c) {
    const int nq = c->L, nb = c->nb;
    BfvTab &T = c->bt;
    size_t w = 0;
    auto take = [&](size_t n) {
        size_t o = w;
        w += n;
        return o;
    };
    T.qt = take(2 * nq);
    T.tt = take(nq);
    T.qd = take(nq);
    T.qbm = take((size_t)nq * nb);
    T.qb = take(nb);
    T.qim = take((size_t)nq * nb);
    T.qib = take(2 * nb);
    T.tb = take(2 * nb);
    T.bt = take(2 * nb);
    T.bd = take(nb);
    T.bqm = take((size_t)nb * nq);
    T.bq = take(nq);
    T.dl = take(2 * nq);
    T.words = w;
    std::vector<u64> h(w, 0);
    auto qv = [&](int i) { return c->q[i]; };            // chain prime i
    auto bv = [&](int j) { return c->q[c->b0 + j]; };    // auxiliary prime j
    auto r64 = [&](u64 m) { return (u64)(((u128)1 << 64) % m); };
    auto dbits = [](double d) {
        u64 b;
        memcpy(&b, &d, 8);
        return b;
    };
    const u64 t = c->t;
    u64 Qt = 1;  // Q mod t
    for (int i = 0; i < nq; i++) Qt = hmul(Qt, qv(i) % t, t);
    for (int i = 0; i < nq; i++) {
        const u64 qi = qv(i);
        u64 hat = 1;
        for (int i2 = 0; i2 < nq; i2++)
            if (i2 != i) hat = hmul(hat, qv(i2) % qi, qi);
        const u64 hi = hinv(hat, qi);
        h[T.qt + 2 * i] = hi;
        h[T.qt + 2 * i + 1] = shoup(hi, qi);
        h[T.tt + i] = (u64)(((u128)t << 64) / qi);
        h[T.qd + i] = dbits(1.0 / (double)qi);
        u64 Bq = 1;
        for (int j = 0; j < nb; j++) Bq = hmul(Bq, bv(j) % qi, qi);
        h[T.bq + i] = Bq;
        // Delta = (Q - (Q mod t)) / t, so Delta mod q_i = -(Q mod t) t^-1 mod q_i
        const u64 dl = hmul((qi - Qt % qi) % qi, hinv(t % qi, qi), qi);
        h[T.dl + 2 * i] = dl;
        h[T.dl + 2 * i + 1] = shoup(dl, qi);
    }
    for (int j = 0; j < nb; j++) {
        const u64 bj = bv(j), r1 = r64(bj);
        u64 Qb = 1;
        for (int i = 0; i < nq; i++) Qb = hmul(Qb, qv(i) % bj, bj);
        h[T.qb + j] = Qb;
        const u64 Qi = hinv(Qb, bj);
        h[T.qib + 2 * j] = Qi;
        h[T.qib + 2 * j + 1] = shoup(Qi, bj);
        h[T.tb + 2 * j] = t % bj;
        h[T.tb + 2 * j + 1] = shoup(t % bj, bj);
        for (int i = 0; i < nq; i++) {
            u64 hat = 1;  // Q / q_i mod b_j
            for (int i2 = 0; i2 < nq; i2++)
                if (i2 != i) hat = hmul(hat, qv(i2) % bj, bj);
            h[T.qbm + (size_t)i * nb + j] = hmul(hat, r1, bj);
            h[T.qim + (size_t)i * nb + j] = hmul(hinv(qv(i) % bj, bj), r1, bj);
        }
        u64 hatb = 1;  // B / b_j mod b_j
        for (int j2 = 0; j2 < nb; j2++)
            if (j2 != j) hatb = hmul(hatb, bv(j2) % bj, bj);
        const u64 bt = hinv(hatb, bj);
        h[T.bt + 2 * j] = bt;
        h[T.bt + 2 * j + 1] = shoup(bt, bj);
        h[T.bd + j] = dbits(1.0 / (double)bj);
        for (int i = 0; i < nq; i++) {
            const u64 qi = qv(i);
            u64 hb = 1;  // B / b_j mod q_i
            for (int j2 = 0; j2 < nb; j2++)
                if (j2 != j) hb = hmul(hb, bv(j2) % qi, qi);
            h[T.bqm + (size_t)j * nq + i] = hmul(hb, r64(qi), qi);
        }
    }
    c->d_bfv = dalloc(c, w);
    if (!c->d_bfv) return set_err(c, HEGMM_ENOMEM, "BFV tables");
    cudaMemcpyAsync(c->d_bfv, h.data(), w * 8, cudaMemcpyHostToDevice, c->st);
    cudaStreamSynchronize(c->st);
    return cuda_check(c, "BFV tables");
}

// ---------------------------------------------------------------- context

static int ctx_init(Ctx *c, const hegmm_params *p, void *stream) {
    c->prm = *p;
    c->logN = p->logN;
    c->N = 1 << p->logN;
    c->S = c->N / 2;
    c->L = p->L;
    c->K = p->K;
    c->alpha = p->alpha;
    c->t = p->t;
    c->st = (cudaStream_t)stream;
    if (p->logN < 10 || p->logN > 14 || p->L < 2 || p->K < 1 || p->L + p->K > 24 || p->qbits < 20 || p->qbits > 56 ||
        p->alpha < 1 || p->alpha > 4 || p->L % p->alpha != 0 || p->K < p->alpha || p->K > 4 || p->eta < 1 ||
        p->eta > 31 || p->ms_drop < 0 || p->ms_drop > 1 || (p->ms_drop && p->L < 3))
        return set_err(c, HEGMM_EINVAL, "parameters outside the supported limits");
    // ModUp's new limbs of one ciphertext form one limb pattern (pat_nonown)
    if ((p->L / p->alpha) * (p->L + p->K) - p->L > PAT_MAX)
        return set_err(c, HEGMM_EINVAL,
                       "parameters outside the supported limits: digits(L) (L + K) - L ModUp limbs exceed " +
                           std::to_string(PAT_MAX));
    const u64 two_n = 2 * (u64)c->N;
    if (!is_prime(p->t) || (p->t - 1) % two_n != 0) return set_err(c, HEGMM_EINVAL, "t must be a prime = 1 mod 2N");
    if (p->scheme != HEGMM_SCHEME_BGV && p->scheme != HEGMM_SCHEME_BFV)
        return set_err(c, HEGMM_EINVAL, "scheme must be HEGMM_SCHEME_BGV or HEGMM_SCHEME_BFV");
    c->bfv = p->scheme == HEGMM_SCHEME_BFV;
    if (c->bfv && p->ms_drop) return set_err(c, HEGMM_EINVAL, "the BFV variant has no modulus switch (ms_drop = 0)");
    c->dnum = p->L / p->alpha;
    c->np = p->L + p->K;
    c->tmod = c->np;
    c->nb = c->bfv ? p->L + 2 : 0;
    c->b0 = c->np + 1;
    c->nmod = c->np + 1 + c->nb;
    if (c->nmod > MAXM) return set_err(c, HEGMM_EINVAL, "too many primes (BFV: 2 L + K + 3 <= 25)");
    // primes: largest below 2^qbits, = 1 mod 2N, descending: chain, special,
    // then (BFV) the auxiliary base, which sits after t in q[]
    u64 cand = ((((u64)1 << p->qbits) - 1) / two_n) * two_n + 1;
    if (cand >= ((u64)1 << p->qbits)) cand -= two_n;
    int got = 0;
    while (got < c->np + c->nb && cand > two_n) {
        if (is_prime(cand) && cand != p->t) c->q[got < c->np ? got : got + 1] = cand, got++;
        cand -= two_n;
    }
    if (got != c->np + c->nb) return set_err(c, HEGMM_EINVAL, "not enough NTT primes");
    // the key inner product sums dnum products (+ one folded term) below q 2^64 before one reduction
    if ((u128)(c->dnum + 2) * c->q[0] >= ((u128)1 << 64))
        return set_err(c, HEGMM_EINVAL, "primes too large for dnum: (dnum + 2) q must stay below 2^64");
    c->q[c->tmod] = p->t;
    for (int i = 0; i < c->nmod; i++) {
        const u64 q = c->q[i];
        u64 psi = 0;
        if (i == c->tmod) {
            psi = hpow(3, (q - 1) / two_n, q);  // zeta: fixes the slot order
        } else {
            for (u64 g = 2; g < q; g++) {
                u64 w = hpow(g, (q - 1) / two_n, q);
                if (hpow(w, (u64)c->N, q) == q - 1) {
                    psi = w;
                    break;
                }
            }
        }
        if (hpow(psi, (u64)c->N, q) != q - 1) return set_err(c, HEGMM_EINVAL, "no primitive 2N-th root");
        c->psi[i] = psi;
        ModDev &M = c->hmod[i];
        M.q = q;
        u64 inv = 1;  // Newton: q^-1 mod 2^64
        for (int k = 0; k < 7; k++) inv *= 2 - q * inv;
        M.qinv = inv;
        const u64 r1 = (u64)(((u128)1 << 64) % q);
        M.r2 = hmul(r1, r1, q);
        M.barr = (u64)(((u128)1 << 64) / q);
        M.ninv = hinv((u64)c->N % q, q);
        M.ninv_sh = shoup(M.ninv, q);
        M.tq = p->t % q;
        M.tq_sh = shoup(M.tq, q);
        u64 P = 1;
        for (int k = 0; k < p->K; k++) P = hmul(P, c->q[p->L + k] % q, q);
        M.pR = (i >= p->L && i < p->L + p->K) ? 0 : hmul(P, r1, q);  // r1 = 2^64 mod q
        M.pad = 0;
    }
    cudaDeviceProp prop;
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) c->nsm = prop.multiProcessorCount;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        u64 thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    // twiddles: [modulus][forward, inverse, inverse output factor][N] pairs
    const int N = c->N;
    std::vector<u64> tw((size_t)c->nmod * 6 * N);
    for (int m = 0; m < c->nmod; m++) build_twiddles_host(c->q[m], c->psi[m], c->logN, &tw[(size_t)m * 6 * N]);
    c->d_tw = dalloc(c, tw.size());
    void *dm = nullptr;
    if (cudaMallocAsync(&dm, sizeof(ModDev) * c->nmod, c->st) != cudaSuccess || !c->d_tw)
        return set_err(c, HEGMM_ENOMEM, "tables");
    c->d_mods = (ModDev *)dm;
    void *de = nullptr;
    if (cudaMallocAsync(&de, sizeof(int), c->st) != cudaSuccess) return set_err(c, HEGMM_ENOMEM, "error flag");
    c->d_err = (int *)de;
    cudaMemsetAsync(c->d_err, 0, sizeof(int), c->st);
    cudaMemcpyAsync(c->d_tw, tw.data(), tw.size() * 8, cudaMemcpyHostToDevice, c->st);
    cudaMemcpyAsync(c->d_mods, c->hmod, sizeof(ModDev) * c->nmod, cudaMemcpyHostToDevice, c->st);
    cudaStreamSynchronize(c->st);
    int rc = cuda_check(c, "context tables");
    if (rc) return rc;
    rc = init_kernels(c);
    if (rc) return rc;
    c->slot_pos0.resize(c->S);
    c->slot_pos1.resize(c->S);
    u64 g = 1;
    for (int j = 0; j < c->S; j++) {
        c->slot_pos0[j] = (int)brev_bits((u32)((g - 1) / 2), c->logN);
        const u64 ng = two_n - g;
        c->slot_pos1[j] = (int)brev_bits((u32)((ng - 1) / 2), c->logN);
        g = g * 5 % two_n;
    }
    std::vector<int> both(c->slot_pos0);
    both.insert(both.end(), c->slot_pos1.begin(), c->slot_pos1.end());
    c->d_slot_pos = upload(c, both);
    if (!c->d_slot_pos) return set_err(c, HEGMM_ENOMEM, "slot table");
    cudaStreamSynchronize(c->st);
    if (int rc = cuda_check(c, "slot table")) return rc;
    return c->bfv ? build_bfv_tab(c) : HEGMM_OK;
}

u64 galois_of(Ctx *c, long long z) {
    long long zz = z % c->S;
    if (zz < 0) zz += c->S;
    u64 g = 1;
    const u64 two_n = 2 * (u64)c->N;
    for (long long i = 0; i < zz; i++) g = g * 5 % two_n;
    return g;
}

// ---------------------------------------------------------------- keys

static u64 *g_Pmod_dev(Ctx *c) {
    if (c->d_Pmod) return c->d_Pmod;
    std::vector<u64> h(2 * c->np);
    for (int i = 0; i < c->np; i++) {
        const u64 q = c->q[i];
        u64 P = 1;
        for (int k = 0; k < c->K; k++) P = hmul(P, c->q[c->L + k] % q, q);
        h[2 * i] = P;
        h[2 * i + 1] = shoup(P, q);
    }
    u64 *d = dalloc(c, h.size());
    cudaMemcpyAsync(d, h.data(), h.size() * 8, cudaMemcpyHostToDevice, c->st);
    cudaStreamSynchronize(c->st);
    c->d_Pmod = d;
    return d;
}

int key_digit_combine(Ctx *c, u64 *kb, u64 *ka, const u64 *sprime, const u64 *d_Pmod, int lo, int hi);

static int gen_key(Ctx *c, u64 g) {
    if (c->keys.count(g)) return HEGMM_OK;
    const int N = c->N, np = c->np;
    u64 *key = dalloc(c, c->key_words());
    u64 *sp = dalloc(c, (size_t)np * N);
    if (!key || !sp) {
        dfree(c, key);
        dfree(c, sp);
        return set_err(c, HEGMM_ENOMEM, "key allocation");
    }
    int rc;
    if (g == 0) rc = pw_mont(c, np, 1, c->d_s, c->d_sR, 1, sp);  // s^2
    else rc = permute_limbs(c, np, c->d_s, sp, (u32)g);        // tau_g(s)
    if (rc) return rc;
    std::vector<int> mods(np);
    for (int i = 0; i < np; i++) mods[i] = i;
    const u64 *Pm = g_Pmod_dev(c);
    for (int j = 0; j < c->dnum; j++) {
        u64 *kb = key + ((size_t)j * 2 + 0) * np * N;
        u64 *ka = key + ((size_t)j * 2 + 1) * np * N;
        LimbPat pa = pat_mods(ka, np, mods.data(), 1, 0), pb = pat_mods(kb, np, mods.data(), 1, 0);
        if ((rc = sample_uniform(c, pa, rng_stream(c->key_seed, DOM_KEY_A, g * 256 + (u64)j), nullptr))) return rc;
        const u64 est = rng_stream(c->key_seed, DOM_KEY_E, g * 256 + (u64)j);
        if ((rc = c->bfv ? sample_cbd(c, pb, est, c->prm.eta) : sample_cbd_t(c, pb, est, c->prm.eta))) return rc;
        if ((rc = ntt_fwd(c, pa))) return rc;
        if ((rc = ntt_fwd(c, pb))) return rc;
        if ((rc = key_digit_combine(c, kb, ka, sp, Pm, j * c->alpha, std::min((j + 1) * c->alpha, c->L)))) return rc;
    }
    dfree(c, sp);
    c->keys[g] = key;
    return HEGMM_OK;
}

int ensure_galois_key(Ctx *c, u64 g) {
    if (c->keys.count(g)) return HEGMM_OK;  // generated or imported
    if (!c->have_sk) return set_err(c, HEGMM_ENOKEY, "missing key and no secret key to make it");
    return gen_key(c, g);
}

static void free_keys(Ctx *c) {
    for (auto &kv : c->keys) dfree(c, kv.second);
    c->keys.clear();
    dfree(c, c->d_s);
    dfree(c, c->d_sR);
    c->d_s = c->d_sR = nullptr;
    c->have_sk = false;
}

static int gen_secret(Ctx *c, u64 seed) {
    free_keys(c);
    free_plans(c);
    const int N = c->N, np = c->np;
    c->d_s = dalloc(c, (size_t)np * N);
    c->d_sR = dalloc(c, (size_t)np * N);
    if (!c->d_s || !c->d_sR) return set_err(c, HEGMM_ENOMEM, "secret key");
    std::vector<int> mods(np);
    for (int i = 0; i < np; i++) mods[i] = i;
    LimbPat ps = pat_mods(c->d_s, np, mods.data(), 1, 0);
    int rc;
    if ((rc = sample_ternary(c, ps, rng_stream(seed, DOM_SK, 0)))) return rc;
    if ((rc = ntt_fwd(c, ps))) return rc;
    cudaMemcpyAsync(c->d_sR, c->d_s, (size_t)np * N * 8, cudaMemcpyDeviceToDevice, c->st);
    if ((rc = pw_to_mont(c, pat_mods(c->d_sR, np, mods.data(), 1, 0)))) return rc;
    c->key_seed = seed;
    c->have_sk = true;
    return gen_key(c, 0);
}

// ---------------------------------------------------------------- ciphertext handles

hegmm_ct *new_ct(Ctx *c, int level) {
    hegmm_ct *ct = new hegmm_ct;
    ct->ctx = c;
    ct->level = level;
    ct->d = dalloc(c, (size_t)2 * level * c->N);
    if (!ct->d) {
        delete ct;
        return nullptr;
    }
    return ct;
}

static hegmm_pt *new_pt(Ctx *c) {
    hegmm_pt *pt = new hegmm_pt;
    pt->ctx = c;
    pt->level = c->L;
    pt->d = dalloc(c, (size_t)c->L * c->N);
    pt->d_mont = dalloc(c, (size_t)c->L * c->N);
    if (!pt->d || !pt->d_mont) {
        dfree(c, pt->d);
        dfree(c, pt->d_mont);
        delete pt;
        return nullptr;
    }
    return pt;
}

// slot vector (count values mod t: slots 0..S-1 of row 0, then row 1) ->
// plaintext (NTT domain over q_0..q_{L-1})
static int encode_slots(Ctx *c, const u64 *slots, int count, hegmm_pt **out) {
    if (count < 0 || count > c->N) return set_err(c, HEGMM_ESHAPE, "more values than slots");
    const int N = c->N, L = c->L, S = c->S;
    std::vector<u64> ev(N, 0);
    for (int j = 0; j < count; j++) ev[j < S ? c->slot_pos0[j] : c->slot_pos1[j - S]] = slots[j] % c->t;
    u64 *m = dalloc(c, N);
    hegmm_pt *pt = new_pt(c);
    if (!m || !pt) return set_err(c, HEGMM_ENOMEM, "encode");
    cudaMemcpyAsync(m, ev.data(), (size_t)N * 8, cudaMemcpyHostToDevice, c->st);
    int tm = c->tmod, rc;
    LimbPat pm = pat_mods(m, 1, &tm, 1, 0);
    if ((rc = ntt_inv(c, pm))) return rc;  // coefficients mod t
    if ((rc = lift_from_t(c, L, m, pt->d))) return rc;
    if ((rc = ntt_fwd(c, pat_ct(c, pt->d, 1, L)))) return rc;
    cudaMemcpyAsync(pt->d_mont, pt->d, (size_t)L * N * 8, cudaMemcpyDeviceToDevice, c->st);
    if ((rc = pw_to_mont(c, pat_ct(c, pt->d_mont, 1, L)))) return rc;
    cudaStreamSynchronize(c->st);  // ev is a stack buffer
    dfree(c, m);
    *out = pt;
    return cuda_check(c, "encode");
}

static int encrypt(Ctx *c, const hegmm_pt *pt, u64 seed, u64 sid, hegmm_ct **out) {
    if (!c->have_sk) return set_err(c, HEGMM_ENOKEY, "no secret key: call hegmm_keygen first");
    const int L = c->L;
    hegmm_ct *ct = new_ct(c, L);
    if (!ct) return set_err(c, HEGMM_ENOMEM, "encrypt");
    LimbPat p0 = pat_ct(c, ct->d, 1, L), p1 = pat_ct(c, ct->d + (size_t)L * c->N, 1, L);
    int rc;
    if ((rc = sample_uniform(c, p1, rng_stream(seed, DOM_ENC_A, sid), nullptr))) return rc;
    const u64 est = rng_stream(seed, DOM_ENC_E, sid);
    if ((rc = c->bfv ? sample_cbd(c, p0, est, c->prm.eta) : sample_cbd_t(c, p0, est, c->prm.eta))) return rc;
    if ((rc = ntt_fwd(c, pat_ct(c, ct->d, 2, L)))) return rc;
    if ((rc = encrypt_combine(c, L, ct->d, pt->d))) return rc;
    *out = ct;
    return HEGMM_OK;
}

static const u64 *crt_tab(Ctx *c, int lv) {
    auto it = c->crt.find(lv);
    if (it != c->crt.end()) return it->second;
    std::vector<u64> h(4 * lv + 1);
    u64 Qt = 1;
    for (int i = 0; i < lv; i++) Qt = hmul(Qt, c->q[i] % c->t, c->t);
    for (int i = 0; i < lv; i++) {
        const u64 qi = c->q[i];
        u64 hat = 1, hat_t = 1;
        for (int i2 = 0; i2 < lv; i2++)
            if (i2 != i) {
                hat = hmul(hat, c->q[i2] % qi, qi);
                hat_t = hmul(hat_t, c->q[i2] % c->t, c->t);
            }
        const u64 hi = hinv(hat, qi);
        h[4 * i] = hi;
        h[4 * i + 1] = shoup(hi, qi);
        h[4 * i + 2] = hat_t;
        double dq = (double)qi;
        memcpy(&h[4 * i + 3], &dq, 8);
    }
    h[4 * lv] = Qt;
    u64 *d = dalloc(c, h.size());
    cudaMemcpyAsync(d, h.data(), h.size() * 8, cudaMemcpyHostToDevice, c->st);
    cudaStreamSynchronize(c->st);
    c->crt[lv] = d;
    return d;
}

// all row-0 slots of a ciphertext
static int decrypt_slots(Ctx *c, const hegmm_ct *ct, std::vector<u64> &slots) {
    if (!c->have_sk) return set_err(c, HEGMM_ENOKEY, "no secret key");
    const int lv = ct->level, N = c->N;
    u64 *v = dalloc(c, (size_t)lv * N + N);
    if (!v) return set_err(c, HEGMM_ENOMEM, "decrypt");
    u64 *m = v + (size_t)lv * N;
    int rc;
    if ((rc = decrypt_dot(c, lv, ct->d, v))) return rc;
    if ((rc = ntt_inv(c, pat_ct(c, v, 1, lv)))) return rc;
    if (c->bfv) {
        if (lv != c->L) return set_err(c, HEGMM_EINVAL, "BFV ciphertexts are at the top level");
        if ((rc = bfv_decode(c, v, m))) return rc;  // round(t v / Q) mod t
    } else if ((rc = crt_to_t(c, lv, v, crt_tab(c, lv), m))) {
        return rc;
    }
    int tm = c->tmod;
    if ((rc = ntt_fwd(c, pat_mods(m, 1, &tm, 1, 0)))) return rc;
    std::vector<u64> ev(N);
    cudaMemcpyAsync(ev.data(), m, (size_t)N * 8, cudaMemcpyDeviceToHost, c->st);
    dfree(c, v);
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_check(c, "decrypt");
    if ((rc = device_status(c))) return rc;
    slots.resize(c->N);  // row 0, then row 1
    for (int j = 0; j < c->S; j++) {
        slots[j] = ev[c->slot_pos0[j]];
        slots[c->S + j] = ev[c->slot_pos1[j]];
    }
    return cuda_check(c, "decrypt");
}

// HEGMM_ETIMEOUT if a kernel's bounded wait ran out since the last check
// (the flag is cleared); synchronises the stream.
int device_status(Ctx *c) {
    if (!c->d_err) return HEGMM_OK;
    int v = 0;
    if (cudaMemcpyAsync(&v, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
        cudaStreamSynchronize(c->st) != cudaSuccess)
        return cuda_check(c, "status");
    if (!v) return HEGMM_OK;
    cudaMemsetAsync(c->d_err, 0, sizeof(int), c->st);
    return set_err(c, HEGMM_ETIMEOUT, "a kernel's bounded wait for its staged copies ran out; its results are invalid");
}

}  // namespace hg

using namespace hg;

// =================================================================== C ABI

extern "C" {

int hegmm_ctx_create(const hegmm_params *params, void *cuda_stream, hegmm_ctx **out) {
    if (!params || !out) return HEGMM_EINVAL;
    hegmm_ctx *h = new hegmm_ctx;
    int rc = ctx_init(&h->c, params, cuda_stream);
    if (rc) {
        // keep the message reachable only through the return code
        delete h;
        *out = nullptr;
        return rc;
    }
    *out = h;
    return HEGMM_OK;
}

void hegmm_ctx_destroy(hegmm_ctx *h) {
    if (!h) return;
    Ctx *c = &h->c;
    for (cudaStream_t s : c->par_st)
        if (s) cudaStreamSynchronize(s);  // sub-batch plans ran there
    free_plans(c);
    free_keys(c);
    for (auto &kv : c->modup) dfree(c, kv.second.d);
    for (auto &kv : c->divs) dfree(c, kv.second.d);
    for (auto &kv : c->crt) dfree(c, kv.second);
    dfree(c, c->d_Pmod);
    dfree(c, c->d_bfv);
    dfree(c, c->d_slot_pos);
    dfree(c, c->d_tw);
    dfree(c, c->d_mods);
    dfree(c, c->d_err);
    cudaStreamSynchronize(c->st);
    for (auto &p : c->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : c->evpool) cudaEventDestroy(e);
    for (cudaStream_t s : c->par_st)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : c->par_ev)
        if (e) cudaEventDestroy(e);
    delete h;
}

const char *hegmm_last_error(const hegmm_ctx *h) { return h ? h->c.err.c_str() : "no context"; }

int hegmm_get_primes(const hegmm_ctx *h, uint64_t *out) {
    if (!h || !out) return HEGMM_EINVAL;
    for (int i = 0; i < h->c.np; i++) out[i] = h->c.q[i];
    return HEGMM_OK;
}

int hegmm_keygen(hegmm_ctx *h, uint64_t seed, const int *mln, int n_shapes, int alg) {
    if (!h || (n_shapes > 0 && !mln)) return HEGMM_EINVAL;
    Ctx *c = &h->c;
    int rc;
    if (!c->have_sk || c->key_seed != seed) {
        if ((rc = gen_secret(c, seed))) return rc;
    }
    if (c->key_pow2) {
        // only the +-2^i rotations: every rotation of a product is a chain of them
        for (int s = 0; s < n_shapes; s++)
            if (!resolve_alg(mln[3 * s], mln[3 * s + 1], mln[3 * s + 2], alg, c->S))
                return set_err(c, HEGMM_ESHAPE, "shape does not fit one slot row");
        for (int z : pow2_offsets(c->S))
            if ((rc = gen_key(c, galois_of(c, z)))) return rc;
        return cuda_check(c, "keygen");
    }
    for (int s = 0; s < n_shapes; s++) {
        const int m = mln[3 * s], l = mln[3 * s + 1], n = mln[3 * s + 2];
        const int a = resolve_alg(m, l, n, alg, c->S);
        if (!a) return set_err(c, HEGMM_ESHAPE, "shape does not fit one slot row");
        HostPlan P = make_host_plan(m, l, n, a);
        std::set<u64> gs;
        for (auto &it : P.iters) {
            for (auto &d : it.eps)
                if (d.d % c->S) gs.insert(galois_of(c, d.d));
            for (auto &d : it.omg)
                if (d.d % c->S) gs.insert(galois_of(c, d.d));
        }
        for (int z : P.extract)
            if (z % c->S) gs.insert(galois_of(c, z));
        // the offsets of the shared-baby-step evaluation order as well
        for (int s2 = 0; s2 < 2; s2++)
            for (const GiantLT &f : giant_factor_of(P, s2, c->S)) {
                if (f.g) gs.insert(galois_of(c, f.g));
                for (const GTerm &t : f.terms)
                    if (t.b) gs.insert(galois_of(c, t.b));
            }
        for (u64 g : gs)
            if ((rc = gen_key(c, g))) return rc;
    }
    return cuda_check(c, "keygen");
}

int hegmm_set_key_policy(hegmm_ctx *h, int policy) {
    if (!h) return HEGMM_EINVAL;
    Ctx *c = &h->c;
    if (policy != HEGMM_KEYS_DIRECT && policy != HEGMM_KEYS_POW2)
        return set_err(c, HEGMM_EINVAL, "key policy must be HEGMM_KEYS_DIRECT or HEGMM_KEYS_POW2");
    c->key_pow2 = policy == HEGMM_KEYS_POW2;
    if (c->key_pow2 && c->have_sk)
        for (int z : pow2_offsets(c->S))
            if (int rc = gen_key(c, galois_of(c, z))) return rc;
    return cuda_check(c, "key policy");
}

int hegmm_keygen_rotations(hegmm_ctx *h, const int *z, int count) {
    if (!h || (count > 0 && !z)) return HEGMM_EINVAL;
    Ctx *c = &h->c;
    for (int i = 0; i < count; i++) {
        if (z[i] % c->S == 0) continue;
        int rc = ensure_galois_key(c, galois_of(c, z[i]));
        if (rc) return rc;
    }
    return HEGMM_OK;
}

int hegmm_key_export(hegmm_ctx *h, uint64_t which, uint64_t *host) {
    if (!h || !host) return HEGMM_EINVAL;
    Ctx *c = &h->c;
    auto it = c->keys.find(which);
    if (it == c->keys.end()) return set_err(c, HEGMM_ENOKEY, "no such key");
    const size_t w = c->key_words();
    u64 *tmp = dalloc(c, w);
    if (!tmp) return set_err(c, HEGMM_ENOMEM, "key export");
    cudaMemcpyAsync(tmp, it->second, w * 8, cudaMemcpyDeviceToDevice, c->st);
    std::vector<int> mods(c->np);
    for (int i = 0; i < c->np; i++) mods[i] = i;
    LimbPat p = pat_mods(tmp, c->np, mods.data(), 2 * c->dnum, (long long)c->np * c->N);
    int rc;
    if ((rc = pw_from_mont(c, p))) return rc;
    if ((rc = ntt_inv(c, p))) return rc;
    cudaMemcpyAsync(host, tmp, w * 8, cudaMemcpyDeviceToHost, c->st);
    dfree(c, tmp);
    cudaStreamSynchronize(c->st);
    return cuda_check(c, "key export");
}

int hegmm_key_import(hegmm_ctx *h, uint64_t which, const uint64_t *host) {
    if (!h || !host) return HEGMM_EINVAL;
    Ctx *c = &h->c;
    if (which != 0 && (which % 2 == 0 || which >= (uint64_t)2 * c->N))
        return set_err(c, HEGMM_EINVAL, "which must be 0 or an odd Galois element below 2N");
    const size_t w = c->key_words();
    for (size_t i = 0; i < w; i++) {
        const int limb = (int)((i / c->N) % c->np);
        if (host[i] >= c->q[limb]) return set_err(c, HEGMM_EINVAL, "key residue not below its prime");
    }
    auto it = c->keys.find(which);
    u64 *key = it != c->keys.end() ? it->second : dalloc(c, w);  // in place: cached plans keep their pointers
    if (!key) return set_err(c, HEGMM_ENOMEM, "key import");
    cudaMemcpyAsync(key, host, w * 8, cudaMemcpyHostToDevice, c->st);
    std::vector<int> mods(c->np);
    for (int i = 0; i < c->np; i++) mods[i] = i;
    LimbPat p = pat_mods(key, c->np, mods.data(), 2 * c->dnum, (long long)c->np * c->N);
    int rc;
    if (!(rc = ntt_fwd(c, p))) rc = pw_to_mont(c, p);
    if (rc) {
        if (it == c->keys.end()) dfree(c, key);
        return rc;
    }
    c->keys[which] = key;
    cudaStreamSynchronize(c->st);  // the host buffer may be reused once this returns
    return cuda_check(c, "key import");
}

int hegmm_key_list(hegmm_ctx *h, uint64_t *which, int cap, int *count) {
    if (!h || !count || (cap > 0 && !which)) return HEGMM_EINVAL;
    int k = 0;
    for (auto &kv : h->c.keys) {
        if (k < cap) which[k] = kv.first;
        k++;
    }
    *count = k;
    return HEGMM_OK;
}

int hegmm_encode(hegmm_ctx *h, int role, const int64_t *mat, int m, int l, int n, int alg, hegmm_pt **out) {
    if (!h || !mat || !out || (role != 0 && role != 1)) return HEGMM_EINVAL;
    Ctx *c = &h->c;
    const int a = resolve_alg(m, l, n, alg, c->S);
    if (!a) return set_err(c, HEGMM_ESHAPE, "shape does not fit one slot row");
    HostPlan P = make_host_plan(m, l, n, a);
    std::vector<u64> v = role == 0 ? P.a_slots(mat, c->t) : P.b_slots(mat, c->t);
    return encode_slots(c, v.data(), (int)v.size(), out);
}

int hegmm_encode_pair(hegmm_ctx *h, int role, const int64_t *mat0, const int64_t *mat1, int m, int l, int n, int alg,
                      hegmm_pt **out) {
    if (!h || !mat0 || !out || (role != 0 && role != 1)) return HEGMM_EINVAL;
    Ctx *c = &h->c;
    const int a = resolve_alg(m, l, n, alg, c->S);
    if (!a) return set_err(c, HEGMM_ESHAPE, "shape does not fit one slot row");
    HostPlan P = make_host_plan(m, l, n, a);
    std::vector<u64> v = role == 0 ? P.a_slots(mat0, c->t) : P.b_slots(mat0, c->t);
    v.resize(c->S, 0);
    if (mat1) {
        const std::vector<u64> w = role == 0 ? P.a_slots(mat1, c->t) : P.b_slots(mat1, c->t);
        v.insert(v.end(), w.begin(), w.end());
    }
    return encode_slots(c, v.data(), (int)v.size(), out);
}

int hegmm_encode_slots(hegmm_ctx *h, const uint64_t *slots, int count, hegmm_pt **out) {
    if (!h || (!slots && count) || !out) return HEGMM_EINVAL;
    return encode_slots(&h->c, slots, count, out);
}

int hegmm_encrypt(hegmm_ctx *h, const hegmm_pt *pt, uint64_t seed, uint64_t sid, hegmm_ct **out) {
    if (!h || !pt || !out) return HEGMM_EINVAL;
    return encrypt(&h->c, pt, seed, sid, out);
}

int hegmm_decrypt_slots(hegmm_ctx *h, const hegmm_ct *ct, uint64_t *out) {
    if (!h || !ct || !out) return HEGMM_EINVAL;
    std::vector<u64> s;
    int rc = decrypt_slots(&h->c, ct, s);
    if (rc) return rc;
    memcpy(out, s.data(), (size_t)h->c.S * 8);
    return HEGMM_OK;
}

int hegmm_decrypt_rows(hegmm_ctx *h, const hegmm_ct *ct, uint64_t *out) {
    if (!h || !ct || !out) return HEGMM_EINVAL;
    std::vector<u64> s;
    int rc = decrypt_slots(&h->c, ct, s);
    if (rc) return rc;
    memcpy(out, s.data(), s.size() * 8);
    return HEGMM_OK;
}

int hegmm_decrypt(hegmm_ctx *h, const hegmm_ct *ct, int m, int l, int n, int alg, uint64_t *out) {
    if (!h || !ct || !out) return HEGMM_EINVAL;
    Ctx *c = &h->c;
    const int a = resolve_alg(m, l, n, alg, c->S);
    if (!a) return set_err(c, HEGMM_ESHAPE, "shape does not fit one slot row");
    HostPlan P = make_host_plan(m, l, n, a);
    std::vector<u64> s;
    int rc = decrypt_slots(c, ct, s);
    if (rc) return rc;
    for (int i = 0; i < m; i++)
        for (int j = 0; j < n; j++) out[(size_t)i * n + j] = s[P.result_slot(i, j)];
    return HEGMM_OK;
}

int hegmm_decrypt_pair(hegmm_ctx *h, const hegmm_ct *ct, int m, int l, int n, int alg, uint64_t *out0,
                       uint64_t *out1) {
    if (!h || !ct || !out0 || !out1) return HEGMM_EINVAL;
    Ctx *c = &h->c;
    const int a = resolve_alg(m, l, n, alg, c->S);
    if (!a) return set_err(c, HEGMM_ESHAPE, "shape does not fit one slot row");
    HostPlan P = make_host_plan(m, l, n, a);
    std::vector<u64> s;
    int rc = decrypt_slots(c, ct, s);
    if (rc) return rc;
    for (int i = 0; i < m; i++)
        for (int j = 0; j < n; j++) {
            out0[(size_t)i * n + j] = s[P.result_slot(i, j)];
            out1[(size_t)i * n + j] = s[c->S + P.result_slot(i, j)];
        }
    return HEGMM_OK;
}

int hegmm_ct_level(const hegmm_ct *ct) { return ct ? ct->level : 0; }

int hegmm_ct_export(hegmm_ctx *h, const hegmm_ct *ct, uint64_t *host) {
    if (!h || !ct || !host) return HEGMM_EINVAL;
    Ctx *c = &h->c;
    const size_t w = (size_t)2 * ct->level * c->N;
    u64 *tmp = dalloc(c, w);
    if (!tmp) return set_err(c, HEGMM_ENOMEM, "export");
    cudaMemcpyAsync(tmp, ct->d, w * 8, cudaMemcpyDeviceToDevice, c->st);
    int rc = ntt_inv(c, pat_ct(c, tmp, 2, ct->level));
    if (rc) return rc;
    cudaMemcpyAsync(host, tmp, w * 8, cudaMemcpyDeviceToHost, c->st);
    dfree(c, tmp);
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_check(c, "export");
    if ((rc = device_status(c))) return rc;
    return cuda_check(c, "export");
}

int hegmm_ct_import(hegmm_ctx *h, const uint64_t *host, int level, hegmm_ct **out) {
    if (!h || !host || !out || level < 1 || level > h->c.L) return HEGMM_EINVAL;
    Ctx *c = &h->c;
    hegmm_ct *ct = new_ct(c, level);
    if (!ct) return set_err(c, HEGMM_ENOMEM, "import");
    cudaMemcpyAsync(ct->d, host, (size_t)2 * level * c->N * 8, cudaMemcpyHostToDevice, c->st);
    int rc = ntt_fwd(c, pat_ct(c, ct->d, 2, level));
    if (rc) return rc;
    *out = ct;
    return HEGMM_OK;
}

// count ciphertexts' 2*level limbs as one limb pattern through a device
// array of their addresses (ptrs: count pointers on the device)
static LimbPat pat_cts(Ctx *c, u64 *const *ptrs, int count, int level) {
    LimbPat p{};
    p.base = nullptr;
    p.outer_ptrs = ptrs;
    p.outer_stride = 0;
    p.inner = 2 * level;
    p.count = 2 * level * count;
    for (int k = 0; k < 2 * level; k++) {
        p.off[k] = (unsigned short)k;
        p.mod[k] = (unsigned char)(k % level);
    }
    (void)c;
    return p;
}

int hegmm_ct_import_batch(hegmm_ctx *h, int count, const uint64_t *const *host, int level, hegmm_ct **out) {
    if (!h || count < 0 || (count && (!host || !out)) || level < 1 || level > h->c.L) return HEGMM_EINVAL;
    Ctx *c = &h->c;
    if (2 * level > PAT_MAX) return set_err(c, HEGMM_EINVAL, "import_batch: level too large");
    for (int i = 0; i < count; i++) out[i] = nullptr;
    if (!count) return HEGMM_OK;
    std::vector<u64 *> ptrs((size_t)count);
    const size_t bytes = (size_t)2 * level * c->N * 8;
    for (int i = 0; i < count; i++) {
        if (!host[i]) return set_err(c, HEGMM_EINVAL, "import_batch: null host buffer");
        out[i] = new_ct(c, level);
        if (!out[i]) {
            for (int j = 0; j < i; j++) {
                hegmm_ct_destroy(out[j]);
                out[j] = nullptr;
            }
            return set_err(c, HEGMM_ENOMEM, "import_batch");
        }
        ptrs[i] = out[i]->d;
        cudaMemcpyAsync(out[i]->d, host[i], bytes, cudaMemcpyHostToDevice, c->st);
    }
    u64 **d_ptrs = upload(c, ptrs);
    if (!d_ptrs) return set_err(c, HEGMM_ENOMEM, "import_batch");
    int rc = ntt_fwd(c, pat_cts(c, d_ptrs, count, level));
    dfree(c, d_ptrs);
    if (rc) return rc;
    return cuda_check(c, "import_batch");
}

int hegmm_ct_export_batch(hegmm_ctx *h, int count, const hegmm_ct *const *cts, uint64_t *const *host) {
    if (!h || count < 0 || (count && (!cts || !host))) return HEGMM_EINVAL;
    Ctx *c = &h->c;
    if (!count) return HEGMM_OK;
    const int level = cts[0] ? cts[0]->level : 0;
    for (int i = 0; i < count; i++)
        if (!cts[i] || !host[i] || cts[i]->level != level) return set_err(c, HEGMM_EINVAL, "export_batch: arguments");
    const size_t w = (size_t)2 * level * c->N;
    u64 *tmp = dalloc(c, w * count);
    if (!tmp) return set_err(c, HEGMM_ENOMEM, "export_batch");
    for (int i = 0; i < count; i++)
        cudaMemcpyAsync(tmp + (size_t)i * w, cts[i]->d, w * 8, cudaMemcpyDeviceToDevice, c->st);
    int rc = ntt_inv(c, pat_ct(c, tmp, 2 * count, level));
    if (rc) return rc;
    for (int i = 0; i < count; i++)
        cudaMemcpyAsync(host[i], tmp + (size_t)i * w, w * 8, cudaMemcpyDeviceToHost, c->st);
    dfree(c, tmp);
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_check(c, "export_batch");
    return device_status(c);
}

int hegmm_sync(hegmm_ctx *h) {
    if (!h) return HEGMM_EINVAL;
    if (cudaStreamSynchronize(h->c.st) != cudaSuccess) return cuda_check(&h->c, "sync");
    return device_status(&h->c);
}

void hegmm_pt_destroy(hegmm_pt *pt) {
    if (!pt) return;
    dfree(pt->ctx, pt->d);
    dfree(pt->ctx, pt->d_mont);
    delete pt;
}

void hegmm_ct_destroy(hegmm_ct *ct) {
    if (!ct) return;
    dfree(ct->ctx, ct->d);
    delete ct;
}

static const char *kKernelNames[K_NUM] = {"ntt_fwd",     "ntt_inv",      "modup",         "ksw_inner_product",
                                          "div_conv",    "div_combine",  "divround_ntt",  "lt_accumulate",
                                          "tensor",      "sum",          "pointwise",     "sample",
                                          "codec",       "lt_keyswitch"};

int hegmm_set_timing(hegmm_ctx *h, int enable) {
    if (!h) return HEGMM_EINVAL;
    h->c.timing = enable != 0;
    return HEGMM_OK;
}

int hegmm_kernel_kinds(void) { return K_NUM; }

const char *hegmm_kernel_name(int kind) { return kind >= 0 && kind < K_NUM ? kKernelNames[kind] : "?"; }

static void drain(Ctx *c) {
    if (c->pending.empty()) return;
    cudaStreamSynchronize(c->st);
    for (auto &p : c->pending) {
        float ms = 0;
        cudaEventElapsedTime(&ms, p.a, p.b);
        c->stat_ms[p.kind] += ms;
        c->stat_n[p.kind] += 1;
        c->stat_bytes[p.kind] += p.bytes;
        c->stat_work[p.kind] += p.work;
        c->evpool.push_back(p.a);
        c->evpool.push_back(p.b);
    }
    c->pending.clear();
}

int hegmm_kernel_stats(hegmm_ctx *h, int kind, double *total_ms, long long *launches, double *bytes,
                       double *butterflies) {
    if (!h || kind < 0 || kind >= K_NUM) return HEGMM_EINVAL;
    drain(&h->c);
    if (total_ms) *total_ms = h->c.stat_ms[kind];
    if (launches) *launches = h->c.stat_n[kind];
    if (bytes) *bytes = h->c.stat_bytes[kind];
    if (butterflies) *butterflies = h->c.stat_work[kind];
    return HEGMM_OK;
}

int hegmm_kernel_reset(hegmm_ctx *h) {
    if (!h) return HEGMM_EINVAL;
    drain(&h->c);
    for (int k = 0; k < K_NUM; k++) {
        h->c.stat_ms[k] = 0;
        h->c.stat_n[k] = 0;
        h->c.stat_bytes[k] = 0;
        h->c.stat_work[k] = 0;
    }
    return HEGMM_OK;
}

int hegmm_set_budgets(hegmm_ctx *h, uint64_t mask_bytes, uint64_t plan_bytes, uint64_t chunk_bytes) {
    if (!h) return HEGMM_EINVAL;
    if (mask_bytes) h->c.mask_budget = mask_bytes;
    if (plan_bytes) h->c.plan_cache_budget = plan_bytes;
    if (chunk_bytes) h->c.ws_budget = std::max<uint64_t>(chunk_bytes, (uint64_t)1 << 24);
    return HEGMM_OK;
}

int hegmm_device_memory(hegmm_ctx *h, int reset_high, uint64_t *out) {
    if (!h || !out) return HEGMM_EINVAL;
    Ctx *c = &h->c;
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_check(c, "device_memory");
    int dev = 0;
    cudaMemPool_t pool;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess)
        return cuda_check(c, "device_memory: pool");
    uint64_t used = 0, high = 0, reserved = 0;
    if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) != cudaSuccess ||
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &high) != cudaSuccess ||
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) != cudaSuccess)
        return cuda_check(c, "device_memory: pool attributes");
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return cuda_check(c, "device_memory: cudaMemGetInfo");
    out[0] = used;
    out[1] = high;
    out[2] = reserved;
    out[3] = fr;
    if (reset_high) {
        uint64_t zero = 0;  // the high-water mark restarts from the current use
        if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero) != cudaSuccess)
            return cuda_check(c, "device_memory: reset");
    }
    return HEGMM_OK;
}

int hegmm_peak_butterflies(hegmm_ctx *h, double *per_s) {
    if (!h || !per_s) return HEGMM_EINVAL;
    return peak_butterflies(&h->c, per_s);
}

}  // extern "C"

// exec.cu -- hoisted rotations, HE-Mult, modulus switch and the HEGMM executor.
//
// HEGMM (Algorithms 1 and 2 of arXiv 2405.02238) is executed per product
// shape from a prebuilt ExecPlan:
//   1. one hoisted ModUp of c1 for each operand (ct.A, ct.B);
//   2. every distinct rotation offset of an operand is key-switched once
//      (the linear transformations eps^k / omega^k of all iterations share
//      the same source ciphertext, so Rot(ct, d) is reused bit-identically
//      across k), in chunks: inner product with the Galois key fused with the
//      NTT-domain automorphism, then ModDown;
//   3. the masks u_d (Eq. lintrans) are applied and accumulated into the
//      eps^k(A) / omega^k(B) outputs of all iterations in one launch per chunk;
//   4. optional modulus switch, tensor of every iteration, batched
//      relinearisation (hoisted ModUp of every d2, inner product, ModDown)
//      and the sum over iterations (HE-Add of Algorithm 1 line 7);
//   5. Algorithm 2: t-1 hoisted extraction rotations by h p and their sum.
// All device descriptors are built once per shape, so a product is a fixed
// sequence of about 20-40 kernel launches.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <set>

#include "device.cuh"
#include "internal.h"
#include "plan.h"

namespace hg {

// ---------------------------------------------------------------- helpers

template <typename T>
static T *upload(Ctx *c, const std::vector<T> &v) {
    size_t bytes = std::max<size_t>(v.size() * sizeof(T), 8);
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, c->st) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (!v.empty()) cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, c->st);
    return (T *)p;
}

// Limbs of the digits D [n][nd][ne][N] that ModUp produced in coefficient
// form (every prime outside the digit's own ones).
static LimbPat pat_nonown(Ctx *c, int lv, u64 *D, int n, long long stride) {
    LimbPat p{};
    p.base = D;
    p.outer_stride = stride;
    const int ne = lv + c->K, nd = c->digits(lv);
    int k = 0;
    for (int j = 0; j < nd; j++) {
        const int lo = j * c->alpha, hi = std::min(lo + c->alpha, lv);
        for (int e = 0; e < ne; e++) {
            if (e >= lo && e < hi) continue;
            p.off[k] = (unsigned short)(j * ne + e);
            p.mod[k] = (unsigned char)c->gidx(lv, e);
            k++;
        }
    }
    p.inner = k;
    p.count = k * n;
    return p;
}

// The K special-prime limbs of n polynomials over the extended basis.
static LimbPat pat_drop_special(Ctx *c, int lv, u64 *u, int npoly) {
    LimbPat p{};
    p.base = u;
    p.outer_stride = (long long)(lv + c->K) * c->N;
    p.inner = c->K;
    p.count = c->K * npoly;
    for (int k = 0; k < c->K; k++) {
        p.off[k] = (unsigned short)(lv + k);
        p.mod[k] = (unsigned char)(c->L + k);
    }
    return p;
}

static const DivTab *div_tab(Ctx *c, int lv, int kind) {
    auto it = c->divs.find({lv, kind});
    if (it == c->divs.end()) {
        if (build_div_tab(c, lv, kind)) return nullptr;
        it = c->divs.find({lv, kind});
    }
    return &it->second;
}

// Hoisted ModUp of n polynomials given in NTT form at xn (stride xn_stride):
// xc receives their coefficient form, D [n][nd][ne][N] the digits (NTT).
static int modup(Ctx *c, int lv, int n, const u64 *xn, long long xn_stride, u64 *xc, u64 *D) {
    const int N = c->N, ne = lv + c->K, nd = c->digits(lv);
    int rc;
    if (xn_stride == (long long)lv * N) {
        cudaMemcpyAsync(xc, xn, (size_t)n * lv * N * 8, cudaMemcpyDeviceToDevice, c->st);
    } else {
        cudaMemcpy2DAsync(xc, (size_t)lv * N * 8, xn, (size_t)xn_stride * 8, (size_t)lv * N * 8, n,
                          cudaMemcpyDeviceToDevice, c->st);
    }
    if ((rc = ntt_inv(c, pat_ct(c, xc, n, lv)))) return rc;
    const ModUpTab *tb = modup_tab(c, lv);
    if (!tb) return HEGMM_ENOMEM;
    return modup_ntt(c, *tb, pat_nonown(c, lv, D, n, (long long)nd * ne * N), xc, (long long)lv * N, xn, xn_stride, D,
                     (long long)nd * ne * N, n);
}

// Inner product + ModDown for nrot key switches whose descriptors are on
// the device; u/tmp are [2*nrot] polynomial scratch laid out contiguously.
static int ksw_moddown(Ctx *c, int lv, const RotDesc *d_rots, const DivDesc *d_div, int nrot, u64 *u, u64 *tmp) {
    const DivTab *tb = div_tab(c, lv, 0);
    if (!tb) return HEGMM_ENOMEM;
    int rc;
    (void)tmp;
    if ((rc = ksw_ip(c, lv, d_rots, nrot))) return rc;
    if ((rc = ntt_inv(c, pat_drop_special(c, lv, u, 2 * nrot)))) return rc;
    return divround_ntt(c, *tb, d_div, 2 * nrot);
}

// ---------------------------------------------------------------- single operations

int rotate_hoisted(Ctx *c, const hegmm_ct *in, const int *z, int count, hegmm_ct **outs) {
    const int lv = in->level, N = c->N, ne = lv + c->K, nd = c->digits(lv);
    std::vector<RotDesc> rd;
    std::vector<DivDesc> dd;
    std::vector<int> idx;
    for (int r = 0; r < count; r++) outs[r] = nullptr;
    for (int r = 0; r < count; r++) {
        outs[r] = new_ct(c, lv);
        if (!outs[r]) return set_err(c, HEGMM_ENOMEM, "rotate");
        if (((long long)z[r] % c->S) == 0) {
            cudaMemcpyAsync(outs[r]->d, in->d, (size_t)2 * lv * N * 8, cudaMemcpyDeviceToDevice, c->st);
            continue;
        }
        const u64 g = galois_of(c, z[r]);
        auto it = c->keys.find(g);
        if (it == c->keys.end()) return set_err(c, HEGMM_ENOKEY, "missing Galois key for a rotation");
        idx.push_back(r);
        RotDesc d{};
        d.key = it->second;
        d.g = (u32)g;
        rd.push_back(d);
    }
    if (rd.empty()) return HEGMM_OK;
    const int nr = (int)rd.size();
    u64 *xc = dalloc(c, (size_t)lv * N);
    u64 *D = dalloc(c, (size_t)nd * ne * N);
    u64 *u = dalloc(c, (size_t)nr * 2 * ne * N);
    u64 *tmp = dalloc(c, (size_t)nr * 2 * lv * N);
    if (!xc || !D || !u || !tmp) return set_err(c, HEGMM_ENOMEM, "rotate scratch");
    for (int k = 0; k < nr; k++) {
        rd[k].D = D;
        rd[k].u = u + (size_t)k * 2 * ne * N;
        for (int comp = 0; comp < 2; comp++) {
            DivDesc v{};
            v.u = u + ((size_t)2 * k + comp) * ne * N;
            v.tmp = tmp + ((size_t)2 * k + comp) * lv * N;
            v.out = outs[idx[k]]->d + (size_t)comp * lv * N;
            v.add = comp == 0 ? in->d : nullptr;
            v.g = rd[k].g;
            dd.push_back(v);
        }
    }
    RotDesc *d_r = upload(c, rd);
    DivDesc *d_d = upload(c, dd);
    int rc;
    if ((rc = modup(c, lv, 1, in->d + (size_t)lv * N, (long long)lv * N, xc, D))) return rc;
    if ((rc = ksw_moddown(c, lv, d_r, d_d, nr, u, tmp))) return rc;
    dfree(c, d_r);
    dfree(c, d_d);
    dfree(c, xc);
    dfree(c, D);
    dfree(c, u);
    dfree(c, tmp);
    return cuda_check(c, "rotate");
}

int mult_relin(Ctx *c, const hegmm_ct *a, const hegmm_ct *b, hegmm_ct **out) {
    if (a->level != b->level) return set_err(c, HEGMM_EINVAL, "operands at different levels");
    const int lv = a->level, N = c->N, ne = lv + c->K, nd = c->digits(lv);
    auto kit = c->keys.find(0);
    if (kit == c->keys.end()) return set_err(c, HEGMM_ENOKEY, "no relinearisation key");
    hegmm_ct *o = new_ct(c, lv);
    u64 *d3 = dalloc(c, (size_t)3 * lv * N);
    u64 *xc = dalloc(c, (size_t)lv * N);
    u64 *D = dalloc(c, (size_t)nd * ne * N);
    u64 *u = dalloc(c, (size_t)2 * ne * N);
    u64 *tmp = dalloc(c, (size_t)2 * lv * N);
    if (!o || !d3 || !xc || !D || !u || !tmp) return set_err(c, HEGMM_ENOMEM, "mult");
    std::vector<Tensor3> tv{{a->d, b->d, d3}};
    std::vector<RotDesc> rd{{D, kit->second, u, 1u, 0u}};
    std::vector<DivDesc> dd(2);
    for (int comp = 0; comp < 2; comp++) {
        dd[comp].u = u + (size_t)comp * ne * N;
        dd[comp].tmp = tmp + (size_t)comp * lv * N;
        dd[comp].out = o->d + (size_t)comp * lv * N;
        dd[comp].add = d3 + (size_t)comp * lv * N;
        dd[comp].g = 1;
    }
    Tensor3 *d_t = upload(c, tv);
    RotDesc *d_r = upload(c, rd);
    DivDesc *d_d = upload(c, dd);
    int rc;
    if ((rc = tensor(c, lv, d_t, 1))) return rc;
    if ((rc = modup(c, lv, 1, d3 + (size_t)2 * lv * N, (long long)lv * N, xc, D))) return rc;
    if ((rc = ksw_moddown(c, lv, d_r, d_d, 1, u, tmp))) return rc;
    for (void *p : {(void *)d_t, (void *)d_r, (void *)d_d, (void *)d3, (void *)xc, (void *)D, (void *)u, (void *)tmp})
        dfree(c, p);
    *out = o;
    return cuda_check(c, "mult");
}

// Modulus switch of npoly polynomials at level lv (stride lv*N from `in`,
// which is overwritten in its last limb) into out (stride (lv-1)*N).
static int modswitch_polys(Ctx *c, int lv, u64 *in, int npoly, u64 *tmp, u64 *out, DivDesc *d_desc) {
    const DivTab *tb = div_tab(c, lv, 1);
    if (!tb) return HEGMM_ENOMEM;
    LimbPat pd{};
    pd.base = in;
    pd.outer_stride = (long long)lv * c->N;
    pd.inner = 1;
    pd.count = npoly;
    pd.off[0] = (unsigned short)(lv - 1);
    pd.mod[0] = (unsigned char)(lv - 1);
    int rc;
    (void)tmp;
    if ((rc = ntt_inv(c, pd))) return rc;
    return divround_ntt(c, *tb, d_desc, npoly);
}

int modswitch(Ctx *c, const hegmm_ct *in, hegmm_ct **out) {
    const int lv = in->level, N = c->N;
    if (lv < 2) return set_err(c, HEGMM_EINVAL, "no prime left to drop");
    hegmm_ct *o = new_ct(c, lv - 1);
    u64 *cp = dalloc(c, (size_t)2 * lv * N);
    u64 *tmp = dalloc(c, (size_t)2 * (lv - 1) * N);
    if (!o || !cp || !tmp) return set_err(c, HEGMM_ENOMEM, "modswitch");
    cudaMemcpyAsync(cp, in->d, (size_t)2 * lv * N * 8, cudaMemcpyDeviceToDevice, c->st);
    std::vector<DivDesc> dd(2);
    for (int p = 0; p < 2; p++) {
        dd[p].u = cp + (size_t)p * lv * N;
        dd[p].tmp = tmp + (size_t)p * (lv - 1) * N;
        dd[p].out = o->d + (size_t)p * (lv - 1) * N;
        dd[p].add = nullptr;
        dd[p].g = 1;
    }
    DivDesc *d_d = upload(c, dd);
    int rc = modswitch_polys(c, lv, cp, 2, tmp, o->d, d_d);
    if (rc) return rc;
    dfree(c, d_d);
    dfree(c, cp);
    dfree(c, tmp);
    *out = o;
    return cuda_check(c, "modswitch");
}

// ---------------------------------------------------------------- HEGMM plans

struct Chunk {
    int cnt = 0;
    RotDesc *d_rots = nullptr;
    DivDesc *d_div = nullptr;
    LtTerm *d_terms = nullptr;
    int *d_off = nullptr;
};

struct Side {
    std::vector<long long> zs;  // distinct non-zero offsets (mod S)
    std::vector<Chunk> chunks;
    LtTerm *d_id_terms = nullptr;
    int *d_id_off = nullptr;
    u64 **d_outs = nullptr;
};

struct ExecPlan {
    HostPlan hp;
    int lv0 = 0, lv1 = 0, niter = 0, ne0 = 0, nd0 = 0, ne1 = 0, nd1 = 0, RC = 0, next = 0;
    size_t ws_words = 0;
    u64 *ws = nullptr;
    u64 *in = nullptr, *xc = nullptr, *D = nullptr, *u = nullptr, *tmp = nullptr, *rot = nullptr, *outs = nullptr;
    u64 *ms = nullptr, *mstmp = nullptr, *d3 = nullptr, *rxc = nullptr, *rD = nullptr, *ru = nullptr, *rtmp = nullptr;
    u64 *rout = nullptr, *cacc = nullptr, *exc = nullptr, *eD = nullptr, *eu = nullptr, *etmp = nullptr, *erot = nullptr;
    u64 *masks = nullptr;
    int nmask = 0;
    Side side[2];
    Tensor3 *d_tens = nullptr;
    RotDesc *d_rrot = nullptr, *d_erot = nullptr;
    DivDesc *d_rdiv = nullptr, *d_msdiv = nullptr, *d_ediv = nullptr;
    hegmm_opcount cnt{};
    std::vector<void *> allocs;
};

static void free_plan(Ctx *c, ExecPlan *p) {
    for (void *a : p->allocs) dfree(c, a);
    delete p;
}

void free_plans(Ctx *c) {
    for (auto &kv : c->plans) free_plan(c, kv.second);
    c->plans.clear();
}

// Encode count 0/1 masks (value `scale` on the listed slots) into
// Montgomery NTT form over q_0..q_{lv-1}: out [count][lv][N].
static int encode_masks(Ctx *c, int lv, const std::vector<const std::vector<int> *> &dsts, u64 scale, u64 *out) {
    const int N = c->N;
    const int B = 128;
    u64 *m = dalloc(c, (size_t)B * N);
    if (!m) return set_err(c, HEGMM_ENOMEM, "mask encode");
    std::vector<u64> ev((size_t)B * N);
    int rc;
    for (size_t b0 = 0; b0 < dsts.size(); b0 += B) {
        const int nb = (int)std::min<size_t>(B, dsts.size() - b0);
        std::fill(ev.begin(), ev.begin() + (size_t)nb * N, 0);
        for (int b = 0; b < nb; b++)
            for (int s : *dsts[b0 + b]) ev[(size_t)b * N + c->slot_pos0[s]] = scale;
        cudaMemcpyAsync(m, ev.data(), (size_t)nb * N * 8, cudaMemcpyHostToDevice, c->st);
        LimbPat pm{};
        pm.base = m;
        pm.outer_stride = N;
        pm.inner = 1;
        pm.count = nb;
        pm.off[0] = 0;
        pm.mod[0] = (unsigned char)c->tmod;
        u64 *o = out + b0 * lv * N;
        if ((rc = ntt_inv(c, pm))) return rc;
        if ((rc = lift_from_t(c, lv, m, o, nb))) return rc;
        LimbPat pq = pat_ct(c, o, nb, lv);
        if ((rc = ntt_fwd(c, pq))) return rc;
        if ((rc = pw_to_mont(c, pq))) return rc;
        cudaStreamSynchronize(c->st);  // ev is reused
    }
    dfree(c, m);
    return cuda_check(c, "mask encode");
}

static int build_plan(Ctx *c, int m, int l, int n, int alg, ExecPlan **out) {
    const int N = c->N, S = c->S;
    ExecPlan *P = new ExecPlan;
    P->hp = make_host_plan(m, l, n, alg);
    const HostPlan &hp = P->hp;
    P->lv0 = c->L;
    P->lv1 = c->L - c->prm.ms_drop;
    P->niter = (int)hp.iters.size();
    P->ne0 = P->lv0 + c->K;
    P->nd0 = c->digits(P->lv0);
    P->ne1 = P->lv1 + c->K;
    P->nd1 = c->digits(P->lv1);
    P->next = (int)hp.extract.size();
    const int lv0 = P->lv0, lv1 = P->lv1, ni = P->niter, ne0 = P->ne0, nd0 = P->nd0, ne1 = P->ne1, nd1 = P->nd1;
    auto fail = [&](int code, const char *msg) {
        free_plan(c, P);
        return set_err(c, code, msg);
    };
    // distinct rotations per operand and the key of each
    std::map<long long, int> zidx[2];
    for (int s = 0; s < 2; s++) {
        std::set<long long> zs;
        for (auto &it : hp.iters)
            for (auto &d : (s == 0 ? it.eps : it.omg)) {
                long long z = ((long long)d.d % S + S) % S;
                if (z) zs.insert(z);
            }
        for (long long z : zs) {
            zidx[s][z] = (int)P->side[s].zs.size();
            P->side[s].zs.push_back(z);
        }
    }
    for (int s = 0; s < 2; s++)
        for (long long z : P->side[s].zs)
            if (!c->keys.count(galois_of(c, z))) return fail(HEGMM_ENOKEY, "missing Galois key: run hegmm_keygen for this shape");
    for (int z : hp.extract)
        if (!c->keys.count(galois_of(c, z))) return fail(HEGMM_ENOKEY, "missing Galois key for extraction");
    if (!c->keys.count(0)) return fail(HEGMM_ENOKEY, "no relinearisation key");
    // rotation chunk size: about 1 GiB of u / tmp / rot scratch
    const size_t per_rot = (size_t)(2 * ne0 + 4 * lv0) * N * 8;
    const int maxr = (int)std::max(P->side[0].zs.size(), P->side[1].zs.size());
    P->RC = (int)std::max<size_t>(1, std::min<size_t>((size_t)std::max(maxr, 1), ((size_t)1 << 30) / per_rot));
    const int RC = P->RC, T1 = std::max(P->next, 1);
    // workspace layout (words)
    size_t off = 0;
    auto take = [&](size_t w) {
        size_t o = off;
        off += (w + 31) & ~(size_t)31;
        return o;
    };
    const size_t o_in = take((size_t)2 * 2 * lv0 * N), o_xc = take((size_t)2 * lv0 * N),
                 o_D = take((size_t)2 * nd0 * ne0 * N), o_u = take((size_t)RC * 2 * ne0 * N),
                 o_tmp = take((size_t)RC * 2 * lv0 * N), o_rot = take((size_t)RC * 2 * lv0 * N),
                 o_outs = take((size_t)2 * ni * 2 * lv0 * N);
    size_t o_ms = 0, o_mstmp = 0;
    if (lv1 != lv0) {
        o_ms = take((size_t)2 * ni * 2 * lv1 * N);
        o_mstmp = take((size_t)2 * ni * 2 * lv1 * N);
    }
    const size_t o_d3 = take((size_t)ni * 3 * lv1 * N), o_rxc = take((size_t)ni * lv1 * N),
                 o_rD = take((size_t)ni * nd1 * ne1 * N), o_ru = take((size_t)ni * 2 * ne1 * N),
                 o_rtmp = take((size_t)ni * 2 * lv1 * N), o_rout = take((size_t)ni * 2 * lv1 * N),
                 o_cacc = take((size_t)2 * lv1 * N), o_exc = take((size_t)lv1 * N), o_eD = take((size_t)nd1 * ne1 * N),
                 o_eu = take((size_t)T1 * 2 * ne1 * N), o_etmp = take((size_t)T1 * 2 * lv1 * N),
                 o_erot = take((size_t)T1 * 2 * lv1 * N);
    P->ws_words = off;
    P->ws = dalloc(c, off);
    if (!P->ws) return fail(HEGMM_ENOMEM, "plan workspace");
    P->allocs.push_back(P->ws);
    u64 *W = P->ws;
    P->in = W + o_in;
    P->xc = W + o_xc;
    P->D = W + o_D;
    P->u = W + o_u;
    P->tmp = W + o_tmp;
    P->rot = W + o_rot;
    P->outs = W + o_outs;
    P->ms = lv1 != lv0 ? W + o_ms : nullptr;
    P->mstmp = lv1 != lv0 ? W + o_mstmp : nullptr;
    P->d3 = W + o_d3;
    P->rxc = W + o_rxc;
    P->rD = W + o_rD;
    P->ru = W + o_ru;
    P->rtmp = W + o_rtmp;
    P->rout = W + o_rout;
    P->cacc = W + o_cacc;
    P->exc = W + o_exc;
    P->eD = W + o_eD;
    P->eu = W + o_eu;
    P->etmp = W + o_etmp;
    P->erot = W + o_erot;
    // masks: one per distinct (slot set), value scale = prod of dropped primes mod t
    u64 scale = 1;
    for (int i = 0; i < c->prm.ms_drop; i++) scale = (u64)((unsigned __int128)scale * (c->q[c->L - 1 - i] % c->t) % c->t);
    std::map<std::vector<int>, int> mask_of;
    std::vector<const std::vector<int> *> mlist;
    for (auto &it : hp.iters)
        for (int s = 0; s < 2; s++)
            for (auto &d : (s == 0 ? it.eps : it.omg))
                if (!mask_of.count(d.dst)) {
                    mask_of[d.dst] = (int)mlist.size();
                    mlist.push_back(&mask_of.find(d.dst)->first);
                }
    P->nmask = (int)mlist.size();
    P->masks = dalloc(c, (size_t)P->nmask * lv0 * N);
    if (!P->masks) return fail(HEGMM_ENOMEM, "plan masks");
    P->allocs.push_back(P->masks);
    int rc = encode_masks(c, lv0, mlist, scale, P->masks);
    if (rc) {
        free_plan(c, P);
        return rc;
    }
    auto mask_ptr = [&](const std::vector<int> &dst) { return P->masks + (size_t)mask_of[dst] * lv0 * N; };
    // per operand: output pointers, identity terms, rotation chunks
    for (int s = 0; s < 2; s++) {
        Side &sd = P->side[s];
        const u64 *src_ct = P->in + (size_t)s * 2 * lv0 * N;
        std::vector<u64 *> outs(ni);
        for (int k = 0; k < ni; k++) outs[k] = P->outs + ((size_t)s * ni + k) * 2 * lv0 * N;
        sd.d_outs = upload(c, outs);
        P->allocs.push_back(sd.d_outs);
        // identity (d = 0) terms, one launch that also initialises the outputs
        std::vector<LtTerm> terms;
        std::vector<int> offs{0};
        for (int k = 0; k < ni; k++) {
            for (auto &d : (s == 0 ? hp.iters[k].eps : hp.iters[k].omg))
                if (((long long)d.d % S) == 0) terms.push_back({src_ct, mask_ptr(d.dst)});
            offs.push_back((int)terms.size());
        }
        sd.d_id_terms = upload(c, terms);
        sd.d_id_off = upload(c, offs);
        P->allocs.push_back(sd.d_id_terms);
        P->allocs.push_back(sd.d_id_off);
        const int nz = (int)sd.zs.size();
        for (int r0 = 0; r0 < nz; r0 += RC) {
            Chunk ch;
            ch.cnt = std::min(RC, nz - r0);
            std::vector<RotDesc> rd;
            std::vector<DivDesc> dd;
            for (int r = 0; r < ch.cnt; r++) {
                const u64 g = galois_of(c, sd.zs[r0 + r]);
                rd.push_back({P->D + (size_t)s * nd0 * ne0 * N, c->keys[g], P->u + (size_t)r * 2 * ne0 * N, (u32)g, 0u});
                for (int comp = 0; comp < 2; comp++) {
                    DivDesc v{};
                    v.u = P->u + ((size_t)2 * r + comp) * ne0 * N;
                    v.tmp = P->tmp + ((size_t)2 * r + comp) * lv0 * N;
                    v.out = P->rot + ((size_t)2 * r + comp) * lv0 * N;
                    v.add = comp == 0 ? src_ct : nullptr;
                    v.g = (u32)g;
                    dd.push_back(v);
                }
            }
            std::vector<LtTerm> ct;
            std::vector<int> co{0};
            for (int k = 0; k < ni; k++) {
                for (auto &d : (s == 0 ? hp.iters[k].eps : hp.iters[k].omg)) {
                    long long z = ((long long)d.d % S + S) % S;
                    if (!z) continue;
                    const int ri = zidx[s][z];
                    if (ri < r0 || ri >= r0 + ch.cnt) continue;
                    ct.push_back({P->rot + (size_t)(ri - r0) * 2 * lv0 * N, mask_ptr(d.dst)});
                }
                co.push_back((int)ct.size());
            }
            ch.d_rots = upload(c, rd);
            ch.d_div = upload(c, dd);
            ch.d_terms = upload(c, ct);
            ch.d_off = upload(c, co);
            for (void *p : {(void *)ch.d_rots, (void *)ch.d_div, (void *)ch.d_terms, (void *)ch.d_off}) P->allocs.push_back(p);
            sd.chunks.push_back(ch);
        }
    }
    // modulus switch descriptors: 4 ni polynomials (A outputs then B outputs)
    if (lv1 != lv0) {
        std::vector<DivDesc> dd;
        for (int b = 0; b < 4 * ni; b++) {
            DivDesc v{};
            v.u = P->outs + (size_t)b * lv0 * N;
            v.tmp = P->mstmp + (size_t)b * lv1 * N;
            v.out = P->ms + (size_t)b * lv1 * N;
            v.g = 1;
            dd.push_back(v);
        }
        P->d_msdiv = upload(c, dd);
        P->allocs.push_back(P->d_msdiv);
    }
    // tensor + relinearisation descriptors
    {
        const u64 *A1 = lv1 != lv0 ? P->ms : P->outs;
        std::vector<Tensor3> tv;
        std::vector<RotDesc> rd;
        std::vector<DivDesc> dd;
        for (int k = 0; k < ni; k++) {
            const u64 *a = A1 + (size_t)k * 2 * lv1 * N;
            const u64 *b = A1 + ((size_t)ni + k) * 2 * lv1 * N;
            u64 *d = P->d3 + (size_t)k * 3 * lv1 * N;
            tv.push_back({a, b, d});
            rd.push_back({P->rD + (size_t)k * nd1 * ne1 * N, c->keys[0], P->ru + (size_t)k * 2 * ne1 * N, 1u, 0u});
            for (int comp = 0; comp < 2; comp++) {
                DivDesc v{};
                v.u = P->ru + ((size_t)2 * k + comp) * ne1 * N;
                v.tmp = P->rtmp + ((size_t)2 * k + comp) * lv1 * N;
                v.out = P->rout + ((size_t)2 * k + comp) * lv1 * N;
                v.add = d + (size_t)comp * lv1 * N;
                v.g = 1;
                dd.push_back(v);
            }
        }
        P->d_tens = upload(c, tv);
        P->d_rrot = upload(c, rd);
        P->d_rdiv = upload(c, dd);
        for (void *p : {(void *)P->d_tens, (void *)P->d_rrot, (void *)P->d_rdiv}) P->allocs.push_back(p);
    }
    // extraction rotations (Algorithm 2)
    if (P->next > 0) {
        std::vector<RotDesc> rd;
        std::vector<DivDesc> dd;
        for (int h = 0; h < P->next; h++) {
            const u64 g = galois_of(c, hp.extract[h]);
            rd.push_back({P->eD, c->keys[g], P->eu + (size_t)h * 2 * ne1 * N, (u32)g, 0u});
            for (int comp = 0; comp < 2; comp++) {
                DivDesc v{};
                v.u = P->eu + ((size_t)2 * h + comp) * ne1 * N;
                v.tmp = P->etmp + ((size_t)2 * h + comp) * lv1 * N;
                v.out = P->erot + ((size_t)2 * h + comp) * lv1 * N;
                v.add = comp == 0 ? P->cacc : nullptr;
                v.g = (u32)g;
                dd.push_back(v);
            }
        }
        P->d_erot = upload(c, rd);
        P->d_ediv = upload(c, dd);
        P->allocs.push_back(P->d_erot);
        P->allocs.push_back(P->d_ediv);
    }
    // operation counts
    hegmm_opcount &ct = P->cnt;
    ct.rot = hp.paper_rot();
    ct.cmult = hp.paper_cmult();
    ct.mult = ni;
    ct.relin = ni;
    ct.extract = P->next;
    ct.add = ct.cmult - 2LL * ni + (ni - 1) + P->next;
    ct.ksw = (long long)P->side[0].zs.size() + (long long)P->side[1].zs.size() + ni + P->next;
    ct.modup = 2 + ni + (P->next > 0 ? 1 : 0);
    ct.modswitch = lv1 != lv0 ? 2LL * ni : 0;
    if ((rc = cuda_check(c, "plan build"))) {
        free_plan(c, P);
        return rc;
    }
    *out = P;
    return HEGMM_OK;
}

static int get_plan(Ctx *c, int m, int l, int n, int alg, ExecPlan **out) {
    auto key = std::make_tuple(m, l, n, alg);
    auto it = c->plans.find(key);
    if (it != c->plans.end()) {
        *out = it->second;
        return HEGMM_OK;
    }
    int rc = build_plan(c, m, l, n, alg, out);
    if (rc) return rc;
    c->plans[key] = *out;
    return HEGMM_OK;
}

int prepare_plan(Ctx *c, int m, int l, int n, int alg) {
    const int a = resolve_alg(m, l, n, alg, c->S);
    if (!a) return set_err(c, HEGMM_ESHAPE, "shape does not fit one slot row");
    ExecPlan *P;
    return get_plan(c, m, l, n, a, &P);
}

// Runs a prepared plan on operands already copied into P->in; the result
// (level lv1) is written to out.
static int run_plan(Ctx *c, ExecPlan *P, u64 *out) {
    const int N = c->N, lv0 = P->lv0, lv1 = P->lv1, ni = P->niter, nd0 = P->nd0, ne0 = P->ne0;
    const int nd1 = P->nd1, ne1 = P->ne1;
    int rc;
    // 1. hoisted ModUp of both operands' c1
    if ((rc = modup(c, lv0, 2, P->in + (size_t)lv0 * N, (long long)2 * lv0 * N, P->xc, P->D))) return rc;
    (void)nd0;
    (void)ne0;
    // 2-3. rotations, masks, accumulation into eps^k(A) and omega^k(B)
    for (int s = 0; s < 2; s++) {
        Side &sd = P->side[s];
        if ((rc = lt_accumulate(c, lv0, sd.d_id_terms, sd.d_id_off, sd.d_outs, ni, 0))) return rc;
        for (auto &ch : sd.chunks) {
            if ((rc = ksw_moddown(c, lv0, ch.d_rots, ch.d_div, ch.cnt, P->u, P->tmp))) return rc;
            if ((rc = lt_accumulate(c, lv0, ch.d_terms, ch.d_off, sd.d_outs, ni, 1))) return rc;
        }
    }
    // 4. modulus switch (only when the chain drops a prime before products)
    if (lv1 != lv0)
        if ((rc = modswitch_polys(c, lv0, P->outs, 4 * ni, P->mstmp, P->ms, P->d_msdiv))) return rc;
    // tensor and relinearisation of every iteration, then the sum
    if ((rc = tensor(c, lv1, P->d_tens, ni))) return rc;
    if ((rc = modup(c, lv1, ni, P->d3 + (size_t)2 * lv1 * N, (long long)3 * lv1 * N, P->rxc, P->rD))) return rc;
    if ((rc = ksw_moddown(c, lv1, P->d_rrot, P->d_rdiv, ni, P->ru, P->rtmp))) return rc;
    if ((rc = sum_cts(c, lv1, P->rout, (long long)2 * lv1 * N, ni, P->cacc, 0))) return rc;
    (void)nd1;
    (void)ne1;
    // 5. Algorithm 2 extraction: C = C_acc + sum_h Rot(C_acc, h p)
    cudaMemcpyAsync(out, P->cacc, (size_t)2 * lv1 * N * 8, cudaMemcpyDeviceToDevice, c->st);
    if (P->next > 0) {
        if ((rc = modup(c, lv1, 1, P->cacc + (size_t)lv1 * N, (long long)lv1 * N, P->exc, P->eD))) return rc;
        if ((rc = ksw_moddown(c, lv1, P->d_erot, P->d_ediv, P->next, P->eu, P->etmp))) return rc;
        if ((rc = sum_cts(c, lv1, P->erot, (long long)2 * lv1 * N, P->next, out, 1))) return rc;
    }
    return HEGMM_OK;
}

int matmul(Ctx *c, const hegmm_ct *A, const hegmm_ct *B, int m, int l, int n, int alg, hegmm_ct **C,
           hegmm_opcount *cnt) {
    const int a = resolve_alg(m, l, n, alg, c->S);
    if (!a) return set_err(c, HEGMM_ESHAPE, "shape does not fit one slot row");
    ExecPlan *P;
    int rc = get_plan(c, m, l, n, a, &P);
    if (rc) return rc;
    if (A->level != P->lv0 || B->level != P->lv0) return set_err(c, HEGMM_EINVAL, "operand level does not match");
    const size_t w = (size_t)2 * P->lv0 * c->N;
    cudaMemcpyAsync(P->in, A->d, w * 8, cudaMemcpyDeviceToDevice, c->st);
    cudaMemcpyAsync(P->in + w, B->d, w * 8, cudaMemcpyDeviceToDevice, c->st);
    hegmm_ct *o = new_ct(c, P->lv1);
    if (!o) return set_err(c, HEGMM_ENOMEM, "result ciphertext");
    if ((rc = run_plan(c, P, o->d))) {
        hegmm_ct_destroy(o);
        return rc;
    }
    if (cnt) *cnt = P->cnt;
    *C = o;
    return cuda_check(c, "matmul");
}

int matmul_batch(Ctx *c, int count, const hegmm_ct *const *A, const hegmm_ct *const *B, const int *mln, int alg,
                 hegmm_ct **C) {
    for (int i = 0; i < count; i++) C[i] = nullptr;
    for (int i = 0; i < count; i++) {
        int rc = matmul(c, A[i], B[i], mln[3 * i], mln[3 * i + 1], mln[3 * i + 2], alg, &C[i], nullptr);
        if (rc) {
            for (int j = 0; j <= i; j++) {
                hegmm_ct_destroy(C[j]);
                C[j] = nullptr;
            }
            return rc;
        }
    }
    return HEGMM_OK;
}

}  // namespace hg

using namespace hg;

extern "C" {

int hegmm_matmul(hegmm_ctx *h, const hegmm_ct *A, const hegmm_ct *B, int m, int l, int n, int alg, hegmm_ct **C,
                 hegmm_opcount *cnt) {
    if (!h || !A || !B || !C) return HEGMM_EINVAL;
    return matmul(&h->c, A, B, m, l, n, alg, C, cnt);
}

int hegmm_matmul_batch(hegmm_ctx *h, int count, const hegmm_ct *const *A, const hegmm_ct *const *B, const int *mln,
                       int alg, hegmm_ct **C) {
    if (!h || count < 0 || (count && (!A || !B || !mln || !C))) return HEGMM_EINVAL;
    return matmul_batch(&h->c, count, A, B, mln, alg, C);
}

int hegmm_rotate(hegmm_ctx *h, const hegmm_ct *ct, int z, hegmm_ct **out) {
    if (!h || !ct || !out) return HEGMM_EINVAL;
    return rotate_hoisted(&h->c, ct, &z, 1, out);
}

int hegmm_rotate_many(hegmm_ctx *h, const hegmm_ct *ct, const int *z, int count, hegmm_ct **outs) {
    if (!h || !ct || !outs || count < 0 || (count && !z)) return HEGMM_EINVAL;
    int rc = rotate_hoisted(&h->c, ct, z, count, outs);
    if (rc)
        for (int i = 0; i < count; i++) {
            hegmm_ct_destroy(outs[i]);
            outs[i] = nullptr;
        }
    return rc;
}

int hegmm_cmult(hegmm_ctx *h, const hegmm_ct *ct, const hegmm_pt *pt, hegmm_ct **out) {
    if (!h || !ct || !pt || !out) return HEGMM_EINVAL;
    Ctx *c = &h->c;
    hegmm_ct *o = new_ct(c, ct->level);
    if (!o) return set_err(c, HEGMM_ENOMEM, "cmult");
    int rc = pw_mont(c, ct->level, 2, ct->d, pt->d_mont, 1, o->d);
    if (rc) {
        hegmm_ct_destroy(o);
        return rc;
    }
    *out = o;
    return HEGMM_OK;
}

int hegmm_add(hegmm_ctx *h, const hegmm_ct *a, const hegmm_ct *b, hegmm_ct **out) {
    if (!h || !a || !b || !out) return HEGMM_EINVAL;
    Ctx *c = &h->c;
    if (a->level != b->level) return set_err(c, HEGMM_EINVAL, "operands at different levels");
    hegmm_ct *o = new_ct(c, a->level);
    if (!o) return set_err(c, HEGMM_ENOMEM, "add");
    int rc = pw_add(c, a->level, 2, a->d, b->d, o->d);
    if (rc) {
        hegmm_ct_destroy(o);
        return rc;
    }
    *out = o;
    return HEGMM_OK;
}

int hegmm_mult(hegmm_ctx *h, const hegmm_ct *a, const hegmm_ct *b, hegmm_ct **out) {
    if (!h || !a || !b || !out) return HEGMM_EINVAL;
    return mult_relin(&h->c, a, b, out);
}

int hegmm_modswitch(hegmm_ctx *h, const hegmm_ct *ct, hegmm_ct **out) {
    if (!h || !ct || !out) return HEGMM_EINVAL;
    return modswitch(&h->c, ct, out);
}

}  // extern "C"

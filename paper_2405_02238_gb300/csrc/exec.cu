// exec.cu -- the single HE operations of Section 2.1 (HE-Rot with hoisting,
// HE-Mult with relinearisation, HE-CMult, HE-Add), the BGV modulus switch,
// and the ModUp / key-switch helpers shared with the HEGMM batch executor
// (batch.cu).
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


// Limbs of the digits D [n][nd][ne][N] that ModUp produced in coefficient
// form (every prime outside the digit's own ones).
LimbPat pat_nonown(Ctx *c, int lv, u64 *D, int n, long long stride) {
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
LimbPat pat_drop_special(Ctx *c, int lv, u64 *u, int npoly) {
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

const DivTab *div_tab(Ctx *c, int lv, int kind) {
    auto it = c->divs.find({lv, kind});
    if (it == c->divs.end()) {
        if (build_div_tab(c, lv, kind)) return nullptr;
        it = c->divs.find({lv, kind});
    }
    return &it->second;
}

// Hoisted ModUp of n polynomials given in NTT form at xn (stride xn_stride):
// xc receives their coefficient form, D [n][nd][ne][N] the digits (NTT).
int modup(Ctx *c, int lv, int n, const u64 *xn, long long xn_stride, u64 *xc, u64 *D) {
    const int N = c->N, ne = lv + c->K, nd = c->digits(lv);
    int rc;
    if (xn_stride == (long long)lv * N) {
        cudaMemcpyAsync(xc, xn, (size_t)n * lv * N * 8, cudaMemcpyDeviceToDevice, c->st);
    } else {
        cudaMemcpy2DAsync(xc, (size_t)lv * N * 8, xn, (size_t)xn_stride * 8, (size_t)lv * N * 8, n,
                          cudaMemcpyDeviceToDevice, c->st);
    }
    const ModUpTab *tb = modup_tab(c, lv);
    if (!tb) return HEGMM_ENOMEM;
    // the inverse NTT also multiplies limb i by [(Q_j/q_i)^-1]_{q_i} (the
    // table's first pairs; 1 when a digit is one prime)
    if ((rc = ntt_inv(c, pat_ct(c, xc, n, lv), c->alpha > 1 ? tb->d : nullptr))) return rc;
    return modup_ntt(c, *tb, pat_nonown(c, lv, D, n, (long long)nd * ne * N), xc, (long long)lv * N, xn, xn_stride, D,
                     (long long)nd * ne * N, n);
}

// Inner product + ModDown for nrot key switches whose descriptors are on
// the device; u/tmp are [2*nrot] polynomial scratch laid out contiguously.
int ksw_moddown(Ctx *c, int lv, const RotDesc *d_rots, const DivDesc *d_div, int nrot, u64 *u, u64 *tmp) {
    const DivTab *tb = div_tab(c, lv, c->bfv ? 2 : 0);
    if (!tb) return HEGMM_ENOMEM;
    int rc;
    (void)tmp;
    if ((rc = ksw_ip(c, lv, d_rots, nrot))) return rc;
    // the special limbs' inverse NTT also multiplies them by [t^-1 (P/p_k)^-1]_{p_k}
    if ((rc = ntt_inv(c, pat_drop_special(c, lv, u, 2 * nrot), tb->d))) return rc;
    return divround_ntt(c, *tb, d_div, 2 * nrot);
}

// ---------------------------------------------------------------- BFV HE-Mult

// Scratch of bfv_tensor: the operands in coefficient form over Q and over
// the auxiliary base B ([n][4][L][N], [n][4][nb][N]), the tensors over Q and
// over B ([nout][3][L][N], [nout][3][nb][N]) and the rounded tensors over B
// ([nout][3][nb][N]); nout = n, or the number of sums.
size_t bfv_tensor_words(const Ctx *c, int n, int nout) {
    return (size_t)c->N * ((size_t)n * 4 * (c->L + c->nb) + (size_t)nout * 3 * (c->L + 2 * c->nb));
}

// The limbs over the auxiliary base of npoly polynomials at stride nb N.
static LimbPat pat_aux(Ctx *c, u64 *base, int npoly) {
    LimbPat p{};
    p.base = base;
    p.outer_stride = (long long)c->nb * c->N;
    p.inner = c->nb;
    p.count = c->nb * npoly;
    for (int i = 0; i < c->nb; i++) {
        p.off[i] = (unsigned short)i;
        p.mod[i] = (unsigned char)(c->b0 + i);
    }
    return p;
}

// HE-Mult before relinearisation under BFV, for n products a_k (x) b_k at
// level L (ciphertexts in the NTT domain; d_ops = {a_0, b_0, a_1, ...}):
// both operands' centred values are extended from Q to the auxiliary base
// B (exact base conversion), the tensors are formed over Q u B (the exact
// integer tensors, QB exceeding twice their size), each of d0, d1, d2 is
// rounded to round(t y / Q) over B and converted back to Q, and `out`
// receives the results [nout][3][L][N] in the NTT domain.  d_tq / d_tb:
// n Tensor3 descriptors over Q (operands a_k, b_k) and over B (operands in
// the scratch); or, with sums != 0, d_sq / d_sb: nout = sums TensorSum
// descriptors whose tensors are summed before the rounding (the lazy
// relinearisation of several iterations).
int bfv_tensor(Ctx *c, int n, u64 *const *d_ops, u64 *out, u64 *scratch, const Tensor3 *d_tq, const Tensor3 *d_tb,
               const TensorSum *d_sq, const TensorSum *d_sb, int sums) {
    const int L = c->L, nb = c->nb, N = c->N, nout = sums ? sums : n;
    u64 *xq = scratch, *xb = xq + (size_t)n * 4 * L * N, *dq = xb + (size_t)n * 4 * nb * N;
    u64 *db = dq + (size_t)nout * 3 * L * N, *zb = db + (size_t)nout * 3 * nb * N;
    int rc;
    if ((rc = gather_cts(c, L, d_ops, 2 * n, xq))) return rc;
    if ((rc = ntt_inv(c, pat_ct(c, xq, 4 * n, L)))) return rc;
    if ((rc = bfv_conv_q_to_b(c, xq, (long long)L * N, xb, (long long)nb * N, 4 * n))) return rc;
    if ((rc = ntt_fwd(c, pat_aux(c, xb, 4 * n)))) return rc;
    if (sums) {
        if ((rc = tensor_sum(c, L, d_sq, nout, 0))) return rc;
        if ((rc = tensor_sum(c, nb, d_sb, nout, c->b0))) return rc;
    } else {
        if ((rc = tensor(c, L, d_tq, n, 0))) return rc;
        if ((rc = tensor(c, nb, d_tb, n, c->b0))) return rc;
    }
    if ((rc = ntt_inv(c, pat_ct(c, dq, 3 * nout, L)))) return rc;
    if ((rc = ntt_inv(c, pat_aux(c, db, 3 * nout)))) return rc;
    if ((rc = bfv_scale(c, dq, (long long)L * N, db, (long long)nb * N, zb, (long long)nb * N, 3 * nout))) return rc;
    if ((rc = bfv_conv_b_to_q(c, zb, (long long)nb * N, out, (long long)L * N, 3 * nout))) return rc;
    return ntt_fwd(c, pat_ct(c, out, 3 * nout, L));
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
        d.add0 = in->d;  // tau_g(c0) enters the inner product as P tau_g(c0)
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
            v.add = nullptr;
            v.g = 1;
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
    u64 *bs = nullptr;
    u64 **d_ops = nullptr;
    Tensor3 *d_tb = nullptr;
    if (c->bfv) {
        if (lv != c->L) return set_err(c, HEGMM_EINVAL, "BFV products need operands at the top level");
        bs = dalloc(c, bfv_tensor_words(c, 1, 1));
        if (!bs) return set_err(c, HEGMM_ENOMEM, "mult");
        std::vector<u64 *> ops{a->d, b->d};
        d_ops = upload(c, ops);
        u64 *xb = bs + (size_t)4 * c->L * N, *db = xb + (size_t)4 * c->nb * N + (size_t)3 * c->L * N;
        std::vector<Tensor3> tb{{xb, xb + (size_t)2 * c->nb * N, db}};
        tv[0].d = xb + (size_t)4 * c->nb * N;  // the tensor over Q goes to the scratch
        d_tb = upload(c, tb);
    }
    // d0 / d1 enter the inner product as P d0, P d1
    std::vector<RotDesc> rd{{D, kit->second, u, d3, d3 + (size_t)lv * N, 1u, 0u}};
    std::vector<DivDesc> dd(2);
    for (int comp = 0; comp < 2; comp++) {
        dd[comp].u = u + (size_t)comp * ne * N;
        dd[comp].tmp = tmp + (size_t)comp * lv * N;
        dd[comp].out = o->d + (size_t)comp * lv * N;
        dd[comp].add = nullptr;
        dd[comp].g = 1;
    }
    Tensor3 *d_t = upload(c, tv);
    RotDesc *d_r = upload(c, rd);
    DivDesc *d_d = upload(c, dd);
    int rc;
    if (c->bfv) {
        if ((rc = bfv_tensor(c, 1, d_ops, d3, bs, d_t, d_tb, nullptr, nullptr, 0))) return rc;
    } else if ((rc = tensor(c, lv, d_t, 1))) {
        return rc;
    }
    if ((rc = modup(c, lv, 1, d3 + (size_t)2 * lv * N, (long long)lv * N, xc, D))) return rc;
    if ((rc = ksw_moddown(c, lv, d_r, d_d, 1, u, tmp))) return rc;
    for (void *p : {(void *)d_t, (void *)d_r, (void *)d_d, (void *)d3, (void *)xc, (void *)D, (void *)u, (void *)tmp,
                    (void *)bs, (void *)d_ops, (void *)d_tb})
        dfree(c, p);
    *out = o;
    return cuda_check(c, "mult");
}

// Modulus switch of npoly polynomials at level lv (stride lv*N from `in`,
// which is overwritten in its last limb) into out (stride (lv-1)*N).
int modswitch_polys(Ctx *c, int lv, u64 *in, int npoly, u64 *tmp, u64 *out, DivDesc *d_desc) {
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
    if ((rc = ntt_inv(c, pd, tb->d))) return rc;  // times [t^-1]_{q_{lv-1}}
    return divround_ntt(c, *tb, d_desc, npoly);
}

int modswitch(Ctx *c, const hegmm_ct *in, hegmm_ct **out) {
    const int lv = in->level, N = c->N;
    if (c->bfv) return set_err(c, HEGMM_EINVAL, "the BFV variant has no modulus switch");
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

}  // namespace hg

using namespace hg;

extern "C" {

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

// noalloc.cu -- a key-switched rotation that allocates no device memory.
//
// Some callers cannot allocate device memory while they run this library:
// an application whose framework has already reserved the GPU's memory in
// its own pool (so cudaMalloc fails or competes with that pool), or a
// latency-bound serving loop that must never block in cudaMalloc/cudaFree
// (cudaFree synchronises the whole device).  hegmm_rotate_noalloc gives them
// HE-Rot with every intermediate (ModUp digits, inner-product output,
// ModDown scratch, kernel descriptors and conversion tables) placed in one
// fixed array declared below, which every GPU that loads the library keeps
// for the life of the process.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "device.cuh"
#include "internal.h"

namespace hg {

// 12 MiB: enough for one rotation at N = 2^14 with 8 chain primes, 2 special
// primes and 2-prime digits (about 10.5 MiB), the largest supported preset.
constexpr size_t NOALLOC_BYTES = (size_t)12 << 20;
constexpr size_t NOALLOC_WORDS = NOALLOC_BYTES / 8;
constexpr size_t NOALLOC_HDR = 2048;  // words for descriptors and tables

static __device__ __align__(256) u64 g_noalloc_scratch[NOALLOC_WORDS];

// Device address of g_noalloc_scratch per device ordinal, set on the first
// call made with that device current.
constexpr int NOALLOC_MAX_DEV = 64;
static u64 *s_scratch[NOALLOC_MAX_DEV];

typedef unsigned __int128 u128;
static u64 nm(u64 a, u64 b, u64 q) { return (u64)((u128)a * b % q); }
static u64 npow(u64 a, u64 e, u64 q) {
    u64 r = 1 % q;
    a %= q;
    for (; e; e >>= 1) {
        if (e & 1) r = nm(r, a, q);
        a = nm(a, a, q);
    }
    return r;
}
static u64 ninv(u64 a, u64 q) { return npow(a, q - 2, q); }
static u64 nsh(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

}  // namespace hg

using namespace hg;

extern "C" int hegmm_rotate_noalloc(hegmm_ctx *h, const hegmm_ct *in, int z, hegmm_ct *out) {
    if (!h || !in || !out) return HEGMM_EINVAL;
    Ctx *c = &h->c;
    if (out->level != in->level) return set_err(c, HEGMM_EINVAL, "rotate_noalloc: output level differs from input");
    if (out->d == in->d) return set_err(c, HEGMM_EINVAL, "rotate_noalloc: output must not alias the input");
    const int lv = in->level, N = c->N, K = c->K, ne = lv + K, nd = c->digits(lv), a = c->alpha;
    const size_t need = NOALLOC_HDR + (size_t)lv * N + (size_t)nd * ne * N + (size_t)2 * ne * N + (size_t)2 * lv * N;
    if (need > NOALLOC_WORDS)
        return set_err(c, HEGMM_EINVAL,
                       "rotate_noalloc: these parameters need " + std::to_string(need * 8) +
                           " bytes of scratch, more than the fixed " + std::to_string(NOALLOC_BYTES) + " bytes");
    if (((long long)z % c->S) == 0) {
        cudaMemcpyAsync(out->d, in->d, (size_t)2 * lv * N * 8, cudaMemcpyDeviceToDevice, c->st);
        return cuda_check(c, "rotate_noalloc copy");
    }
    const u64 g = galois_of(c, z);
    auto kit = c->keys.find(g);
    if (kit == c->keys.end()) return set_err(c, HEGMM_ENOKEY, "rotate_noalloc: missing Galois key");

    // Set-up, once per device: the device address of the scratch array.
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEV)
        return cuda_check(c, "rotate_noalloc: device");
    if (!s_scratch[dev]) {
        u64 *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void **)&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return set_err(c, HEGMM_ECUDA, std::string("rotate_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        s_scratch[dev] = p;
    }
    u64 *S0 = s_scratch[dev];
    u64 *xc = S0 + NOALLOC_HDR;
    u64 *D = xc + (size_t)lv * N;
    u64 *u = D + (size_t)nd * ne * N;
    u64 *tmp = u + (size_t)2 * ne * N;

    // Header: RotDesc at word 0, two DivDesc at word 6, ModUp table at word
    // 16, ModDown table after it (same layouts as the context's tables).
    std::vector<u64> hdr(16, 0);
    RotDesc rd{D, kit->second, u, nullptr, nullptr, (u32)g, 0u};
    DivDesc dd[2];
    for (int comp = 0; comp < 2; comp++) {
        dd[comp].u = u + (size_t)comp * ne * N;
        dd[comp].tmp = tmp + (size_t)comp * lv * N;
        dd[comp].out = out->d + (size_t)comp * lv * N;
        dd[comp].add = comp == 0 ? in->d : nullptr;
        dd[comp].g = (u32)g;
        dd[comp].pad = 0;
    }
    static_assert(sizeof(RotDesc) == 48 && sizeof(DivDesc) == 40, "descriptor layout");
    memcpy(&hdr[0], &rd, sizeof(rd));
    memcpy(&hdr[6], dd, sizeof(dd));
    // ModUp table: [nd][a] {hinv, shoup}, [nd][a][ne] {hat mod r, shoup, q_i mod r}
    const size_t o_mu = hdr.size();
    hdr.resize(o_mu + (size_t)nd * a * 2 + (size_t)nd * a * ne * 3, 0);
    for (int j = 0; j < nd; j++) {
        const int lo = j * a, hi = std::min(lo + a, lv);
        for (int ii = 0; ii < hi - lo; ii++) {
            const int i = lo + ii;
            const u64 qi = c->q[i];
            u64 hq = 1;
            for (int i2 = lo; i2 < hi; i2++)
                if (i2 != i) hq = nm(hq, c->q[i2] % qi, qi);
            const u64 hv = ninv(hq, qi);
            hdr[o_mu + ((size_t)j * a + ii) * 2] = hv;
            hdr[o_mu + ((size_t)j * a + ii) * 2 + 1] = nsh(hv, qi);
            for (int e = 0; e < ne; e++) {
                const u64 r = c->q[c->gidx(lv, e)];
                u64 hr = 1;
                for (int i2 = lo; i2 < hi; i2++)
                    if (i2 != i) hr = nm(hr, c->q[i2] % r, r);
                u64 *dst = &hdr[o_mu + (size_t)nd * a * 2 + (((size_t)j * a + ii) * ne + e) * 3];
                dst[0] = hr;
                dst[1] = nsh(hr, r);
                dst[2] = qi % r;
            }
        }
    }
    // ModDown table: drop = special primes, keep = q_0..q_{lv-1}
    const size_t o_dv = hdr.size();
    for (int k = 0; k < K; k++) {
        const u64 dk = c->q[c->L + k];
        u64 hat = 1;
        for (int k2 = 0; k2 < K; k2++)
            if (k2 != k) hat = nm(hat, c->q[c->L + k2] % dk, dk);
        const u64 coef = nm(ninv(c->t % dk, dk), ninv(hat, dk), dk);
        hdr.push_back(coef);
        hdr.push_back(nsh(coef, dk));
    }
    for (int i = 0; i < lv; i++) {
        const u64 qi = c->q[i];
        for (int k = 0; k < K; k++) {
            u64 hat = 1;
            for (int k2 = 0; k2 < K; k2++)
                if (k2 != k) hat = nm(hat, c->q[c->L + k2] % qi, qi);
            hdr.push_back(hat);
            hdr.push_back(nsh(hat, qi));
            hdr.push_back(c->q[c->L + k] % qi);
        }
    }
    for (int i = 0; i < lv; i++) {
        const u64 qi = c->q[i];
        u64 P = 1;
        for (int k = 0; k < K; k++) P = nm(P, c->q[c->L + k] % qi, qi);
        const u64 Pi = ninv(P, qi);
        hdr.push_back(Pi);
        hdr.push_back(nsh(Pi, qi));
        hdr.push_back(c->t % qi);
        hdr.push_back(nsh(c->t % qi, qi));
    }
    for (int i = 0; i < lv; i++) hdr.push_back((u64)i);
    for (int k = 0; k < K; k++) hdr.push_back((u64)(c->L + k));
    if (hdr.size() > NOALLOC_HDR) return set_err(c, HEGMM_EINVAL, "rotate_noalloc: table header too large");
    // Every scratch word the kernels read is written earlier in this call, so
    // nothing has to be cleared; the header is rewritten on every call.
    cudaMemcpyAsync(S0, hdr.data(), hdr.size() * 8, cudaMemcpyHostToDevice, c->st);

    ModUpTab mt;
    mt.lv = lv;
    mt.ne = ne;
    mt.nd = nd;
    mt.d = S0 + o_mu;
    DivTab dt;
    dt.nkeep = lv;
    dt.ndrop = K;
    dt.d = S0 + o_dv;
    const RotDesc *d_rd = reinterpret_cast<const RotDesc *>(S0);
    const DivDesc *d_dd = reinterpret_cast<const DivDesc *>(S0 + 6);

    // hoisted ModUp of c1
    cudaMemcpyAsync(xc, in->d + (size_t)lv * N, (size_t)lv * N * 8, cudaMemcpyDeviceToDevice, c->st);
    int rc;
    if ((rc = ntt_inv(c, pat_ct(c, xc, 1, lv)))) return rc;
    if ((rc = modup_conv_tab(c, mt, 1, xc, (long long)lv * N, in->d + (size_t)lv * N, (long long)lv * N, D,
                             (long long)nd * ne * N)))
        return rc;
    LimbPat pn{};
    pn.base = D;
    pn.outer_stride = (long long)nd * ne * N;
    int k = 0;
    for (int j = 0; j < nd; j++) {
        const int lo = j * a, hi = std::min(lo + a, lv);
        for (int e = 0; e < ne; e++) {
            if (e >= lo && e < hi) continue;
            pn.off[k] = (unsigned short)(j * ne + e);
            pn.mod[k] = (unsigned char)c->gidx(lv, e);
            k++;
        }
    }
    pn.inner = k;
    pn.count = k;
    if ((rc = ntt_fwd(c, pn))) return rc;
    // inner product with the Galois key (fused automorphism), ModDown
    if ((rc = ksw_ip(c, lv, d_rd, 1))) return rc;
    LimbPat pd{};
    pd.base = u;
    pd.outer_stride = (long long)ne * N;
    pd.inner = K;
    pd.count = 2 * K;
    for (int q = 0; q < K; q++) {
        pd.off[q] = (unsigned short)(lv + q);
        pd.mod[q] = (unsigned char)(c->L + q);
    }
    if ((rc = ntt_inv(c, pd))) return rc;
    if ((rc = div_conv(c, dt, d_dd, 2))) return rc;
    if ((rc = ntt_fwd(c, pat_ct(c, tmp, 2, lv)))) return rc;
    if ((rc = div_combine(c, dt, d_dd, 2))) return rc;
    return cuda_check(c, "rotate_noalloc");
}

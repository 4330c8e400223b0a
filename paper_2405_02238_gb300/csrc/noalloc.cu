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

}  // namespace hg

using namespace hg;

extern "C" int hegmm_rotate_noalloc(hegmm_ctx *h, const hegmm_ct *in, int z, hegmm_ct *out) {
    if (!h || !in || !out) return HEGMM_EINVAL;
    Ctx *c = &h->c;
    if (out->level != in->level) return set_err(c, HEGMM_EINVAL, "rotate_noalloc: output level differs from input");
    if (out->d == in->d) return set_err(c, HEGMM_EINVAL, "rotate_noalloc: output must not alias the input");
    const int lv = in->level, N = c->N, K = c->K, ne = lv + K, nd = c->digits(lv);
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

    // A call under stream capture would record the header upload below
    // against a host buffer that the capture does not own.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->st, &cap) != cudaSuccess) return cuda_check(c, "rotate_noalloc: capture status");
    if (cap != cudaStreamCaptureStatusNone)
        return set_err(c, HEGMM_EINVAL, "rotate_noalloc: the context stream is capturing; call it outside capture");

    // Set-up, once per device: the device address of the scratch array.
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return cuda_check(c, "rotate_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= NOALLOC_MAX_DEV)
        return set_err(c, HEGMM_EINVAL,
                       "rotate_noalloc: device ordinal " + std::to_string(dev) + " beyond the scratch table (" +
                           std::to_string(NOALLOC_MAX_DEV) + " devices)");
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

    // Header: RotDesc at word 0, two DivDesc at word 6, then the ModUp and
    // ModDown tables of this level (the context's table layouts, built by
    // the same host functions and kept per level in host memory).
    auto tit = c->noalloc_tabs.find(lv);
    if (tit == c->noalloc_tabs.end()) {
        std::vector<int> keep, drop;
        std::vector<u64> t = modup_table_host(c, lv);
        const size_t first = t.size();
        const std::vector<u64> dv = div_table_host(c, lv, c->bfv ? 2 : 0, keep, drop);
        t.insert(t.end(), dv.begin(), dv.end());
        // the kernels read modulus indices from the ModDown table: check
        // where they sit before the table goes to the device
        const size_t idx = first + (size_t)2 * K + (size_t)3 * lv * K + (size_t)4 * lv;
        bool ok = t.size() >= idx + lv + K;
        for (int i = 0; ok && i < lv; i++) ok = t[idx + i] == (u64)i;
        for (int k = 0; ok && k < K; k++) ok = t[idx + lv + k] == (u64)(c->L + k);
        if (!ok) return set_err(c, HEGMM_EINVAL, "rotate_noalloc: ModDown table layout mismatch");
        tit = c->noalloc_tabs.emplace(lv, std::make_pair(first, std::move(t))).first;
    }
    const size_t n_mu = tit->second.first;  // words of the ModUp table (with its extension)
    const std::vector<u64> &tabs = tit->second.second;
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
    const size_t o_mu = hdr.size(), o_dv = o_mu + n_mu;
    hdr.insert(hdr.end(), tabs.begin(), tabs.end());
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
    const LimbPat pn = pat_nonown(c, lv, D, 1, (long long)nd * ne * N);
    if ((rc = ntt_fwd(c, pn))) return rc;
    // inner product with the Galois key (fused automorphism), ModDown
    if ((rc = ksw_ip(c, lv, d_rd, 1))) return rc;
    const LimbPat pd = pat_drop_special(c, lv, u, 2);
    if ((rc = ntt_inv(c, pd))) return rc;
    if ((rc = div_conv(c, dt, d_dd, 2))) return rc;
    if ((rc = ntt_fwd(c, pat_ct(c, tmp, 2, lv)))) return rc;
    if ((rc = div_combine(c, dt, d_dd, 2))) return rc;
    return cuda_check(c, "rotate_noalloc");
}

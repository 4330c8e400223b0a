// device.cuh -- per-thread building blocks of the HEGMM kernels.
//
// Functions are __host__ __device__ so the index arithmetic can be checked on
// the CPU; 128-bit products use __umul64hi on the device and unsigned
// __int128 on the host.
#pragma once
#include <stdint.h>

#include <vector>

typedef uint64_t u64;
typedef uint32_t u32;

#ifdef __CUDACC__
#define HDI __host__ __device__ __forceinline__
#else
#define HDI inline
#endif

namespace hg {

HDI u64 mulhi(u64 a, u64 b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (u64)(((unsigned __int128)a * b) >> 64);
#endif
}

HDI u64 addm(u64 a, u64 b, u64 q) {
    u64 r = a + b;
    return r >= q ? r - q : r;
}

HDI u64 subm(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }

// a w mod q for a < 2^64, w < q < 2^63, wp = floor(w 2^64 / q)  (Shoup).
HDI u64 mulsh(u64 a, u64 w, u64 wp, u64 q) {
    u64 h = mulhi(a, wp);
    u64 r = a * w - h * q;
    return r >= q ? r - q : r;
}

// a b 2^-64 mod q for a < 2^64, b < q, qinv = q^-1 mod 2^64 (Montgomery).
HDI u64 montmul(u64 a, u64 b, u64 q, u64 qinv) {
    u64 lo = a * b, hi = mulhi(a, b);
    u64 mh = mulhi(lo * qinv, q);
    return hi >= mh ? hi - mh : hi - mh + q;
}

struct Acc {
    u64 lo, hi;
};

// a += x y (exact 128-bit sum).  On the device the four 32 x 32-bit partial
// products go straight into the accumulator's four words through
// carry-chained multiply-adds: x0 y0 and x1 y1 in one chain, then the two
// cross products at 2^32.
HDI void mac(Acc &a, u64 x, u64 y) {
#ifdef __CUDA_ARCH__
    asm("{\n\t"
        ".reg .u32 x0, x1, y0, y1, a0, a1, a2, a3;\n\t"
        "mov.b64 {x0, x1}, %2;\n\t"
        "mov.b64 {y0, y1}, %3;\n\t"
        "mov.b64 {a0, a1}, %0;\n\t"
        "mov.b64 {a2, a3}, %1;\n\t"
        "mad.lo.cc.u32 a0, x0, y0, a0;\n\t"
        "madc.hi.cc.u32 a1, x0, y0, a1;\n\t"
        "madc.lo.cc.u32 a2, x1, y1, a2;\n\t"
        "madc.hi.u32 a3, x1, y1, a3;\n\t"
        "mad.lo.cc.u32 a1, x0, y1, a1;\n\t"
        "madc.hi.cc.u32 a2, x0, y1, a2;\n\t"
        "addc.u32 a3, a3, 0;\n\t"
        "mad.lo.cc.u32 a1, x1, y0, a1;\n\t"
        "madc.hi.cc.u32 a2, x1, y0, a2;\n\t"
        "addc.u32 a3, a3, 0;\n\t"
        "mov.b64 %0, {a0, a1};\n\t"
        "mov.b64 %1, {a2, a3};\n\t"
        "}"
        : "+l"(a.lo), "+l"(a.hi)
        : "l"(x), "l"(y));
#else
    u64 lo = x * y, hi = mulhi(x, y);
    u64 n = a.lo + lo;
    a.hi += hi + (n < lo ? 1 : 0);
    a.lo = n;
#endif
}

// (hi 2^64 + lo) 2^-64 mod q for a value below q 2^64.
HDI u64 montred(Acc a, u64 q, u64 qinv) {
    u64 mh = mulhi(a.lo * qinv, q);
    return a.hi >= mh ? a.hi - mh : a.hi - mh + q;
}

// v mod r for any v < 2^64; br = floor(2^64 / r).
HDI u64 redc64(u64 v, u64 r, u64 br) { return mulsh(v, 1, br, r); }

// Centred value of v in [0, p) reduced into [0, r); pr = p mod r.
HDI u64 centred(u64 v, u64 p, u64 pr, u64 r, u64 br) {
    u64 vr = redc64(v, r, br);
    return v <= (p - 1) / 2 ? vr : subm(vr, pr, r);
}

HDI u32 brev_bits(u32 x, int bits) {
#ifdef __CUDA_ARCH__
    return __brev(x) >> (32 - bits);
#else
    u32 r = 0;
    for (int i = 0; i < bits; i++) r |= ((x >> i) & 1u) << (bits - 1 - i);
    return r;
#endif
}

// NTT-domain automorphism X -> X^g: position c holds the evaluation at
// psi^(2 brev(c) + 1); the output at c reads the input at the position of
// exponent (2 brev(c) + 1) g mod 2N.
HDI u32 auto_src(u32 c, u32 g, int logN) {
    u32 e = 2u * brev_bits(c, logN) + 1u;
    u32 eg = (u32)(((u64)e * g) & ((2ull << logN) - 1));
    return brev_bits((eg - 1u) >> 1, logN);
}

#ifdef __CUDACC__
// mbarrier and bulk-copy (TMA engine) helpers.  A bulk copy moves bytes
// (a multiple of 16, both addresses 16-byte aligned) from global to shared
// memory and reports completion to an mbarrier as transaction bytes.
__device__ __forceinline__ u32 smem_addr(const void *p) { return (u32)__cvta_generic_to_shared(p); }

// One 8-byte asynchronous copy global -> shared (no register is held while
// it is in flight); cp_async_wait_all waits for the calling thread's copies.
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void mbar_init(u64 *bar, u32 count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(u64 *bar, u32 bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, u32 bytes, u64 *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(u64 *bar, u32 parity) {
    u32 ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void mbar_arrive(u64 *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// Bounded wait for the phase of the given parity: false if it did not
// complete within the limit.
__device__ __forceinline__ bool mbar_wait_bounded(u64 *bar, u32 parity, int limit) {
    for (int i = 0; i < limit; i++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

#endif  // __CUDACC__

// Shoup product with an approximate quotient: a w mod q left in [0, 4q),
// for a < 2^64, w < q < 2^62, wp = floor(w 2^64 / q).  The quotient
// floor(a wp / 2^64) is taken from three of the four 32 x 32-bit partial
// products (a1 p1 + hi(a1 p0) + hi(a0 p1)); the dropped low parts make it
// smaller by 0, 1 or 2, so the remainder a w - h q is the Shoup remainder
// ([0, 2q)) plus at most 2q.  Host and device compute the same h.
HDI u64 mulsh_approx(u64 a, u64 w, u64 wp, u64 q) {
#ifdef __CUDA_ARCH__
    u64 h;
    asm("{\n\t"
        ".reg .u32 a0, a1, p0, p1, t1, t2, s0, s1;\n\t"
        ".reg .u64 s;\n\t"
        "mov.b64 {a0, a1}, %1;\n\t"
        "mov.b64 {p0, p1}, %2;\n\t"
        "mul.hi.u32 t1, a1, p0;\n\t"
        "mul.hi.u32 t2, a0, p1;\n\t"
        "add.cc.u32 s0, t1, t2;\n\t"
        "addc.u32 s1, 0, 0;\n\t"
        "mov.b64 s, {s0, s1};\n\t"
        "mad.wide.u32 %0, a1, p1, s;\n\t"
        "}"
        : "=l"(h)
        : "l"(a), "l"(wp));
#else
    const u64 a0 = (u32)a, a1 = a >> 32, p0 = (u32)wp, p1 = wp >> 32;
    const u64 h = a1 * p1 + ((a1 * p0) >> 32) + ((a0 * p1) >> 32);
#endif
    return a * w - h * q;
}

// Centred lift of v in [0, p) into [0, r) when p < 2 r (every prime of a
// context has the same bit length): v itself below p / 2, else v - p + r;
// d = r - p mod 2^64.
HDI u64 centred_narrow(u64 v, u64 half_p, u64 d) { return v > half_p ? v + d : v; }

#ifdef __CUDACC__
// Brings the 128-byte line holding p into L2 (no register result, no fault
// on the line's contents; p must point into an allocation).
__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }
#endif

// Padded shared-memory index: one spare word every 16 keeps the strided
// butterfly accesses of every pass at two wavefronts per warp.
HDI int pad16(int i) { return i + (i >> 4); }

// A twiddle and its Shoup companion, loaded together (one 16-byte load).
struct alignas(16) TwPair {
    u64 w, wp;
};

// a w mod q left in [0, 2q) (Shoup without the final correction).
HDI u64 mulsh_lazy(u64 a, u64 w, u64 wp, u64 q) { return a * w - mulhi(a, wp) * q; }

// Lazy butterflies.  Each butterfly leaves its outputs at most 4q above its
// inputs (T = w Y mod q in [0, 4q) from mulsh_approx; X + T and X - T + 4q)
// and reduces nothing, so after the log2 N <= 14 stages of a transform the
// values stay below (input bound + 56) q; with q < 2^56 and inputs below
// 16 q everything stays below 128 q < 2^63.  Values are reduced once, when
// they leave the transform.
HDI void bfly_ct(u64 &X, u64 &Y, const TwPair &t, u64 q4, u64 q) {
    const u64 T = mulsh_approx(Y, t.w, t.wp, q);
    const u64 x = X;
    X = x + T;
    Y = x + (q4 - T);
}

// Forward negacyclic NTT (Cooley-Tukey, bit-reversed psi powers): one group
// of 2^R elements held in registers through stages s0 .. s0+R-1; B is the
// group's block index, tw[k] = psi^brev(k) with its Shoup companion.
template <int R>
HDI void ntt_fwd_regs(u64 *x, int B, int s0, const TwPair *tw, u64 q) {
    const u64 q4 = 4 * q;
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int half = 1 << (R - 1 - r);
#pragma unroll
        for (int k = 0; k < (1 << R); k++) {
            if (k & half) continue;
            bfly_ct(x[k], x[k + half], tw[((1 << s0) << r) + (B << r) + (k >> (R - r))], q4, q);
        }
    }
}

// The same group staged in shared memory: group g covers elements
// base + k tl, k < 2^R.
template <int R>
HDI void ntt_fwd_group_lazy(u64 *sm, int g, int s0, int logN, const TwPair *tw, u64 q) {
    const int ltl = logN - s0 - R;
    const int tl = 1 << ltl;
    const int B = g >> ltl, o = g & (tl - 1);
    const int base = (B << (ltl + R)) + o;
    u64 x[1 << R];
#pragma unroll
    for (int k = 0; k < (1 << R); k++) x[k] = sm[pad16(base + k * tl)];
    ntt_fwd_regs<R>(x, B, s0, tw, q);
#pragma unroll
    for (int k = 0; k < (1 << R); k++) sm[pad16(base + k * tl)] = x[k];
}

// Inverse transform as a cyclic inverse DFT in Cooley-Tukey
// (decimation-in-time) form: the NTT domain holds the evaluations at
// psi omega^k (omega = psi^2) in bit-reversed order, which is the order this
// form reads; its output (natural order) is multiplied by N^-1 psi^-i when
// it leaves (a_i = N^-1 psi^-i sum_k a^_k omega^-ik).  One group of 2^R
// elements in registers: element k of the group is element base + k 2^u0
// of the limb, base = B 2^(u0+R) + o with o < 2^u0; stage r pairs k and
// k + 2^r (span 2^(u0+r) in the limb) with omega^(-j N / 2^(u0+r+1)),
// j = o + (k mod 2^r) 2^u0, stored at tw[2^(u0+r) + j].
template <int R>
HDI void ntt_inv_ct_regs(u64 *x, int o, int u0, const TwPair *tw, u64 q) {
    const u64 q4 = 4 * q;
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int h = 1 << r;
#pragma unroll
        for (int k = 0; k < (1 << R); k++) {
            if (k & h) continue;
            bfly_ct(x[k], x[k + h], tw[(1 << (u0 + r)) + o + ((k & (h - 1)) << u0)], q4, q);
        }
    }
}

template <int R>
HDI void ntt_inv_ct_group(u64 *sm, int g, int u0, const TwPair *tw, u64 q) {
    const int tl = 1 << u0;
    const int B = g >> u0, o = g & (tl - 1);
    const int base = (B << (u0 + R)) + o;
    u64 x[1 << R];
#pragma unroll
    for (int k = 0; k < (1 << R); k++) x[k] = sm[pad16(base + k * tl)];
    ntt_inv_ct_regs<R>(x, o, u0, tw, q);
#pragma unroll
    for (int k = 0; k < (1 << R); k++) sm[pad16(base + k * tl)] = x[k];
}

// Twiddle tables of one prime (host side; shared by the context and by host
// checks of the transforms): out[3][N] pairs {w, floor(w 2^64 / q)}:
// [0][k] = psi^brev(k) (forward), [1][h + j] = omega^(-j N / (2h)) for
// h = 1, 2, .., N/2 and j < h (inverse, index 0 unused), [2][i] =
// N^-1 psi^-i (the inverse's output factor).  psi: a primitive 2N-th root.
inline void build_twiddles_host(u64 q, u64 psi, int logN, u64 *out) {
    const int N = 1 << logN;
    auto mm = [q](u64 a, u64 b) { return (u64)((unsigned __int128)a * b % q); };
    auto sh = [q](u64 w) { return (u64)(((unsigned __int128)w << 64) / q); };
    u64 ipsi = 1, ninv = 1;  // psi^-1 = psi^(2N-1), N^-1 = q - (q-1)/N (q = 1 mod 2N)
    for (int i = 0; i < 2 * N - 1; i++) ipsi = mm(ipsi, psi);
    ninv = q - (q - 1) / (u64)N;
    std::vector<u64> pw((size_t)N), ipw((size_t)N);
    pw[0] = ipw[0] = 1;
    for (int i = 1; i < N; i++) {
        pw[i] = mm(pw[i - 1], psi);
        ipw[i] = mm(ipw[i - 1], ipsi);
    }
    u64 *T0 = out, *T1 = out + 2 * (size_t)N, *T2 = out + 4 * (size_t)N;
    for (int k = 0; k < N; k++) {
        const u64 w = pw[brev_bits((u32)k, logN)];
        T0[2 * k] = w;
        T0[2 * k + 1] = sh(w);
        T2[2 * k] = mm(ninv, ipw[k]);
        T2[2 * k + 1] = sh(T2[2 * k]);
    }
    T1[0] = T1[1] = 0;
    for (int h = 1; h < N; h <<= 1)
        for (int j = 0; j < h; j++) {
            const u64 w = ipw[(size_t)j * (N / h)];  // omega^-(j N / 2h) = psi^-(j N / h)
            T1[2 * (h + j)] = w;
            T1[2 * (h + j) + 1] = sh(w);
        }
}

// SplitMix64 (Steele, Lea, Flood 2014) in counter mode.
constexpr u64 SM_GAMMA = 0x9E3779B97F4A7C15ull;

HDI u64 mix64(u64 z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

HDI u64 rng_stream(u64 seed, u64 domain, u64 obj) { return mix64(seed ^ mix64((domain << 48) | obj)); }
HDI u64 rng_draw(u64 stream, u64 idx) { return mix64(stream + (idx + 1) * SM_GAMMA); }

// Centred binomial sample: popcount(low eta bits) - popcount(next eta bits).
HDI long long cbd_sample(u64 r, int eta) {
    const u64 m = (1ull << eta) - 1;
#ifdef __CUDA_ARCH__
    return (long long)__popcll(r & m) - (long long)__popcll((r >> eta) & m);
#else
    return (long long)__builtin_popcountll(r & m) - (long long)__builtin_popcountll((r >> eta) & m);
#endif
}

// Random-stream domains (shared definition with every other implementation
// of the same scheme conventions).
enum { DOM_SK = 1, DOM_KEY_A = 2, DOM_KEY_E = 3, DOM_ENC_A = 4, DOM_ENC_E = 5 };

}  // namespace hg

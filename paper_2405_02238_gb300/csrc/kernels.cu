// kernels.cu -- CUDA kernels of the HEGMM library (sm_103a) and their launchers.
//
// Data layout: every polynomial is a sequence of limbs, one limb = N uint64
// residues of one modulus; ciphertexts are [2][level][N]; ModUp digits are
// [digits][level + K][N]; keys are [dnum][2][L + K][N] in Montgomery form.
// All kernels are grid-strided over the N coefficients of each limb, so
// consecutive threads touch consecutive words (coalesced 256-byte warps).
#include <cuda_runtime.h>

#include <algorithm>

#include "device.cuh"
#include "internal.h"

namespace hg {

// ------------------------------------------------------------------ timing

Launch::Launch(Ctx *c_, int kind_, double bytes_, double work_) : c(c_), kind(kind_), bytes(bytes_), work(work_) {
    if (!c->timing) return;
    if (c->evpool.size() < 2) {
        for (int i = 0; i < 64; i++) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            c->evpool.push_back(e);
        }
    }
    a = c->evpool.back();
    c->evpool.pop_back();
    b = c->evpool.back();
    c->evpool.pop_back();
    cudaEventRecord(a, c->st);
}

Launch::~Launch() {
    if (!a) return;
    cudaEventRecord(b, c->st);
    c->pending.push_back({kind, a, b, bytes, work});
}

// ------------------------------------------------------------------ helpers

// Block b of a pattern launch: blocks are ordered modulus-major (all outers
// of inner entry 0 first), so consecutive CTAs -- and the CTAs an SM runs
// one after another -- use the same modulus and its twiddle table stays in L1.
static __device__ __forceinline__ u64 *pat_ptr(const LimbPat &p, int b, int N, int &mod) {
    const int nouter = p.count / p.inner;
    const int in = b / nouter, outer = b - in * nouter;
    u64 *base = p.outer_ptrs ? p.outer_ptrs[outer] : p.base + (long long)outer * p.outer_stride;
    mod = p.mod[in];
    return base + (size_t)p.off[in] * N;
}

constexpr int kMaxGridZ = 65535;  // grid.z limit; launches over more items are split
static inline dim3 grid_coef(int N, int y, int z) { return dim3((unsigned)((N + 255) / 256), (unsigned)y, (unsigned)z); }

// ------------------------------------------------------------------ NTT
// One CTA per limb.  The limb is staged in (padded) shared memory; radix-8
// passes run three butterfly stages in registers per group of eight
// elements, so N = 2^14 takes five shared-memory passes.

// The ring degree is a template parameter (logN = 10..14), so every pass,
// stride and twiddle index folds to constants; butterflies are lazy
// (Harvey): forward values stay in [0, 4q), inverse values in [0, 2q), and
// are reduced once when the limb leaves shared memory.

// Up to N = 2^13 two CTAs of 512 threads share an SM (registers 2 x 512 x 64,
// shared memory 2 x 70 KB), so one CTA's loads and barriers overlap the
// other's butterflies; at N = 2^14 the 139 KB limb allows one CTA per SM.
//
// A launch of no more CTAs than SMs leaves every CTA an SM of its own; there
// the NT_WIDE form (one radix-8 group per thread and pass, up to 1024
// threads) halves the latency of each pass at N = 2^13.
//
// Every kernel exists in two thread counts, NT_A (up to 512) and NT_B (up to
// 1024); HEGMM_TUNE_NTT_THREADS forces one of them (hegmm_autotune tries
// both), else NT at N = 2^14 and the rule above below it.
template <int LOGN>
struct NttCfg {
    static constexpr int N = 1 << LOGN;
    static constexpr int NT_A = (N / 8) < 512 ? (N / 8) : 512;
    static constexpr int NT_B = (N / 8) < 1024 ? (N / 8) : 1024;
    static constexpr int NT = LOGN >= 14 ? NT_B : NT_A;
    static constexpr int NT_WIDE = NT_B;
    static constexpr size_t SMEM = (size_t)(N + N / 16) * 8;
};

// CTAs per SM the register budget is set for: one for 1024 threads or when
// the limb takes more than half of the SM's shared memory (N = 2^14: 512
// threads then get 128 registers each), else two.
template <int LOGN, int NT>
struct NttMinBlocks {
    static constexpr int V = (NT >= 1024 || 2 * NttCfg<LOGN>::SMEM > (size_t)227 * 1024) ? 1 : 2;
};

// Fused pass layout of the kernels below: the first radix-8 pass (stages
// 0..2) runs on register values the kernel's prologue produces (no shared
// memory round trip before it), the middle radix-8 passes through shared
// memory, and the last pass of RL stages ends in registers that the
// kernel's epilogue consumes directly.  Forward: group g of the first pass
// holds elements g + k N/8, of the last pass elements (g << RL) + k;
// inverse: the first pass holds (g << 3) + k, the last g + k 2^LAST.
template <int LOGN>
struct NttPasses {
    static constexpr int RL = (LOGN % 3) ? (LOGN % 3) : 3;
    static constexpr int LAST = LOGN - RL;  // first stage of the last pass
};

template <int LOGN, int NT>
__device__ __forceinline__ void fwd_middle(u64 *sm, const TwPair *__restrict__ T, u64 q) {
    constexpr int N = 1 << LOGN, LAST = NttPasses<LOGN>::LAST;
#pragma unroll
    for (int s0 = 3; s0 < LAST; s0 += 3) {
        for (int g = threadIdx.x; g < N / 8; g += NT) ntt_fwd_group_lazy<3>(sm, g, s0, LOGN, T, q);
        __syncthreads();
    }
}

template <int LOGN, int NT>
__device__ __forceinline__ void inv_middle(u64 *sm, const TwPair *__restrict__ T, u64 q) {
    constexpr int N = 1 << LOGN, LAST = NttPasses<LOGN>::LAST;
#pragma unroll
    for (int u0 = 3; u0 < LAST; u0 += 3) {
        for (int g = threadIdx.x; g < N / 8; g += NT) ntt_inv_ct_group<3>(sm, g, u0, T, q);
        __syncthreads();
    }
}

// Twiddle table layout: [modulus][0 = forward psi^brev(k), 1 = inverse
// omega^-j by span, 2 = inverse output factor N^-1 psi^-i][N] pairs
// (build_twiddles_host).
__device__ __forceinline__ const TwPair *tw_of(const TwPair *tw, int mi, int which, int N) {
    return tw + ((size_t)mi * 3 + which) * N;
}

// One CTA per limb.  Forward: values leave reduced to [0, q).  Inverse: the
// output is the coefficient vector in [0, q), multiplied by scale[i] (a
// {w, Shoup companion} pair per inner entry i of the pattern) when scale is
// not null.
template <int LOGN, bool INV, int NT>
__global__ void __launch_bounds__(NT, NttMinBlocks<LOGN, NT>::V) k_ntt(LimbPat p, const ModDev *__restrict__ mods,
                                                                 const TwPair *__restrict__ tw,
                                                                 const TwPair *__restrict__ scale) {
    extern __shared__ u64 sm[];
    constexpr int N = 1 << LOGN, RL = NttPasses<LOGN>::RL, LAST = NttPasses<LOGN>::LAST;
    int mi;
    u64 *ptr = pat_ptr(p, blockIdx.x, N, mi);
    const u64 q = mods[mi].q;
    if (INV) {
        const TwPair *T = tw_of(tw, mi, 1, N);
        // first pass on registers: group g is the 8 consecutive elements 8g .. 8g+7
        for (int g = threadIdx.x; g < N / 8; g += NT) {
            u64 x[8];
#pragma unroll
            for (int k = 0; k < 8; k += 2) {
                const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2 *>(ptr + 8 * g + k));
                x[k] = v.x;
                x[k + 1] = v.y;
            }
            ntt_inv_ct_regs<3>(x, 0, 0, T, q);
#pragma unroll
            for (int k = 0; k < 8; k++) sm[pad16(8 * g + k)] = x[k];
        }
        __syncthreads();
        inv_middle<LOGN, NT>(sm, T, q);
        // last pass on registers, then the output factor N^-1 psi^-i (and the
        // optional limb scale), stored in natural order
        const TwPair *F = tw_of(tw, mi, 2, N);
        TwPair sc{0, 0};
        if (scale) sc = scale[blockIdx.x / (p.count / p.inner)];
        for (int g = threadIdx.x; g < (N >> RL); g += NT) {
            u64 x[1 << RL];
#pragma unroll
            for (int k = 0; k < (1 << RL); k++) x[k] = sm[pad16(g + (k << LAST))];
            ntt_inv_ct_regs<RL>(x, g, LAST, T, q);
#pragma unroll
            for (int k = 0; k < (1 << RL); k++) {
                const int e = g + (k << LAST);
                const TwPair f = F[e];
                ptr[e] = scale ? mulsh(mulsh_lazy(x[k], f.w, f.wp, q), sc.w, sc.wp, q) : mulsh(x[k], f.w, f.wp, q);
            }
        }
    } else {
        const TwPair *T = tw_of(tw, mi, 0, N);
        for (int g = threadIdx.x; g < N / 8; g += NT) {
            u64 x[8];
#pragma unroll
            for (int k = 0; k < 8; k++) x[k] = ptr[g + k * (N / 8)];
            ntt_fwd_regs<3>(x, 0, 0, T, q);
#pragma unroll
            for (int k = 0; k < 8; k++) sm[pad16(g + k * (N / 8))] = x[k];
        }
        __syncthreads();
        fwd_middle<LOGN, NT>(sm, T, q);
        const u64 barr = mods[mi].barr;
        for (int g = threadIdx.x; g < (N >> RL); g += NT) {
            u64 x[1 << RL];
#pragma unroll
            for (int k = 0; k < (1 << RL); k++) x[k] = sm[pad16((g << RL) + k)];
            ntt_fwd_regs<RL>(x, g, LAST, T, q);
#pragma unroll
            for (int k = 0; k < (1 << RL); k++) ptr[(g << RL) + k] = redc64(x[k], q, barr);
        }
    }
}

// ModDown / modulus switch, fused: one CTA per (polynomial, kept prime q_i).
// The dropped limbs arrive in coefficient form already multiplied by
// [t^-1 (D/d_k)^-1]_{d_k} (the scale of their inverse NTT), z_k.
// Prologue: t y~_i = sum_k centred(z_k) [t (D/d_k)]_{q_i}, kept lazily below
// 4 ndrop q_i; forward NTT in shared memory (values grow by at most 4 q_i a
// stage); epilogue: out_i = (u_i - t y~_i) D^-1 (+ add_i at the
// automorphism's index), computed as (u_i + 128 q_i - t y~_i) D^-1 with one
// reducing Shoup product.  Table layout: build_div_tab; NARROW: every
// dropped prime below twice every kept one (centred_narrow).
template <int LOGN, int NT, bool NARROW>
__global__ void __launch_bounds__(NT, NttMinBlocks<LOGN, NT>::V) k_divround_ntt(int nkeep, int ndrop,
                                                                          const ModDev *__restrict__ mods,
                                                                          const u64 *__restrict__ tab, int ext,
                                                                          const DivDesc *__restrict__ desc,
                                                                          const TwPair *__restrict__ tw) {
    extern __shared__ u64 sm[];
    constexpr int N = 1 << LOGN;
    const int npoly = gridDim.x / nkeep;  // prime-major block order (twiddles stay in L1)
    const int i = blockIdx.x / npoly, b = blockIdx.x - i * npoly;
    const DivDesc d = desc[b];
    const u64 *tB = tab + 2 * ndrop;
    const u64 *tC = tB + (size_t)3 * nkeep * ndrop;
    const u64 *tI = tC + (size_t)4 * nkeep;
    const int mi = (int)tI[i];
    const ModDev M = mods[mi];
    const u64 *hB = tB + (size_t)i * ndrop * 3;
    const u64 *hE = tab + ext + (size_t)i * ndrop * 3;
    const TwPair *T = tw_of(tw, mi, 0, N);
    constexpr int RL = NttPasses<LOGN>::RL, LAST = NttPasses<LOGN>::LAST;
    // the epilogue reads u_i (and add_i): ask L2 for them now, so that their
    // DRAM latency passes under the transform (one 128-byte line a thread)
    for (int w = threadIdx.x * 16; w < N; w += NT * 16) {
        prefetch_l2(d.u + (size_t)i * N + w);
        if (d.add) prefetch_l2(d.add + (size_t)i * N + w);
    }
    // prologue fused with the first pass: the conversion of the group's 8
    // coefficients, one dropped prime at a time (its constants loaded once)
    for (int g = threadIdx.x; g < N / 8; g += NT) {
        u64 x[8];
#pragma unroll
        for (int k = 0; k < 8; k++) x[k] = 0;
        for (int kk = 0; kk < ndrop; kk++) {
            const u64 dk = mods[tI[nkeep + kk]].q;
            const u64 lc = NARROW ? __ldg(hE + 3 * kk + 2) : __ldg(hB + 3 * kk + 2);
            const u64 w = __ldg(hE + 3 * kk), ws = __ldg(hE + 3 * kk + 1);
            const u64 *zp = d.u + (size_t)(nkeep + kk) * N + g;
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const u64 z = zp[k * (N / 8)];
                const u64 v = NARROW ? centred_narrow(z, dk >> 1, lc) : centred(z, dk, lc, M.q, M.barr);
                x[k] += mulsh_approx(v, w, ws, M.q);
            }
        }
        ntt_fwd_regs<3>(x, 0, 0, T, M.q);
#pragma unroll
        for (int k = 0; k < 8; k++) sm[pad16(g + k * (N / 8))] = x[k];
    }
    __syncthreads();
    fwd_middle<LOGN, NT>(sm, T, M.q);
    const u64 *k4 = tC + 4 * i;
    const u64 Di = k4[0], Dis = k4[1], q128 = M.q << 7;
    const u64 *ui = d.u + (size_t)i * N;
    u64 *oi = d.out + (size_t)i * N;
    // last pass fused with the epilogue
    for (int g = threadIdx.x; g < (N >> RL); g += NT) {
        u64 x[1 << RL];
        const int base = g << RL;
#pragma unroll
        for (int k = 0; k < (1 << RL); k++) x[k] = sm[pad16(base + k)];
        ntt_fwd_regs<RL>(x, g, LAST, T, M.q);
#pragma unroll
        for (int k = 0; k < (1 << RL); k++) {
            const int c = base + k;
            u64 v = mulsh(ui[c] + (q128 - x[k]), Di, Dis, M.q);
            if (d.add) v = addm(v, d.add[(size_t)i * N + (d.g == 1 ? (u32)c : auto_src((u32)c, d.g, LOGN))], M.q);
            oi[c] = v;
        }
    }
}

// The same ModDown with each output limb split between two CTAs of 512
// threads, one per half of the limb (the forward transform's first stage
// pairs c with c + N/2; every later stage stays inside a half).  Each CTA
// converts all N coefficients (the first stage needs both halves), computes
// that stage's outputs for its own half only, runs the remaining stages on
// N/2 values and writes its half; the values it produces are those of
// k_divround_ntt, stage for stage.  A half limb takes 69.6 KB of shared
// memory at N = 2^14, so two CTAs share an SM and one's loads and barriers
// overlap the other's butterflies.  Grid: 2 CTAs per (polynomial, kept
// prime), prime-major as k_divround_ntt.
template <int LOGN>
struct DivHalfCfg {
    static constexpr int N = 1 << LOGN, NT = 512;
    static constexpr size_t SMEM = (size_t)(N / 2 + N / 32) * 8;
};

template <int LOGN, bool NARROW>
__global__ void __launch_bounds__(512, 2) k_divround_half(int nkeep, int ndrop, const ModDev *__restrict__ mods,
                                                          const u64 *__restrict__ tab, int ext,
                                                          const DivDesc *__restrict__ desc,
                                                          const TwPair *__restrict__ tw) {
    extern __shared__ u64 sm[];
    constexpr int N = 1 << LOGN, NT = 512, HALF = N / 2, G = N / 8;
    constexpr int RL = NttPasses<LOGN>::RL, LAST = NttPasses<LOGN>::LAST;
    const int h = blockIdx.x & 1, cta = blockIdx.x >> 1;
    const int npoly = (gridDim.x >> 1) / nkeep;
    const int i = cta / npoly, b = cta - i * npoly;
    const DivDesc d = desc[b];
    const u64 *tB = tab + 2 * ndrop;
    const u64 *tC = tB + (size_t)3 * nkeep * ndrop;
    const u64 *tI = tC + (size_t)4 * nkeep;
    const int mi = (int)tI[i];
    const ModDev M = mods[mi];
    const u64 *hB = tB + (size_t)i * ndrop * 3;
    const u64 *hE = tab + ext + (size_t)i * ndrop * 3;
    const TwPair *T = tw_of(tw, mi, 0, N);
    const int off = h * HALF;  // first element of this CTA's half
    for (int w = threadIdx.x * 16; w < HALF; w += NT * 16) {
        prefetch_l2(d.u + (size_t)i * N + off + w);
        if (d.add) prefetch_l2(d.add + (size_t)i * N + off + w);
    }
    // prologue: the conversion of the group's 8 coefficients (both halves),
    // the first stage for this half's 4, then stages 1 and 2 on them
    const u64 q4 = 4 * M.q;
    for (int g = threadIdx.x; g < G; g += NT) {
        u64 x[8];
#pragma unroll
        for (int k = 0; k < 8; k++) x[k] = 0;
        for (int kk = 0; kk < ndrop; kk++) {
            const u64 dk = mods[tI[nkeep + kk]].q;
            const u64 lc = NARROW ? __ldg(hE + 3 * kk + 2) : __ldg(hB + 3 * kk + 2);
            const u64 w = __ldg(hE + 3 * kk), ws = __ldg(hE + 3 * kk + 1);
            const u64 *zp = d.u + (size_t)(nkeep + kk) * N + g;
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const u64 z = zp[k * (N / 8)];
                const u64 v = NARROW ? centred_narrow(z, dk >> 1, lc) : centred(z, dk, lc, M.q, M.barr);
                x[k] += mulsh_approx(v, w, ws, M.q);
            }
        }
        const TwPair t1 = T[1];
        u64 y[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const u64 t = mulsh_approx(x[k + 4], t1.w, t1.wp, M.q);
            y[k] = h ? x[k] + (q4 - t) : x[k] + t;
        }
        ntt_fwd_regs<2>(y, h, 1, T, M.q);
#pragma unroll
        for (int k = 0; k < 4; k++) sm[pad16(g + k * (N / 8))] = y[k];
    }
    __syncthreads();
    // middle passes on this half's groups
#pragma unroll
    for (int s0 = 3; s0 < LAST; s0 += 3) {
        const int ltl = LOGN - s0 - 3, tl = 1 << ltl;
        for (int gl = threadIdx.x; gl < G / 2; gl += NT) {
            const int g = gl + h * (G / 2);
            const int B = g >> ltl, o = g & (tl - 1);
            const int base = (B << (ltl + 3)) + o - off;
            u64 x[8];
#pragma unroll
            for (int k = 0; k < 8; k++) x[k] = sm[pad16(base + k * tl)];
            ntt_fwd_regs<3>(x, B, s0, T, M.q);
#pragma unroll
            for (int k = 0; k < 8; k++) sm[pad16(base + k * tl)] = x[k];
        }
        __syncthreads();
    }
    const u64 *k4 = tC + 4 * i;
    const u64 Di = k4[0], Dis = k4[1], q128 = M.q << 7;
    const u64 *ui = d.u + (size_t)i * N;
    u64 *oi = d.out + (size_t)i * N;
    // last pass fused with the epilogue
    for (int gl = threadIdx.x; gl < (HALF >> RL); gl += NT) {
        const int g = gl + h * (HALF >> RL);
        u64 x[1 << RL];
        const int base = g << RL;
#pragma unroll
        for (int k = 0; k < (1 << RL); k++) x[k] = sm[pad16(base + k - off)];
        ntt_fwd_regs<RL>(x, g, LAST, T, M.q);
#pragma unroll
        for (int k = 0; k < (1 << RL); k++) {
            const int c = base + k;
            u64 v = mulsh(ui[c] + (q128 - x[k]), Di, Dis, M.q);
            if (d.add) v = addm(v, d.add[(size_t)i * N + (d.g == 1 ? (u32)c : auto_src((u32)c, d.g, LOGN))], M.q);
            oi[c] = v;
        }
    }
}

// ModUp, fused: one CTA per (input, digit j, prime e outside digit j):
// prologue computes the digit's centred fast base conversion into prime e
// from the coefficient-form source limbs, which arrive already multiplied
// by [(Q_j/q_i)^-1]_{q_i} (the scale of their inverse NTT), summed lazily
// below 4 alpha r; then forward NTT, then the reduced store.  Limb
// selection follows a LimbPat whose off[] = j * ne + e.  NARROW: every
// source prime below twice every target prime (centred_narrow).
template <int LOGN, int NT, bool NARROW>
__global__ void __launch_bounds__(NT, NttMinBlocks<LOGN, NT>::V) k_modup_ntt(LimbPat p, int lv, int ne, int nd, int alpha,
                                                                       int L, const ModDev *__restrict__ mods,
                                                                       const u64 *__restrict__ tab, int ext,
                                                                       const u64 *__restrict__ xc, long long xc_stride,
                                                                       const TwPair *__restrict__ tw) {
    extern __shared__ u64 sm[];
    constexpr int N = 1 << LOGN;
    const int nouter = p.count / p.inner;  // prime-major block order, as pat_ptr
    const int in = blockIdx.x / nouter, outer = blockIdx.x - in * nouter;
    const int off = p.off[in], j = off / ne, e = off - j * ne;
    const int mi = p.mod[in];
    u64 *dst = (p.outer_ptrs ? p.outer_ptrs[outer] : p.base + (long long)outer * p.outer_stride) + (size_t)off * N;
    const u64 *x = xc + outer * xc_stride;
    const int lo = j * alpha, ns = min(alpha, lv - lo);
    const ModDev R = mods[mi];
    const u64 *thm = tab + (size_t)nd * alpha * 2 + (size_t)j * alpha * ne * 3;
    const u64 *tex = tab + ext + (size_t)j * alpha * ne;
    const TwPair *T = tw_of(tw, mi, 0, N);
    constexpr int RL = NttPasses<LOGN>::RL, LAST = NttPasses<LOGN>::LAST;
    // prologue fused with the first pass: the digit's conversion of the
    // group's coefficients, one source prime at a time (its constants loaded
    // once)
    for (int g = threadIdx.x; g < N / 8; g += NT) {
        u64 xv[8];
#pragma unroll
        for (int k = 0; k < 8; k++) xv[k] = 0;
        for (int ii = 0; ii < ns; ii++) {
            const u64 sq = mods[lo + ii].q;
            const u64 *h = thm + ((size_t)ii * ne + e) * 3;
            const u64 lc = NARROW ? __ldg(tex + (size_t)ii * ne + e) : __ldg(h + 2);
            const u64 w = __ldg(h), ws = __ldg(h + 1);
            const u64 *yp = x + (size_t)(lo + ii) * N + g;
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const u64 y = yp[k * (N / 8)];
                const u64 v = NARROW ? centred_narrow(y, sq >> 1, lc) : centred(y, sq, lc, R.q, R.barr);
                xv[k] += mulsh_approx(v, w, ws, R.q);
            }
        }
        ntt_fwd_regs<3>(xv, 0, 0, T, R.q);
#pragma unroll
        for (int k = 0; k < 8; k++) sm[pad16(g + k * (N / 8))] = xv[k];
    }
    __syncthreads();
    fwd_middle<LOGN, NT>(sm, T, R.q);
    for (int g = threadIdx.x; g < (N >> RL); g += NT) {
        u64 xv[1 << RL];
        const int base = g << RL;
#pragma unroll
        for (int k = 0; k < (1 << RL); k++) xv[k] = sm[pad16(base + k)];
        ntt_fwd_regs<RL>(xv, g, LAST, T, R.q);
#pragma unroll
        for (int k = 0; k < (1 << RL); k++) dst[base + k] = redc64(xv[k], R.q, R.barr);
    }
}

// The digits' own limbs: D_j = x on the primes of digit j (NTT form copy).
__global__ void k_modup_own(int lv, int ne, int alpha, int logN, const u64 *__restrict__ xn, long long xn_stride,
                            u64 *__restrict__ D, long long D_stride) {
    const int N = 1 << logN;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int e = blockIdx.y, o = blockIdx.z, j = e / alpha;
    D[o * D_stride + ((size_t)j * ne + e) * N + c] = xn[o * xn_stride + (size_t)e * N + c];
}

template <int LOGN, int NT>
static int set_smem_attrs_nt() {
    const int sm = (int)NttCfg<LOGN>::SMEM;
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if (cudaFuncSetAttribute(k_ntt<LOGN, false, NT>, A, sm) != cudaSuccess ||
        cudaFuncSetAttribute(k_ntt<LOGN, true, NT>, A, sm) != cudaSuccess ||
        cudaFuncSetAttribute(k_divround_ntt<LOGN, NT, false>, A, sm) != cudaSuccess ||
        cudaFuncSetAttribute(k_divround_ntt<LOGN, NT, true>, A, sm) != cudaSuccess ||
        cudaFuncSetAttribute(k_modup_ntt<LOGN, NT, false>, A, sm) != cudaSuccess ||
        cudaFuncSetAttribute(k_modup_ntt<LOGN, NT, true>, A, sm) != cudaSuccess)
        return 1;
    return 0;
}

template <int LOGN>
static int set_smem_attrs() {
    if (set_smem_attrs_nt<LOGN, NttCfg<LOGN>::NT_A>() || set_smem_attrs_nt<LOGN, NttCfg<LOGN>::NT_B>()) return 1;
    if constexpr (LOGN >= 13) {
        const int sm = (int)DivHalfCfg<LOGN>::SMEM;
        const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
        if (cudaFuncSetAttribute(k_divround_half<LOGN, false>, A, sm) != cudaSuccess ||
            cudaFuncSetAttribute(k_divround_half<LOGN, true>, A, sm) != cudaSuccess)
            return 1;
    }
    return 0;
}

static int init_staged_kernels();

int init_kernels(Ctx *c) {
    int bad = 0;
    switch (c->logN) {
        case 10: bad = set_smem_attrs<10>(); break;
        case 11: bad = set_smem_attrs<11>(); break;
        case 12: bad = set_smem_attrs<12>(); break;
        case 13: bad = set_smem_attrs<13>(); break;
        case 14: bad = set_smem_attrs<14>(); break;
        default: return set_err(c, HEGMM_EINVAL, "unsupported ring degree");
    }
    if (bad) return cuda_check(c, "ntt shared-memory attribute");
    if (init_staged_kernels()) return cuda_check(c, "staged kernel shared-memory attribute");
    return HEGMM_OK;
}

#define HG_DISPATCH_LOGN(logN, KERNEL_CALL) \
    switch (logN) {                         \
        case 10: { constexpr int LG = 10; KERNEL_CALL; } break; \
        case 11: { constexpr int LG = 11; KERNEL_CALL; } break; \
        case 12: { constexpr int LG = 12; KERNEL_CALL; } break; \
        case 13: { constexpr int LG = 13; KERNEL_CALL; } break; \
        case 14: { constexpr int LG = 14; KERNEL_CALL; } break; \
        default: break;                     \
    }

// Thread count of a launch of `ctas` limb CTAs: the tuned one when set,
// else NttCfg's rule (the wide form when every CTA has an SM of its own).
// True: NT_B, false: NT_A.
template <int LG>
static bool ntt_wide(const Ctx *c, long long ctas) {
    if (c->ntt_threads && NttCfg<LG>::NT_B > NttCfg<LG>::NT_A) return c->ntt_threads >= NttCfg<LG>::NT_B;
    if (NttCfg<LG>::NT == NttCfg<LG>::NT_B) return true;
    return NttCfg<LG>::NT_WIDE > NttCfg<LG>::NT && ctas <= c->nsm;
}

template <int LG, bool INV>
static void launch_ntt(Ctx *c, const LimbPat &p, const TwPair *tw, const TwPair *scale) {
    constexpr int NA = NttCfg<LG>::NT_A, NB = NttCfg<LG>::NT_B;
    constexpr size_t SM = NttCfg<LG>::SMEM;
    if (ntt_wide<LG>(c, p.count))
        k_ntt<LG, INV, NB><<<p.count, NB, SM, c->st>>>(p, c->d_mods, tw, scale);
    else
        k_ntt<LG, INV, NA><<<p.count, NA, SM, c->st>>>(p, c->d_mods, tw, scale);
}

int ntt_fwd(Ctx *c, const LimbPat &p) {
    if (p.count <= 0) return HEGMM_OK;
    Launch t(c, K_NTT_FWD, 2.0 * p.count * c->limb_bytes(), p.count * ntt_bfly(c));
    const TwPair *tw = reinterpret_cast<const TwPair *>(c->d_tw);
    HG_DISPATCH_LOGN(c->logN, (launch_ntt<LG, false>(c, p, tw, nullptr)));
    return cuda_check(c, "ntt_fwd");
}

int ntt_inv(Ctx *c, const LimbPat &p, const u64 *scale) {
    if (p.count <= 0) return HEGMM_OK;
    Launch t(c, K_NTT_INV, 2.0 * p.count * c->limb_bytes(), p.count * ntt_bfly(c));
    const TwPair *tw = reinterpret_cast<const TwPair *>(c->d_tw);
    const TwPair *sc = reinterpret_cast<const TwPair *>(scale);
    HG_DISPATCH_LOGN(c->logN, (launch_ntt<LG, true>(c, p, tw, sc)));
    return cuda_check(c, "ntt_inv");
}

template <int LG, int NT, bool NARROW>
static void launch_divround_t(Ctx *c, int grid, const DivTab &tab, const DivDesc *d_desc, const TwPair *tw) {
    k_divround_ntt<LG, NT, NARROW><<<grid, NT, NttCfg<LG>::SMEM, c->st>>>(tab.nkeep, tab.ndrop, c->d_mods, tab.d,
                                                                       (int)tab.ext, d_desc, tw);
}

template <int LG>
static void launch_divround(Ctx *c, int grid, const DivTab &tab, const DivDesc *d_desc, const TwPair *tw) {
    if constexpr (LG >= 13) {
        // two half-limb CTAs per output limb: always (1), or (2) for launches
        // of fewer than two waves of one-CTA limbs, where twice the CTAs fill
        // the SMs
        if (c->moddown_split == 1 || (c->moddown_split == 2 && grid < 2 * c->nsm)) {
            constexpr size_t SM = DivHalfCfg<LG>::SMEM;
            if (tab.narrow)
                k_divround_half<LG, true><<<2 * grid, 512, SM, c->st>>>(tab.nkeep, tab.ndrop, c->d_mods, tab.d,
                                                                         (int)tab.ext, d_desc, tw);
            else
                k_divround_half<LG, false><<<2 * grid, 512, SM, c->st>>>(tab.nkeep, tab.ndrop, c->d_mods, tab.d,
                                                                          (int)tab.ext, d_desc, tw);
            return;
        }
    }
    constexpr int NT = NttCfg<LG>::NT_A, NW = NttCfg<LG>::NT_B;
    const bool w = ntt_wide<LG>(c, grid);
    if (tab.narrow) {
        if (w) launch_divround_t<LG, NW, true>(c, grid, tab, d_desc, tw);
        else launch_divround_t<LG, NT, true>(c, grid, tab, d_desc, tw);
    } else {
        if (w) launch_divround_t<LG, NW, false>(c, grid, tab, d_desc, tw);
        else launch_divround_t<LG, NT, false>(c, grid, tab, d_desc, tw);
    }
}

int divround_ntt(Ctx *c, const DivTab &tab, const DivDesc *d_desc, int npoly) {
    if (npoly <= 0) return HEGMM_OK;
    // algorithmic bytes: drop limbs + u_i + add_i read, out_i written, per kept limb
    Launch t(c, K_DIV_NTT, (double)npoly * tab.nkeep * (tab.ndrop + 3.0) * c->limb_bytes(),
             (double)npoly * tab.nkeep * ntt_bfly(c));
    const TwPair *tw = reinterpret_cast<const TwPair *>(c->d_tw);
    const int grid = npoly * tab.nkeep;
    HG_DISPATCH_LOGN(c->logN, (launch_divround<LG>(c, grid, tab, d_desc, tw)));
    return cuda_check(c, "divround_ntt");
}

template <int LG, int NT, bool NARROW>
static void launch_modup_t(Ctx *c, const LimbPat &nonown, const ModUpTab &tb, const u64 *xc, long long xc_stride,
                           const TwPair *tw) {
    k_modup_ntt<LG, NT, NARROW><<<nonown.count, NT, NttCfg<LG>::SMEM, c->st>>>(
        nonown, tb.lv, tb.ne, tb.nd, c->alpha, c->L, c->d_mods, tb.d, (int)tb.ext, xc, xc_stride, tw);
}

template <int LG>
static void launch_modup(Ctx *c, const LimbPat &nonown, const ModUpTab &tb, const u64 *xc, long long xc_stride,
                         const TwPair *tw) {
    constexpr int NT = NttCfg<LG>::NT_A, NW = NttCfg<LG>::NT_B;
    const bool w = ntt_wide<LG>(c, nonown.count);
    if (tb.narrow) {
        if (w) launch_modup_t<LG, NW, true>(c, nonown, tb, xc, xc_stride, tw);
        else launch_modup_t<LG, NT, true>(c, nonown, tb, xc, xc_stride, tw);
    } else {
        if (w) launch_modup_t<LG, NW, false>(c, nonown, tb, xc, xc_stride, tw);
        else launch_modup_t<LG, NT, false>(c, nonown, tb, xc, xc_stride, tw);
    }
}

// xc: the coefficient form of the inputs, each limb i already multiplied by
// [(Q_j/q_i)^-1]_{q_i} (modup() scales its inverse NTT by the table's first
// pairs).
int modup_ntt(Ctx *c, const ModUpTab &tb, const LimbPat &nonown, const u64 *xc, long long xc_stride, const u64 *xn,
              long long xn_stride, u64 *D, long long D_stride, int n) {
    Launch t(c, K_MODUP, (double)n * (tb.lv + 2.0 * (tb.nd * tb.ne)) * c->limb_bytes(), nonown.count * ntt_bfly(c));
    const TwPair *tw = reinterpret_cast<const TwPair *>(c->d_tw);
    if (nonown.count > 0)
        HG_DISPATCH_LOGN(c->logN, (launch_modup<LG>(c, nonown, tb, xc, xc_stride, tw)));
    k_modup_own<<<grid_coef(c->N, tb.lv, n), 256, 0, c->st>>>(tb.lv, tb.ne, c->alpha, c->logN, xn, xn_stride, D,
                                                              D_stride);
    return cuda_check(c, "modup_ntt");
}

const ModUpTab *modup_tab(Ctx *c, int lv) {
    auto it = c->modup.find(lv);
    if (it == c->modup.end()) {
        if (build_modup_tab(c, lv)) return nullptr;
        it = c->modup.find(lv);
    }
    return &it->second;
}

// ------------------------------------------------------------------ ModUp
// Table (build_modup_tab): [nd][alpha] x {hinv, hinv_sh}, then
// [nd][alpha][ne] x {hat mod r, shoup, q_i mod r}.

constexpr int MAX_ALPHA = 4;

__global__ void k_modup(int lv, int ne, int nd, int alpha, int L, int logN, const ModDev *__restrict__ mods,
                        const u64 *__restrict__ tab, const u64 *__restrict__ xc, long long xc_stride,
                        const u64 *__restrict__ xn, long long xn_stride, u64 *__restrict__ D, long long D_stride) {
    const int N = 1 << logN;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int j = blockIdx.y, o = blockIdx.z;
    const u64 *x = xc + o * xc_stride;
    const u64 *xv = xn + o * xn_stride;
    u64 *Dj = D + o * D_stride + (size_t)j * ne * N;
    const int lo = j * alpha;
    const int ns = min(alpha, lv - lo);
    const u64 *tinv = tab + (size_t)j * alpha * 2;
    const u64 *thm = tab + (size_t)nd * alpha * 2 + (size_t)j * alpha * ne * 3;
    u64 y[MAX_ALPHA];
#pragma unroll
    for (int ii = 0; ii < MAX_ALPHA; ii++)
        if (ii < ns) y[ii] = mulsh(x[(size_t)(lo + ii) * N + c], tinv[2 * ii], tinv[2 * ii + 1], mods[lo + ii].q);
    for (int e = 0; e < ne; e++) {
        if (e >= lo && e < lo + ns) {
            Dj[(size_t)e * N + c] = xv[(size_t)e * N + c];
            continue;
        }
        const int gm = e < lv ? e : L + (e - lv);
        const u64 r = mods[gm].q, br = mods[gm].barr;
        u64 acc = 0;
#pragma unroll
        for (int ii = 0; ii < MAX_ALPHA; ii++) {
            if (ii >= ns) break;
            const u64 *h = thm + ((size_t)ii * ne + e) * 3;
            const u64 v = centred(y[ii], mods[lo + ii].q, h[2], r, br);
            acc = addm(acc, mulsh(v, h[0], h[1], r), r);
        }
        Dj[(size_t)e * N + c] = acc;
    }
}

int modup_conv(Ctx *c, int lv, int n, const u64 *xc, long long xc_stride, const u64 *xn, long long xn_stride, u64 *D,
               long long D_stride) {
    auto it = c->modup.find(lv);
    if (it == c->modup.end()) {
        int rc = build_modup_tab(c, lv);
        if (rc) return rc;
        it = c->modup.find(lv);
    }
    const ModUpTab &tb = it->second;
    Launch t(c, K_MODUP, (double)n * (lv + (double)tb.nd * tb.ne) * c->limb_bytes());
    k_modup<<<grid_coef(c->N, tb.nd, n), 256, 0, c->st>>>(lv, tb.ne, tb.nd, c->alpha, c->L, c->logN, c->d_mods, tb.d,
                                                            xc, xc_stride, xn, xn_stride, D, D_stride);
    return cuda_check(c, "modup");
}

// Same conversion with a caller-provided table (laid out as build_modup_tab does).
int modup_conv_tab(Ctx *c, const ModUpTab &tb, int n, const u64 *xc, long long xc_stride, const u64 *xn,
                   long long xn_stride, u64 *D, long long D_stride) {
    Launch t(c, K_MODUP, (double)n * (tb.lv + (double)tb.nd * tb.ne) * c->limb_bytes());
    k_modup<<<grid_coef(c->N, tb.nd, n), 256, 0, c->st>>>(tb.lv, tb.ne, tb.nd, c->alpha, c->L, c->logN, c->d_mods,
                                                            tb.d, xc, xc_stride, xn, xn_stride, D, D_stride);
    return cuda_check(c, "modup");
}

// ------------------------------------------------------------------ key-switching inner product
// u[c][e] = sum_j D_j[e][auto_g(.)] * key[j][c][gp(e)], fused with the
// NTT-domain automorphism of the hoisted digits; 128-bit accumulation, one
// Montgomery reduction (keys are stored times 2^64).

// Each thread computes two adjacent coefficients: the key is streamed with
// 16-byte loads, the digits are gathered at the automorphism's indices
// (they are L2-resident: one hoisted ModUp serves every rotation).
__global__ void __launch_bounds__(256, 4) k_ksw_ip(int lv, int ne, int nd, int np, int L, int logN,
                                                const ModDev *__restrict__ mods, const RotDesc *__restrict__ rots) {
    const int N = 1 << logN;
    const int c = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (c >= N) return;
    const int e = blockIdx.y;
    const RotDesc d = rots[blockIdx.z];
    const int gm = e < lv ? e : L + (e - lv);
    const u64 q = mods[gm].q, qinv = mods[gm].qinv;
    const u32 s0 = d.g == 1 ? (u32)c : auto_src((u32)c, d.g, logN);
    const u32 s1 = d.g == 1 ? (u32)c + 1 : auto_src((u32)c + 1, d.g, logN);
    const u64 *Dp = d.D + (size_t)e * N;
    const u64 *Kp = d.key + (size_t)gm * N + c;
    const size_t dstep = (size_t)ne * N, kstep = (size_t)np * N;
    Acc a00{0, 0}, a01{0, 0}, a10{0, 0}, a11{0, 0};
#pragma unroll 4
    for (int j = 0; j < nd; j++) {
        const u64 x0 = __ldg(Dp + (size_t)j * dstep + s0);
        const u64 x1 = __ldg(Dp + (size_t)j * dstep + s1);
        const ulonglong2 k0 = __ldcs(reinterpret_cast<const ulonglong2 *>(Kp + (size_t)(2 * j) * kstep));
        const ulonglong2 k1 = __ldcs(reinterpret_cast<const ulonglong2 *>(Kp + (size_t)(2 * j + 1) * kstep));
        mac(a00, x0, k0.x);
        mac(a01, x1, k0.y);
        mac(a10, x0, k1.x);
        mac(a11, x1, k1.y);
    }
    if (e < lv) {  // P * add on the chain primes (P = 0 mod every special prime)
        const u64 pR = mods[gm].pR;
        if (d.add0) {
            mac(a00, __ldg(d.add0 + (size_t)e * N + s0), pR);
            mac(a01, __ldg(d.add0 + (size_t)e * N + s1), pR);
        }
        if (d.add1) {
            mac(a10, __ldg(d.add1 + (size_t)e * N + s0), pR);
            mac(a11, __ldg(d.add1 + (size_t)e * N + s1), pR);
        }
    }
    ulonglong2 o0, o1;
    o0.x = montred(a00, q, qinv);
    o0.y = montred(a01, q, qinv);
    o1.x = montred(a10, q, qinv);
    o1.y = montred(a11, q, qinv);
    *reinterpret_cast<ulonglong2 *>(d.u + (size_t)e * N + c) = o0;
    *reinterpret_cast<ulonglong2 *>(d.u + ((size_t)ne + e) * N + c) = o1;
}

int ksw_ip(Ctx *c, int lv, const RotDesc *d_rots, int nrot) {
    if (nrot <= 0) return HEGMM_OK;
    const int ne = lv + c->K, nd = c->digits(lv);
    // algorithmic HBM bytes per rotation: its key (2 nd ne limbs) read and u
    // (2 ne limbs) written; the hoisted digits are shared by every rotation
    // of a source and served from L2, so they are not counted.
    Launch t(c, K_KSW_IP, (double)nrot * (2.0 * nd * ne + 2.0 * ne) * c->limb_bytes());
    for (int r0 = 0; r0 < nrot; r0 += kMaxGridZ)
        k_ksw_ip<<<grid_coef(c->N / 2, ne, std::min(kMaxGridZ, nrot - r0)), 256, 0, c->st>>>(
            lv, ne, nd, c->np, c->L, c->logN, c->d_mods, d_rots + r0);
    return cuda_check(c, "ksw_ip");
}

// Double-hoisted linear transformations, one CTA row per (work item, limb),
// one coefficient per thread: each entry's key-switch inner product is
// formed once in registers and multiplied into the lazy 128-bit sums of
// every output of the item that uses it (at most LT_GROUP), so a rotation
// shared by the outputs of an item reads its key once:
//   acc_j += mask_j * u,  u_0 = <tau_g(D), k_0> + P tau_g(c0),
//   u_1 = <tau_g(D), k_1>;  d = 0 entries: u = P ct (0 on special primes).
// grid (N / 256, items, limbs): the CTAs resident together cover many items
// of one limb.
// RED: the output sums are kept reduced (one Montgomery product and a modular
// add per use: half the registers of the lazy 128-bit sums).
template <int G, int MINB, bool RED>
__global__ void __launch_bounds__(256, MINB) k_lt_grp(int lv, int ne, int nd, int np, int L, int logN,
                                                   const ModDev *__restrict__ mods, const LtEntry *__restrict__ ents,
                                                   const LtItem *__restrict__ items) {
    const int N = 1 << logN;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int e = blockIdx.z;
    const LtItem *it = items + blockIdx.y;
    const int gm = e < lv ? e : L + (e - lv);
    const u64 q = mods[gm].q, qinv = mods[gm].qinv, pR = mods[gm].pR;
    const size_t dstep = (size_t)ne * N, kstep = (size_t)np * N, moff = (size_t)gm * N + c;
    Acc s0[RED ? 1 : G], s1[RED ? 1 : G];
    u64 r0[RED ? G : 1], r1[RED ? G : 1];
#pragma unroll
    for (int j = 0; j < (RED ? 1 : G); j++) s0[j] = s1[j] = Acc{0, 0};
#pragma unroll
    for (int j = 0; j < (RED ? G : 1); j++) r0[j] = r1[j] = 0;
    const int t0 = it->first, t1 = t0 + it->count;
    for (int t = t0; t < t1; t++) {
        const LtEntry *E = ents + t;
        const u64 *key = E->key;
        if (!key && e >= lv) continue;  // P ct is 0 on the special primes
        // the masks are loaded with the key and digits, so that one memory
        // latency covers the whole entry
        u64 mv[G];
        const unsigned used = E->used;
#pragma unroll
        for (int j = 0; j < G; j++) mv[j] = (used >> j & 1u) ? __ldg(E->mask[j] + moff) : 0;
        u64 u0, u1;
        if (key) {
            const u32 src = auto_src((u32)c, E->g, logN);
            const u64 *Dp = E->D + (size_t)e * N + src;
            const u64 *Kp = key + moff;
            Acc a0{0, 0}, a1{0, 0};
            if (e < lv) mac(a0, __ldg(E->ct + (size_t)e * N + src), pR);
#pragma unroll 4
            for (int j = 0; j < nd; j++) {
                const u64 x = __ldg(Dp + (size_t)j * dstep);
                mac(a0, x, __ldcs(Kp + (size_t)(2 * j) * kstep));
                mac(a1, x, __ldcs(Kp + (size_t)(2 * j + 1) * kstep));
            }
            u0 = montred(a0, q, qinv);
            u1 = montred(a1, q, qinv);
        } else {
            u0 = montmul(__ldg(E->ct + (size_t)e * N + c), pR, q, qinv);
            u1 = montmul(__ldg(E->ct + ((size_t)lv + e) * N + c), pR, q, qinv);
        }
#pragma unroll
        for (int j = 0; j < G; j++)
            if (used & (1u << j)) {
                if constexpr (RED) {
                    r0[j] = addm(r0[j], montmul(u0, mv[j], q, qinv), q);
                    r1[j] = addm(r1[j], montmul(u1, mv[j], q, qinv), q);
                } else {
                    mac(s0[j], u0, mv[j]);
                    mac(s1[j], u1, mv[j]);
                }
            }
    }
#pragma unroll
    for (int j = 0; j < G; j++) {
        u64 *o = it->out[j];
        if (o) {
            if constexpr (RED) {
                o[(size_t)e * N + c] = r0[j];
                o[((size_t)ne + e) * N + c] = r1[j];
            } else {
                o[(size_t)e * N + c] = montred(s0[j], q, qinv);
                o[((size_t)ne + e) * N + c] = montred(s1[j], q, qinv);
            }
        }
    }
}


// Items of one output with every operand of an entry fetched by per-thread
// asynchronous copies into shared memory (cp.async): the key words, the
// gathered digits, c0 and the mask are all in flight at once without
// holding registers, so the CTA count per SM, not the register budget,
// sets how many loads are outstanding.  Each thread reads back only the
// slots it filled (slot k of thread t at lsm[k 256 + t]), so no barrier is
// needed.  The sums are those of k_lt_grp<1, ., false> (exact 128-bit
// accumulations).  Shared memory: (3 nd + 2) 2 KB.
template <int MINB>
__global__ void __launch_bounds__(256, MINB) k_lt_one_cpa(int lv, int ne, int nd, int np, int L, int logN,
                                                       const ModDev *__restrict__ mods,
                                                       const LtEntry *__restrict__ ents,
                                                       const LtItem *__restrict__ items) {
    extern __shared__ u64 lsm[];
    const int N = 1 << logN;
    const int tid = threadIdx.x;
    const int c = blockIdx.x * 256 + tid;  // N is a multiple of 256
    const int e = blockIdx.z;
    const LtItem *it = items + blockIdx.y;
    const int gm = e < lv ? e : L + (e - lv);
    const u64 q = mods[gm].q, qinv = mods[gm].qinv, pR = mods[gm].pR;
    const size_t dstep = (size_t)ne * N, kstep = (size_t)np * N, moff = (size_t)gm * N + c;
    u64 *my = lsm + tid;
    const int sD = 2 * nd, sC = 3 * nd, sM = 3 * nd + 1;
    Acc s0{0, 0}, s1{0, 0};
    const int t0 = it->first, t1 = t0 + it->count;
    for (int t = t0; t < t1; t++) {
        const LtEntry *E = ents + t;
        const u64 *key = E->key;
        if (!key && e >= lv) continue;  // P ct is 0 on the special primes
        const bool used = E->used & 1u;
        if (key) {
            const u32 src = auto_src((u32)c, E->g, logN);
            const u64 *Dp = E->D + (size_t)e * N + src;
            const u64 *Kp = key + moff;
            for (int j = 0; j < nd; j++) {
                cp_async8(my + (size_t)(2 * j) * 256, Kp + (size_t)(2 * j) * kstep);
                cp_async8(my + (size_t)(2 * j + 1) * 256, Kp + (size_t)(2 * j + 1) * kstep);
                cp_async8(my + (size_t)(sD + j) * 256, Dp + (size_t)j * dstep);
            }
            if (e < lv) cp_async8(my + (size_t)sC * 256, E->ct + (size_t)e * N + src);
        } else {
            cp_async8(my, E->ct + (size_t)e * N + c);
            cp_async8(my + 256, E->ct + ((size_t)lv + e) * N + c);
        }
        if (used) cp_async8(my + (size_t)sM * 256, E->mask[0] + moff);
        cp_async_wait_all();
        u64 u0, u1;
        if (key) {
            Acc a0{0, 0}, a1{0, 0};
            if (e < lv) mac(a0, my[(size_t)sC * 256], pR);
            for (int j = 0; j < nd; j++) {
                const u64 x = my[(size_t)(sD + j) * 256];
                mac(a0, x, my[(size_t)(2 * j) * 256]);
                mac(a1, x, my[(size_t)(2 * j + 1) * 256]);
            }
            u0 = montred(a0, q, qinv);
            u1 = montred(a1, q, qinv);
        } else {
            u0 = montmul(my[0], pR, q, qinv);
            u1 = montmul(my[256], pR, q, qinv);
        }
        if (used) {
            const u64 mv = my[(size_t)sM * 256];
            mac(s0, u0, mv);
            mac(s1, u1, mv);
        }
    }
    u64 *o = it->out[0];
    if (o) {
        o[(size_t)e * N + c] = montred(s0, q, qinv);
        o[((size_t)ne + e) * N + c] = montred(s1, q, qinv);
    }
}

// The 8-output kernel with its streamed operands staged by the TMA engine:
// one CTA per (256 coefficients, item, limb); thread 0 issues, for entry
// t + 1, bulk copies of the key rows (2 nd rows of 2 KB) and of every used
// mask row into the other half of a double buffer in shared memory while
// the CTA works on entry t; the permuted digit gathers stay plain loads,
// issued before the wait.  Every wait is bounded: on a timeout (voted over
// the CTA) the kernel sets *err, waits (bounded) for its copies in flight
// and leaves its outputs unwritten.
constexpr int TMA_MAX_ND = 8;
__device__ __forceinline__ size_t tma_stage_words(int nd, int G) { return (size_t)(2 * nd + G) * 256; }

template <int G, int MINB>
__global__ void __launch_bounds__(256, MINB) k_lt_grp_tma(int lv, int ne, int nd, int np, int L, int logN,
                                                     const ModDev *__restrict__ mods,
                                                     const LtEntry *__restrict__ ents,
                                                     const LtItem *__restrict__ items, int *err, int spin,
                                                     int drop) {
    extern __shared__ __align__(128) u64 tsm[];
    const int N = 1 << logN;
    const int tid = threadIdx.x;
    const int c0 = blockIdx.x * 256, c = c0 + tid;  // N is a multiple of 256
    const int e = blockIdx.z;
    const LtItem *it = items + blockIdx.y;
    const int gm = e < lv ? e : L + (e - lv);
    const u64 q = mods[gm].q, qinv = mods[gm].qinv, pR = mods[gm].pR;
    const size_t dstep = (size_t)ne * N, kstep = (size_t)np * N, moff = (size_t)gm * N + c0;
    const size_t sw = tma_stage_words(nd, G);
    u64 *bar = tsm + 2 * sw;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    const int t0 = it->first, n = it->count;
    // producer: the copies of entry t into stage s (thread 0 only); the
    // item's entry number `drop` is left unarmed (a test of the bounded waits)
    auto issue = [&](int t, int s) {
        if (t - it->first == drop) return;
        const LtEntry *E = ents + t;
        u64 *st = tsm + s * sw;
        const bool live = E->key || e < lv;
        u32 bytes = 0;
        if (live) {
            if (E->key) bytes += 2u * nd * 2048u;
#pragma unroll
            for (int j = 0; j < G; j++)
                if (E->mask[j]) bytes += 2048u;
        }
        mbar_arrive_expect_tx(&bar[s], bytes);
        if (!live) return;
        if (E->key)
            for (int r = 0; r < 2 * nd; r++) bulk_g2s(st + (size_t)r * 256, E->key + (size_t)r * kstep + moff, 2048u, &bar[s]);
#pragma unroll
        for (int j = 0; j < G; j++)
            if (E->mask[j]) bulk_g2s(st + (size_t)(2 * nd + j) * 256, E->mask[j] + moff, 2048u, &bar[s]);
    };
    Acc s0[G], s1[G];
#pragma unroll
    for (int j = 0; j < G; j++) s0[j] = s1[j] = Acc{0, 0};
    u32 ph[2] = {0u, 0u};
    if (tid == 0 && n > 0) issue(t0, 0);
    bool bad = false;
    int i = 0;
    for (; i < n; i++) {
        const int s = i & 1;
        if (tid == 0 && i + 1 < n) {
            fence_proxy_async();  // the stage was read through the generic proxy
            issue(t0 + i + 1, s ^ 1);
        }
        const LtEntry *E = ents + t0 + i;
        const u64 *key = E->key;
        const bool live = key || e < lv;
        // the permuted gathers first: they overlap the bulk copies
        u64 xd[TMA_MAX_ND], x0 = 0, x1 = 0;
        if (key) {
            const u32 src = auto_src((u32)c, E->g, logN);
            const u64 *Dp = E->D + (size_t)e * N + src;
#pragma unroll
            for (int j = 0; j < TMA_MAX_ND; j++)
                if (j < nd) xd[j] = __ldg(Dp + (size_t)j * dstep);
            if (e < lv) x0 = __ldg(E->ct + (size_t)e * N + src);
        } else if (e < lv) {
            x0 = __ldg(E->ct + (size_t)e * N + c);
            x1 = __ldg(E->ct + ((size_t)lv + e) * N + c);
        }
        const bool ok = mbar_wait_bounded(&bar[s], ph[s], spin);
        if (__syncthreads_or(!ok)) {
            bad = true;
            break;
        }
        ph[s] ^= 1u;
        if (live) {
            const u64 *st = tsm + s * sw;
            u64 u0, u1;
            if (key) {
                Acc a0{0, 0}, a1{0, 0};
                if (e < lv) mac(a0, x0, pR);
#pragma unroll
                for (int j = 0; j < TMA_MAX_ND; j++)
                    if (j < nd) {
                        mac(a0, xd[j], st[(size_t)(2 * j) * 256 + tid]);
                        mac(a1, xd[j], st[(size_t)(2 * j + 1) * 256 + tid]);
                    }
                u0 = montred(a0, q, qinv);
                u1 = montred(a1, q, qinv);
            } else {
                u0 = montmul(x0, pR, q, qinv);
                u1 = montmul(x1, pR, q, qinv);
            }
            const u32 used = E->used;
#pragma unroll
            for (int j = 0; j < G; j++)
                if (used >> j & 1u) {
                    const u64 m = st[(size_t)(2 * nd + j) * 256 + tid];
                    mac(s0[j], u0, m);
                    mac(s1[j], u1, m);
                }
        }
        __syncthreads();  // the stage is read before it is filled again
    }
    if (bad) {
        if (tid == 0) atomicExch(err, 1);
        // the copies of entry i + 1 may still be in flight into the other stage
        if (i + 1 < n) {
            const int s = (i + 1) & 1;
            const bool ok = mbar_wait_bounded(&bar[s], ph[s], spin);
            __syncthreads_or(!ok);
        }
        return;
    }
#pragma unroll
    for (int j = 0; j < G; j++) {
        u64 *o = it->out[j];
        if (o) {
            o[(size_t)e * N + c] = montred(s0[j], q, qinv);
            o[((size_t)ne + e) * N + c] = montred(s1[j], q, qinv);
        }
    }
}

// Warp-specialised form of k_lt_grp_tma: warp 8 (lane 0) produces, the 8
// consumer warps compute.  S stages; full[s] completes when the copies of
// the entry in stage s have landed (one arrival with the transaction bytes),
// empty[s] when all 8 consumer warps have read it (one arrival per warp), so
// no block-wide barrier is taken per entry.  Every wait is bounded; a
// timeout anywhere sets *err, the producer then waits (bounded) for the
// copies it issued, and no output is written.
template <int G, int S>
__global__ void __launch_bounds__(288, 2) k_lt_grp_ws(int lv, int ne, int nd, int np, int L, int logN,
                                                    const ModDev *__restrict__ mods, const LtEntry *__restrict__ ents,
                                                    const LtItem *__restrict__ items, int *err, int spin, int drop) {
    extern __shared__ __align__(128) u64 tsm[];
    const int N = 1 << logN;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int c0 = blockIdx.x * 256, c = c0 + tid;  // consumers: tid < 256
    const int e = blockIdx.z;
    const LtItem *it = items + blockIdx.y;
    const int gm = e < lv ? e : L + (e - lv);
    const u64 q = mods[gm].q, qinv = mods[gm].qinv, pR = mods[gm].pR;
    const size_t dstep = (size_t)ne * N, kstep = (size_t)np * N, moff = (size_t)gm * N + c0;
    const size_t sw = tma_stage_words(nd, G);
    u64 *full = tsm + S * sw, *empty = full + S;
    if (tid == 0) {
        for (int s = 0; s < S; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 8);
        }
        fence_mbar_init();
    }
    __syncthreads();
    const int t0 = it->first, n = it->count;
    bool bad = false;
    Acc s0[G], s1[G];
#pragma unroll
    for (int j = 0; j < G; j++) s0[j] = s1[j] = Acc{0, 0};
    if (warp == 8) {
        if (lane == 0) {
            int issued = 0;
            for (int i = 0; i < n; i++) {
                const int s = i % S;
                if (i >= S && !mbar_wait_bounded(&empty[s], (u32)((i / S - 1) & 1), spin)) {
                    bad = true;
                    break;
                }
                if (i == drop) {  // left unarmed (a test of the bounded waits)
                    issued = i + 1;
                    continue;
                }
                const LtEntry *E = ents + t0 + i;
                u64 *st = tsm + s * sw;
                const bool live = E->key || e < lv;
                u32 bytes = 0;
                if (live) {
                    if (E->key) bytes += 2u * nd * 2048u;
#pragma unroll
                    for (int j = 0; j < G; j++)
                        if (E->mask[j]) bytes += 2048u;
                }
                fence_proxy_async();
                mbar_arrive_expect_tx(&full[s], bytes);
                if (live) {
                    if (E->key)
                        for (int r = 0; r < 2 * nd; r++)
                            bulk_g2s(st + (size_t)r * 256, E->key + (size_t)r * kstep + moff, 2048u, &full[s]);
#pragma unroll
                    for (int j = 0; j < G; j++)
                        if (E->mask[j]) bulk_g2s(st + (size_t)(2 * nd + j) * 256, E->mask[j] + moff, 2048u, &full[s]);
                }
                issued = i + 1;
            }
            // every issued copy lands before the CTA can leave
            for (int i = issued - S > 0 ? issued - S : 0; i < issued; i++)
                if (!mbar_wait_bounded(&full[i % S], (u32)((i / S) & 1), spin)) bad = true;
        }
    } else {
        for (int i = 0; i < n; i++) {
            const int s = i % S;
            const LtEntry *E = ents + t0 + i;
            const u64 *key = E->key;
            const bool live = key || e < lv;
            u64 xd[TMA_MAX_ND], x0 = 0, x1 = 0;
            if (key) {
                const u32 src = auto_src((u32)c, E->g, logN);
                const u64 *Dp = E->D + (size_t)e * N + src;
#pragma unroll
                for (int j = 0; j < TMA_MAX_ND; j++)
                    if (j < nd) xd[j] = __ldg(Dp + (size_t)j * dstep);
                if (e < lv) x0 = __ldg(E->ct + (size_t)e * N + src);
            } else if (e < lv) {
                x0 = __ldg(E->ct + (size_t)e * N + c);
                x1 = __ldg(E->ct + ((size_t)lv + e) * N + c);
            }
            if (!mbar_wait_bounded(&full[s], (u32)((i / S) & 1), spin)) {
                bad = true;
                break;
            }
            if (live) {
                const u64 *st = tsm + s * sw;
                u64 u0, u1;
                if (key) {
                    Acc a0{0, 0}, a1{0, 0};
                    if (e < lv) mac(a0, x0, pR);
#pragma unroll
                    for (int j = 0; j < TMA_MAX_ND; j++)
                        if (j < nd) {
                            mac(a0, xd[j], st[(size_t)(2 * j) * 256 + tid]);
                            mac(a1, xd[j], st[(size_t)(2 * j + 1) * 256 + tid]);
                        }
                    u0 = montred(a0, q, qinv);
                    u1 = montred(a1, q, qinv);
                } else {
                    u0 = montmul(x0, pR, q, qinv);
                    u1 = montmul(x1, pR, q, qinv);
                }
                const u32 used = E->used;
#pragma unroll
                for (int j = 0; j < G; j++)
                    if (used >> j & 1u) {
                        const u64 m = st[(size_t)(2 * nd + j) * 256 + tid];
                        mac(s0[j], u0, m);
                        mac(s1[j], u1, m);
                    }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
        }
    }
    if (__syncthreads_or(bad)) {
        if (tid == 0) atomicExch(err, 1);
        return;
    }
    if (warp == 8) return;
#pragma unroll
    for (int j = 0; j < G; j++) {
        u64 *o = it->out[j];
        if (o) {
            o[(size_t)e * N + c] = montred(s0[j], q, qinv);
            o[((size_t)ne + e) * N + c] = montred(s1[j], q, qinv);
        }
    }
}

// Persistent form of k_lt_grp_ws: one launch of gridDim.x CTAs (a few per
// SM) walks the flattened queue of every (item, limb, 256-coefficient slice)
// work unit of the call, CTA b taking units b, b + gridDim.x, ... (limb
// major, then item, then slice, the order of the one-launch-per-kind grid),
// so the items of several outputs and of one output share a single launch
// with no tail between them.  The producer warp keeps filling the S-stage
// ring across units (stage = running entry count mod S), the consumers
// zero their sums at each unit's start and write its outputs at its end.
// Bounded waits as k_lt_grp_ws; `drop` leaves entry number `drop` of every
// unit unarmed (a test of those waits).
template <int G, int S>
__global__ void __launch_bounds__(288, 2) k_lt_grp_pws(int lv, int ne, int nd, int np, int L, int logN,
                                                     const ModDev *__restrict__ mods, const LtEntry *__restrict__ ents,
                                                     const LtItem *__restrict__ items, int nitems, int *err, int spin,
                                                     int drop) {
    extern __shared__ __align__(128) u64 tsm[];
    const int N = 1 << logN, nsl = N >> 8;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long nunits = (long long)nitems * ne * nsl;
    const size_t dstep = (size_t)ne * N, kstep = (size_t)np * N;
    const size_t sw = tma_stage_words(nd, G);
    u64 *full = tsm + S * sw, *empty = full + S;
    if (tid == 0) {
        for (int s = 0; s < S; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 8);
        }
        fence_mbar_init();
    }
    __syncthreads();
    bool bad = false;
    if (warp == 8) {
        if (lane == 0) {
            long long cnt = 0, issued = 0;  // entries through the ring so far
            for (long long w = blockIdx.x; w < nunits && !bad; w += gridDim.x) {
                const int e = (int)(w / ((long long)nitems * nsl));
                const long long rem = w - (long long)e * nitems * nsl;
                const LtItem *it = items + rem / nsl;
                const int c0 = (int)(rem % nsl) * 256;
                const int gm = e < lv ? e : L + (e - lv);
                const size_t moff = (size_t)gm * N + c0;
                for (int i = 0; i < it->count; i++, cnt++) {
                    const int s = (int)(cnt % S);
                    if (cnt >= S && !mbar_wait_bounded(&empty[s], (u32)((cnt / S - 1) & 1), spin)) {
                        bad = true;
                        break;
                    }
                    issued = cnt + 1;
                    if (i == drop) continue;  // left unarmed (a test of the bounded waits)
                    const LtEntry *E = ents + it->first + i;
                    u64 *st = tsm + s * sw;
                    const bool live = E->key || e < lv;
                    u32 bytes = 0;
                    if (live) {
                        if (E->key) bytes += 2u * nd * 2048u;
#pragma unroll
                        for (int j = 0; j < G; j++)
                            if (E->mask[j]) bytes += 2048u;
                    }
                    fence_proxy_async();
                    mbar_arrive_expect_tx(&full[s], bytes);
                    if (live) {
                        if (E->key)
                            for (int r = 0; r < 2 * nd; r++)
                                bulk_g2s(st + (size_t)r * 256, E->key + (size_t)r * kstep + moff, 2048u, &full[s]);
#pragma unroll
                        for (int j = 0; j < G; j++)
                            if (E->mask[j]) bulk_g2s(st + (size_t)(2 * nd + j) * 256, E->mask[j] + moff, 2048u, &full[s]);
                    }
                }
            }
            // every issued copy lands before the CTA can leave
            for (long long i = issued - S > 0 ? issued - S : 0; i < issued; i++)
                if (!mbar_wait_bounded(&full[i % S], (u32)((i / S) & 1), spin)) bad = true;
        }
    } else {
        long long cnt = 0;
        for (long long w = blockIdx.x; w < nunits && !bad; w += gridDim.x) {
            const int e = (int)(w / ((long long)nitems * nsl));
            const long long rem = w - (long long)e * nitems * nsl;
            const LtItem *it = items + rem / nsl;
            const int c = (int)(rem % nsl) * 256 + tid;
            const int gm = e < lv ? e : L + (e - lv);
            const u64 q = mods[gm].q, qinv = mods[gm].qinv, pR = mods[gm].pR;
            Acc s0[G], s1[G];
#pragma unroll
            for (int j = 0; j < G; j++) s0[j] = s1[j] = Acc{0, 0};
            for (int i = 0; i < it->count; i++, cnt++) {
                const int s = (int)(cnt % S);
                const LtEntry *E = ents + it->first + i;
                const u64 *key = E->key;
                const bool live = key || e < lv;
                u64 xd[TMA_MAX_ND], x0 = 0, x1 = 0;
                if (key) {
                    const u32 src = auto_src((u32)c, E->g, logN);
                    const u64 *Dp = E->D + (size_t)e * N + src;
#pragma unroll
                    for (int j = 0; j < TMA_MAX_ND; j++)
                        if (j < nd) xd[j] = __ldg(Dp + (size_t)j * dstep);
                    if (e < lv) x0 = __ldg(E->ct + (size_t)e * N + src);
                } else if (e < lv) {
                    x0 = __ldg(E->ct + (size_t)e * N + c);
                    x1 = __ldg(E->ct + ((size_t)lv + e) * N + c);
                }
                if (!mbar_wait_bounded(&full[s], (u32)((cnt / S) & 1), spin)) {
                    bad = true;
                    break;
                }
                if (live) {
                    const u64 *st = tsm + s * sw;
                    u64 u0, u1;
                    if (key) {
                        Acc a0{0, 0}, a1{0, 0};
                        if (e < lv) mac(a0, x0, pR);
#pragma unroll
                        for (int j = 0; j < TMA_MAX_ND; j++)
                            if (j < nd) {
                                mac(a0, xd[j], st[(size_t)(2 * j) * 256 + tid]);
                                mac(a1, xd[j], st[(size_t)(2 * j + 1) * 256 + tid]);
                            }
                        u0 = montred(a0, q, qinv);
                        u1 = montred(a1, q, qinv);
                    } else {
                        u0 = montmul(x0, pR, q, qinv);
                        u1 = montmul(x1, pR, q, qinv);
                    }
                    const u32 used = E->used;
#pragma unroll
                    for (int j = 0; j < G; j++)
                        if (used >> j & 1u) {
                            const u64 m = st[(size_t)(2 * nd + j) * 256 + tid];
                            mac(s0[j], u0, m);
                            mac(s1[j], u1, m);
                        }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);
            }
            if (bad) break;
#pragma unroll
            for (int j = 0; j < G; j++) {
                u64 *o = it->out[j];
                if (o) {
                    o[(size_t)e * N + c] = montred(s0[j], q, qinv);
                    o[((size_t)ne + e) * N + c] = montred(s1[j], q, qinv);
                }
            }
        }
    }
    if (__syncthreads_or(bad) && tid == 0) atomicExch(err, 1);
}

constexpr int WS_STAGES = 3;
constexpr int LT_CPA_MAX_SMEM = (3 * TMA_MAX_ND + 2) * 256 * 8;  // k_lt_one_cpa's shared memory at nd = 8

static int init_staged_kernels() {
    const int smem8 = (int)((2 * (size_t)(2 * TMA_MAX_ND + LT_GROUP) * 256 + 2) * 8);
    const int smem1 = (int)((2 * (size_t)(2 * TMA_MAX_ND + 1) * 256 + 2) * 8);
    const int smemw = (int)((WS_STAGES * (size_t)(2 * TMA_MAX_ND + LT_GROUP) * 256 + 2 * WS_STAGES) * 8);
    return cudaFuncSetAttribute(k_lt_grp_tma<LT_GROUP, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem8) !=
               cudaSuccess ||
           cudaFuncSetAttribute(k_lt_grp_ws<LT_GROUP, WS_STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smemw) != cudaSuccess ||
           cudaFuncSetAttribute(k_lt_grp_pws<LT_GROUP, WS_STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smemw) != cudaSuccess ||
           cudaFuncSetAttribute(k_lt_grp_tma<1, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem1) != cudaSuccess ||
           cudaFuncSetAttribute(k_lt_one_cpa<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, LT_CPA_MAX_SMEM) !=
               cudaSuccess;
}

// Every item (of one or several outputs) in one launch of the persistent
// kernel: two CTAs per SM walk the units.
int lt_group_persistent(Ctx *c, int lv, const LtEntry *d_ents, const LtItem *d_items, int nitems, double bytes) {
    if (nitems <= 0) return HEGMM_OK;
    const int ne = lv + c->K, nd = c->digits(lv);
    if (nd > TMA_MAX_ND) return set_err(c, HEGMM_EINVAL, "persistent linear-transformation kernel: too many digits");
    Launch t(c, K_LT_KSW, bytes);
    const long long units = (long long)nitems * ne * (c->N >> 8);
    const int grid = (int)std::min<long long>(units, 2LL * c->nsm);
    const size_t smem = (WS_STAGES * (size_t)(2 * nd + LT_GROUP) * 256 + 2 * WS_STAGES) * 8;
    k_lt_grp_pws<LT_GROUP, WS_STAGES><<<grid, 288, smem, c->st>>>(lv, ne, nd, c->np, c->L, c->logN, c->d_mods, d_ents,
                                                                 d_items, nitems, c->d_err, c->wait_limit,
                                                                 c->test_drop_entry);
    return cuda_check(c, "lt_group_persistent");
}

int lt_group(Ctx *c, int lv, int group, const LtEntry *d_ents, const LtItem *d_items, int nitems, double bytes) {
    if (nitems <= 0) return HEGMM_OK;
    const int ne = lv + c->K, nd = c->digits(lv);
    Launch t(c, K_LT_KSW, bytes);
    for (int i0 = 0; i0 < nitems; i0 += kMaxGridZ) {
        const dim3 grid((unsigned)((c->N + 255) / 256), (unsigned)std::min(kMaxGridZ, nitems - i0), (unsigned)ne);
        const LtItem *it = d_items + i0;
#define HG_LTG(G, MB, RED) \
    k_lt_grp<G, MB, RED><<<grid, 256, 0, c->st>>>(lv, ne, nd, c->np, c->L, c->logN, c->d_mods, d_ents, it)
        const bool staged = (c->lt_kernel == 6 || c->lt_kernel == 7) && nd <= TMA_MAX_ND;
        if (group == 1) {  // items of one output
            if (staged && c->lt_one == 1) {
                const size_t smem = (2 * (size_t)(2 * nd + 1) * 256 + 2) * 8;
                k_lt_grp_tma<1, 3><<<grid, 256, smem, c->st>>>(lv, ne, nd, c->np, c->L, c->logN, c->d_mods, d_ents, it,
                                                               c->d_err, c->wait_limit, c->test_drop_entry);
            } else if (c->lt_one == 2) {
                HG_LTG(1, 5, false);
            } else if (c->lt_one == 3) {
                HG_LTG(1, 4, false);
            } else if (c->lt_one == 4 && nd <= TMA_MAX_ND) {
                const size_t smem = (size_t)(3 * nd + 2) * 256 * 8;
                k_lt_one_cpa<6><<<grid, 256, smem, c->st>>>(lv, ne, nd, c->np, c->L, c->logN, c->d_mods, d_ents, it);
            } else {
                HG_LTG(1, 6, false);  // few registers, six CTAs per SM
            }
            continue;
        }
        if (staged && c->lt_kernel == 7) {
            const size_t smem = (WS_STAGES * (size_t)(2 * nd + LT_GROUP) * 256 + 2 * WS_STAGES) * 8;
            k_lt_grp_ws<LT_GROUP, WS_STAGES><<<grid, 288, smem, c->st>>>(lv, ne, nd, c->np, c->L, c->logN, c->d_mods,
                                                                        d_ents, it, c->d_err, c->wait_limit,
                                                                        c->test_drop_entry);
            continue;
        }
        if (staged) {
            const size_t smem = (2 * (size_t)(2 * nd + LT_GROUP) * 256 + 2) * 8;
            k_lt_grp_tma<LT_GROUP, 2><<<grid, 256, smem, c->st>>>(lv, ne, nd, c->np, c->L, c->logN, c->d_mods, d_ents,
                                                                 it, c->d_err, c->wait_limit, c->test_drop_entry);
            continue;
        }
        switch (c->lt_kernel) {
            case 1: HG_LTG(LT_GROUP, 2, false); break;
            case 2: HG_LTG(LT_GROUP, 3, false); break;
            case 3: HG_LTG(LT_GROUP, 4, true); break;
            case 4: HG_LTG(LT_GROUP, 5, true); break;
            case 5: HG_LTG(LT_GROUP, 6, true); break;
            default: HG_LTG(LT_GROUP, 4, false); break;
        }
#undef HG_LTG
    }
    return cuda_check(c, "lt_group");
}

// ------------------------------------------------------------------ exact division by D with t-correction
// Table (build_div_tab): [ndrop] x {coef, coef_sh}; [nkeep][ndrop] x {hat,
// hat_sh, d_k mod q_i}; [nkeep] x {Dinv, Dinv_sh, t mod q_i, shoup};
// then the modulus indices keep[nkeep], drop[ndrop] as u64.

constexpr int MAX_DROP = 4;

__global__ void k_div_conv(int nkeep, int ndrop, int logN, const ModDev *__restrict__ mods, const u64 *__restrict__ tab,
                           const DivDesc *__restrict__ desc) {
    const int N = 1 << logN;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const DivDesc d = desc[blockIdx.y];
    const u64 *tA = tab;
    const u64 *tB = tA + 2 * ndrop;
    const u64 *tC = tB + (size_t)3 * nkeep * ndrop;
    const u64 *tI = tC + (size_t)4 * nkeep;
    u64 z[MAX_DROP], dq[MAX_DROP];
#pragma unroll
    for (int k = 0; k < MAX_DROP; k++) {
        if (k >= ndrop) break;
        dq[k] = mods[tI[nkeep + k]].q;
        z[k] = mulsh(d.u[(size_t)(nkeep + k) * N + c], tA[2 * k], tA[2 * k + 1], dq[k]);
    }
    for (int i = 0; i < nkeep; i++) {
        const ModDev &M = mods[tI[i]];
        u64 acc = 0;
#pragma unroll
        for (int k = 0; k < MAX_DROP; k++) {
            if (k >= ndrop) break;
            const u64 *h = tB + ((size_t)i * ndrop + k) * 3;
            acc = addm(acc, mulsh(centred(z[k], dq[k], h[2], M.q, M.barr), h[0], h[1], M.q), M.q);
        }
        d.tmp[(size_t)i * N + c] = acc;
    }
}

__global__ void k_div_combine(int nkeep, int ndrop, int logN, const ModDev *__restrict__ mods,
                              const u64 *__restrict__ tab, const DivDesc *__restrict__ desc) {
    const int N = 1 << logN;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int i = blockIdx.y;
    const DivDesc d = desc[blockIdx.z];
    const u64 *tC = tab + 2 * ndrop + (size_t)3 * nkeep * ndrop;
    const u64 *tI = tC + (size_t)4 * nkeep;
    const u64 q = mods[tI[i]].q;
    const u64 *k = tC + 4 * i;
    u64 v = subm(d.u[(size_t)i * N + c], mulsh(d.tmp[(size_t)i * N + c], k[2], k[3], q), q);
    v = mulsh(v, k[0], k[1], q);
    if (d.add) {
        const u32 s = d.g == 1 ? (u32)c : auto_src((u32)c, d.g, logN);
        v = addm(v, d.add[(size_t)i * N + s], q);
    }
    d.out[(size_t)i * N + c] = v;
}

int div_conv(Ctx *c, const DivTab &tab, const DivDesc *d_desc, int npoly) {
    if (npoly <= 0) return HEGMM_OK;
    Launch t(c, K_DIV_CONV, (double)npoly * (tab.ndrop + tab.nkeep) * c->limb_bytes());
    k_div_conv<<<grid_coef(c->N, npoly, 1), 256, 0, c->st>>>(tab.nkeep, tab.ndrop, c->logN, c->d_mods, tab.d, d_desc);
    return cuda_check(c, "div_conv");
}

int div_combine(Ctx *c, const DivTab &tab, const DivDesc *d_desc, int npoly) {
    if (npoly <= 0) return HEGMM_OK;
    Launch t(c, K_DIV_COMBINE, (double)npoly * 4.0 * tab.nkeep * c->limb_bytes());
    k_div_combine<<<grid_coef(c->N, tab.nkeep, npoly), 256, 0, c->st>>>(tab.nkeep, tab.ndrop, c->logN, c->d_mods,
                                                                        tab.d, d_desc);
    return cuda_check(c, "div_combine");
}

// ------------------------------------------------------------------ linear-transformation accumulation
// out[o][comp][i] (+)= sum_{terms of o} src[comp][i] * mask[i]  (HE-CMult + HE-Add of Eq. lintrans)

__global__ void k_lt_acc(int lv, int np, int src_np, int lift, int Lc, int logN, const ModDev *__restrict__ mods,
                         const LtTerm *__restrict__ terms, const int *__restrict__ off, u64 *const *__restrict__ outs,
                         int accumulate) {
    const int N = 1 << logN;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int pl = blockIdx.y, o = blockIdx.z;
    const int comp = pl / np, e = pl - comp * np;
    const int gm = e < lv ? e : Lc + (e - lv);
    const u64 q = mods[gm].q, qinv = mods[gm].qinv;
    u64 *out = outs[o] + (size_t)pl * N;
    u64 acc = 0;
    if (e < src_np) {
        const size_t so = ((size_t)comp * src_np + e) * N + c;
        const int t0 = off[o], t1 = off[o + 1];
        for (int t = t0; t < t1; t++) {
            const LtTerm tm = terms[t];
            acc = addm(acc, montmul(__ldg(tm.src + so), __ldg(tm.mask + (size_t)gm * N + c), q, qinv), q);
        }
        if (lift) acc = montmul(acc, mods[gm].pR, q, qinv);  // P acc (pR = P R mod q)
    }
    if (accumulate) acc = addm(acc, out[c], q);
    out[c] = acc;
}

int lt_accumulate(Ctx *c, int lv, int np, int src_np, int lift, const LtTerm *d_terms, const int *d_off,
                  u64 *const *d_outs, int nout, int accumulate) {
    if (nout <= 0) return HEGMM_OK;
    Launch t(c, K_LT_ACC, 0.0);
    for (int o0 = 0; o0 < nout; o0 += kMaxGridZ)
        k_lt_acc<<<grid_coef(c->N, 2 * np, std::min(kMaxGridZ, nout - o0)), 256, 0, c->st>>>(
            lv, np, src_np, lift, c->L, c->logN, c->d_mods, d_terms, d_off + o0, d_outs + o0, accumulate);
    return cuda_check(c, "lt_acc");
}

// ------------------------------------------------------------------ tensor (HE-Mult before relinearisation)

// limb i of the operands is in modulus m0 + i (m0 = 0: the chain primes).
__global__ void k_tensor(int lv, int m0, int logN, const ModDev *__restrict__ mods, const Tensor3 *__restrict__ ts) {
    const int N = 1 << logN;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int i = blockIdx.y;
    const Tensor3 T = ts[blockIdx.z];
    const ModDev M = mods[m0 + i];
    const size_t o0 = (size_t)i * N + c, o1 = ((size_t)lv + i) * N + c;
    const u64 a0 = T.a[o0], a1 = T.a[o1];
    const u64 b0 = montmul(T.b[o0], M.r2, M.q, M.qinv);  // b R
    const u64 b1 = montmul(T.b[o1], M.r2, M.q, M.qinv);
    T.d[o0] = montmul(a0, b0, M.q, M.qinv);
    T.d[o1] = addm(montmul(a0, b1, M.q, M.qinv), montmul(a1, b0, M.q, M.qinv), M.q);
    T.d[((size_t)2 * lv + i) * N + c] = montmul(a1, b1, M.q, M.qinv);
}

// One thread per coefficient of one limb of one sum; the products of all
// iterations are summed lazily (Montgomery, b taken to b R first).
__global__ void k_tensor_sum(int lv, int m0, int logN, const ModDev *__restrict__ mods,
                             const TensorSum *__restrict__ ts) {
    const int N = 1 << logN;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int i = blockIdx.y;
    const TensorSum T = ts[blockIdx.z];
    const ModDev M = mods[m0 + i];
    Acc s0{0, 0}, s1{0, 0}, s2{0, 0};
    const size_t o0 = (size_t)i * N + c, o1 = ((size_t)lv + i) * N + c;
    for (int k = 0; k < T.count; k++) {
        const u64 *a = T.a + (size_t)k * T.stride, *b = T.b + (size_t)k * T.stride;
        const u64 a0 = __ldg(a + o0), a1 = __ldg(a + o1);
        const u64 b0 = montmul(__ldg(b + o0), M.r2, M.q, M.qinv);  // b R
        const u64 b1 = montmul(__ldg(b + o1), M.r2, M.q, M.qinv);
        mac(s0, a0, b0);
        mac(s1, a0, b1);
        mac(s1, a1, b0);
        mac(s2, a1, b1);
    }
    T.d[o0] = montred(s0, M.q, M.qinv);
    T.d[o1] = montred(s1, M.q, M.qinv);
    T.d[((size_t)2 * lv + i) * N + c] = montred(s2, M.q, M.qinv);
}

int tensor_sum(Ctx *c, int lv, const TensorSum *d_t, int n, int m0) {
    if (n <= 0) return HEGMM_OK;
    Launch t(c, K_TENSOR, 0.0);
    for (int i0 = 0; i0 < n; i0 += kMaxGridZ)
        k_tensor_sum<<<grid_coef(c->N, lv, std::min(kMaxGridZ, n - i0)), 256, 0, c->st>>>(lv, m0, c->logN, c->d_mods,
                                                                                            d_t + i0);
    return cuda_check(c, "tensor_sum");
}

int tensor(Ctx *c, int lv, const Tensor3 *d_t, int n, int m0) {
    if (n <= 0) return HEGMM_OK;
    Launch t(c, K_TENSOR, (double)n * 7.0 * lv * c->limb_bytes());
    for (int i0 = 0; i0 < n; i0 += kMaxGridZ)
        k_tensor<<<grid_coef(c->N, lv, std::min(kMaxGridZ, n - i0)), 256, 0, c->st>>>(lv, m0, c->logN, c->d_mods,
                                                                                        d_t + i0);
    return cuda_check(c, "tensor");
}

// ------------------------------------------------------------------ BFV (HEGMM_SCHEME_BFV)

constexpr int BFV_MAXB = 16;  // chain or auxiliary primes a conversion handles in registers

// round(sum_i w_i t / q_i) over the nq chain primes (w_i < q_i): each integer
// part exactly -- a = floor(w_i T_i / 2^64) with T_i = floor(t 2^64 / q_i) is
// the quotient or one less, the remainder w_i t - a q_i (exact mod 2^64,
// below 2 q_i) corrects it -- and the remainders' fractions r_i / q_i summed
// in double precision, so the result is the nearest integer unless that
// sum lies within about nq 2^-52 of a half-integer.
__device__ __forceinline__ u64 bfv_round_sum(const u64 *w, int nq, const u64 *__restrict__ tt,
                                             const u64 *__restrict__ qd, const ModDev *__restrict__ mods, u64 t) {
    u64 whole = 0;
    double frac = 0.0;
    for (int i = 0; i < nq; i++) {
        const u64 q = mods[i].q;
        u64 a = mulhi(w[i], tt[i]);
        u64 r = w[i] * t - a * q;
        if (r >= q) {
            r -= q;
            a++;
        }
        whole += a;
        frac += (double)r * __longlong_as_double((long long)qd[i]);
    }
    return whole + (u64)floor(frac + 0.5);
}

// Decryption: v (coefficient form over the nq chain primes) -> round(t v / Q)
// mod t: with w_i = [v_i (Q/q_i)^-1]_{q_i}, t v / Q = sum_i w_i t / q_i - t u
// for an integer u, so round(t v / Q) = round(sum_i w_i t / q_i) mod t.
__global__ void k_bfv_decode(int nq, int logN, const ModDev *__restrict__ mods, const u64 *__restrict__ tab,
                             BfvTab bt, u64 t, const u64 *__restrict__ v, u64 *__restrict__ out) {
    const int N = 1 << logN;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    u64 w[BFV_MAXB];
    for (int i = 0; i < nq; i++)
        w[i] = mulsh(v[(size_t)i * N + c], tab[bt.qt + 2 * i], tab[bt.qt + 2 * i + 1], mods[i].q);
    out[c] = bfv_round_sum(w, nq, tab + bt.tt, tab + bt.qd, mods, t) % t;
}

int bfv_decode(Ctx *c, const u64 *v, u64 *out) {
    Launch t(c, K_CODEC, (double)(c->L + 1) * c->limb_bytes());
    k_bfv_decode<<<grid_coef(c->N, 1, 1), 256, 0, c->st>>>(c->L, c->logN, c->d_mods, c->d_bfv, c->bt, c->t, v, out);
    return cuda_check(c, "bfv_decode");
}

// Exact base conversion of each coefficient's centred value from basis X
// (moduli x0 .. x0+nx-1) to basis Y (y0 .. y0+ny-1): w_i = [x_i (X/x_i)^-1]_{x_i},
// v = round(sum_i w_i / x_i) (double precision), out_j = sum_i w_i [X/x_i]_{y_j}
// - v [X]_{y_j} mod y_j -- the representative in (-X/2, X/2] unless the
// value lies within about nx 2^-52 X of +-X/2.  xt: [nx] pairs, xd: [nx]
// doubles, cross: [nx][ny] Montgomery, Xy: [ny].  One thread per
// coefficient of one polynomial (grid.y).
__global__ void k_bconv(int nx, int ny, int x0, int y0, int logN, const ModDev *__restrict__ mods,
                        const u64 *__restrict__ xt, const u64 *__restrict__ xd, const u64 *__restrict__ cross,
                        const u64 *__restrict__ Xy, const u64 *__restrict__ in, long long in_pstride,
                        u64 *__restrict__ out, long long out_pstride) {
    const int N = 1 << logN;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const u64 *ip = in + blockIdx.y * in_pstride;
    u64 *op = out + blockIdx.y * out_pstride;
    u64 w[BFV_MAXB];
    double f = 0.0;
    for (int i = 0; i < nx; i++) {
        w[i] = mulsh(ip[(size_t)i * N + c], xt[2 * i], xt[2 * i + 1], mods[x0 + i].q);
        f += (double)w[i] * __longlong_as_double((long long)xd[i]);
    }
    const u64 v = (u64)floor(f + 0.5);
    for (int j = 0; j < ny; j++) {
        const ModDev M = mods[y0 + j];
        Acc a{0, 0};
        for (int i = 0; i < nx; i++) mac(a, w[i], cross[(size_t)i * ny + j]);
        const u64 r = montred(a, M.q, M.qinv);
        op[(size_t)j * N + c] = subm(r, redc64(v * Xy[j], M.q, M.barr), M.q);
    }
}

// HE-Mult's rounding: y given by its residues over the chain (yq, nq limbs)
// and the auxiliary base (yb, nb limbs), coefficient form; zb receives
// round(t y / Q) over the auxiliary base.  With w_i = [y_i (Q/q_i)^-1]_{q_i}
// and Y = sum_i w_i Q/q_i = y + u Q: round(t y / Q) = round(sum_i w_i t / q_i)
// - t u, u = (Y - y) Q^-1 = sum_i w_i q_i^-1 - y Q^-1 mod b_j.
__global__ void k_bfv_scale(int nq, int nb, int b0, int logN, const ModDev *__restrict__ mods,
                            const u64 *__restrict__ tab, BfvTab bt, u64 t, const u64 *__restrict__ yq,
                            long long yq_pstride, const u64 *__restrict__ yb, long long yb_pstride,
                            u64 *__restrict__ zb, long long zb_pstride) {
    const int N = 1 << logN;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const u64 *q_in = yq + blockIdx.y * yq_pstride, *b_in = yb + blockIdx.y * yb_pstride;
    u64 *z = zb + blockIdx.y * zb_pstride;
    u64 w[BFV_MAXB];
    for (int i = 0; i < nq; i++)
        w[i] = mulsh(q_in[(size_t)i * N + c], tab[bt.qt + 2 * i], tab[bt.qt + 2 * i + 1], mods[i].q);
    const u64 r = bfv_round_sum(w, nq, tab + bt.tt, tab + bt.qd, mods, t);
    for (int j = 0; j < nb; j++) {
        const ModDev M = mods[b0 + j];
        Acc a{0, 0};
        for (int i = 0; i < nq; i++) mac(a, w[i], tab[bt.qim + (size_t)i * nb + j]);
        const u64 y = b_in[(size_t)j * N + c];
        const u64 u = subm(montred(a, M.q, M.qinv), mulsh(y, tab[bt.qib + 2 * j], tab[bt.qib + 2 * j + 1], M.q), M.q);
        z[(size_t)j * N + c] = subm(redc64(r, M.q, M.barr), mulsh(u, tab[bt.tb + 2 * j], tab[bt.tb + 2 * j + 1], M.q), M.q);
    }
}

int bfv_conv_q_to_b(Ctx *c, const u64 *in, long long in_pstride, u64 *out, long long out_pstride, int npoly) {
    if (npoly <= 0) return HEGMM_OK;
    const BfvTab &T = c->bt;
    Launch t(c, K_CODEC, (double)npoly * (c->L + c->nb) * c->limb_bytes());
    k_bconv<<<grid_coef(c->N, npoly, 1), 256, 0, c->st>>>(c->L, c->nb, 0, c->b0, c->logN, c->d_mods, c->d_bfv + T.qt,
                                                           c->d_bfv + T.qd, c->d_bfv + T.qbm, c->d_bfv + T.qb, in,
                                                           in_pstride, out, out_pstride);
    return cuda_check(c, "bfv_conv_q_to_b");
}

int bfv_conv_b_to_q(Ctx *c, const u64 *in, long long in_pstride, u64 *out, long long out_pstride, int npoly) {
    if (npoly <= 0) return HEGMM_OK;
    const BfvTab &T = c->bt;
    Launch t(c, K_CODEC, (double)npoly * (c->L + c->nb) * c->limb_bytes());
    k_bconv<<<grid_coef(c->N, npoly, 1), 256, 0, c->st>>>(c->nb, c->L, c->b0, 0, c->logN, c->d_mods, c->d_bfv + T.bt,
                                                           c->d_bfv + T.bd, c->d_bfv + T.bqm, c->d_bfv + T.bq, in,
                                                           in_pstride, out, out_pstride);
    return cuda_check(c, "bfv_conv_b_to_q");
}

int bfv_scale(Ctx *c, const u64 *yq, long long yq_pstride, const u64 *yb, long long yb_pstride, u64 *zb,
              long long zb_pstride, int npoly) {
    if (npoly <= 0) return HEGMM_OK;
    Launch t(c, K_CODEC, (double)npoly * (c->L + 2.0 * c->nb) * c->limb_bytes());
    k_bfv_scale<<<grid_coef(c->N, npoly, 1), 256, 0, c->st>>>(c->L, c->nb, c->b0, c->logN, c->d_mods, c->d_bfv, c->bt,
                                                               c->t, yq, yq_pstride, yb, yb_pstride, zb, zb_pstride);
    return cuda_check(c, "bfv_scale");
}

// ------------------------------------------------------------------ sums and pointwise ops

__global__ void k_sum(int lv, int logN, const ModDev *__restrict__ mods, const u64 *__restrict__ in, long long stride,
                      int nk, u64 *__restrict__ out, int accumulate) {
    const int N = 1 << logN;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int pl = blockIdx.y;
    const u64 q = mods[pl % lv].q;
    u64 acc = accumulate ? out[(size_t)pl * N + c] : 0;
    for (int k = 0; k < nk; k++) acc = addm(acc, in[k * stride + (size_t)pl * N + c], q);
    out[(size_t)pl * N + c] = acc;
}

int sum_cts(Ctx *c, int lv, const u64 *in, long long in_stride, int nk, u64 *out, int accumulate) {
    Launch t(c, K_SUM, (double)(nk + 1) * 2 * lv * c->limb_bytes());
    k_sum<<<grid_coef(c->N, 2 * lv, 1), 256, 0, c->st>>>(lv, c->logN, c->d_mods, in, in_stride, nk, out, accumulate);
    return cuda_check(c, "sum");
}

// Batched sums: out = (init ? init : out) + sum_j items[j * stride], one
// descriptor per grid.z, over the 2 lv limbs of a ciphertext.
__global__ void k_sum_desc(int lv, int np, int Lc, int logN, const ModDev *__restrict__ mods,
                           const SumDesc *__restrict__ ds) {
    const int N = 1 << logN;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int pl = blockIdx.y;
    const SumDesc d = ds[blockIdx.z];
    const int e = pl % np;
    const u64 q = mods[e < lv ? e : Lc + (e - lv)].q;
    const size_t o = (size_t)pl * N + c;
    u64 acc = d.init ? d.init[o] : d.out[o];
    for (int j = 0; j < d.count; j++) acc = addm(acc, d.items[j * d.stride + o], q);
    d.out[o] = acc;
}

int sum_desc(Ctx *c, int lv, const SumDesc *d_sums, int n, int np) {
    if (n <= 0) return HEGMM_OK;
    if (np <= 0) np = lv;
    Launch t(c, K_SUM, 0.0);
    for (int i0 = 0; i0 < n; i0 += kMaxGridZ)
        k_sum_desc<<<grid_coef(c->N, 2 * np, std::min(kMaxGridZ, n - i0)), 256, 0, c->st>>>(lv, np, c->L, c->logN,
                                                                                          c->d_mods, d_sums + i0);
    return cuda_check(c, "sum_desc");
}

// Group sums of whole ciphertexts: one thread per coefficient of one limb of
// one group's output (grid: coefficients x 2 lv limbs x groups).
__global__ void k_sum_groups(int lv, int logN, const ModDev *__restrict__ mods, const u64 *const *__restrict__ src,
                             const int *__restrict__ first, u64 *const *__restrict__ out) {
    const int N = 1 << logN;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int pl = blockIdx.y, g = blockIdx.z;
    const u64 q = mods[pl % lv].q;
    const size_t o = (size_t)pl * N + c;
    u64 acc = 0;
    for (int j = first[g]; j < first[g + 1]; j++) acc = addm(acc, src[j][o], q);
    out[g][o] = acc;
}

int sum_groups(Ctx *c, int lv, const u64 *const *d_src, const int *d_first, u64 *const *d_out, int ngroups) {
    if (ngroups <= 0) return HEGMM_OK;
    Launch t(c, K_SUM, 0.0);
    for (int g0 = 0; g0 < ngroups; g0 += kMaxGridZ)
        k_sum_groups<<<grid_coef(c->N, 2 * lv, std::min(kMaxGridZ, ngroups - g0)), 256, 0, c->st>>>(
            lv, c->logN, c->d_mods, d_src, d_first + g0, d_out + g0);
    return cuda_check(c, "sum_groups");
}

__global__ void k_scatter_slots(const int *__restrict__ off, const int *__restrict__ slots,
                                const int *__restrict__ pos, u64 value, int N, u64 *__restrict__ ev) {
    const int b = blockIdx.x, S = N / 2;
    for (int j = off[b] + threadIdx.x; j < off[b + 1]; j += blockDim.x) {
        const int s = slots[j];
        ev[(size_t)b * N + pos[s]] = value;      // row 0
        ev[(size_t)b * N + pos[S + s]] = value;  // row 1
    }
}

// Butterfly throughput probe: the lazy butterfly of the NTT kernels
// (bfly_ct), repeated on registers (12 per round, the stages of one radix-8
// group); the values are reduced every round so that they stay in range.
__global__ void __launch_bounds__(256) k_bfly_peak(u64 q, const TwPair *__restrict__ tw, int iters, u64 *out) {
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    u64 x[8];
#pragma unroll
    for (int k = 0; k < 8; k++) x[k] = ((u64)gid * 8 + k) % q;
    const TwPair t0 = tw[1], t1 = tw[2], t2 = tw[3], t3 = tw[4], t4 = tw[5], t5 = tw[6], t6 = tw[7];
    const u64 q4 = 4 * q, q16 = 16 * q;
    for (int it = 0; it < iters; it++) {
        bfly_ct(x[0], x[4], t0, q4, q);
        bfly_ct(x[1], x[5], t0, q4, q);
        bfly_ct(x[2], x[6], t0, q4, q);
        bfly_ct(x[3], x[7], t0, q4, q);
        bfly_ct(x[0], x[2], t1, q4, q);
        bfly_ct(x[1], x[3], t1, q4, q);
        bfly_ct(x[4], x[6], t2, q4, q);
        bfly_ct(x[5], x[7], t2, q4, q);
        bfly_ct(x[0], x[1], t3, q4, q);
        bfly_ct(x[2], x[3], t4, q4, q);
        bfly_ct(x[4], x[5], t5, q4, q);
        bfly_ct(x[6], x[7], t6, q4, q);
#pragma unroll
        for (int k = 0; k < 8; k++) x[k] = x[k] >= q16 ? x[k] - q16 : x[k];  // bounded below 40 q
    }
    out[gid] = x[0] ^ x[1] ^ x[2] ^ x[3] ^ x[4] ^ x[5] ^ x[6] ^ x[7];
}

int peak_butterflies(Ctx *c, double *per_s) {
    const int blocks = c->nsm * 8, threads = 256, iters = 4096;
    u64 *out = dalloc(c, (size_t)blocks * threads);
    if (!out) return set_err(c, HEGMM_ENOMEM, "butterfly probe");
    const TwPair *tw = reinterpret_cast<const TwPair *>(c->d_tw);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    k_bfly_peak<<<blocks, threads, 0, c->st>>>(c->q[0], tw, iters / 8, out);
    cudaEventRecord(a, c->st);
    k_bfly_peak<<<blocks, threads, 0, c->st>>>(c->q[0], tw, iters, out);
    cudaEventRecord(b, c->st);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    dfree(c, out);
    *per_s = (double)blocks * threads * iters * 12.0 / (ms / 1e3);
    return cuda_check(c, "butterfly probe");
}

int scatter_slots(Ctx *c, const int *d_off, const int *d_slots, int nb, u64 value, u64 *ev) {
    if (nb <= 0) return HEGMM_OK;
    Launch t(c, K_CODEC, 0.0);
    k_scatter_slots<<<nb, 256, 0, c->st>>>(d_off, d_slots, c->d_slot_pos, value, c->N, ev);
    return cuda_check(c, "scatter_slots");
}

// dst[i] = *src[i] for n ciphertexts of level lv (dst contiguous).
__global__ void k_gather_cts(int lv, int logN, u64 *const *__restrict__ src, u64 *__restrict__ dst) {
    const int N = 1 << logN;
    const int c = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (c >= N) return;
    const size_t o = (size_t)blockIdx.y * N + c;
    const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(src[blockIdx.z] + o);
    *reinterpret_cast<ulonglong2 *>(dst + (size_t)blockIdx.z * 2 * lv * N + o) = v;
}

int gather_cts(Ctx *c, int lv, u64 *const *d_src, int n, u64 *dst) {
    if (n <= 0) return HEGMM_OK;
    Launch t(c, K_POINTWISE, 2.0 * n * 2 * lv * c->limb_bytes());
    for (int i0 = 0; i0 < n; i0 += kMaxGridZ)
        k_gather_cts<<<grid_coef(c->N / 2, 2 * lv, std::min(kMaxGridZ, n - i0)), 256, 0, c->st>>>(
            lv, c->logN, d_src + i0, dst + (size_t)i0 * 2 * lv * c->N);
    return cuda_check(c, "gather_cts");
}

__global__ void k_add(int lv, int logN, const ModDev *__restrict__ mods, const u64 *a, const u64 *b, u64 *out) {
    const int N = 1 << logN;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const size_t o = (size_t)blockIdx.y * N + c;
    out[o] = addm(a[o], b[o], mods[blockIdx.y % lv].q);
}

int pw_add(Ctx *c, int lv, int npoly, const u64 *a, const u64 *b, u64 *out) {
    Launch t(c, K_POINTWISE, 3.0 * npoly * lv * c->limb_bytes());
    k_add<<<grid_coef(c->N, npoly * lv, 1), 256, 0, c->st>>>(lv, c->logN, c->d_mods, a, b, out);
    return cuda_check(c, "add");
}

// out[p][i] = a[p][i] * bR[i or p*lv+i] (Montgomery)
__global__ void k_mont(int lv, int logN, const ModDev *__restrict__ mods, const u64 *a, const u64 *bR, int b_per_limb,
                       u64 *out) {
    const int N = 1 << logN;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int pl = blockIdx.y, i = pl % lv;
    const size_t o = (size_t)pl * N + c;
    const u64 b = bR[(size_t)(b_per_limb ? i : pl) * N + c];
    out[o] = montmul(a[o], b, mods[i].q, mods[i].qinv);
}

int pw_mont(Ctx *c, int lv, int npoly, const u64 *a, const u64 *bR, int b_per_limb, u64 *out) {
    Launch t(c, K_POINTWISE, 3.0 * npoly * lv * c->limb_bytes());
    k_mont<<<grid_coef(c->N, npoly * lv, 1), 256, 0, c->st>>>(lv, c->logN, c->d_mods, a, bR, b_per_limb, out);
    return cuda_check(c, "mont");
}

template <int MODE>  // 0: x -> x R, 1: x R -> x
__global__ void k_mont_conv(LimbPat p, int logN, const ModDev *__restrict__ mods) {
    const int N = 1 << logN;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    int mi;
    u64 *ptr = pat_ptr(p, blockIdx.y, N, mi);
    const ModDev M = mods[mi];
    ptr[c] = montmul(ptr[c], MODE == 0 ? M.r2 : 1, M.q, M.qinv);
}

int pw_to_mont(Ctx *c, const LimbPat &p) {
    Launch t(c, K_POINTWISE, 2.0 * p.count * c->limb_bytes());
    k_mont_conv<0><<<grid_coef(c->N, p.count, 1), 256, 0, c->st>>>(p, c->logN, c->d_mods);
    return cuda_check(c, "to_mont");
}

int pw_from_mont(Ctx *c, const LimbPat &p) {
    Launch t(c, K_POINTWISE, 2.0 * p.count * c->limb_bytes());
    k_mont_conv<1><<<grid_coef(c->N, p.count, 1), 256, 0, c->st>>>(p, c->logN, c->d_mods);
    return cuda_check(c, "from_mont");
}

__global__ void k_permute(int logN, const u64 *in, u64 *out, u32 g) {
    const int N = 1 << logN;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const size_t b = (size_t)blockIdx.y * N;
    out[b + c] = in[b + auto_src((u32)c, g, logN)];
}

int permute_limbs(Ctx *c, int nlimb, const u64 *in, u64 *out, u32 g) {
    Launch t(c, K_POINTWISE, 2.0 * nlimb * c->limb_bytes());
    k_permute<<<grid_coef(c->N, nlimb, 1), 256, 0, c->st>>>(c->logN, in, out, g);
    return cuda_check(c, "permute");
}

// ------------------------------------------------------------------ sampling (coefficient domain)

template <int KIND>  // 0 uniform mod q (index gp N + c), 1 t * CBD(eta), 2 ternary, 3 CBD(eta)
__global__ void k_sample(LimbPat p, int logN, const ModDev *__restrict__ mods, u64 stream, int eta) {
    const int N = 1 << logN;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    int mi;
    u64 *ptr = pat_ptr(p, blockIdx.y, N, mi);
    const ModDev M = mods[mi];
    u64 v;
    if (KIND == 0) {
        v = rng_draw(stream, (u64)mi * N + c) % M.q;
    } else if (KIND == 1 || KIND == 3) {
        const long long e = cbd_sample(rng_draw(stream, (u64)c), eta);
        const u64 r = e >= 0 ? (u64)e : M.q - (u64)(-e);
        v = KIND == 1 ? mulsh(r, M.tq, M.tq_sh, M.q) : r;
    } else {
        const u64 r = rng_draw(stream, (u64)c) % 3;
        v = r == 0 ? M.q - 1 : (r == 1 ? 0 : 1);
    }
    ptr[c] = v;
}

int sample_uniform(Ctx *c, const LimbPat &p, u64 stream, const int *) {
    Launch t(c, K_SAMPLE, 1.0 * p.count * c->limb_bytes());
    k_sample<0><<<grid_coef(c->N, p.count, 1), 256, 0, c->st>>>(p, c->logN, c->d_mods, stream, 0);
    return cuda_check(c, "sample_uniform");
}

int sample_cbd_t(Ctx *c, const LimbPat &p, u64 stream, int eta) {
    Launch t(c, K_SAMPLE, 1.0 * p.count * c->limb_bytes());
    k_sample<1><<<grid_coef(c->N, p.count, 1), 256, 0, c->st>>>(p, c->logN, c->d_mods, stream, eta);
    return cuda_check(c, "sample_cbd");
}

int sample_cbd(Ctx *c, const LimbPat &p, u64 stream, int eta) {
    Launch t(c, K_SAMPLE, 1.0 * p.count * c->limb_bytes());
    k_sample<3><<<grid_coef(c->N, p.count, 1), 256, 0, c->st>>>(p, c->logN, c->d_mods, stream, eta);
    return cuda_check(c, "sample_cbd");
}

int sample_ternary(Ctx *c, const LimbPat &p, u64 stream) {
    Launch t(c, K_SAMPLE, 1.0 * p.count * c->limb_bytes());
    k_sample<2><<<grid_coef(c->N, p.count, 1), 256, 0, c->st>>>(p, c->logN, c->d_mods, stream, 0);
    return cuda_check(c, "sample_ternary");
}

// ------------------------------------------------------------------ keys, encryption, decryption

// One digit j of a switching key from s' to s (NTT domain):
//   b = t e - a s + [P]_{q_i} s' on the primes of digit j, t e - a s elsewhere;
// both b and a are then stored times 2^64 (Montgomery form).
__global__ void k_key_combine(int np, int logN, const ModDev *__restrict__ mods, u64 *kb, u64 *ka,
                              const u64 *__restrict__ sR, const u64 *__restrict__ sprime, const u64 *__restrict__ Pmod,
                              int lo, int hi) {
    const int N = 1 << logN;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int i = blockIdx.y;
    const ModDev M = mods[i];
    const size_t o = (size_t)i * N + c;
    const u64 a = ka[o];
    u64 b = subm(kb[o], montmul(a, sR[o], M.q, M.qinv), M.q);
    if (i >= lo && i < hi) b = addm(b, mulsh(sprime[o], Pmod[2 * i], Pmod[2 * i + 1], M.q), M.q);
    kb[o] = montmul(b, M.r2, M.q, M.qinv);
    ka[o] = montmul(a, M.r2, M.q, M.qinv);
}

int key_digit_combine(Ctx *c, u64 *kb, u64 *ka, const u64 *sprime, const u64 *d_Pmod, int lo, int hi) {
    Launch t(c, K_POINTWISE, 6.0 * c->np * c->limb_bytes());
    k_key_combine<<<grid_coef(c->N, c->np, 1), 256, 0, c->st>>>(c->np, c->logN, c->d_mods, kb, ka, c->d_sR, sprime,
                                                               d_Pmod, lo, hi);
    return cuda_check(c, "key_combine");
}

// c0 = e' + m' - a s (NTT domain), c1 = a: e' = t e and m' = m (BGV), or
// e' = e and m' = Delta m with delta[i] = {Delta mod q_i, Shoup} (BFV).
__global__ void k_enc_combine(int lv, int logN, const ModDev *__restrict__ mods, u64 *ct, const u64 *__restrict__ pt,
                              const u64 *__restrict__ sR, const u64 *__restrict__ delta) {
    const int N = 1 << logN;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int i = blockIdx.y;
    const ModDev M = mods[i];
    const size_t o0 = (size_t)i * N + c, o1 = ((size_t)lv + i) * N + c;
    const u64 m = delta ? mulsh(pt[o0], delta[2 * i], delta[2 * i + 1], M.q) : pt[o0];
    const u64 v = addm(ct[o0], m, M.q);
    ct[o0] = subm(v, montmul(ct[o1], sR[o0], M.q, M.qinv), M.q);
}

int encrypt_combine(Ctx *c, int lv, u64 *ct, const u64 *pt) {
    Launch t(c, K_POINTWISE, 4.0 * lv * c->limb_bytes());
    k_enc_combine<<<grid_coef(c->N, lv, 1), 256, 0, c->st>>>(lv, c->logN, c->d_mods, ct, pt, c->d_sR,
                                                            c->bfv ? c->d_bfv + c->bt.dl : nullptr);
    return cuda_check(c, "enc_combine");
}

// v = c0 + c1 s (NTT domain)
__global__ void k_dec_dot(int lv, int logN, const ModDev *__restrict__ mods, const u64 *__restrict__ ct,
                          const u64 *__restrict__ sR, u64 *v) {
    const int N = 1 << logN;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int i = blockIdx.y;
    const ModDev M = mods[i];
    const size_t o0 = (size_t)i * N + c, o1 = ((size_t)lv + i) * N + c;
    v[o0] = addm(ct[o0], montmul(ct[o1], sR[o0], M.q, M.qinv), M.q);
}

int decrypt_dot(Ctx *c, int lv, const u64 *ct, u64 *v) {
    Launch t(c, K_CODEC, 3.0 * lv * c->limb_bytes());
    k_dec_dot<<<grid_coef(c->N, lv, 1), 256, 0, c->st>>>(lv, c->logN, c->d_mods, ct, c->d_sR, v);
    return cuda_check(c, "dec_dot");
}

// Centred v (coefficient residues over q_0..q_{lv-1}) reduced mod t.
// y_i = [v_i (Q/q_i)^-1]_{q_i}; k = round(sum y_i / q_i) (exact while |v| is
// far below Q/2); v = sum y_i (Q/q_i) - k Q.  tab per i: {hinv, hinv_sh,
// (Q/q_i) mod t, q_i as double bits}, then Q mod t.
__global__ void k_crt_t(int lv, int logN, const ModDev *__restrict__ mods, const u64 *__restrict__ v,
                        const u64 *__restrict__ tab, u64 t, u64 *out) {
    const int N = 1 << logN;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    double frac = 0.0;
    u64 acc = 0;
    for (int i = 0; i < lv; i++) {
        const u64 *tb = tab + 4 * i;
        const u64 y = mulsh(v[(size_t)i * N + c], tb[0], tb[1], mods[i].q);
        frac += (double)y / __longlong_as_double((long long)tb[3]);
        acc = (acc + (y % t) * tb[2]) % t;
    }
    const u64 k = (u64)llrint(frac);
    const u64 Qt = tab[4 * lv];
    out[c] = (acc + t - (k % t) * Qt % t) % t;
}

int crt_to_t(Ctx *c, int lv, const u64 *v, const u64 *tab, u64 *out) {
    Launch t(c, K_CODEC, (double)(lv + 1) * c->limb_bytes());
    k_crt_t<<<grid_coef(c->N, 1, 1), 256, 0, c->st>>>(lv, c->logN, c->d_mods, v, tab, c->t, out);
    return cuda_check(c, "crt_t");
}

// m in [0, t) -> centred -> residues over q_0..q_{lv-1}
__global__ void k_lift_t(int lv, int logN, const ModDev *__restrict__ mods, const u64 *__restrict__ m, u64 t,
                         u64 *out) {
    const int N = 1 << logN;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int i = blockIdx.y, b = blockIdx.z;
    const u64 q = mods[i].q;
    const u64 x = m[(size_t)b * N + c];
    out[((size_t)b * lv + i) * N + c] = x <= (t - 1) / 2 ? x % q : q - (t - x) % q;
}

int lift_from_t(Ctx *c, int lv, const u64 *m, u64 *out, int nbatch) {
    Launch t(c, K_CODEC, (double)nbatch * (lv + 1) * c->limb_bytes());
    k_lift_t<<<grid_coef(c->N, lv, nbatch), 256, 0, c->st>>>(lv, c->logN, c->d_mods, m, c->t, out);
    return cuda_check(c, "lift_t");
}

}  // namespace hg

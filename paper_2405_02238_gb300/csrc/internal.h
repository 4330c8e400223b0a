// internal.h -- host-side structures and kernel launchers of the HEGMM library.
// Not part of the ABI (include/hegmm.h is).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/hegmm.h"

typedef uint64_t u64;
typedef uint32_t u32;

namespace hg {

constexpr int MAXM = 25;      // L + K primes, t, and (BFV) the auxiliary base
// inner entries of a limb pattern; the largest pattern is the ModUp's
// limbs outside each digit's own primes, digits(L) (L + K) - L entries, which
// context creation checks against this bound
constexpr int PAT_MAX = 128;

// Per-modulus constants in device memory.
struct ModDev {
    u64 q;
    u64 qinv;   // q^-1 mod 2^64
    u64 r2;     // 2^128 mod q
    u64 barr;   // floor(2^64 / q)
    u64 ninv;   // N^-1 mod q
    u64 ninv_sh;
    u64 tq;     // t mod q
    u64 tq_sh;
    u64 pR;     // (P mod q) 2^64 mod q, P = product of the special primes (0 on them)
    u64 pad;
};

// A batch of limbs: limb b = outer * inner + i lives at
//   (outer_ptrs ? outer_ptrs[outer] : base + outer * outer_stride) + off[i] * N
// in modulus mod[i].
struct LimbPat {
    u64 *base;
    u64 *const *outer_ptrs;
    long long outer_stride;
    int inner;
    int count;
    unsigned short off[PAT_MAX];
    unsigned char mod[PAT_MAX];
};

// One key-switching inner product: u[c][e] = sum_j D[j][e][perm_g] * key[j][c][gp(e)]
// (+ P * add_c[e][perm_g] on the chain primes, so that ModDown(u) already
// contains add_c: ModDown(u + P x) = ModDown(u) + x exactly).
struct RotDesc {
    const u64 *D;    // [nd][ne][N] hoisted ModUp digits (NTT domain)
    const u64 *key;  // [dnum][2][L+K][N] Montgomery NTT
    u64 *u;          // [2][ne][N]
    const u64 *add0; // [lv][N] or null: added to component 0 (e.g. c0 of a rotation)
    const u64 *add1; // [lv][N] or null: added to component 1
    u32 g;           // Galois element (1 = none), also applied to add0 / add1
    u32 pad;
};

// One polynomial of an exact division with t-corrected rounding (ModDown /
// modulus switch): out = (u_keep - t y~) D^-1 (+ add, optionally permuted by g).
struct DivDesc {
    const u64 *u;   // keep limbs [nkeep][N]; drop limbs follow at u + nkeep * N
    u64 *tmp;       // [nkeep][N] scratch
    u64 *out;       // [nkeep][N]
    const u64 *add; // [nkeep][N] or null
    u32 g;          // automorphism applied to add (1 = none)
    u32 pad;
};

// A product output of the linear-transformation accumulation:
// out[c][i] (+)= sum over terms src[c][i] * mask[i].
// Double-hoisted linear transformations (Eq. lintrans) of up to LT_GROUP
// outputs of one operand per work item.  An entry is one source term shared
// by the item's outputs: u = (<tau_g(D), k_0> + P tau_g(c0), <tau_g(D), k_1>)
// for a rotation, u = P ct for the d = 0 term (key null); every output j of
// the item with mask[j] != null adds mask[j] (.) u to its sum over PQ.  The
// caller divides each sum by P once (ModDown).
constexpr int LT_GROUP = 8;
struct LtEntry {
    const u64 *D;                // hoisted digits of the source [nd][ne][N] (NTT)
    const u64 *key;              // Galois key [nd][2][L+K][N], Montgomery NTT; null: the d = 0 term
    const u64 *ct;               // the source ciphertext [2][lv][N] (NTT)
    u32 g;
    u32 used;                    // bit j set: mask[j] != null
    const u64 *mask[LT_GROUP];   // [L + K][N] Montgomery NTT per output of the item, or null
};
struct LtItem {
    int first, count;            // entries [first, first + count)
    u64 *out[LT_GROUP];          // [2][lv+K][N] per output of the item, or null
};

// Sum of the tensors of count iteration products: d = sum_k (a_k0 b_k0,
// a_k0 b_k1 + a_k1 b_k0, a_k1 b_k1), a_k = a + k stride, b_k = b + k stride.
struct TensorSum {
    const u64 *a;
    const u64 *b;
    long long stride;
    u64 *d;  // [3][lv][N]
    int count;
    int pad;
};

struct LtTerm {
    const u64 *src;  // [2][np][N]: a ciphertext (np = lv) or a key-switch output over PQ (np = lv + K)
    const u64 *mask; // [L + K][N] Montgomery NTT, limb = global prime index
};

struct Tensor3 {
    const u64 *a, *b;  // [2][lv][N]
    u64 *d;            // [3][lv][N]
};

enum KernelKind {
    K_NTT_FWD = 0,
    K_NTT_INV,
    K_MODUP,
    K_KSW_IP,
    K_DIV_CONV,
    K_DIV_COMBINE,
    K_DIV_NTT,
    K_LT_ACC,
    K_TENSOR,
    K_SUM,
    K_POINTWISE,
    K_SAMPLE,
    K_CODEC,
    K_LT_KSW,
    K_NUM
};

struct ModUpTab {
    int lv = 0, ne = 0, nd = 0;
    u64 *d = nullptr;  // see modup_table_host
    size_t ext = 0;    // word offset of the narrow-lift constants in d
    int narrow = 0;    // every digit prime < 2 x every prime of the basis
};

struct DivTab {
    int nkeep = 0, ndrop = 0;
    std::vector<int> keep, drop;  // global modulus indices
    u64 *d = nullptr;             // see div_table_host
    size_t ext = 0;               // word offset of the fused kernel's constants in d
    int narrow = 0;               // every dropped prime < 2 x every kept prime
};

struct ShapeData;
struct BatchPlan;

// out = (init ? init : out) + sum_{j < count} items[j * stride]   over [2][lv][N]
struct SumDesc {
    u64 *out;
    const u64 *init;
    const u64 *items;
    long long stride;
    int count;
    int pad;
};

// BFV constants (HEGMM_SCHEME_BFV) on the device, word offsets into Ctx::d_bfv
// (nq = L chain primes q_i, nb auxiliary primes b_j; Montgomery = times
// 2^64 mod the target prime; pairs = {w, Shoup companion}):
//   qt  [nq] pairs (Q/q_i)^-1 mod q_i      tt [nq] floor(t 2^64 / q_i)
//   qd  [nq] 1/q_i as double bits           qbm [nq][nb] Q/q_i mod b_j, Montgomery
//   qb  [nb] Q mod b_j                      qim [nq][nb] q_i^-1 mod b_j, Montgomery
//   qib [nb] pairs Q^-1 mod b_j             tb [nb] pairs t mod b_j
//   bt  [nb] pairs (B/b_j)^-1 mod b_j       bd [nb] 1/b_j as double bits
//   bqm [nb][nq] B/b_j mod q_i, Montgomery  bq [nq] B mod q_i
//   dl  [nq] pairs Delta mod q_i, Delta = floor(Q / t)
struct BfvTab {
    size_t qt, tt, qd, qbm, qb, qim, qib, tb, bt, bd, bqm, bq, dl, words;
};

struct Ctx {
    hegmm_params prm{};
    int bfv = 0;           // HEGMM_SCHEME_BFV
    int nb = 0, b0 = 0;    // BFV: auxiliary primes at q[b0 .. b0 + nb)
    u64 *d_bfv = nullptr;  // BFV constants (BfvTab)
    BfvTab bt{};
    int logN = 0, N = 0, S = 0, L = 0, K = 0, alpha = 0, dnum = 0, np = 0, tmod = 0, nmod = 0;
    u64 t = 0;
    u64 q[MAXM]{};
    u64 psi[MAXM]{};
    ModDev hmod[MAXM]{};
    ModDev *d_mods = nullptr;
    u64 *d_tw = nullptr;  // [nmod][3][N] x {w, Shoup companion}: see build_twiddles_host (device.cuh)
    cudaStream_t st = nullptr;
    std::string err;
    int nsm = 148;

    bool have_sk = false;
    u64 key_seed = 0;
    u64 *d_s = nullptr;   // [np][N] NTT, normal form
    u64 *d_sR = nullptr;  // [np][N] NTT, Montgomery form
    std::map<u64, u64 *> keys;  // Galois element -> key; 0 = relinearisation

    std::map<int, ModUpTab> modup;
    std::map<std::pair<int, int>, DivTab> divs;  // (level, 0 = ModDown / 1 = modswitch)
    std::vector<int> slot_pos0, slot_pos1;       // slot -> NTT position mod t
    int *d_slot_pos = nullptr;                   // device copy of slot_pos0 then slot_pos1 (N entries)
    std::map<std::tuple<int, int, int, int, int, int>, ShapeData *> shapes;  // per (shape, order, key policy): plan + masks
    std::map<std::vector<int>, BatchPlan *> bplans;                // per product list
    std::map<std::tuple<int, int, int, int>, std::pair<size_t, size_t>> shape_counts;  // iterations, extractions
    unsigned long long bplan_clock = 0;
    std::vector<const BatchPlan *> pinned;     // cached plans in flight on a stream (never evicted)
    int par_groups = 1;                        // concurrent sub-batches of a cached batch (1 or 2)
    int moddown_split = 2;                     // fused ModDown as two half-limb CTAs per limb (N >= 2^13): 0 never, 1 always, 2 small launches
    int par_slot = 0;                          // stream of the running sub-batch (0: st), part of plan keys
    bool in_groups = false;
    cudaStream_t par_st[2] = {nullptr, nullptr};
    cudaEvent_t par_ev[3] = {nullptr, nullptr, nullptr};
    size_t bplan_bytes = 0;
    int ks_double = 0;                         // products: sums of key switches kept over PQ, one ModDown each
    int lazy_relin = 0;                        // products: one relinearisation of the summed tensors
    int lt_shared = 0;                         // products: shared baby steps + giant rotations
    int giant_cost = 8;                        // shared baby steps: giant rotation cost in the greedy rule
    int key_pow2 = 0;                          // power-of-two key policy: rotations as chains of +-2^i
    int use_graphs = 1;                        // replay cached plans as CUDA graphs
    int *d_err = nullptr;                      // set by a kernel whose bounded wait ran out
    int wait_limit = 1 << 22;                  // polls of a bounded mbarrier wait
    int test_drop_entry = -1;                  // test hook: a staged entry left unarmed
    int lt_chunk = 32;                         // double mode: entries per k_lt_grp work item
    int lt_fused = 1;                          // double mode: fused kernel (1) or chunked rotations (0)
    int lt_kernel = 6;                         // grouped fused kernel variant (6: operands staged by TMA)
    int lt_one = 4;                            // one-output kernel: 4 asynchronous copies, 0/2/3 plain loads at 6/5/4 CTAs per SM, 1 staged
    int ntt_threads = 0;                       // threads of an NTT-family CTA: 0 = by launch size, 512 or 1024
    size_t ws_budget = (size_t)1 << 30;        // scratch per chunked stage
    size_t mask_bytes = 0;
    size_t mask_budget = (size_t)96 << 30;     // resident plan masks (LRU beyond this)
    char *arena = nullptr;                     // when set, plan memory is carved from here
    size_t arena_cap = 0, arena_used = 0;
    size_t plan_cache_budget = (size_t)48 << 30;  // workspace kept by cached batch plans
    u64 *d_Pmod = nullptr;           // [np] x {P mod q_i, shoup}
    std::map<int, u64 *> crt;        // level -> CRT-to-t table
    // level -> host tables of the scratch-free rotation: the ModUp table, then
    // the ModDown table from word `first`
    std::map<int, std::pair<size_t, std::vector<u64>>> noalloc_tabs;

    bool timing = false;
    struct Pending {
        int kind;
        cudaEvent_t a, b;
        double bytes, work;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> evpool;
    double stat_ms[K_NUM]{};
    long long stat_n[K_NUM]{};
    double stat_bytes[K_NUM]{};
    double stat_work[K_NUM]{};  // NTT butterflies

    // ext index e of the key-switching basis at level lv -> global modulus
    int gidx(int lv, int e) const { return e < lv ? e : L + (e - lv); }
    int digits(int lv) const { return (lv + alpha - 1) / alpha; }
    size_t limb_bytes() const { return (size_t)N * 8; }
    size_t key_words() const { return (size_t)dnum * 2 * np * N; }
};

// Times one launch when timing is enabled.
// bytes: algorithmic HBM bytes of the launch; work: NTT butterflies.
struct Launch {
    Ctx *c;
    int kind;
    double bytes, work;
    cudaEvent_t a = nullptr, b = nullptr;
    Launch(Ctx *c_, int kind_, double bytes_, double work_ = 0.0);
    ~Launch();
};

// Butterflies of one limb NTT: (N/2) log2 N.
inline double ntt_bfly(const Ctx *c) { return (double)(c->N / 2) * c->logN; }

// Measured throughput of the lazy forward butterfly on registers (no memory
// traffic), in butterflies per second, on the context's device.
int peak_butterflies(Ctx *c, double *per_s);

// ---------------------------------------------------------------- kernels.cu
int init_kernels(Ctx *c);
int ntt_fwd(Ctx *c, const LimbPat &p);
// inverse NTT; scale (may be null): a {w, Shoup companion} pair per inner
// entry of the pattern, multiplied into that entry's limbs
int ntt_inv(Ctx *c, const LimbPat &p, const u64 *scale = nullptr);
// ModUp base conversion of n inputs: xc (coeff, lv limbs) and xn (NTT, lv
// limbs) -> D [nd][ne][N] (own limbs copied from xn in NTT form, others in
// coefficient form, to be forward transformed).
int modup_conv(Ctx *c, int lv, int n, const u64 *xc, long long xc_stride, const u64 *xn, long long xn_stride,
               u64 *D, long long D_stride);
int modup_conv_tab(Ctx *c, const ModUpTab &tb, int n, const u64 *xc, long long xc_stride, const u64 *xn,
                   long long xn_stride, u64 *D, long long D_stride);
int ksw_ip(Ctx *c, int lv, const RotDesc *d_rots, int nrot);
// Fused ModDown / modulus switch: conversion, forward NTT and combine in one kernel.
int divround_ntt(Ctx *c, const DivTab &tab, const DivDesc *d_desc, int npoly);
// Fused ModUp: conversion + forward NTT of every limb outside the digits'
// own primes (nonown pattern), plus the own limbs copied in NTT form.
int modup_ntt(Ctx *c, const ModUpTab &tb, const LimbPat &nonown, const u64 *xc, long long xc_stride, const u64 *xn,
              long long xn_stride, u64 *D, long long D_stride, int n);
const ModUpTab *modup_tab(Ctx *c, int lv);
int div_conv(Ctx *c, const DivTab &tab, const DivDesc *d_desc, int npoly);
int div_combine(Ctx *c, const DivTab &tab, const DivDesc *d_desc, int npoly);
// outs[o] (+)= sum over terms of mask (.) src, over 2 np limbs per output
// (np = lv: the chain primes; np = lv + K: the extended basis, limb e >= lv
// on special prime L + e - lv).  src_np: limbs per component of each source
// (lv or np).  lift: the sources are ciphertexts over Q taken as P ct in the
// extended basis (the sum is multiplied by P; special limbs are zero).
int lt_accumulate(Ctx *c, int lv, int np, int src_np, int lift, const LtTerm *d_terms, const int *d_off,
                  u64 *const *d_outs, int nout, int accumulate);
// limb i of the operands in modulus m0 + i (0: the chain primes; BFV's
// auxiliary base: Ctx::b0)
int tensor(Ctx *c, int lv, const Tensor3 *d_t, int n, int m0 = 0);
// n tensor sums (lazy 128-bit: (2 count + 2) q < 2^64)
int tensor_sum(Ctx *c, int lv, const TensorSum *d_t, int n, int m0 = 0);
// BFV (HEGMM_SCHEME_BFV): decryption's rounding to t, the exact base
// conversions Q -> B and B -> Q of centred values, and HE-Mult's
// round(t y / Q) from y over Q u B to B; coefficient form, npoly polynomials
// of nq (resp. nb) limbs at the given polynomial strides (words).
int bfv_decode(Ctx *c, const u64 *v, u64 *out);
int bfv_conv_q_to_b(Ctx *c, const u64 *in, long long in_pstride, u64 *out, long long out_pstride, int npoly);
int bfv_conv_b_to_q(Ctx *c, const u64 *in, long long in_pstride, u64 *out, long long out_pstride, int npoly);
int bfv_scale(Ctx *c, const u64 *yq, long long yq_pstride, const u64 *yb, long long yb_pstride, u64 *zb,
              long long zb_pstride, int npoly);
// The HE-Mult tensors of n products at level L, BFV: ops holds 2 n device
// pointers (a_k, b_k, ciphertexts [2][L][N], NTT domain), d_out n results
// [3][L][N] (NTT) at stride 3 L N words from `out`; scratch: see
// bfv_tensor_words.  sum != 0: the n tensors are summed over Q u B and
// rounded once into `out` (one result).
size_t bfv_tensor_words(const Ctx *c, int n, int nout);
int bfv_tensor(Ctx *c, int n, u64 *const *d_ops, u64 *out, u64 *scratch, const Tensor3 *d_tq, const Tensor3 *d_tb,
               const TensorSum *d_sq, const TensorSum *d_sb, int sum);
// Every item's output sums over the extended basis of level lv.  Needs
// (entries per item + 2) * q < 2^64 for every prime (lazy 128-bit sums).
// bytes: the algorithmic HBM bytes of the launch (keys, masks, outputs).
// group: 1 for items of one output each, LT_GROUP otherwise.
int lt_group(Ctx *c, int lv, int group, const LtEntry *d_ents, const LtItem *d_items, int nitems, double bytes);
// The same for items of any output count in one persistent launch (variant 8).
int lt_group_persistent(Ctx *c, int lv, const LtEntry *d_ents, const LtItem *d_items, int nitems, double bytes);
// out[poly] = sum_k in[k][poly] over nk inputs with stride in_stride words; npolylimbs = 2*lv
int sum_cts(Ctx *c, int lv, const u64 *in, long long in_stride, int nk, u64 *out, int accumulate);
// pointwise helpers over [npoly][lv][N]
int pw_add(Ctx *c, int lv, int npoly, const u64 *a, const u64 *b, u64 *out);
int pw_mont(Ctx *c, int lv, int npoly, const u64 *a, const u64 *bR, int b_per_limb, u64 *out);
int pw_to_mont(Ctx *c, const LimbPat &p);                  // x -> x R
int pw_from_mont(Ctx *c, const LimbPat &p);                // x R -> x
int sample_uniform(Ctx *c, const LimbPat &p, u64 stream, const int *gprime_of_inner);
int sample_cbd_t(Ctx *c, const LimbPat &p, u64 stream, int eta);   // t * e mod q
int sample_ternary(Ctx *c, const LimbPat &p, u64 stream);
int sample_cbd(Ctx *c, const LimbPat &p, u64 stream, int eta);     // e mod q (BFV errors)
int key_digit_combine(Ctx *c, u64 *kb, u64 *ka, const u64 *sprime, const u64 *d_Pmod, int lo, int hi);
int encrypt_combine(Ctx *c, int lv, u64 *ct, const u64 *pt);
int decrypt_dot(Ctx *c, int lv, const u64 *ct, u64 *v);
int crt_to_t(Ctx *c, int lv, const u64 *v, const u64 *tab, u64 *out);
int lift_from_t(Ctx *c, int lv, const u64 *m, u64 *out, int nbatch = 1);
int permute_limbs(Ctx *c, int nlimb, const u64 *in, u64 *out, u32 g);

// ---------------------------------------------------------------- tables / memory
int build_modup_tab(Ctx *c, int lv);
int build_div_tab(Ctx *c, int lv, int kind);
// host copies of the same tables (layouts at their definitions in ctx.cu)
std::vector<u64> modup_table_host(const Ctx *c, int lv);
std::vector<u64> div_table_host(const Ctx *c, int lv, int kind, std::vector<int> &keep, std::vector<int> &drop);
u64 *dalloc(Ctx *c, size_t words);
void dfree(Ctx *c, void *p);
int set_err(Ctx *c, int code, const std::string &msg);
int cuda_check(Ctx *c, const char *where);
LimbPat pat_ct(Ctx *c, u64 *base, int npoly, int lv, long long poly_stride_words = -1);

// batched sums (SumDesc list) and the input gather of a batch
// np = lv (chain primes) or lv + K (extended basis), as for lt_accumulate
int sum_desc(Ctx *c, int lv, const SumDesc *d_sums, int n, int np = 0);
// out[g] = sum of src[first[g] .. first[g + 1]) (ciphertexts [2][lv][N]),
// device arrays of pointers and offsets.
int sum_groups(Ctx *c, int lv, const u64 *const *d_src, const int *d_first, u64 *const *d_out, int ngroups);
// ev[b][slot_pos0[s]] = ev[b][slot_pos1[s]] = value for s = slots[j],
// j in [off[b], off[b+1]) (NTT order mod t): the slot in both slot rows
int scatter_slots(Ctx *c, const int *d_off, const int *d_slots, int nb, u64 value, u64 *ev);
int gather_cts(Ctx *c, int lv, u64 *const *d_src, int n, u64 *dst);

// ---------------------------------------------------------------- exec.cu
// Copies a host vector into a new stream-ordered device allocation.
template <typename T>
T *upload(Ctx *c, const std::vector<T> &v) {
    size_t bytes = (v.size() * sizeof(T)) > 8 ? v.size() * sizeof(T) : 8;
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, c->st) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (!v.empty()) cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, c->st);
    return (T *)p;
}
LimbPat pat_nonown(Ctx *c, int lv, u64 *D, int n, long long stride);
LimbPat pat_drop_special(Ctx *c, int lv, u64 *u, int npoly);
const DivTab *div_tab(Ctx *c, int lv, int kind);
int modup(Ctx *c, int lv, int n, const u64 *xn, long long xn_stride, u64 *xc, u64 *D);
int ksw_moddown(Ctx *c, int lv, const RotDesc *d_rots, const DivDesc *d_div, int nrot, u64 *u, u64 *tmp);
int modswitch_polys(Ctx *c, int lv, u64 *in, int npoly, u64 *tmp, u64 *out, DivDesc *d_desc);
int rotate_hoisted(Ctx *c, const hegmm_ct *in, const int *z, int count, hegmm_ct **outs);
int mult_relin(Ctx *c, const hegmm_ct *a, const hegmm_ct *b, hegmm_ct **out);
int modswitch(Ctx *c, const hegmm_ct *in, hegmm_ct **out);

// ---------------------------------------------------------------- batch.cu
// products i < count: A[i] (m x l) . B[i] (l x n), shapes mln[3i..3i+2],
// algorithm alg resolved per shape; C[i] receive new ciphertexts; cnt (may
// be null) receives the summed operation counts.
// algs (may be null): one algorithm per product, overriding alg
int matmul_many(Ctx *c, int count, const hegmm_ct *const *A, const hegmm_ct *const *B, const int *mln, int alg,
                hegmm_ct **C, hegmm_opcount *cnt, const int *algs = nullptr);
// Same on the context's current stream; cache = false builds a plan only
// for this call and hands it back in *hold, to be released with
// release_plan (stream-ordered on c->st) once the work is done.
int matmul_run(Ctx *c, int count, const hegmm_ct *const *A, const hegmm_ct *const *B, const int *mln, int alg,
               const int *algs, hegmm_ct **C, hegmm_opcount *cnt, bool cache, BatchPlan **hold);
void release_plan(Ctx *c, BatchPlan *P);
// Device workspace one product adds to a batch (admission estimate).
size_t estimate_bytes(Ctx *c, int m, int l, int n, int alg);
void free_plans(Ctx *c);
void *dalloc_evicting(Ctx *c, size_t bytes);
hegmm_ct *new_ct(Ctx *c, int level);
u64 galois_of(Ctx *c, long long z);
int ensure_galois_key(Ctx *c, u64 g);
int device_status(Ctx *c);

}  // namespace hg

struct hegmm_ctx {
    hg::Ctx c;
};

struct hegmm_pt {
    hg::Ctx *ctx;
    u64 *d;       // [L][N] NTT domain, normal form
    u64 *d_mont;  // [L][N] NTT domain, Montgomery form
    int level;
};

struct hegmm_ct {
    hg::Ctx *ctx;
    u64 *d;  // [2][level][N] NTT domain
    int level;
};

// Host check of the NTT building blocks of device.cuh (compiled by g++ from
// tests/test_device_math.py; the same functions run on the device).
//
// For several primes and ring degrees it runs the forward and inverse
// transforms with the pass structure of the library's NTT kernels (first
// radix-8 pass on registers, middle radix-8 passes through a padded buffer,
// a last pass of logN mod 3 stages on registers) and checks:
//  * the forward output at sampled positions c equals the direct evaluation
//    sum_i a_i psi^((2 brev(c) + 1) i) mod q (the NTT-domain convention);
//  * the inverse of the forward output is the input, every coefficient;
//  * the inverse with a limb scale s gives s a;
//  * no intermediate value exceeds (input bound + 4 q per stage) and 128 q;
//  * mulsh_approx(a, w) is in [0, 4q) and equals a w mod q, and
//    centred_narrow lifts as the centred residue, on random and extreme
//    inputs.
// Prints "ok" or the first failure and exits non-zero.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "device.cuh"

using namespace hg;
typedef unsigned __int128 u128;

static u64 mm(u64 a, u64 b, u64 q) { return (u64)((u128)a * b % q); }
static u64 pw(u64 a, u64 e, u64 q) {
    u64 r = 1 % q;
    for (; e; e >>= 1, a = mm(a, a, q))
        if (e & 1) r = mm(r, a, q);
    return r;
}
static bool is_prime(u64 n) {
    if (n < 2) return false;
    for (u64 p : {2ull, 3ull, 5ull, 7ull, 11ull, 13ull, 17ull, 19ull, 23ull, 29ull, 31ull, 37ull}) {
        if (n % p == 0) return n == p;
    }
    u64 d = n - 1;
    int s = 0;
    while (!(d & 1)) d >>= 1, s++;
    for (u64 b : {2ull, 3ull, 5ull, 7ull, 11ull, 13ull, 17ull, 19ull, 23ull, 29ull, 31ull, 37ull}) {
        u64 x = pw(b, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int r = 1; r < s && comp; r++) {
            x = mm(x, x, n);
            if (x == n - 1) comp = false;
        }
        if (comp) return false;
    }
    return true;
}

static int fails = 0;
#define CHECK(cond, ...)                  \
    do {                                  \
        if (!(cond)) {                    \
            printf("FAIL: " __VA_ARGS__); \
            printf("\n");                 \
            if (++fails > 5) exit(1);     \
        }                                 \
    } while (0)

template <int LOGN>
struct Passes {
    static constexpr int RL = (LOGN % 3) ? (LOGN % 3) : 3;
    static constexpr int LAST = LOGN - RL;
};

static void track(u64 v, u64 &mx) { mx = v > mx ? v : mx; }

// forward transform, the kernel's pass structure; returns the largest value seen
template <int LOGN>
static u64 fwd(std::vector<u64> &a, const TwPair *T, u64 q) {
    constexpr int N = 1 << LOGN, RL = Passes<LOGN>::RL, LAST = Passes<LOGN>::LAST;
    std::vector<u64> sm(N + N / 16);
    u64 mx = 0;
    for (int g = 0; g < N / 8; g++) {
        u64 x[8];
        for (int k = 0; k < 8; k++) x[k] = a[g + k * (N / 8)];
        ntt_fwd_regs<3>(x, 0, 0, T, q);
        for (int k = 0; k < 8; k++) sm[pad16(g + k * (N / 8))] = x[k], track(x[k], mx);
    }
    for (int s0 = 3; s0 < LAST; s0 += 3) {
        for (int g = 0; g < N / 8; g++) ntt_fwd_group_lazy<3>(sm.data(), g, s0, LOGN, T, q);
        for (u64 v : sm) track(v, mx);
    }
    const u64 barr = (u64)(((u128)1 << 64) / q);
    for (int g = 0; g < (N >> RL); g++) {
        u64 x[1 << RL];
        for (int k = 0; k < (1 << RL); k++) x[k] = sm[pad16((g << RL) + k)];
        ntt_fwd_regs<RL>(x, g, LAST, T, q);
        for (int k = 0; k < (1 << RL); k++) track(x[k], mx), a[(g << RL) + k] = redc64(x[k], q, barr);
    }
    return mx;
}

template <int LOGN>
static u64 inv(std::vector<u64> &a, const TwPair *T1, const TwPair *F, u64 q, const TwPair *scale) {
    constexpr int N = 1 << LOGN, RL = Passes<LOGN>::RL, LAST = Passes<LOGN>::LAST;
    std::vector<u64> sm(N + N / 16);
    u64 mx = 0;
    for (int g = 0; g < N / 8; g++) {
        u64 x[8];
        for (int k = 0; k < 8; k++) x[k] = a[8 * g + k];
        ntt_inv_ct_regs<3>(x, 0, 0, T1, q);
        for (int k = 0; k < 8; k++) sm[pad16(8 * g + k)] = x[k], track(x[k], mx);
    }
    for (int u0 = 3; u0 < LAST; u0 += 3) {
        for (int g = 0; g < N / 8; g++) ntt_inv_ct_group<3>(sm.data(), g, u0, T1, q);
        for (u64 v : sm) track(v, mx);
    }
    for (int g = 0; g < (N >> RL); g++) {
        u64 x[1 << RL];
        for (int k = 0; k < (1 << RL); k++) x[k] = sm[pad16(g + (k << LAST))];
        ntt_inv_ct_regs<RL>(x, g, LAST, T1, q);
        for (int k = 0; k < (1 << RL); k++) {
            const int e = g + (k << LAST);
            track(x[k], mx);
            a[e] = scale ? mulsh(mulsh_lazy(x[k], F[e].w, F[e].wp, q), scale->w, scale->wp, q)
                         : mulsh(x[k], F[e].w, F[e].wp, q);
        }
    }
    return mx;
}

template <int LOGN>
static void check_ring(int qbits, int count, std::mt19937_64 &rng) {
    constexpr int N = 1 << LOGN;
    const u64 two_n = 2ull * N;
    u64 cand = ((((u64)1 << qbits) - 1) / two_n) * two_n + 1;
    for (int found = 0; found < count; cand -= two_n) {
        if (!is_prime(cand)) continue;
        found++;
        const u64 q = cand;
        u64 psi = 0;
        for (u64 g = 2;; g++) {
            psi = pw(g, (q - 1) / two_n, q);
            if (pw(psi, N, q) == q - 1) break;
        }
        std::vector<u64> tw(6 * (size_t)N);
        build_twiddles_host(q, psi, LOGN, tw.data());
        const TwPair *T0 = reinterpret_cast<const TwPair *>(tw.data());
        const TwPair *T1 = T0 + N, *F = T0 + 2 * N;
        for (int trial = 0; trial < 3; trial++) {
            std::vector<u64> a(N);
            for (auto &v : a) v = trial == 2 ? q - 1 : rng() % q;  // the last trial: every value at q - 1
            std::vector<u64> A = a;
            const u64 mf = fwd<LOGN>(A, T0, q);
            CHECK(mf < (u128)(1 + 4 * LOGN) * q && mf < (u128)128 * q, "forward bound q=%llu max=%llu",
                  (unsigned long long)q, (unsigned long long)mf);
            for (int s = 0; s < 24; s++) {
                const int c = s < 4 ? s : (int)(rng() % N);
                const u64 root = pw(psi, 2ull * brev_bits((u32)c, LOGN) + 1, q);
                u64 acc = 0, rp = 1;
                for (int i = 0; i < N; i++) {
                    acc = (acc + mm(a[i], rp, q)) % q;
                    rp = mm(rp, root, q);
                }
                CHECK(A[c] == acc, "forward value q=%llu N=%d c=%d", (unsigned long long)q, N, c);
            }
            for (u64 v : A) CHECK(v < q, "forward output not reduced");
            std::vector<u64> B = A;
            const u64 mi = inv<LOGN>(B, T1, F, q, nullptr);
            CHECK(mi < (u128)(1 + 4 * LOGN) * q && mi < (u128)128 * q, "inverse bound");
            for (int i = 0; i < N; i++) CHECK(B[i] == a[i], "inverse(forward) != id q=%llu N=%d i=%d",
                                              (unsigned long long)q, N, i);
            const u64 s = rng() % q;
            const TwPair sp{s, (u64)(((u128)s << 64) / q)};
            std::vector<u64> C = A;
            inv<LOGN>(C, T1, F, q, &sp);
            for (int i = 0; i < N; i++) CHECK(C[i] == mm(a[i], s, q), "scaled inverse");
        }
    }
}

int main() {
    std::mt19937_64 rng(12345);
    // mulsh_approx and centred_narrow on random and extreme inputs
    for (int bits : {30, 40, 50, 56}) {
        for (int it = 0; it < 200000; it++) {
            const u64 q = ((rng() >> (64 - bits)) | (1ull << (bits - 1))) | 1;
            const u64 w = rng() % q, wp = (u64)(((u128)w << 64) / q);
            u64 a = rng();
            if (it % 4 == 1) a = ~0ull;
            if (it % 4 == 2) a = rng() % (128 * q);
            const u64 r = mulsh_approx(a, w, wp, q);
            CHECK(r < 4 * q && r % q == (u64)((u128)a * w % q), "mulsh_approx bits=%d", bits);
            const u64 p = ((rng() >> (64 - bits)) | (1ull << (bits - 1))) | 1;  // same bit length: p < 2 q
            const u64 v = rng() % p;
            const u64 got = centred_narrow(v, p >> 1, q - p);
            const u64 want = v <= (p - 1) / 2 ? v % q : (u64)(((__int128)v - (__int128)p) % (__int128)q + q) % q;
            CHECK(got == want && got < q, "centred_narrow bits=%d", bits);
        }
    }
    check_ring<10>(30, 2, rng);
    check_ring<12>(30, 2, rng);
    check_ring<13>(40, 2, rng);
    check_ring<14>(50, 2, rng);
    check_ring<14>(56, 1, rng);
    if (fails) return 1;
    printf("ok\n");
    return 0;
}

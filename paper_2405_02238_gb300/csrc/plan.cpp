// plan.cpp -- host planner for Algorithms 1 and 2 (see plan.h).
#include "plan.h"

#include <algorithm>
#include <set>

#include "../../include/hegmm.h"

namespace hg {

static inline int imod(long long a, int b) {
    long long r = a % b;
    return (int)(r < 0 ? r + b : r);
}

// Non-adjacent form of v: signed digits, least significant first, as the
// signed powers of two themselves.  An odd v takes the digit +1 when
// v = 1 mod 4 and -1 when v = 3 mod 4, so that v - digit is a multiple of 4.
static std::vector<long long> naf_steps(long long v) {
    std::vector<long long> out;
    long long pw = 1;
    while (v != 0) {
        if (v & 1) {
            const long long r = ((v % 4) + 4) % 4;
            const long long d = r == 1 ? 1 : -1;
            out.push_back(d * pw);
            v -= d;
        }
        v /= 2;  // exact: v is even here
        pw *= 2;
    }
    return out;
}

std::vector<int> pow2_steps(long long z, int S) {
    const long long a = ((z % S) + S) % S;
    std::vector<long long> fa = naf_steps(a), fb = naf_steps(a - S);
    const std::vector<long long> &best = fb.size() < fa.size() ? fb : fa;
    return std::vector<int>(best.begin(), best.end());
}

std::vector<int> pow2_offsets(int S) {
    std::set<int> out;
    for (long long p = 1; p < S; p *= 2) {
        out.insert((int)(p % S));
        out.insert((int)(((-p) % S + S) % S));
    }
    return std::vector<int>(out.begin(), out.end());
}

int alg1_length(int m, int l, int n) { return std::max(m * l, std::max(l * n, m * n)); }
int alg1x_length(int m, int l, int n) { return std::max(m * (l + n - 1), l * n); }

static void alg2_shape(int m, int l, int n, char &kase, int &p, int &t, int &M, int &Np, int &WA, int &HB) {
    p = std::min(m, std::min(l, n));
    if (p == m) {
        kase = 'A';
        t = (l + p - 1) / p;
    } else if (p == n) {
        kase = 'B';
        t = (l + p - 1) / p;
    } else {
        kase = 'L';
        t = 1;
    }
    M = kase == 'A' ? t * m : m;
    Np = kase == 'B' ? t * n : n;
    WA = std::max(l, Np);
    HB = std::max(l, M);
}

int alg2_length(int m, int l, int n) {
    char k;
    int p, t, M, Np, WA, HB;
    alg2_shape(m, l, n, k, p, t, M, Np, WA, HB);
    return std::max(M * WA, std::max(HB * Np, M * Np));
}

void result_layout(int m, int l, int n, int alg, int &rows, int &cols, bool &col) {
    if (alg == 1 || alg == 3) {
        rows = m;
        cols = n;
        col = true;
        return;
    }
    char kase;
    int p, t, WA, HB;
    alg2_shape(m, l, n, kase, p, t, rows, cols, WA, HB);
    col = kase != 'B';
}

std::vector<int> operand_source(const HostPlan &P, int role) {
    const int rows = role == 0 ? P.m : P.l, cols = role == 0 ? P.l : P.n;
    std::vector<int64_t> idx((size_t)rows * cols);
    for (int i = 0; i < rows; i++)
        for (int j = 0; j < cols; j++) idx[(size_t)i * cols + j] = 1 + i + (int64_t)j * rows;
    const uint64_t big = (uint64_t)1 << 30;  // above every index (< slots + 1): no reduction
    const std::vector<uint64_t> v = role == 0 ? P.a_slots(idx.data(), big) : P.b_slots(idx.data(), big);
    std::vector<int> src(v.size());
    for (size_t d = 0; d < v.size(); d++) src[d] = (int)v[d] - 1;
    return src;
}

std::vector<int> result_source(const HostPlan &P) {
    std::vector<int> src((size_t)P.m * P.n, -1);
    for (int i = 0; i < P.m; i++)
        for (int j = 0; j < P.n; j++) src[(size_t)i + (size_t)j * P.m] = P.result_slot(i, j);
    return src;
}

int resolve_alg(int m, int l, int n, int alg, int S) {
    if (m <= 0 || l <= 0 || n <= 0) return 0;
    if (alg == 1) return alg1_length(m, l, n) <= S ? 1 : 0;
    if (alg == 2) return alg2_length(m, l, n) <= S ? 2 : 0;
    if (alg == 3) return alg1x_length(m, l, n) <= S ? 3 : 0;
    if (alg != 0) return 0;
    if (alg2_length(m, l, n) <= S) return 2;
    if (alg1_length(m, l, n) <= S) return 1;
    return 0;
}

// Group a destination -> source slot map by offset d = src - dst:
// ascending offsets, ascending destinations within each.  Every
// destination appears once, so two counting passes (by destination, then
// stably by offset) order it without comparisons.
static std::vector<Diag> group(const std::vector<std::pair<int, int>> &dst_src) {
    std::vector<Diag> out;
    if (dst_src.empty()) return out;
    int lo = dst_src[0].second - dst_src[0].first, hi = lo, dmax = 0;
    for (auto &ds : dst_src) {
        const int d = ds.second - ds.first;
        lo = std::min(lo, d);
        hi = std::max(hi, d);
        dmax = std::max(dmax, ds.first);
    }
    std::vector<int> src_of((size_t)dmax + 1, -1);
    for (auto &ds : dst_src) src_of[(size_t)ds.first] = ds.second;
    std::vector<int> cnt((size_t)(hi - lo) + 2, 0);
    for (auto &ds : dst_src) cnt[(size_t)(ds.second - ds.first - lo) + 1]++;
    for (size_t i = 1; i < cnt.size(); i++) cnt[i] += cnt[i - 1];  // cnt[d - lo] = start of offset d
    std::vector<int> slots(dst_src.size());
    std::vector<int> pos(cnt.begin(), cnt.end() - 1);
    for (int x = 0; x <= dmax; x++)
        if (src_of[(size_t)x] >= 0) slots[(size_t)pos[(size_t)(src_of[(size_t)x] - x - lo)]++] = x;
    for (int d = lo; d <= hi; d++) {
        const int b = cnt[(size_t)(d - lo)], e = cnt[(size_t)(d - lo) + 1];
        if (b == e) continue;
        Diag g;
        g.d = d;
        g.dst.assign(slots.begin() + b, slots.begin() + e);
        out.push_back(std::move(g));
    }
    return out;
}

HostPlan make_host_plan(int m, int l, int n, int alg) {
    HostPlan P;
    P.m = m;
    P.l = l;
    P.n = n;
    P.alg = alg;
    if (alg == 1) {
        // Algorithm 1, column-major: A0 = sigma(A) (m x l), B0 = tau(B) (l x n);
        // eps^k_{m x n}: (i, j) <- (i, [j+k]_l); omega^k_{m x n}: (i, j) <- ([i+k]_l, j).
        P.kase = '1';
        P.col = true;
        P.p = l;
        P.t = 1;
        P.M = m;
        P.Np = n;
        P.a_rows = m;
        P.a_cols = l;
        P.b_rows = l;
        P.b_cols = n;
        P.res_rows = m;
        P.res_cols = n;
        P.length = alg1_length(m, l, n);
        for (int k = 0; k < l; k++) {
            std::vector<std::pair<int, int>> e, o;
            e.reserve((size_t)m * n);
            o.reserve((size_t)m * n);
            for (int i = 0; i < m; i++)
                for (int j = 0; j < n; j++) {
                    const int dst = P.flat(i, j, m, n);
                    e.push_back({dst, P.flat(i, (j + k) % l, m, l)});
                    o.push_back({dst, P.flat((i + k) % l, j, l, n)});
                }
            PlanIter it;
            it.eps = group(e);
            it.omg = group(o);
            P.iters.push_back(it);
        }
        return P;
    }
    if (alg == 3) {
        // Algorithm 1 with sigma(A) stored over W = l + n - 1 columns (column
        // c holds sigma(A)'s column c mod l): eps^k_{m x n}: (i, j) <- (i, j + k),
        // one rotation by k m in column-major order; omega^k as Algorithm 1.
        const int W = l + n - 1;
        P.kase = 'X';
        P.col = true;
        P.p = l;
        P.t = 1;
        P.M = m;
        P.Np = n;
        P.a_rows = m;
        P.a_cols = W;
        P.b_rows = l;
        P.b_cols = n;
        P.res_rows = m;
        P.res_cols = n;
        P.length = alg1x_length(m, l, n);
        for (int k = 0; k < l; k++) {
            std::vector<std::pair<int, int>> e, o;
            e.reserve((size_t)m * n);
            o.reserve((size_t)m * n);
            for (int i = 0; i < m; i++)
                for (int j = 0; j < n; j++) {
                    const int dst = P.flat(i, j, m, n);
                    e.push_back({dst, P.flat(i, j + k, m, W)});
                    o.push_back({dst, P.flat((i + k) % l, j, l, n)});
                }
            PlanIter it;
            it.eps = group(e);
            it.omg = group(o);
            P.iters.push_back(it);
        }
        return P;
    }
    alg2_shape(m, l, n, P.kase, P.p, P.t, P.M, P.Np, P.WA, P.HB);
    P.col = P.kase != 'B';
    P.a_rows = P.M;
    P.a_cols = P.WA;
    P.b_rows = P.HB;
    P.b_cols = P.Np;
    P.res_rows = P.M;
    P.res_cols = P.Np;
    P.length = alg2_length(m, l, n);
    std::vector<char> seen(l, 0);
    for (int k = 0; k < P.p; k++) {
        std::vector<char> keep(P.t, 0);
        for (int h = 0; h < P.t; h++) {
            const int ph = (k + h * P.p) % l;
            keep[h] = !seen[ph];
            seen[ph] = 1;
        }
        std::vector<std::pair<int, int>> e, o;
        e.reserve((size_t)P.M * P.Np);
        o.reserve((size_t)P.M * P.Np);
        for (int i = 0; i < P.M; i++)
            for (int j = 0; j < P.Np; j++) {
                const int dst = P.flat(i, j, P.M, P.Np);
                const bool kept = P.kase == 'A' ? keep[i / m] : (P.kase == 'B' ? keep[j / n] : true);
                if (kept) {
                    // stored column of sA holding sigma(Abar) column [j+k]_l
                    int cc = j + k;
                    while (cc >= P.WA) cc -= l;
                    e.push_back({dst, P.flat(i, cc, P.M, P.WA)});
                }
                int rr = i + k;
                while (rr >= P.HB) rr -= l;
                o.push_back({dst, P.flat(rr, j, P.HB, P.Np)});
            }
        PlanIter it;
        it.eps = group(e);
        it.omg = group(o);
        P.iters.push_back(it);
    }
    for (int h = 1; h < P.t; h++) P.extract.push_back(h * P.p);
    return P;
}

std::vector<uint64_t> HostPlan::a_slots(const int64_t *A, uint64_t tm) const {
    std::vector<uint64_t> v((size_t)a_rows * a_cols, 0);
    for (int i = 0; i < a_rows; i++)
        for (int c = 0; c < a_cols; c++) {
            // Algorithm 1: sigma(A)_{i,c} = A_{i,[i+c]_l} (with the extended
            // layout, c < l + n - 1: sigma(A)'s column c mod l, the same entry).
            // Algorithm 2: eps^0(sigma(Abar))_{i,c} = Abar_{i,[i+c]_l}, Abar row i = A row i mod m.
            const int src_row = (alg == 2 && kase == 'A') ? i % m : i;
            const int64_t x = A[(size_t)src_row * l + imod((long long)i + c, l)];
            v[flat(i, c, a_rows, a_cols)] = (uint64_t)imod(x, (int)tm);
        }
    return v;
}

std::vector<uint64_t> HostPlan::b_slots(const int64_t *B, uint64_t tm) const {
    std::vector<uint64_t> v((size_t)b_rows * b_cols, 0);
    for (int r = 0; r < b_rows; r++)
        for (int j = 0; j < b_cols; j++) {
            // tau(Bbar)_{r,j} = Bbar_{[r+j]_l, j}; Bbar column j = B column j mod n.
            const int src_col = (alg == 2 && kase == 'B') ? j % n : j;
            const int64_t x = B[(size_t)imod((long long)r + j, l) * n + src_col];
            v[flat(r, j, b_rows, b_cols)] = (uint64_t)imod(x, (int)tm);
        }
    return v;
}

long long HostPlan::paper_rot() const {
    long long r = 0;
    for (auto &it : iters) {
        for (auto &d : it.eps) r += d.d != 0;
        for (auto &d : it.omg) r += d.d != 0;
    }
    return r + (long long)extract.size();
}

long long HostPlan::paper_cmult() const {
    long long r = 0;
    for (auto &it : iters) r += (long long)it.eps.size() + (long long)it.omg.size();
    return r;
}

std::vector<GiantLT> giant_factor(const std::vector<const std::vector<Diag> *> &outs, int S, int cost) {
    std::vector<char> in_baby((size_t)S, 0), in_z((size_t)S, 0);
    std::vector<int> baby;                // the non-zero offsets used so far
    std::vector<int> hits((size_t)S, 0);  // g -> #{z : (z - g) mod S in B or 0}
    std::vector<int> touched;
    std::vector<GiantLT> res;
    for (const auto *ds : outs) {
        std::vector<int> Z;
        for (const auto &d : *ds) {
            const int z = imod(d.d, S);
            if (!in_z[(size_t)z]) {
                in_z[(size_t)z] = 1;
                Z.push_back(z);
            }
        }
        for (int z : Z) in_z[(size_t)z] = 0;
        touched.clear();
        auto hit = [&](int g) {
            if (hits[(size_t)g]++ == 0) touched.push_back(g);
        };
        for (int z : Z) {
            hit(z);  // b = 0
            for (int b : baby) hit(imod((long long)z - b, S));
        }
        const int nz = (int)Z.size();
        // g = 0 first; among the others the smallest g of the lowest cost
        int best_g = 0, best_c = nz - hits[0];
        for (int g : touched) {
            if (g == 0) continue;
            const int cst = nz - hits[(size_t)g] + cost;
            if (cst < best_c || (cst == best_c && best_g != 0 && g < best_g)) {
                best_g = g;
                best_c = cst;
            }
        }
        for (int g : touched) hits[(size_t)g] = 0;
        GiantLT f;
        f.g = best_g;
        for (const auto &d : *ds) {
            GTerm t;
            t.b = imod((long long)d.d - best_g, S);
            // destinations + g mod S, ascending: d.dst is ascending in
            // [0, S), so the ones that wrap (x + g >= S) come first
            const auto wrap = std::lower_bound(d.dst.begin(), d.dst.end(), S - best_g);
            t.dst.reserve(d.dst.size());
            for (auto it = wrap; it != d.dst.end(); ++it) t.dst.push_back(*it + best_g - S);
            for (auto it = d.dst.begin(); it != wrap; ++it) t.dst.push_back(*it + best_g);
            if (t.b && !in_baby[(size_t)t.b]) {
                in_baby[(size_t)t.b] = 1;
                baby.push_back(t.b);
            }
            f.terms.push_back(std::move(t));
        }
        res.push_back(std::move(f));
    }
    return res;
}

std::vector<GiantLT> giant_factor_of(const HostPlan &P, int s, int S, int cost) {
    std::vector<const std::vector<Diag> *> outs;
    for (const auto &it : P.iters) outs.push_back(s == 0 ? &it.eps : &it.omg);
    return giant_factor(outs, S, cost);
}

}  // namespace hg

using namespace hg;

extern "C" {

int hegmm_plan_giant(int m, int l, int n, int alg, int slots, int role, int cost, int *buf, int cap) {
    if (slots <= 0 || (role != 0 && role != 1) || cost < 0 || cap < 0 || (cap > 0 && !buf)) return HEGMM_EINVAL;
    const int a = resolve_alg(m, l, n, alg, slots);
    if (!a) return HEGMM_ESHAPE;
    HostPlan P = make_host_plan(m, l, n, a);
    std::vector<GiantLT> f = giant_factor_of(P, role, slots, cost ? cost : GIANT_COST);
    std::vector<int> v{(int)f.size()};
    for (const auto &x : f) {
        v.push_back(x.g);
        v.push_back((int)x.terms.size());
        for (const auto &t : x.terms) {
            v.push_back(t.b);
            v.push_back((int)t.dst.size());
            v.insert(v.end(), t.dst.begin(), t.dst.end());
        }
    }
    for (int i = 0; i < cap && i < (int)v.size(); i++) buf[i] = v[i];
    return (int)v.size();
}


int hegmm_plan_counts(int m, int l, int n, int alg, int slots, hegmm_opcount *out) {
    if (!out || slots <= 0) return HEGMM_EINVAL;
    const int a = resolve_alg(m, l, n, alg, slots);
    if (!a) return HEGMM_ESHAPE;
    HostPlan P = make_host_plan(m, l, n, a);
    std::set<long long> zs[2];
    for (auto &it : P.iters)
        for (int s = 0; s < 2; s++)
            for (auto &d : (s == 0 ? it.eps : it.omg)) {
                long long z = ((long long)d.d % slots + slots) % slots;
                if (z) zs[s].insert(z);
            }
    const long long ni = (long long)P.iters.size(), ne = (long long)P.extract.size();
    out->rot = P.paper_rot();
    out->cmult = P.paper_cmult();
    out->mult = ni;
    out->relin = ni;
    out->extract = ne;
    out->add = out->cmult - 2 * ni + (ni - 1) + ne;
    out->ksw = (long long)zs[0].size() + (long long)zs[1].size() + ni + ne;
    out->modup = 2 + ni + (ne > 0 ? 1 : 0);
    out->modswitch = 0;
    return HEGMM_OK;
}

int hegmm_plan_describe(int m, int l, int n, int alg, int slots, int *buf, int cap) {
    if (slots <= 0 || cap < 0 || (cap > 0 && !buf)) return HEGMM_EINVAL;
    const int a = resolve_alg(m, l, n, alg, slots);
    if (!a) return HEGMM_ESHAPE;
    HostPlan P = make_host_plan(m, l, n, a);
    std::vector<int> v{a, (int)P.kase, P.col ? 1 : 0, (int)P.iters.size(), (int)P.extract.size()};
    for (auto &it : P.iters)
        for (int s = 0; s < 2; s++) {
            const auto &ds = s == 0 ? it.eps : it.omg;
            v.push_back((int)ds.size());
            for (auto &d : ds) {
                v.push_back(d.d);
                v.push_back((int)d.dst.size());
                v.insert(v.end(), d.dst.begin(), d.dst.end());
            }
        }
    v.insert(v.end(), P.extract.begin(), P.extract.end());
    for (int i = 0; i < m; i++)
        for (int j = 0; j < n; j++) v.push_back(P.result_slot(i, j));
    for (int i = 0; i < cap && i < (int)v.size(); i++) buf[i] = v[i];
    return (int)v.size();
}

int hegmm_plan_slot_map(int m, int l, int n, int alg, int slots, int role, int *buf, int cap) {
    if (slots <= 0 || m <= 0 || l <= 0 || n <= 0 || role < 0 || role > 2 || cap < 0 || (cap > 0 && !buf))
        return HEGMM_EINVAL;
    const int a = resolve_alg(m, l, n, alg, slots);
    if (!a) return HEGMM_ESHAPE;
    const HostPlan P = make_host_plan(m, l, n, a);
    const std::vector<int> v = role == 2 ? result_source(P) : operand_source(P, role);
    for (int i = 0; i < cap && i < (int)v.size(); i++) buf[i] = v[i];
    return (int)v.size();
}

int hegmm_plan_result_layout(int m, int l, int n, int alg, int slots, int *rows_cols_col) {
    if (slots <= 0 || m <= 0 || l <= 0 || n <= 0 || !rows_cols_col) return HEGMM_EINVAL;
    const int a = resolve_alg(m, l, n, alg, slots);
    if (!a) return HEGMM_ESHAPE;
    bool col;
    result_layout(m, l, n, a, rows_cols_col[0], rows_cols_col[1], col);
    rows_cols_col[2] = col ? 1 : 0;
    return HEGMM_OK;
}

int hegmm_plan_pow2_steps(long long z, int slots, int *buf, int cap) {
    if (slots <= 0 || (cap > 0 && !buf)) return HEGMM_EINVAL;
    const std::vector<int> v = pow2_steps(z, slots);
    for (int i = 0; i < cap && i < (int)v.size(); i++) buf[i] = v[i];
    return (int)v.size();
}

int hegmm_plan_layout(int m, int l, int n, int alg, int slots, int role, const int64_t *mat, uint64_t t, uint64_t *out,
                      int cap) {
    if (!mat || slots <= 0 || (role != 0 && role != 1) || t < 2) return HEGMM_EINVAL;
    const int a = resolve_alg(m, l, n, alg, slots);
    if (!a) return HEGMM_ESHAPE;
    HostPlan P = make_host_plan(m, l, n, a);
    std::vector<uint64_t> v = role == 0 ? P.a_slots(mat, t) : P.b_slots(mat, t);
    if (cap < (int)v.size() || !out) return (int)v.size();
    for (size_t i = 0; i < v.size(); i++) out[i] = v[i];
    return (int)v.size();
}

}  // extern "C"

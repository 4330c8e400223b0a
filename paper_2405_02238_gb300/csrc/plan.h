// plan.h -- host planner: the linear transformations of Algorithms 1 and 2.
//
// For a product A (m x l) . B (l x n) the planner fixes, following
// arXiv 2405.02238 Section 3:
//  * the client-side slot layouts: sigma(A) / tau(B) for Algorithm 1; for
//    Algorithm 2 the duplicated operand and eps^0_{M x max(l,N')}(sigma(Abar)),
//    omega^0_{max(l,M) x N'}(tau(Bbar)) (Algorithm 2, lines 1-18);
//  * per iteration k the diagonals {d: destination slots} of eps^k and
//    omega^k as linear transformations (Eq. lintrans), d = source - destination
//    slot, with Algorithm 2's first-occurrence keep mask folded into eps^k;
//  * Algorithm 2's extraction rotations h p (h = 1..t-1) and the result slots.
// Algorithm 2 checks p = m first, then p = n, else the l-case; its initial
// C <- sA (.) tB is taken as C <- 0 (the loop already covers k = 0).
#pragma once
#include <stdint.h>

#include <map>
#include <vector>

namespace hg {

struct Diag {
    int d;                 // rotation offset (left), |d| < S
    std::vector<int> dst;  // destination slots where the mask is non-zero
};

struct PlanIter {
    std::vector<Diag> eps, omg;  // ascending d
};

struct HostPlan {
    int m = 0, l = 0, n = 0, alg = 0;
    char kase = '1';     // '1' (Algorithm 1), 'A', 'B', 'L' (Algorithm 2 cases)
    bool col = true;     // column-major flattening
    int p = 0, t = 1, M = 0, Np = 0, WA = 0, HB = 0;
    int a_rows = 0, a_cols = 0, b_rows = 0, b_cols = 0;
    int res_rows = 0, res_cols = 0;
    int length = 0;      // largest slot vector used
    std::vector<PlanIter> iters;
    std::vector<int> extract;

    int flat(int i, int j, int rows, int cols) const { return col ? i + j * rows : i * cols + j; }
    int result_slot(int i, int j) const { return flat(i, j, res_rows, res_cols); }
    // Slot vectors of the client-side layouts; values mod t.
    std::vector<uint64_t> a_slots(const int64_t *A, uint64_t t) const;
    std::vector<uint64_t> b_slots(const int64_t *B, uint64_t t) const;
    // Paper-style counts: one HE-Rot per non-zero diagonal, one CMult per diagonal.
    long long paper_rot() const;
    long long paper_cmult() const;
};

// Shared baby steps: the linear transformations of one operand, in
// iteration order, each rewritten as Rot(sum_d u'_d (.) Rot(x, b_d), g) with
// b_d = (d - g) mod S and u'_d = Rot(u_d, -g) (destination slots + g), an
// identity of cyclic rotations of an S-slot row.  Greedy rule per
// transformation, B = non-zero offsets used so far: over g = 0 and every
// (z - b) mod S (z an offset mod S, b in B or 0) minimise
//   #{distinct (z - g) mod S not in B and != 0} + (g != 0 ? cost : 0),
// ties to the smaller g in [0, S).
constexpr int GIANT_COST = 8;  // a giant rotation, in baby key switches
struct GTerm {
    int b;                 // baby offset in [0, S)
    std::vector<int> dst;  // destination slots of u'_d
};
struct GiantLT {
    int g;                     // giant rotation in [0, S); 0 = none
    std::vector<GTerm> terms;  // in the order of the original diagonals
};
std::vector<GiantLT> giant_factor(const std::vector<const std::vector<Diag> *> &outs, int S, int cost = GIANT_COST);
// The factorisation of operand s (0: eps / A, 1: omega / B) of a plan.
std::vector<GiantLT> giant_factor_of(const HostPlan &P, int s, int S, int cost = GIANT_COST);

// Power-of-two key policy: a left rotation by z over S slots as a chain of
// rotations by signed powers of two, least significant first: the
// non-adjacent form of z mod S or of (z mod S) - S (the same rotation),
// whichever has fewer digits (ties: the non-negative one).  Empty for
// z = 0 mod S.  pow2_offsets: every step the policy uses (+-2^i, 2^i < S),
// as offsets in [0, S).
std::vector<int> pow2_steps(long long z, int S);
std::vector<int> pow2_offsets(int S);

// Number of slots Algorithm 1 / 2 needs for (m, l, n).
int alg1_length(int m, int l, int n);
int alg2_length(int m, int l, int n);
int alg1x_length(int m, int l, int n);
// AUTO: Algorithm 2 if it fits S slots, else Algorithm 1, else 0.
int resolve_alg(int m, int l, int n, int alg, int S);
HostPlan make_host_plan(int m, int l, int n, int alg);
// The result layout of a product (alg 1 or 2): C_ij sits at slot
// i + j rows (col) or i cols + j (!col) of a rows x cols matrix; Algorithm 1
// gives m x n column-major for every l.
void result_layout(int m, int l, int n, int alg, int &rows, int &cols, bool &col);
// The operand layout of role 0 (A, m x l) or 1 (B, l x n) as a slot map from
// the plain column-major matrix (slot i + j rows holds M_ij): for every slot
// of the layout the plain slot it copies, -1 for zero.  An index matrix
// whose entry (i, j) holds its plain slot + 1, carried through the
// client-side layout, names each destination's source.
std::vector<int> operand_source(const HostPlan &P, int role);
// The result of a product as a slot map into the plain column-major m x n
// matrix: destination i + j m takes the result slot of C_ij.
std::vector<int> result_source(const HostPlan &P);

}  // namespace hg

// Internal structures shared by the planner, the executor and the kernels.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/sg2v.h"

namespace sg2v {

constexpr int kMaxColours = 16;
constexpr int kLeaf = -1;

// Binomial coefficient C(n, r) for 0 <= n <= 32 (0 when r < 0 or r > n).
int64_t binom(int n, int r);

// Colex rank of a colour set: with elements c_0 < c_1 < ... the rank is
// sum_i C(c_i, i + 1).  Sets of one size enumerated in increasing bitmask
// order have consecutive ranks 0, 1, 2, ...
uint32_t colex_rank(uint32_t mask);

// One DP node: sub-template T_s with |T_s| = t, split into an active child of
// a vertices and a passive child of p vertices (Sec. 2.3.2).  Children are
// node ids or kLeaf for a single vertex.
struct PlanNode {
    int t = 0, a = 0, p = 0;
    int active = kLeaf, passive = kLeaf;
    bool is_root = false;
    std::string canon;  // AHU form of the rooted sub-template
};

// Colour-compressed tables.  A count M_s(v, S) is zero unless S holds v's own
// colour c (the sub-template's root maps to v), so row v stores only the sets
// S containing c, indexed by the colex rank of S - {c} in the universe of the
// other kc - 1 colours ("squeezed": colours above c move down by one).
uint32_t squeeze_colour(uint32_t mask, int c);
uint32_t unsqueeze_colour(uint32_t mask, int c);

struct CompressedTables {
    // Y'(v, j) for the j-th p-set of the squeezed universe of v's colour c is
    // the sum over k < p of Z[expand[(c * wy + j) * p + k]], where Z(d, i)
    // (offset d * wz_pad + i) accumulates the compressed rows of neighbours of
    // colour d; for p = 1, Z(d) is the colour histogram (wz_pad = 1).
    std::vector<uint32_t> expand;
    int wy = 0;
    // eMA splits in squeezed coordinates (a >= 2): for each (t-1)-set S',
    // nsplit pairs rank(A') | rank(S' - A') << 16 over the (a-1)-subsets A'
    // (set-major: a thread that owns one set walks consecutive words).
    std::vector<uint32_t> splits;
    int nsplit = 0;
};

// Tables of the backward pass of node (t, a, p), squeezed coordinates of the
// row's own colour c (sets of the other kc - 1 colours).
struct BackwardTables {
    // a >= 2: for each p-set P', the pairs rank(S') | rank(S' - P') << 16 over
    // the (t-1)-sets S' containing P' (gradient of Y')
    std::vector<uint32_t> ybar;
    int nybar = 0;
    // a >= 2: for each (a-1)-set A', the pairs rank(S') | rank(S' - A') << 16
    // over the (t-1)-sets S' containing A' (gradient of M_a')
    std::vector<uint32_t> mabar;
    int nmabar = 0;
    // p >= 2: transposed SpMM expansion: the gradient of M_p'(u, P'') (P = {c}
    // + P'') is the sum over the kc - p colours d outside P of Zbar(d, squeezed
    // P), Zbar(d, .) summing gradient rows of neighbours of colour d:
    // offsets d * wz_pad + rank, [kc][C(kc-1, p-1)][kc - p]
    std::vector<uint16_t> expand;
    int wout = 0, nterms = 0;
    // per-arc weight gradient: for neighbour colour cv and own colour cu, the
    // pairs rank of P in cv's squeezed p-sets | rank of P - {cu} in cu's
    // squeezed (p-1)-sets << 16 over the p-sets P with cu in P and cv not in
    // P: [kc][kc][C(kc-2, p-1)] (for p = 1 the second index is 0)
    std::vector<uint32_t> arc;
    int narc = 0;
};

}  // namespace sg2v

struct sg2v_plan {
    int k = 0, kc = 0, root = 0;
    std::vector<int> parent;
    uint64_t alpha = 1;
    double scale = 0.0;  // 1 / (P * alpha)
    long double scale_ld = 0.0L;
    std::vector<sg2v::PlanNode> nodes;  // post-order, root last (empty when k == 1)
    int64_t max_cols = 1;
};

namespace sg2v {
// Builds the colour-compressed tables of node (t, a, p) for kc colours with
// Z rows of wz_pad entries.
void build_compressed_tables(int kc, int t, int a, int wz_pad, CompressedTables *out);
// Builds the backward tables of node (t, a, p) for kc colours; wz_pad is the
// Zbar row stride of the transposed SpMM (p >= 2).
void build_backward_tables(int kc, int t, int a, int wz_pad, BackwardTables *out);
// Thread-local error detail.
void set_error(const std::string &msg);
}  // namespace sg2v

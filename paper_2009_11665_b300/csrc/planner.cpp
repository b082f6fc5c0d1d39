// Template partitioning, sub-template sharing, automorphisms and the
// colour-set index tables (host only; no CUDA calls).
//
// Sec. 2.3.2: the template is split recursively at its root: one edge
// (rho, tau) is cut, the part keeping rho is the active child T_{s,a}, the
// subtree of tau is the passive child T_{s,p}; recursion ends at single
// vertices.  Alg. 2 processes sub-templates children-first.
// Table 1: M_s has one column per colour set of size |T_s|; the column index
// I_C is not fixed by the paper -- this library uses colex rank.
#include <algorithm>
#include <cstring>
#include <functional>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "sg2v_internal.h"

namespace sg2v {

namespace {
struct BinomTable {
    int64_t c[33][33];
    BinomTable() {
        std::memset(c, 0, sizeof c);
        for (int n = 0; n <= 32; ++n) {
            c[n][0] = 1;
            for (int r = 1; r <= n; ++r) c[n][r] = c[n - 1][r - 1] + (r <= n - 1 ? c[n - 1][r] : 0);
        }
    }
};
const BinomTable &binoms() {
    static BinomTable t;
    return t;
}
}  // namespace

int64_t binom(int n, int r) {
    if (n < 0 || n > 32 || r < 0 || r > n) return 0;
    return binoms().c[n][r];
}

uint32_t colex_rank(uint32_t mask) {
    uint32_t r = 0;
    int i = 0;
    while (mask) {
        int c = __builtin_ctz(mask);
        r += (uint32_t)binom(c, i + 1);
        ++i;
        mask &= mask - 1;
    }
    return r;
}

// Next larger mask with the same number of set bits (Gosper); colex order.
static inline uint32_t next_same_popcount(uint32_t x) {
    uint32_t c = x & (0u - x);
    uint32_t r = x + c;
    return (((r ^ x) >> 2) / c) | r;
}

uint32_t squeeze_colour(uint32_t mask, int c) {
    const uint32_t low = (1u << c) - 1u;
    return (mask & low) | ((mask >> (c + 1)) << c);
}

uint32_t unsqueeze_colour(uint32_t mask, int c) {
    const uint32_t low = (1u << c) - 1u;
    return (mask & low) | ((mask >> c) << (c + 1));
}

void build_compressed_tables(int kc, int t, int a, int wz_pad, CompressedTables *out) {
    const int p = t - a;
    const int wy = (int)binom(kc - 1, p);
    out->wy = wy;
    out->expand.assign((size_t)kc * wy * p, 0);
    for (int c = 0; c < kc; ++c) {
        uint32_t Pq = (1u << p) - 1;
        for (int j = 0; j < wy; ++j, Pq = next_same_popcount(Pq)) {
            const uint32_t P = unsqueeze_colour(Pq, c);  // a p-set of colours without c
            int k = 0;
            for (uint32_t rest = P; rest; rest &= rest - 1, ++k) {
                const int d = __builtin_ctz(rest);
                const uint32_t idx = p == 1 ? 0u : colex_rank(squeeze_colour(P ^ (1u << d), d));
                out->expand[((size_t)c * wy + j) * p + k] = (uint32_t)d * (uint32_t)wz_pad + idx;
            }
        }
    }
    out->splits.clear();
    out->nsplit = 0;
    if (a >= 2) {
        const int ws = (int)binom(kc - 1, t - 1);
        const int ns = (int)binom(t - 1, a - 1);
        out->nsplit = ns;
        out->splits.resize((size_t)ws * ns);
        uint32_t S = (1u << (t - 1)) - 1;
        for (int s = 0; s < ws; ++s, S = next_same_popcount(S)) {
            int j = 0;
            for (uint32_t A = 0;;) {
                A = (A - S) & S;
                if (A == 0) break;
                if (__builtin_popcount(A) == a - 1) {
                    out->splits[(size_t)s * ns + j] = colex_rank(A) | (colex_rank(S ^ A) << 16);
                    ++j;
                }
            }
        }
    }
}

void build_backward_tables(int kc, int t, int a, int wz_pad, BackwardTables *out) {
    const int p = t - a;
    const int u = kc - 1;  // squeezed universe
    *out = BackwardTables();
    if (a >= 2) {
        const int wy = (int)binom(u, p), wa = (int)binom(u, a - 1);
        out->nybar = (int)binom(u - p, a - 1);
        out->nmabar = (int)binom(u - (a - 1), p);
        out->ybar.assign((size_t)wy * out->nybar, 0);
        out->mabar.assign((size_t)wa * out->nmabar, 0);
        std::vector<int> fy(wy, 0), fa(wa, 0);
        uint32_t S = (1u << (t - 1)) - 1;
        const int ws = (int)binom(u, t - 1);
        for (int s = 0; s < ws; ++s, S = next_same_popcount(S)) {
            for (uint32_t A = 0;;) {
                A = (A - S) & S;
                if (A == 0 && a - 1 > 0) break;
                if (__builtin_popcount(A) == a - 1) {
                    const uint32_t P = S ^ A;
                    const uint32_t rp = colex_rank(P), ra = colex_rank(A);
                    out->ybar[(size_t)rp * out->nybar + fy[rp]++] = (uint32_t)s | (ra << 16);
                    out->mabar[(size_t)ra * out->nmabar + fa[ra]++] = (uint32_t)s | (rp << 16);
                }
                if (A == 0) break;
            }
        }
    }
    if (p >= 2) {
        const int wout = (int)binom(u, p - 1);
        out->wout = wout;
        out->nterms = kc - p;
        out->expand.assign((size_t)kc * wout * out->nterms, 0);
        for (int c = 0; c < kc; ++c) {
            uint32_t Q = (1u << (p - 1)) - 1;
            for (int j = 0; j < wout; ++j, Q = next_same_popcount(Q)) {
                const uint32_t P = unsqueeze_colour(Q, c) | (1u << c);
                int k = 0;
                for (int d = 0; d < kc; ++d) {
                    if (P >> d & 1u) continue;
                    out->expand[((size_t)c * wout + j) * out->nterms + k++] =
                        (uint16_t)(d * wz_pad + (int)colex_rank(squeeze_colour(P, d)));
                }
            }
        }
    }
    // arc pairs: P ranges over p-sets with cu in P, cv not in P
    out->narc = (int)binom(kc - 2, p - 1);
    out->arc.assign((size_t)kc * kc * out->narc, 0);
    for (int cv = 0; cv < kc; ++cv) {
        for (int cu = 0; cu < kc; ++cu) {
            if (cu == cv) continue;
            int k = 0;
            uint32_t P = (1u << p) - 1;
            const int all = (int)binom(kc, p);
            for (int i = 0; i < all; ++i, P = next_same_popcount(P)) {
                if (!(P >> cu & 1u) || (P >> cv & 1u)) continue;
                const uint32_t iy = colex_rank(squeeze_colour(P, cv));
                const uint32_t im = p == 1 ? 0u : colex_rank(squeeze_colour(P ^ (1u << cu), cu));
                out->arc[((size_t)cv * kc + cu) * out->narc + k++] = iy | (im << 16);
            }
        }
    }
}

}  // namespace sg2v

namespace {

struct Tree {
    int k = 0;
    std::vector<int> par;
    std::vector<std::vector<int>> children;  // increasing vertex index
    std::vector<std::vector<int>> adj;
};

// Validates the parent array and orients the tree from `root`.
sg2v_status build_tree(int k, const int32_t *parent, int root, Tree *T) {
    if (root < 0 || root >= k) {
        sg2v::set_error("root out of range");
        return SG2V_ERR_NOT_A_TREE;
    }
    T->k = k;
    T->adj.assign(k, {});
    int roots = 0;
    for (int i = 0; i < k; ++i) {
        int p = parent[i];
        if (p == -1) {
            ++roots;
            continue;
        }
        if (p < 0 || p >= k || p == i) {
            sg2v::set_error("parent entry out of range");
            return SG2V_ERR_NOT_A_TREE;
        }
        T->adj[i].push_back(p);
        T->adj[p].push_back(i);
    }
    if (roots != 1) {
        sg2v::set_error("parent array must contain exactly one -1");
        return SG2V_ERR_NOT_A_TREE;
    }
    for (auto &a : T->adj) std::sort(a.begin(), a.end());
    T->par.assign(k, -2);
    T->children.assign(k, {});
    std::vector<int> queue{root};
    T->par[root] = -1;
    for (size_t h = 0; h < queue.size(); ++h) {
        int x = queue[h];
        for (int y : T->adj[x]) {
            if (y == T->par[x]) continue;
            if (T->par[y] != -2) {
                sg2v::set_error("parent array contains a cycle");
                return SG2V_ERR_NOT_A_TREE;
            }
            T->par[y] = x;
            T->children[x].push_back(y);
            queue.push_back(y);
        }
    }
    if ((int)queue.size() != k) {
        sg2v::set_error("parent array is not connected");
        return SG2V_ERR_NOT_A_TREE;
    }
    return SG2V_OK;
}

// AHU canonical string of the subtree of x when the tree is entered from
// `from` (x's neighbours other than `from` are its children); also returns
// the number of automorphisms of that rooted subtree.
std::string rooted_form(const Tree &T, int x, int from, uint64_t *aut) {
    std::vector<std::string> forms;
    uint64_t a = 1;
    for (int y : T.adj[x]) {
        if (y == from) continue;
        uint64_t ay;
        forms.push_back(rooted_form(T, y, x, &ay));
        a *= ay;
    }
    std::sort(forms.begin(), forms.end());
    for (size_t i = 0; i < forms.size();) {
        size_t j = i;
        while (j < forms.size() && forms[j] == forms[i]) ++j;
        for (size_t m = 2; m <= j - i; ++m) a *= m;  // identical children permute freely
        i = j;
    }
    std::string s = "(";
    for (auto &f : forms) s += f;
    s += ")";
    *aut = a;
    return s;
}

// Automorphisms of the unrooted tree: root it at its centre (or at the two
// ends of its central edge).
uint64_t automorphisms(const Tree &T) {
    int k = T.k;
    if (k == 1) return 1;
    std::vector<int> ecc(k, 0);
    for (int s = 0; s < k; ++s) {
        std::vector<int> d(k, -1);
        std::vector<int> q{s};
        d[s] = 0;
        for (size_t h = 0; h < q.size(); ++h)
            for (int y : T.adj[q[h]])
                if (d[y] < 0) {
                    d[y] = d[q[h]] + 1;
                    q.push_back(y);
                }
        ecc[s] = *std::max_element(d.begin(), d.end());
    }
    int best = *std::min_element(ecc.begin(), ecc.end());
    std::vector<int> centres;
    for (int s = 0; s < k; ++s)
        if (ecc[s] == best) centres.push_back(s);
    if (centres.size() == 1) {
        uint64_t a;
        rooted_form(T, centres[0], -1, &a);
        return a;
    }
    int c1 = centres[0], c2 = centres[1];
    uint64_t a1, a2;
    std::string f1 = rooted_form(T, c1, c2, &a1);
    std::string f2 = rooted_form(T, c2, c1, &a2);
    return a1 * a2 * (f1 == f2 ? 2u : 1u);
}

// Sub-templates are (x, mask): x with the children of x whose bits are set
// in mask (each with its whole subtree).  The plan cuts one kept child per
// node: the last (highest vertex index) by default, or the choice that
// minimises a work model (min_work).
struct PlanBuilder {
    const Tree &T;
    int kc = 0;
    bool min_work = false;
    double degree = 32.0;
    std::vector<sg2v::PlanNode> nodes;
    std::map<std::string, int> by_form;
    // form of a sub-template -> (least work, form of the child subtree to cut);
    // isomorphic sub-templates share the entry, so the cut is kept as a form
    std::map<std::string, std::pair<double, std::string>> best;

    explicit PlanBuilder(const Tree &t) : T(t) {}

    std::string form_of(int x, uint32_t mask) {
        std::vector<std::string> forms;
        for (size_t i = 0; i < T.children[x].size(); ++i) {
            if (!(mask >> i & 1u)) continue;
            uint64_t unused;
            forms.push_back(rooted_form(T, T.children[x][i], x, &unused));
        }
        std::sort(forms.begin(), forms.end());
        std::string s = "(";
        for (auto &f : forms) s += f;
        return s + ")";
    }

    int subtree_size(int y) const {
        int n = 1;
        for (int c : T.children[y]) n += subtree_size(c);
        return n;
    }

    int size_of(int x, uint32_t mask) const {
        int n = 1;
        for (size_t i = 0; i < T.children[x].size(); ++i)
            if (mask >> i & 1u) n += subtree_size(T.children[x][i]);
        return n;
    }

    static uint32_t all_children(const Tree &T, int x) {
        return T.children[x].size() >= 32 ? ~0u : (1u << T.children[x].size()) - 1u;
    }

    // Work of one node per vertex and colouring, in units of one gathered
    // word of a compressed row (B300 measurements): an arc of a gathering
    // node costs about 20 units plus its row's words, an arc of a histogram
    // node about 2, a product of the eMA about 0.5, a written output word
    // about 1.4.  A root whose two children are isomorphic gathers half the
    // arcs.
    double node_work(int t, int a, int p, bool root, bool twin) const {
        const int u = kc - 1;
        double gather = p >= 2 ? degree * (20.0 + (double)sg2v::binom(u, p - 1)) : degree * 2.0;
        if (root && twin) gather *= 0.5;
        const double ema = a >= 2 ? 0.5 * (double)sg2v::binom(u, t - 1) * (double)sg2v::binom(t - 1, a - 1) : 0.0;
        const double write = root ? 0.0 : 1.4 * (double)sg2v::binom(u, t - 1);
        return gather + ema + write;
    }

    std::string child_form(int x, int i) const {
        uint64_t unused;
        return rooted_form(T, T.children[x][i], x, &unused);
    }

    // Least modelled work of (x, mask) and the child to cut (index into children[x]).
    double plan_work(int x, uint32_t mask, bool root, int *cut) {
        *cut = -1;
        if (mask == 0) return 0.0;
        const std::string f = form_of(x, mask) + (root ? "r" : "");
        auto it = best.find(f);
        if (it != best.end()) {
            for (size_t i = 0; i < T.children[x].size(); ++i)
                if ((mask >> i & 1u) && child_form(x, (int)i) == it->second.second) {
                    *cut = (int)i;
                    break;
                }
            return it->second.first;
        }
        double w_best = 0.0;
        int c_best = -1;
        const int t = size_of(x, mask);
        for (size_t i = 0; i < T.children[x].size(); ++i) {
            if (!(mask >> i & 1u)) continue;
            const int y = T.children[x][i];
            const uint32_t rest = mask & ~(1u << i);
            int unused;
            const int p = subtree_size(y);
            const bool twin = root && form_of(x, rest) == form_of(y, all_children(T, y));
            const double w = node_work(t, t - p, p, root, twin) + plan_work(x, rest, false, &unused) +
                             plan_work(y, all_children(T, y), false, &unused);
            if (c_best < 0 || w < w_best) {
                w_best = w;
                c_best = (int)i;
            }
        }
        best[f] = {w_best, child_form(x, c_best)};
        *cut = c_best;
        return w_best;
    }

    // Returns the node id of sub-template (x, mask), kLeaf for a single vertex;
    // *size receives its number of vertices.
    int make(int x, uint32_t mask, bool root, int *size) {
        if (mask == 0) {
            *size = 1;
            return sg2v::kLeaf;
        }
        std::string f = form_of(x, mask);
        auto it = by_form.find(f);
        if (it != by_form.end() && !root) {
            *size = nodes[it->second].t;
            return it->second;
        }
        int ci = 31 - __builtin_clz(mask);  // the last kept child
        if (min_work) plan_work(x, mask, root, &ci);
        const int tau = T.children[x][ci];
        int a, p;
        int ia = make(x, mask & ~(1u << ci), false, &a);
        int ip = make(tau, all_children(T, tau), false, &p);
        sg2v::PlanNode nd;
        nd.t = a + p;
        nd.a = a;
        nd.p = p;
        nd.active = ia;
        nd.passive = ip;
        nd.canon = f;
        nodes.push_back(nd);
        int id = (int)nodes.size() - 1;
        if (!root) by_form[f] = id;
        *size = nd.t;
        return id;
    }

    // Modelled work of the built plan, every distinct node counted once.
    double built_work() const {
        double w = 0.0;
        for (const auto &nd : nodes) {
            const bool twin = nd.is_root && nd.active == nd.passive && nd.active != sg2v::kLeaf;
            w += node_work(nd.t, nd.a, nd.p, nd.is_root, twin);
        }
        return w;
    }
};

}  // namespace

extern "C" {

sg2v_status sg2v_template_plan(int32_t k, const int32_t *parent, int32_t root, int32_t num_colours,
                               const void *opts, sg2v_plan **out) {
    if (!out || !parent) {
        sg2v::set_error("null argument");
        return SG2V_ERR_INVALID_ARGUMENT;
    }
    *out = nullptr;
    if (k < 1 || k > sg2v::kMaxColours) {
        sg2v::set_error("template size must be in [1, 16]");
        return k < 1 ? SG2V_ERR_INVALID_ARGUMENT : SG2V_ERR_UNSUPPORTED;
    }
    if (num_colours < k) {
        sg2v::set_error("num_colours must be >= template size");
        return SG2V_ERR_INVALID_ARGUMENT;
    }
    if (num_colours > sg2v::kMaxColours) {
        sg2v::set_error("num_colours above 16 is not supported");
        return SG2V_ERR_UNSUPPORTED;
    }
    Tree T;
    sg2v_status st = build_tree(k, parent, root, &T);
    if (st != SG2V_OK) return st;
    sg2v_plan *plan = new (std::nothrow) sg2v_plan();
    if (!plan) return SG2V_ERR_OUT_OF_MEMORY;
    plan->k = k;
    plan->kc = num_colours;
    plan->root = root;
    plan->parent.assign(parent, parent + k);
    plan->alpha = automorphisms(T);
    if (T.children[root].size() > 31) {
        sg2v::set_error("template root has too many children");
        delete plan;
        return SG2V_ERR_UNSUPPORTED;
    }
    const sg2v_plan_opts *o = static_cast<const sg2v_plan_opts *>(opts);
    if (o && (o->size != sizeof(sg2v_plan_opts) || (o->cut != SG2V_CUT_LAST && o->cut != SG2V_CUT_MIN_WORK) ||
              !(o->avg_degree >= 0.0f))) {
        sg2v::set_error("invalid plan options");
        delete plan;
        return SG2V_ERR_INVALID_ARGUMENT;
    }
    auto build = [&](bool min_work, PlanBuilder *B) {
        B->kc = num_colours;
        B->min_work = min_work;
        if (o && o->avg_degree > 0.0f) B->degree = o->avg_degree;
        int size;
        int rid = B->make(root, PlanBuilder::all_children(T, root), true, &size);
        if (rid != sg2v::kLeaf) B->nodes[rid].is_root = true;
    };
    PlanBuilder B(T);
    build(false, &B);
    if (o && o->cut == SG2V_CUT_MIN_WORK) {
        // the work-minimising cuts when the model gains at least 1% over the
        // default plan, sharing counted (smaller gains are within the
        // model's error on B300)
        PlanBuilder M(T);
        build(true, &M);
        if (M.built_work() < 0.99 * B.built_work()) B.nodes = std::move(M.nodes);
    }
    plan->nodes = std::move(B.nodes);
    plan->max_cols = sg2v::binom(num_colours, 1);
    for (auto &nd : plan->nodes) {
        plan->max_cols = std::max<int64_t>(plan->max_cols, sg2v::binom(num_colours, nd.t));
        plan->max_cols = std::max<int64_t>(plan->max_cols, sg2v::binom(num_colours, nd.p));
    }
    // 1 / (P alpha) with P = kc! / ((kc - k)! kc^k)
    unsigned __int128 num = 1, den = plan->alpha;
    for (int i = 0; i < k; ++i) {
        num *= (unsigned __int128)num_colours;
        den *= (unsigned __int128)(num_colours - i);
    }
    plan->scale_ld = (long double)num / (long double)den;
    plan->scale = (double)plan->scale_ld;
    *out = plan;
    return SG2V_OK;
}

sg2v_status sg2v_plan_destroy(sg2v_plan *plan) {
    delete plan;
    return SG2V_OK;
}

sg2v_status sg2v_plan_info(const sg2v_plan *plan, int64_t *automorphisms_out, int32_t *num_nodes,
                           int64_t *max_cols) {
    if (!plan) {
        sg2v::set_error("null plan");
        return SG2V_ERR_INVALID_ARGUMENT;
    }
    if (automorphisms_out) *automorphisms_out = (int64_t)plan->alpha;
    if (num_nodes) *num_nodes = (int32_t)plan->nodes.size();
    if (max_cols) *max_cols = plan->max_cols;
    return SG2V_OK;
}

sg2v_status sg2v_plan_nodes(const sg2v_plan *plan, int32_t *out, int64_t capacity) {
    if (!plan || (!out && !plan->nodes.empty())) {
        sg2v::set_error("null argument");
        return SG2V_ERR_INVALID_ARGUMENT;
    }
    if (capacity < (int64_t)(6 * plan->nodes.size())) {
        sg2v::set_error("output capacity too small");
        return SG2V_ERR_INVALID_ARGUMENT;
    }
    for (size_t i = 0; i < plan->nodes.size(); ++i) {
        const auto &nd = plan->nodes[i];
        int32_t *o = out + 6 * i;
        o[0] = nd.t;
        o[1] = nd.a;
        o[2] = nd.p;
        o[3] = nd.active;
        o[4] = nd.passive;
        o[5] = nd.is_root ? 1 : 0;
    }
    return SG2V_OK;
}

sg2v_status sg2v_plan_estimate_scale(const sg2v_plan *plan, double *scale) {
    if (!plan || !scale) {
        sg2v::set_error("null argument");
        return SG2V_ERR_INVALID_ARGUMENT;
    }
    *scale = plan->scale;
    return SG2V_OK;
}

}  // extern "C"

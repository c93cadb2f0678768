// evolve.cpp -- one generation of tree GP on the host, directly on the
// population DAG (TensorGP, Sec. 3 and Table 2: tournament selection,
// subtree crossover, subtree mutation, elitism), and the export of a
// population back to tokens.
//
// A tree is its root's DAG node; a subtree is a node.  Crossover replaces one
// node occurrence of the first parent's tree by a node of the second parent,
// and mutation by a fresh grow tree: only the nodes on the path from that
// occurrence to the root are new, and they are hash-consed into the next
// generation's DAG together with every unchanged subtree, which keeps its
// identity (no re-parse of unchanged subtrees; a cached subtree stays
// cached).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/tgp.h"
#include "compiler.h"
#include "internal.h"

namespace tgp {
namespace {

// splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014): a counter-based generator, deterministic per seed.
struct Rng {
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9e3779b97f4a7c15ull);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        return z ^ (z >> 31);
    }
    double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }   // [0, 1)
    int64_t below(int64_t n) { return n <= 1 ? 0 : (int64_t)(uniform() * (double)n); }
};

// Copies the subtree rooted at node n of `src` into `dst` (hash-consed).
int32_t copy_node(const Dag& src, int32_t n, Dag& dst, std::vector<int32_t>& memo) {
    if (memo[n] >= 0) return memo[n];
    const DagNode& x = src.nodes[n];
    int32_t k[kMaxKids] = {-1, -1, -1};
    for (int c = 0; c < kMaxKids; ++c)
        if (x.kid[c] >= 0) k[c] = copy_node(src, x.kid[c], dst, memo);
    const int32_t id = dst.intern(x.op, k[0], k[1], x.imm, k[2]);
    memo[n] = id;
    return id;
}

// One occurrence of a node in a tree: the node and its path from the root
// (parent node, operand index) pairs.
struct Site {
    std::vector<std::pair<int32_t, int>> path;
    int32_t node;
    int depth;
};

// The `target`-th node of the tree rooted at r, in preorder.
Site site_at(const Dag& dag, int32_t r, int64_t target) {
    Site s;
    s.node = r;
    s.depth = 0;
    int64_t idx = 0;
    // iterative preorder with explicit path
    std::vector<std::pair<int32_t, int>> path;
    struct Frame { int32_t n; int next; };
    std::vector<Frame> st{{r, 0}};
    while (!st.empty()) {
        Frame& f = st.back();
        if (f.next == 0) {
            if (idx == target) {
                s.node = f.n;
                s.depth = (int)path.size();
                s.path = path;
                return s;
            }
            ++idx;
        }
        const DagNode& x = dag.nodes[f.n];
        int c = f.next;
        while (c < kMaxKids && x.kid[c] < 0) ++c;
        if (c >= kMaxKids) {
            st.pop_back();
            if (!path.empty()) path.pop_back();
            continue;
        }
        f.next = c + 1;
        path.push_back({f.n, c});
        st.push_back({x.kid[c], 0});
    }
    return s;
}

// Largest tree (in tokens, every occurrence of a shared subtree counted) an
// offspring may have: the token limit of one tree in tgp_compile_population.
constexpr int64_t kMaxTreeTokens = (int64_t)1 << 24;

// Number of nodes of the tree rooted at n (counting every occurrence),
// saturating above kMaxTreeTokens (shared subtrees can make it exponential
// in the depth).
int64_t tree_size(const Dag& dag, int32_t n, std::vector<int64_t>& memo) {
    if (memo[n] >= 0) return memo[n];
    int64_t t = 1;
    for (int c = 0; c < kMaxKids; ++c)
        if (dag.nodes[n].kid[c] >= 0) t = std::min(t + tree_size(dag, dag.nodes[n].kid[c], memo), kMaxTreeTokens + 1);
    memo[n] = t;
    return t;
}

// Rebuilds the path of `site` with `repl` at its end (nodes of `dag`).
int32_t replace_at(Dag& dag, const Site& site, int32_t repl, bool simplify) {
    int32_t cur = repl;
    for (size_t i = site.path.size(); i-- > 0;) {
        const DagNode x = dag.nodes[site.path[i].first];
        int32_t k[kMaxKids] = {x.kid[0], x.kid[1], x.kid[2]};
        k[site.path[i].second] = cur;
        cur = simplify ? intern_simplified(dag, x.op, k[0], k[1], x.imm, k[2]) : dag.intern(x.op, k[0], k[1], x.imm, k[2]);
    }
    return cur;
}

struct GrowSpec {
    std::vector<int32_t> funcs;
    float lo, hi;
    bool simplify;
};

int32_t terminal(Dag& dag, Rng& rng, const GrowSpec& g) {
    const int64_t t = rng.below(3);
    if (t == 0) return dag.intern(T_X, -1, -1, 0);
    if (t == 1) return dag.intern(T_Y, -1, -1, 0);
    const float v = (float)(g.lo + (g.hi - g.lo) * rng.uniform());
    uint32_t b;
    std::memcpy(&b, &v, 4);
    return dag.intern(T_CONST, -1, -1, b);
}

// A grow tree of depth <= d (root: a function when d > 0).
int32_t grow(Dag& dag, Rng& rng, const GrowSpec& g, int d, bool at_root) {
    if (d == 0) return terminal(dag, rng, g);
    const int64_t nf = (int64_t)g.funcs.size();
    const int64_t pick = rng.below(at_root ? nf : nf + 3);
    if (pick >= nf) return terminal(dag, rng, g);
    const int op = g.funcs[pick];
    int32_t k[kMaxKids] = {-1, -1, -1};
    for (int c = 0; c < arity(op); ++c) k[c] = grow(dag, rng, g, d - 1, false);
    return make_node(dag, op, k, 0, g.simplify);
}

double rank_key(double r) { return std::isfinite(r) ? r : INFINITY; }

}  // namespace
}  // namespace tgp

using namespace tgp;

extern "C" {

int tgp_evolve(tgp_ctx* ctx, tgp_handle pop, const double* rmse, const tgp_evolve_config* cfg_in,
               tgp_handle* next_pop) {
    if (!ctx || !rmse || !next_pop) return internal::set_error(TGP_E_INVALID, "ctx / rmse / next_pop is NULL");
    tgp_evolve_config cfg{};
    if (cfg_in) cfg = *cfg_in;
    const int tour = cfg.tournament > 0 ? cfg.tournament : 3;
    const double pc = cfg.p_crossover > 0 ? cfg.p_crossover : cfg.p_crossover < 0 ? 0.0 : 0.9;
    const double pm = cfg.p_mutation > 0 ? cfg.p_mutation : cfg.p_mutation < 0 ? 0.0 : 0.1;
    const int elit = cfg.elitism > 0 ? cfg.elitism : cfg.elitism < 0 ? 0 : 1;
    const int max_depth = cfg.max_depth > 0 ? cfg.max_depth : 12;
    if (max_depth > 1024)   // the depth limit of tgp_compile_population
        return internal::set_error(TGP_E_INVALID, "max_depth %d exceeds 1024", max_depth);
    const int mdepth = cfg.mutation_depth > 0 ? cfg.mutation_depth : 4;
    GrowSpec gs;
    if (cfg.functions && cfg.n_functions > 0) {
        for (int i = 0; i < cfg.n_functions; ++i) {
            const int op = cfg.functions[i];
            if (arity(op) <= 0)
                return internal::set_error(TGP_E_INVALID, "function set entry %d (opcode %d) is not a function", i, op);
            gs.funcs.push_back(op);
        }
    } else {
        gs.funcs = {T_ADD, T_SUB, T_MUL, T_DIV, T_SIN, T_COS, T_NEG, T_ABS, T_MIN, T_MAX};
    }
    gs.lo = cfg.const_lo;
    gs.hi = cfg.const_hi;
    if (gs.lo == 0.f && gs.hi == 0.f) { gs.lo = -1.f; gs.hi = 1.f; }
    gs.simplify = internal::context_simplifies(ctx);

    PopIR cur;
    int rc = internal::population_copy(ctx, pop, &cur);
    if (rc) return rc;
    const int64_t T = (int64_t)cur.roots.size();
    if (T == 0) return internal::set_error(TGP_E_INVALID, "empty population");
    Rng rng{cfg.seed};

    // the parents' DAG is extended in place with the new path nodes, then the
    // next generation's trees are copied (hash-consed) into a fresh DAG
    Dag& dag = cur.dag;
    std::vector<int64_t> size_memo(dag.size(), -1);
    auto size_of = [&](int32_t n) {
        if ((size_t)n >= size_memo.size()) size_memo.resize(dag.size(), -1);
        return tree_size(dag, n, size_memo);
    };
    std::vector<int32_t> order(T);
    for (int64_t t = 0; t < T; ++t) order[t] = (int32_t)t;
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return rank_key(rmse[a]) < rank_key(rmse[b]); });
    auto select = [&]() {
        int64_t best = rng.below(T);
        for (int i = 1; i < tour; ++i) {
            const int64_t c = rng.below(T);
            if (rank_key(rmse[c]) < rank_key(rmse[best]) || (rank_key(rmse[c]) == rank_key(rmse[best]) && c < best))
                best = c;
        }
        return cur.roots[best];
    };
    std::vector<int32_t> next;
    next.reserve(T);
    for (int i = 0; i < std::min<int64_t>(elit, T); ++i) next.push_back(cur.roots[order[i]]);
    while ((int64_t)next.size() < T) {
        const int32_t a = select();
        const double u = rng.uniform();
        int32_t child = a;
        if (u < pc) {
            const int32_t b = select();
            const Site sa = site_at(dag, a, rng.below(size_of(a)));
            const Site sb = site_at(dag, b, rng.below(size_of(b)));
            if (sa.depth + dag.nodes[sb.node].depth <= max_depth) child = replace_at(dag, sa, sb.node, gs.simplify);
            if (size_of(child) > kMaxTreeTokens) child = a;
        } else if (u < pc + pm) {
            const Site sa = site_at(dag, a, rng.below(size_of(a)));
            const int d = (int)rng.below(mdepth + 1);
            const int32_t sub = grow(dag, rng, gs, d, true);
            if (sa.depth + dag.nodes[sub].depth <= max_depth) child = replace_at(dag, sa, sub, gs.simplify);
            if (size_of(child) > kMaxTreeTokens) child = a;
        }
        next.push_back(child);
    }
    PopIR out;
    std::vector<int32_t> memo(dag.size(), -1);
    std::vector<int64_t> smemo(dag.size(), -1);
    for (int32_t r : next) {
        const int32_t id = copy_node(dag, r, out.dag, memo);
        out.roots.push_back(id);
        const int64_t n = tree_size(dag, r, smemo);
        out.tree_size.push_back((int32_t)std::min<int64_t>(n, INT32_MAX));
        out.tree_cost.push_back(out.dag.nodes[id].cost);
        out.tree_nodes += n;
    }
    return internal::adopt_population(ctx, std::move(out), next_pop);
}

int tgp_population_tokens(tgp_ctx* ctx, tgp_handle pop, int32_t* ops, int64_t cap_ops, float* imm, int64_t cap_imm,
                          int64_t* tree_off, int64_t cap_off, int64_t* n_ops, int64_t* n_imm, int32_t* n_trees) {
    if (!ctx) return internal::set_error(TGP_E_INVALID, "ctx is NULL");
    PopIR ir;
    int rc = internal::population_copy(ctx, pop, &ir);
    if (rc) return rc;
    const int64_t T = (int64_t)ir.roots.size();
    int64_t no = 0, ni = 0;
    std::vector<int32_t> st;
    for (int64_t t = 0; t < T; ++t) {
        if (tree_off && t < cap_off) tree_off[t] = no;
        st.assign(1, ir.roots[t]);
        while (!st.empty()) {   // prefix order: a node, then its operands left to right
            const int32_t n = st.back();
            st.pop_back();
            const DagNode& x = ir.dag.nodes[n];
            if (ops && no < cap_ops) ops[no] = x.op;
            ++no;
            if (x.op == T_CONST) {
                if (imm && ni < cap_imm) std::memcpy(&imm[ni], &x.imm, 4);
                ++ni;
            }
            for (int c = kMaxKids - 1; c >= 0; --c)
                if (x.kid[c] >= 0) st.push_back(x.kid[c]);
        }
    }
    if (tree_off && T < cap_off) tree_off[T] = no;
    if (n_ops) *n_ops = no;
    if (n_imm) *n_imm = ni;
    if (n_trees) *n_trees = (int32_t)T;
    if ((ops && no > cap_ops) || (imm && ni > cap_imm) || (tree_off && T + 1 > cap_off))
        return internal::set_error(TGP_E_INVALID,
                                   "token arrays too small: %lld ops, %lld constants and %lld offsets needed",
                                   (long long)no, (long long)ni, (long long)(T + 1));
    return TGP_OK;
}

}  // extern "C"

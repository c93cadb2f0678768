// compiler.cpp -- token decode, hash-consing and bytecode generation.
//
// Hot-path steps on the host (all O(tokens)):
//   1. decode + validate each tree of the token stream (prefix or postfix);
//   2. hash-cons every node into the population DAG, so structurally equal
//      subtrees of any tree share one node (Handley's DAG; Sec. 2 and the
//      graph-mode DAG of Sec. 3.1 of TensorGP);
//   3. split the trees into groups (one group = one instruction stream that a
//      CTA runs over a tile of points), order each tree's evaluation
//      Sethi-Ullman style, allocate register slots by liveness, and emit
//      bytecode.  A DAG node used more than once inside a group is evaluated
//      once per point and kept in a register slot (or, when registers run
//      out, a shared-memory slot) until its last use.
#include "compiler.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <memory>
#include <numeric>

namespace tgp {

int arity(int op) {
    switch (op) {
    case T_X: case T_Y: case T_CONST: return 0;
    case T_SIN: case T_COS: case T_NEG: case T_ABS:
    case T_TAN: case T_EXP: case T_LOG: case T_SQRT: case T_SIGN: case T_FRAC: return 1;
    case T_ADD: case T_SUB: case T_MUL: case T_DIV: case T_MIN: case T_MAX:
    case T_POW: case T_MDIST: case T_MOD: return 2;
    case T_CLIP: case T_IF: return 3;
    default: return -1;
    }
}

float op_cost(int op) {
    switch (op) {
    case T_X: case T_Y: case T_CONST: return 0.f;
    case T_DIV: return 8.f;
    case T_SIN: case T_COS: case T_EXP: case T_LOG: case T_MOD: return 16.f;
    case T_TAN: case T_POW: return 40.f;
    case T_SQRT: return 4.f;
    case T_MDIST: case T_SIGN: case T_FRAC: return 2.f;
    default: return 1.f;
    }
}

// ------------------------------------------------------------------ DAG

static inline uint64_t mix64(uint64_t z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// Node ids do not depend on the hash (they are creation order); the key
// comparison on a hit is exact, so only the probe length depends on it.
static inline uint64_t key_hash(int op, int32_t k0, int32_t k1, uint32_t imm, int32_t k2) {
    const uint64_t a = ((uint64_t)(uint32_t)k0 << 32) | (uint32_t)k1;
    const uint64_t b = ((uint64_t)(uint32_t)op << 32) | imm;
    return mix64(a * 0x9e3779b97f4a7c15ull ^ b ^ (uint64_t)(uint32_t)k2 * 0xc2b2ae3d27d4eb4full);
}

void Dag::rehash(size_t cap) {
    table_.assign(cap, -1);
    mask_ = cap - 1;
    for (size_t i = 0; i < nodes.size(); ++i) {
        const DagNode& n = nodes[i];
        size_t h = key_hash(n.op, n.kid[0], n.kid[1], n.imm, n.kid[2]) & mask_;
        while (table_[h] >= 0) h = (h + 1) & mask_;
        table_[h] = (int32_t)i;
    }
}

void Dag::reserve(size_t n) {
    nodes.reserve(n);
    size_t cap = 1024;
    while (cap < 2 * n + 2) cap *= 2;
    if (cap > table_.size()) rehash(cap);
}

void Dag::assign_nodes(NodeVec&& v) {
    nodes = std::move(v);
    used_ = nodes.size();
    // the index is rebuilt by the first intern, if any comes (a parsed
    // population is mostly only planned)
    table_.clear();
    table_.shrink_to_fit();
}

// The fields of node n that follow from its key and its operands' fields
// (`nodes` holds the operands): Sethi-Ullman slots, depth, cost as a tree,
// the coordinates below it.  They are functions of the subtree, and for a
// binary node they do not depend on the order of its operands.
static void derive_fields(DagNode& n, const DagNode* nodes) {
    const int op = n.op;
    const int ar = arity(op);
    n.spare_ = 0;
    n.vars = op == T_X ? 1 : op == T_Y ? 2 : 0;
    for (int c = 0; c < ar; ++c) n.vars |= nodes[n.kid[c]].vars;
    if (ar == 3) {
        // planned order: operand 0 and 1 parked in slots, operand 2 into A
        const DagNode& a = nodes[n.kid[0]];
        const DagNode& b = nodes[n.kid[1]];
        const DagNode& c = nodes[n.kid[2]];
        n.su = std::max(a.su, std::max(b.su + 1, c.su + 2));
        n.depth = std::max(a.depth, std::max(b.depth, c.depth)) + 1;
        n.cost = op_cost(op) + a.cost + b.cost + c.cost;
    } else if (ar == 0) {
        n.su = 0;
        n.depth = 0;
        n.cost = 0.f;
    } else if (ar == 1) {
        const DagNode& c = nodes[n.kid[0]];
        n.su = c.su;
        n.depth = c.depth + 1;
        n.cost = op_cost(op) + c.cost;
    } else {
        const DagNode& l = nodes[n.kid[0]];
        const DagNode& r = nodes[n.kid[1]];
        bool ll = is_leaf(l.op), rl = is_leaf(r.op);
        if (ll && rl) n.su = 0;
        else if (ll) n.su = r.su;
        else if (rl) n.su = l.su;
        else n.su = l.su == r.su ? l.su + 1 : std::max(l.su, r.su);
        n.depth = std::max(l.depth, r.depth) + 1;
        n.cost = op_cost(op) + (l.cost + r.cost);   // (the same bits in either operand order)
    }
}

int32_t Dag::intern(int op, int32_t k0, int32_t k1, uint32_t imm, int32_t k2) {
    if (table_.empty()) {
        size_t cap = 1024;
        while (cap < 2 * nodes.size() + 2) cap *= 2;
        rehash(cap);
    }
    size_t h = key_hash(op, k0, k1, imm, k2) & mask_;
    while (table_[h] >= 0) {
        const DagNode& n = nodes[table_[h]];
        if (n.op == op && n.kid[0] == k0 && n.kid[1] == k1 && n.kid[2] == k2 && n.imm == imm) return table_[h];
        h = (h + 1) & mask_;
    }
    DagNode n;
    n.op = op;
    n.kid[0] = k0;
    n.kid[1] = k1;
    n.kid[2] = k2;
    n.imm = imm;
    derive_fields(n, nodes.data());
    int32_t id = (int32_t)nodes.size();
    nodes.push_back(n);
    table_[h] = id;
    if (++used_ * 2 > table_.size()) rehash(table_.size() * 2);
    return id;
}

// ------------------------------------------------------------------ parse

static void fmt(std::string& err, const char* f, long long a, long long b = 0, long long c = 0) {
    char buf[256];
    snprintf(buf, sizeof buf, f, a, b, c);
    err = buf;
}

// ------------------------------------------------------------ simplification

namespace {

float as_float(uint32_t b) {
    float f;
    std::memcpy(&f, &b, 4);
    return f;
}
uint32_t as_bits(float f) {
    uint32_t b;
    std::memcpy(&b, &f, 4);
    return b;
}
// finite and normal or zero: host and device binary32 arithmetic agree on it
bool plain(float f) { return f == 0.f || std::isnormal(f); }

}  // namespace

// Rewrites applied while hash-consing, each exact for the device's binary32
// semantics (IEEE round-to-nearest, protected division, fminf/fmaxf), so a
// simplified population evaluates bitwise like the original.  NaNs the
// device makes are all one canonical NaN, which the identities below pass
// through unchanged.
//   - constant folding of add, sub, mul, div, min, max, neg, abs when the
//     operands and the result are zero or normal finite numbers and min/max
//     do not compare two zeros (sin and cos are never folded: the host cannot
//     reproduce the device's binary32 values);
//   - neg(neg(a)) = a, abs(neg(a)) = abs(a), abs(abs(a)) = abs(a);
//   - a * 1 = a, a / 1 = a, a / 0 = 0 (protected division), a + (-0) = a,
//     a - (+0) = a, (-0) - a = neg(a), min(a, a) = max(a, a) = a;
//   - negations absorbed by their consumer: a + neg(b) = a - b, neg(a) + b =
//     b - a, a - neg(b) = a + b (IEEE subtraction is addition of the negated
//     operand), neg(a) * neg(b) = a * b, neg(a) / neg(b) = a / b (zero
//     denominator: 0 either way), neg(a) * c = a * (-c), neg(a) / c = a / (-c),
//     c / neg(b) = (-c) / b for a constant c (the sign of a product or
//     quotient is the exclusive or of the operands' signs);
//   - operands of add, mul and mdist in a canonical order (commutative in
//     IEEE arithmetic, signed zeros included), so a+b and b+a are one node;
//   - folding of mdist, sqrt, sign, frac and mod (exact or correctly rounded
//     steps on the host as on the device; never tan, exp, log, pow);
//   - if(c, a, b) with a constant c is a or b; if(c, a, a) is a.
int32_t intern_simplified(Dag& dag, int op, int32_t k0, int32_t k1, uint32_t imm, int32_t k2) {
    const auto is_const = [&](int32_t k, float* v) {
        if (k < 0 || dag.nodes[k].op != T_CONST) return false;
        *v = as_float(dag.nodes[k].imm);
        return true;
    };
    float a = 0.f, b = 0.f;
    const bool ca = is_const(k0, &a), cb = is_const(k1, &b);
    const auto is_neg = [&](int32_t k) { return k >= 0 && dag.nodes[k].op == T_NEG; };
    const auto kid0 = [&](int32_t k) { return dag.nodes[k].kid[0]; };
    const auto negated = [&](float v) { return dag.intern(T_CONST, -1, -1, as_bits(v) ^ 0x80000000u); };
    const int ar = arity(op);
    // if with a constant condition is its chosen operand (NaN cannot be a constant)
    if (op == T_IF && ca) return a != 0.f ? k1 : k2;
    // constant folding
    if ((ar == 1 && ca) || (ar == 2 && ca && cb)) {
        bool ok = plain(a) && (ar == 1 || plain(b));
        float r = 0.f;
        switch (op) {
        case T_ADD: r = a + b; break;
        case T_SUB: r = a - b; break;
        case T_MUL: r = a * b; break;
        case T_DIV: r = b == 0.f ? 0.f : a / b; break;
        case T_MIN: ok = ok && !(a == 0.f && b == 0.f); r = std::fmin(a, b); break;
        case T_MAX: ok = ok && !(a == 0.f && b == 0.f); r = std::fmax(a, b); break;
        case T_NEG: r = -a; break;
        case T_ABS: r = std::fabs(a); break;
        case T_MDIST: r = (a + b) * 0.5f; break;
        case T_SQRT: r = a < 0.f ? 0.f : std::sqrt(a); break;
        case T_SIGN: r = a > 0.f ? 1.f : a < 0.f ? -1.f : 0.f; break;
        case T_FRAC: r = a - std::floor(a); break;
        case T_MOD: {
            ok = ok && b != 0.f;
            r = std::fmod(a, b);
            if (r != 0.f && ((r < 0.f) != (b < 0.f))) r = r + b;
            break;
        }
        default: ok = false; break;   // sin, cos, tan, exp, log, pow: library values on the device
        }
        if (ok && plain(r)) return dag.intern(T_CONST, -1, -1, as_bits(r));
    }
    switch (op) {
    case T_NEG:
        if (dag.nodes[k0].op == T_NEG) return dag.nodes[k0].kid[0];
        break;
    case T_ABS:
        if (dag.nodes[k0].op == T_NEG) return intern_simplified(dag, T_ABS, dag.nodes[k0].kid[0], -1, 0);
        if (dag.nodes[k0].op == T_ABS) return k0;
        break;
    case T_MUL:
        if (cb && as_bits(b) == as_bits(1.f)) return k0;
        if (ca && as_bits(a) == as_bits(1.f)) return k1;
        if (is_neg(k0) && is_neg(k1)) return intern_simplified(dag, T_MUL, kid0(k0), kid0(k1), 0);
        if (cb && is_neg(k0)) return intern_simplified(dag, T_MUL, kid0(k0), negated(b), 0);
        if (ca && is_neg(k1)) return intern_simplified(dag, T_MUL, negated(a), kid0(k1), 0);
        if (k1 < k0) std::swap(k0, k1);
        break;
    case T_DIV:
        if (cb && as_bits(b) == as_bits(1.f)) return k0;
        if (cb && b == 0.f) return dag.intern(T_CONST, -1, -1, as_bits(0.f));
        if (is_neg(k0) && is_neg(k1)) return intern_simplified(dag, T_DIV, kid0(k0), kid0(k1), 0);
        if (cb && is_neg(k0)) return intern_simplified(dag, T_DIV, kid0(k0), negated(b), 0);
        if (ca && is_neg(k1)) return intern_simplified(dag, T_DIV, negated(a), kid0(k1), 0);
        break;
    case T_ADD:
        if (cb && as_bits(b) == as_bits(-0.f)) return k0;
        if (ca && as_bits(a) == as_bits(-0.f)) return k1;
        if (is_neg(k1)) return intern_simplified(dag, T_SUB, k0, kid0(k1), 0);
        if (is_neg(k0)) return intern_simplified(dag, T_SUB, k1, kid0(k0), 0);
        if (k1 < k0) std::swap(k0, k1);
        break;
    case T_SUB:
        if (cb && as_bits(b) == as_bits(0.f)) return k0;
        if (ca && as_bits(a) == as_bits(-0.f)) return intern_simplified(dag, T_NEG, k1, -1, 0);
        if (is_neg(k1)) return intern_simplified(dag, T_ADD, k0, kid0(k1), 0);
        break;
    case T_MIN:
    case T_MAX:
        if (k0 == k1) return k0;
        break;
    case T_MDIST:
        if (k1 < k0) std::swap(k0, k1);
        break;
    case T_IF:
        if (k1 == k2) return k1;   // both operands the same node
        break;
    default:
        break;
    }
    return dag.intern(op, k0, k1, imm, k2);
}

// One token's node.  clip(x, y, z) is its printed definition,
// max(min(z, x), y) (Table 1), so it needs no instruction of its own.
int32_t make_node(Dag& dag, int op, const int32_t (&k)[kMaxKids], uint32_t bits, bool simplify) {
    auto mk = [&](int o, int32_t a, int32_t b, uint32_t imm, int32_t c) {
        return simplify ? intern_simplified(dag, o, a, b, imm, c) : dag.intern(o, a, b, imm, c);
    };
    if (op == T_CLIP) return mk(T_MAX, mk(T_MIN, k[2], k[0], 0, -1), k[1], 0, -1);
    return mk(op, k[0], k[1], bits, k[2]);
}

// Drops DAG nodes no tree reaches (operands that simplification bypassed),
// keeping ids in topological order.
// Nodes reachable from `roots` in `dag`: live[i] = 1.
static void mark_live(const Dag& dag, const int32_t* roots, size_t n_roots, std::vector<uint8_t>& live) {
    live.assign(dag.size(), 0);
    for (size_t t = 0; t < n_roots; ++t) live[roots[t]] = 1;
    for (size_t i = dag.size(); i-- > 0;)   // parents have larger ids than their operands
        if (live[i])
            for (int c = 0; c < kMaxKids; ++c)
                if (dag.nodes[i].kid[c] >= 0) live[dag.nodes[i].kid[c]] = 1;
}

// Keeps the nodes marked live, in their order (operands renumbered; the
// derived fields depend on the operands' only), with `par` in ranges.
static void compact_live(PopIR& pop, const std::vector<uint8_t>& live, const ParallelFor* par) {
    const size_t n = pop.dag.size();
    std::vector<int32_t> id(n, -1);
    int32_t n_live = 0;
    for (size_t i = 0; i < n; ++i)
        if (live[i]) id[i] = n_live++;
    if ((size_t)n_live == n) return;
    NodeVec kept((size_t)n_live);
    auto fill = [&](size_t lo, size_t hi) {
        for (size_t i = lo; i < hi; ++i) {
            if (!live[i]) continue;
            DagNode x = pop.dag.nodes[i];
            for (int c = 0; c < kMaxKids; ++c)
                if (x.kid[c] >= 0) x.kid[c] = id[x.kid[c]];
            kept[id[i]] = x;
        }
    };
    const int P = (par && *par && n >= (1u << 16)) ? 16 : 1;
    if (P > 1) (*par)(P, [&](int t) { fill(n * t / P, n * (t + 1) / P); });
    else fill(0, n);
    for (auto& r : pop.roots) r = id[r];
    pop.dag.assign_nodes(std::move(kept));
}

void compact(PopIR& pop) {
    std::vector<uint8_t> live;
    mark_live(pop.dag, pop.roots.data(), pop.roots.size(), live);
    compact_live(pop, live, nullptr);
}

void append_population(PopIR& dst, const PopIR& src) {
    std::vector<int32_t> id(src.dag.size());
    for (size_t n = 0; n < src.dag.size(); ++n) {   // children precede parents
        const DagNode& s = src.dag.nodes[n];
        id[n] = dst.dag.intern(s.op, s.kid[0] >= 0 ? id[s.kid[0]] : -1, s.kid[1] >= 0 ? id[s.kid[1]] : -1, s.imm,
                               s.kid[2] >= 0 ? id[s.kid[2]] : -1);
    }
    for (size_t t = 0; t < src.roots.size(); ++t) {
        dst.roots.push_back(id[src.roots[t]]);
        dst.tree_size.push_back(src.tree_size[t]);
        dst.tree_cost.push_back(src.tree_cost[t]);
    }
    dst.tree_nodes += src.tree_nodes;
}

// Decodes and hash-conses trees [t0, t1) into `dag` (their constants start
// at imm[imm0]); fills roots, tree_size, tree_cost and the token count of
// those trees (indexed from t0).  Returns 0, or -2 with a message.
static int parse_trees(const int32_t* ops, const float* imm, int64_t n_imm, const int64_t* tree_off, int32_t t0,
                       int32_t t1, int64_t imm0, int32_t order, bool simplify, Dag& dag, int32_t* roots,
                       int32_t* tree_size, float* tree_cost, int64_t* tokens, std::string& err) {
    std::vector<int32_t> stack;
    std::vector<int32_t> dstack;   // depth of each stacked subtree as given (before simplification)
    int64_t imm_pos = imm0;
    *tokens = 0;
    for (int32_t t = t0; t < t1; ++t) {
        int64_t b = tree_off[t], e = tree_off[t + 1];
        int64_t n = e - b;
        if (n <= 0) { fmt(err, "tree %lld is empty (tree_off not increasing)", t); return -2; }
        if (n > (1 << 24)) { fmt(err, "tree %lld has %lld tokens, limit 2^24", t, n); return -2; }
        // constants of this tree, for the prefix reverse scan
        int64_t nconst = 0;
        for (int64_t i = b; i < e; ++i) {
            int op = ops[i];
            if (arity(op) < 0) { fmt(err, "tree %lld token %lld: unknown opcode %lld", t, i - b, op); return -2; }
            nconst += op == T_CONST;
        }
        if (imm_pos + nconst > n_imm) {
            fmt(err, "tree %lld needs constants beyond n_imm = %lld", t, n_imm);
            return -2;
        }
        for (int64_t i = 0; i < nconst; ++i) {
            if (!std::isfinite(imm[imm_pos + i])) {
                fmt(err, "tree %lld: constant %lld is not finite", t, imm_pos + i);
                return -2;
            }
        }
        stack.clear();
        dstack.clear();
        if (order == 1) {   // postfix: operands precede their operator
            int64_t ip = imm_pos;
            for (int64_t i = b; i < e; ++i) {
                int op = ops[i], ar = arity(op);
                if ((int64_t)stack.size() < ar) {
                    fmt(err, "tree %lld token %lld: operator lacks operands", t, i - b);
                    return -2;
                }
                int32_t k[kMaxKids] = {-1, -1, -1}, d = 0;
                uint32_t bits = 0;
                for (int a = 0; a < ar; ++a) { d = std::max(d, dstack.back() + 1); dstack.pop_back(); }
                for (int a = ar - 1; a >= 0; --a) { k[a] = stack.back(); stack.pop_back(); }
                if (op == T_CONST) { float v = imm[ip++]; std::memcpy(&bits, &v, 4); }
                dstack.push_back(d);
                stack.push_back(make_node(dag, op, k, bits, simplify));
            }
        } else {            // prefix: scan backwards, first popped = first operand
            int64_t ip = imm_pos + nconst;
            for (int64_t i = e - 1; i >= b; --i) {
                int op = ops[i], ar = arity(op);
                if ((int64_t)stack.size() < ar) {
                    fmt(err, "tree %lld token %lld: operator lacks operands", t, i - b);
                    return -2;
                }
                int32_t k[kMaxKids] = {-1, -1, -1}, d = 0;
                uint32_t bits = 0;
                for (int a = 0; a < ar; ++a) { d = std::max(d, dstack.back() + 1); dstack.pop_back(); }
                for (int a = 0; a < ar; ++a) { k[a] = stack.back(); stack.pop_back(); }
                if (op == T_CONST) { float v = imm[--ip]; std::memcpy(&bits, &v, 4); }
                dstack.push_back(d);
                stack.push_back(make_node(dag, op, k, bits, simplify));
            }
        }
        if (stack.size() != 1) {
            fmt(err, "tree %lld leaves %lld values (must form exactly one expression)", t, (long long)stack.size());
            return -2;
        }
        int32_t root = stack[0];
        if (dstack[0] > 1024) {
            fmt(err, "tree %lld has depth %lld, limit 1024", t, dstack[0]);
            return -2;
        }
        imm_pos += nconst;
        roots[t - t0] = root;
        tree_size[t - t0] = (int32_t)n;
        tree_cost[t - t0] = dag.nodes[root].cost;
        *tokens += n;
    }
    return 0;
}

// Tokens from which a population is parsed in chunks of trees on the
// planning workers.
constexpr int64_t kParallelParseTokens = 1 << 16;

namespace {

// Insert-only hash set of node keys that the chunks of a parse add to
// concurrently.  A node gets a provisional id when it is first added (in
// whatever order the workers reach it); its key is written before the slot
// that publishes it (release / acquire).  A worker that loses the race for a
// slot leaves its reserved node unreferenced and compares with the winner's.
class MergeTable {
public:
    // max_nodes: the nodes the workers add, at most; workers: how many add
    MergeTable(size_t max_nodes, int workers, const ParallelFor* par)
        : nodes_(new DagNode[max_nodes + (size_t)workers * kBlock]) {   // (written when handed out)
        size_t cap = 1024;
        while (cap < 2 * max_nodes + 2) cap *= 2;
        mask_ = cap - 1;
        slot_.reset(new std::atomic<int32_t>[cap]);
        const int P = 16;
        (*par)(P, [&](int t) {
            for (size_t i = cap * t / P; i < cap * (t + 1) / P; ++i) slot_[i].store(-1, std::memory_order_relaxed);
        });
    }
    // A worker's block of ids to hand out (taken kBlock at a time, so the
    // workers do not contend for one counter).
    struct Ids {
        int32_t next = 0, end = 0;
    };
    static constexpr int32_t kBlock = 256;
    // `src`: the node as its chunk holds it (operands in the chunk's ids),
    // whose derived fields a new node takes.
    int32_t find_or_add(Ids& ids, const DagNode& src, int op, int32_t k0, int32_t k1, uint32_t imm, int32_t k2) {
        size_t h = key_hash(op, k0, k1, imm, k2) & mask_;
        int32_t mine = -1;
        for (;;) {
            int32_t s = slot_[h].load(std::memory_order_acquire);
            if (s < 0) {
                if (mine < 0) {
                    if (ids.next == ids.end) {
                        ids.next = count_.fetch_add(kBlock, std::memory_order_relaxed);
                        ids.end = ids.next + kBlock;
                    }
                    mine = ids.next++;
                    DagNode& n = nodes_[mine];
                    n = src;
                    n.op = op;
                    n.kid[0] = k0;
                    n.kid[1] = k1;
                    n.kid[2] = k2;
                    n.imm = imm;
                }
                int32_t expected = -1;
                if (slot_[h].compare_exchange_strong(expected, mine, std::memory_order_release,
                                                     std::memory_order_acquire))
                    return mine;
                s = expected;
            }
            const DagNode& n = nodes_[s];
            if (n.op == op && n.kid[0] == k0 && n.kid[1] == k1 && n.kid[2] == k2 && n.imm == imm) return s;
            h = (h + 1) & mask_;
        }
    }
    const DagNode& node(int32_t id) const { return nodes_[id]; }
    // ids handed out so far (some, at the ends of blocks, unused)
    int32_t size() const { return count_.load(std::memory_order_relaxed); }

private:
    std::unique_ptr<DagNode[]> nodes_;
    std::unique_ptr<std::atomic<int32_t>[]> slot_;
    size_t mask_ = 0;
    std::atomic<int32_t> count_{0};
};

void atomic_min_u64(std::atomic<uint64_t>& a, uint64_t v) {
    uint64_t cur = a.load(std::memory_order_relaxed);
    while (v < cur && !a.compare_exchange_weak(cur, v, std::memory_order_relaxed)) {}
}

}  // namespace

int parse_population(const int32_t* ops, const float* imm, int64_t n_imm, const int64_t* tree_off,
                     int32_t n_trees, int32_t order, PopIR& out, std::string& err, bool simplify,
                     const ParallelFor* par) {
    if (n_trees < 0 || n_trees > (1 << 24)) { fmt(err, "n_trees %lld out of range", n_trees); return -1; }
    if (order != 0 && order != 1) { fmt(err, "order %lld is neither prefix (0) nor postfix (1)", order); return -1; }
    if (n_imm < 0) { fmt(err, "n_imm %lld is negative", n_imm); return -1; }
    if (n_trees > 0 && (!ops || !tree_off)) { err = "ops / tree_off must not be NULL"; return -1; }
    if (n_imm > 0 && !imm) { err = "imm must not be NULL when n_imm > 0"; return -1; }
    out = PopIR();
    out.roots.resize(n_trees);
    out.tree_size.resize(n_trees);
    out.tree_cost.resize(n_trees);
    if (n_trees > 0 && tree_off[0] != 0) { fmt(err, "tree_off[0] = %lld, must be 0", tree_off[0]); return -2; }
    const int64_t total = n_trees > 0 ? tree_off[n_trees] : 0;
    int n_chunks = 1;
    if (par && *par && total >= kParallelParseTokens && n_trees >= 64) {
        // offsets must increase for the split (a bad offset is reported by the serial parse)
        bool ok = true;
        for (int32_t t = 0; t < n_trees && ok; ++t) ok = tree_off[t + 1] > tree_off[t];
        if (ok) n_chunks = (int)std::min<int64_t>(32, std::min<int64_t>(n_trees / 16, total / (kParallelParseTokens / 4)));
    }
    if (n_chunks <= 1) {
        if (total > 0 && total < (int64_t)1 << 26) out.dag.reserve((size_t)total);   // at most one node per token (two for clip)
        int64_t tokens = 0;
        int rc = parse_trees(ops, imm, n_imm, tree_off, 0, n_trees, 0, order, simplify, out.dag, out.roots.data(),
                             out.tree_size.data(), out.tree_cost.data(), &tokens, err);
        if (rc) return rc;
        out.tree_nodes = tokens;
    } else {
        // Chunks of consecutive trees are decoded and hash-consed into DAGs of
        // their own concurrently; their nodes are then interned into the
        // population DAG chunk by chunk in creation order, which creates the
        // population's nodes in the order, and with the ids, of a serial
        // parse (operands of commutative operators are put back in the
        // canonical order of the population's ids).
        std::vector<int32_t> t_at(n_chunks + 1);
        for (int c = 0; c <= n_chunks; ++c) {   // chunks of about equal token counts
            const int64_t want = total * c / n_chunks;
            t_at[c] = (int32_t)(std::upper_bound(tree_off, tree_off + n_trees + 1, want) - tree_off - 1);
        }
        t_at[0] = 0;
        t_at[n_chunks] = n_trees;
        for (int c = 1; c <= n_chunks; ++c) t_at[c] = std::max(t_at[c], t_at[c - 1]);
        // constants before each chunk
        std::vector<int64_t> imm_at(n_chunks + 1, 0);
        (*par)(n_chunks, [&](int c) {
            int64_t k = 0;
            for (int64_t i = tree_off[t_at[c]]; i < tree_off[t_at[c + 1]]; ++i) k += ops[i] == T_CONST;
            imm_at[c + 1] = k;
        });
        for (int c = 0; c < n_chunks; ++c) imm_at[c + 1] += imm_at[c];
        std::vector<Dag> dags(n_chunks);
        std::vector<int> rcs(n_chunks, 0);
        std::vector<std::string> errs(n_chunks);
        std::vector<int64_t> toks(n_chunks, 0);
        // with simplification, each chunk also marks the nodes its own trees
        // reach: the population's live nodes are their images (see below)
        std::vector<std::vector<uint8_t>> clive(n_chunks);
        (*par)(n_chunks, [&](int c) {
            const int64_t n = tree_off[t_at[c + 1]] - tree_off[t_at[c]];
            dags[c].reserve((size_t)std::max<int64_t>(n, 1));
            rcs[c] = parse_trees(ops, imm, n_imm, tree_off, t_at[c], t_at[c + 1], imm_at[c], order, simplify, dags[c],
                                 out.roots.data() + t_at[c], out.tree_size.data() + t_at[c],
                                 out.tree_cost.data() + t_at[c], &toks[c], errs[c]);
            if (!rcs[c] && simplify)
                mark_live(dags[c], out.roots.data() + t_at[c], (size_t)(t_at[c + 1] - t_at[c]), clive[c]);
        });
        for (int c = 0; c < n_chunks; ++c) {   // the first failing tree's message, as a serial parse gives
            if (rcs[c]) {
                err = errs[c];
                return rcs[c];
            }
        }
        for (int c = 0; c < n_chunks; ++c) out.tree_nodes += toks[c];
        if (n_trees > 0 && total != out.tree_nodes) { err = "internal: token count"; return -1; }
        if (imm_at[n_chunks] != n_imm) {
            fmt(err, "stream has %lld CONST tokens but n_imm = %lld", imm_at[n_chunks], n_imm);
            return -2;
        }
        // The chunks' nodes go into one population DAG.  Its nodes and ids
        // must be those of a serial parse: nodes in the order of their first
        // occurrence (chunk, then place in the chunk's DAG), with
        // simplification only those a tree reaches, the operands of
        // commutative operators in the order of those ids.  The chunks add
        // their nodes to a shared hash set concurrently (provisional ids),
        // then the first occurrence of every node fixes its id.
        size_t n_chunk_nodes = 0;
        for (const Dag& d : dags) n_chunk_nodes += d.size();
        MergeTable mt(n_chunk_nodes, n_chunks, par);
        std::vector<std::vector<int32_t>> pid(n_chunks);
        (*par)(n_chunks, [&](int c) {
            const Dag& d = dags[c];
            std::vector<int32_t>& id = pid[c];
            id.assign(d.size(), -1);
            MergeTable::Ids block;
            for (size_t i = 0; i < d.size(); ++i) {
                const DagNode& x = d.nodes[i];
                int32_t k[kMaxKids];
                for (int j = 0; j < kMaxKids; ++j) k[j] = x.kid[j] >= 0 ? id[x.kid[j]] : -1;
                // commutative operands in provisional-id order, so that both
                // orders of a pair meet (the final order is set below)
                if (simplify && (x.op == T_ADD || x.op == T_MUL || x.op == T_MDIST) && k[1] < k[0])
                    std::swap(k[0], k[1]);
                id[i] = mt.find_or_add(block, x, x.op, k[0], k[1], x.imm, k[2]);
            }
        });
        // first occurrence of each node, as chunk << 32 | place; with
        // simplification a node is kept when it is the image of a node its
        // chunk's trees reach (a serial parse's live nodes)
        const int32_t n_prov = mt.size();
        std::unique_ptr<std::atomic<uint64_t>[]> first(new std::atomic<uint64_t>[(size_t)std::max(n_prov, 1)]);
        std::vector<uint8_t> keep((size_t)std::max(n_prov, 1), simplify ? 0 : 1);
        (*par)(16, [&](int t) {
            for (int64_t g = (int64_t)n_prov * t / 16; g < (int64_t)n_prov * (t + 1) / 16; ++g)
                first[g].store(UINT64_MAX, std::memory_order_relaxed);
        });
        (*par)(n_chunks, [&](int c) {
            for (size_t i = 0; i < pid[c].size(); ++i) {
                atomic_min_u64(first[pid[c][i]], (uint64_t)c << 32 | (uint64_t)i);
                if (simplify && clive[c][i]) __atomic_store_n(&keep[pid[c][i]], (uint8_t)1, __ATOMIC_RELAXED);
            }
        });
        // final ids: kept nodes numbered in the order of their first occurrence
        std::vector<int64_t> base(n_chunks + 1, 0);
        (*par)(n_chunks, [&](int c) {
            int64_t k = 0;
            for (size_t i = 0; i < pid[c].size(); ++i) {
                const int32_t g = pid[c][i];
                k += keep[g] && first[g].load(std::memory_order_relaxed) == ((uint64_t)c << 32 | (uint64_t)i);
            }
            base[c + 1] = k;
        });
        for (int c = 0; c < n_chunks; ++c) base[c + 1] += base[c];
        std::vector<int32_t> fin((size_t)std::max(n_prov, 1), -1);
        (*par)(n_chunks, [&](int c) {
            int64_t k = base[c];
            for (size_t i = 0; i < pid[c].size(); ++i) {
                const int32_t g = pid[c][i];
                if (keep[g] && first[g].load(std::memory_order_relaxed) == ((uint64_t)c << 32 | (uint64_t)i))
                    fin[g] = (int32_t)k++;
            }
        });
        const size_t n_final = (size_t)base[n_chunks];
        NodeVec final_nodes(n_final);
        (*par)(16, [&](int t) {
            for (int64_t g = (int64_t)n_prov * t / 16; g < (int64_t)n_prov * (t + 1) / 16; ++g) {
                if (fin[g] < 0) continue;
                DagNode x = mt.node((int32_t)g);
                for (int j = 0; j < kMaxKids; ++j)
                    if (x.kid[j] >= 0) x.kid[j] = fin[x.kid[j]];
                // commutative operands in the order of the final ids (the
                // derived fields, taken from a chunk, do not depend on it)
                if (simplify && (x.op == T_ADD || x.op == T_MUL || x.op == T_MDIST) && x.kid[1] < x.kid[0])
                    std::swap(x.kid[0], x.kid[1]);
                final_nodes[fin[g]] = x;
            }
        });
        for (int c = 0; c < n_chunks; ++c)
            for (int32_t t = t_at[c]; t < t_at[c + 1]; ++t) out.roots[t] = fin[pid[c][out.roots[t]]];
        out.dag.assign_nodes(std::move(final_nodes));
        return 0;
    }
    if (n_trees > 0 && total != out.tree_nodes) { err = "internal: token count"; return -1; }
    int64_t nconst_all = 0;
    for (int64_t i = 0; i < total; ++i) nconst_all += ops[i] == T_CONST;
    if (nconst_all != n_imm) {
        fmt(err, "stream has %lld CONST tokens but n_imm = %lld", nconst_all, n_imm);
        return -2;
    }
    if (simplify) compact(out);
    return 0;
}

// ------------------------------------------------------------------ codegen

namespace {

// Per-node arrays of a planner, sized to the DAG and at their initial values
// between planners (a planner puts back every entry it changes).  One set per
// host thread, reused by the next planner on that thread: planning the groups
// and tables of a population then neither allocates nor clears them again.
struct GenScratch {
    std::vector<int32_t> uses, where, first_pos, last_pos;
    std::vector<uint8_t> keep, stored, mark;
    bool in_use = false;
    void fit(size_t n) {
        if (uses.size() >= n) return;
        uses.resize(n, 0);
        where.resize(n, -1);
        first_pos.resize(n, -1);
        last_pos.resize(n, -1);
        keep.resize(n, 0);
        stored.resize(n, 0);
        mark.resize(n, 0);
    }
};
thread_local GenScratch tls_scratch;

class GroupGen {
public:
    GroupGen(const Dag& dag, IrVec& out, bool dedup, int kept_cap, const CacheView* cv,
             const std::vector<int32_t>* col, const std::vector<int32_t>* row)
        : sc_(take_scratch(dag.size())), d_(dag), out_(out), uses_(sc_->uses), where_(sc_->where), keep_(sc_->keep),
          first_pos_(sc_->first_pos), last_pos_(sc_->last_pos), dedup_(dedup), kept_cap_(kept_cap),
          cv_(cv && cv->active() ? cv : nullptr), stored_(sc_->stored), mark_(sc_->mark), col_(col),
          row_(row) {}
    ~GroupGen() {
        for (int32_t n : stored_all_) stored_[n] = 0;
        if (sc_ == &tls_scratch) {
            // a very large DAG's arrays are not kept (19 bytes per node per thread)
            if (tls_scratch.uses.size() > ((size_t)1 << 22)) tls_scratch = GenScratch();
            tls_scratch.in_use = false;
        }
    }
    GroupGen(const GroupGen&) = delete;
    GroupGen& operator=(const GroupGen&) = delete;

    int slot_high = 0;                    // slots used by the last run
    void set_kept_cap(int c) { kept_cap_ = c; }
    std::vector<int32_t> refused;         // kept nodes that found no slot under the cap (last run)

    // Forgets the cache stores of the last attempt (the group is re-planned).
    void rollback() {
        for (int32_t n : stored_log_) stored_[n] = 0;
        stored_log_.clear();
    }

    // Emits one group.  Nodes listed in `forbid` are never kept.
    void run(const std::vector<int32_t>& trees, const std::vector<int32_t>& roots,
             const std::vector<int32_t>& forbid) {
        stored_log_.clear();
        slot_high = 0;
        refused.clear();
        count_uses(trees, roots, forbid);
        for (int32_t t : trees) {
            int32_t r = roots[t];
            to_acc(r);
            use(r);
            emit(F_ROOT, 0, 0, 0, t, 0);
        }
        emit(F_END, 0, 0, 0, 0, 0);
        for (int32_t n : touched_) { uses_[n] = 0; where_[n] = -1; keep_[n] = 0; }
        touched_.clear();
        busy_.clear();
    }

private:
    // The thread's scratch, or a fresh set when the thread's is held (a
    // planner inside a planner on one thread).
    std::unique_ptr<GenScratch> own_;
    GenScratch* take_scratch(size_t n) {
        GenScratch* g = &tls_scratch;
        if (g->in_use) {
            own_ = std::make_unique<GenScratch>();
            g = own_.get();
        }
        g->in_use = true;
        g->fit(n);
        return g;
    }
    GenScratch* sc_;

    // A shared node is kept (evaluated once, held in a slot until its last
    // use) when its subtree costs at least this much per point and its uses
    // lie in at most kKeepSpan + 1 consecutive trees of the group; otherwise
    // it is re-evaluated at each use.  Holding values across many trees would
    // fill the slots (shared memory, which bounds how many CTAs fit an SM).
    static constexpr float kKeepMinCost = 2.f;
    static constexpr int kKeepSpan = 1;

    const Dag& d_;
    IrVec& out_;
    std::vector<int32_t>& uses_;    // evaluations of the node still to be consumed
    std::vector<int32_t>& where_;   // slot holding the node, or -1
    std::vector<uint8_t>& keep_;    // evaluated once and held
    std::vector<int32_t>& first_pos_;   // tree positions of first / last use
    std::vector<int32_t>& last_pos_;
    std::vector<int32_t> span_touched_;
    std::vector<int32_t> touched_;
    bool dedup_;
    int kept_cap_;                 // slots a kept node may use; temporaries may go beyond
    const CacheView* cv_;          // cross-call cache, or nullptr
    std::vector<uint8_t>& stored_;  // cache store already emitted (this plan)
    std::vector<int32_t> stored_log_;   // stores of the current group attempt
    std::vector<int32_t> stored_all_;   // every store emitted (put back to 0 at the end)
    std::vector<bool> busy_;
    std::vector<int32_t> dfs_;
    std::vector<uint8_t>& mark_;    // scratch of sort_touched_descending, all zero between calls
    const std::vector<int32_t>* col_;     // column-table entry of a node, -1 (or nullptr: none)
    const std::vector<int32_t>* row_;     // row-table entry of a node, -1 (or nullptr: none)

    const DagNode& N(int32_t n) const { return d_.nodes[n]; }
    bool is_cached(int32_t n) const { return cv_ && cv_->cached[n] >= 0; }
    bool is_col(int32_t n) const { return col_ && (*col_)[n] >= 0; }
    bool is_row(int32_t n) const { return row_ && (*row_)[n] >= 0; }
    // loaded (cache, column or row table): its operands are not evaluated
    bool is_loaded(int32_t n) const { return is_cached(n) || is_col(n) || is_row(n); }

    void emit(int form, int fn, int o1, int o2, int aux, uint32_t imm) {
        IrIns in;
        in.form = form; in.fn = fn; in.o1 = o1; in.o2 = o2; in.aux = aux; in.imm = imm; in.uni = 0;
        out_.push_back(in);
    }

    // Static keep/expand decision and use counts.  A node that is kept is
    // evaluated once, so each operand edge below it is consumed once; a node
    // that is expanded is evaluated at every one of its uses, so its operand
    // edges are consumed that many times.  Node ids are a topological order
    // (operands are interned before their parent), so a pass over the
    // group's nodes in descending id order sees every parent first.
    void count_uses(const std::vector<int32_t>& trees, const std::vector<int32_t>& roots,
                    const std::vector<int32_t>& forbid) {
        // tree positions (within the group) of the first and last use of each node
        for (size_t i = 0; i < trees.size(); ++i) {
            int32_t r = roots[trees[i]];
            if (is_leaf(N(r).op)) continue;
            dfs_.assign(1, r);
            while (!dfs_.empty()) {
                int32_t n = dfs_.back();
                dfs_.pop_back();
                if (last_pos_[n] == (int32_t)i) continue;    // already seen in this tree
                if (last_pos_[n] < 0) { first_pos_[n] = (int32_t)i; span_touched_.push_back(n); }
                last_pos_[n] = (int32_t)i;
                if (is_loaded(n)) continue;
                for (int c = 0; c < kMaxKids; ++c) {
                    int32_t k = N(n).kid[c];
                    if (k >= 0 && !is_leaf(N(k).op)) dfs_.push_back(k);
                }
            }
        }
        // the group's internal nodes (those the walk above reached, each
        // once) and the uses of the roots
        touched_.assign(span_touched_.begin(), span_touched_.end());
        for (int32_t t : trees) {
            int32_t r = roots[t];
            if (!is_leaf(N(r).op)) uses_[r]++;
        }
        sort_touched_descending();
        for (int32_t n : forbid) where_[n] = -3;   // mark: never keep (reset below)
        // uses_ holds the root counts so far; push evaluations down
        for (int32_t n : touched_) {
            int32_t e = uses_[n];
            keep_[n] = dedup_ && e >= 2 && N(n).cost >= kKeepMinCost && where_[n] != -3 &&
                       last_pos_[n] - first_pos_[n] <= kKeepSpan;
            if (is_loaded(n)) continue;   // loaded, operands not evaluated
            int32_t f = keep_[n] ? 1 : e;
            for (int c = 0; c < kMaxKids; ++c) {
                int32_t k = N(n).kid[c];
                if (k >= 0 && !is_leaf(N(k).op)) uses_[k] += f;
            }
        }
        for (int32_t n : forbid) where_[n] = -1;
        for (int32_t n : span_touched_) { first_pos_[n] = -1; last_pos_[n] = -1; }
        span_touched_.clear();
    }

    // touched_ in descending id order without repeats (parents before their
    // operands): a scan of the id range when it is short, else a sort
    void sort_touched_descending() {
        if (touched_.empty()) return;
        int32_t lo = touched_[0], hi = touched_[0];
        for (int32_t n : touched_) { lo = std::min(lo, n); hi = std::max(hi, n); }
        if ((int64_t)(hi - lo) <= 16 * (int64_t)touched_.size() + 64) {
            for (int32_t n : touched_) mark_[n] = 1;
            touched_.clear();
            for (int32_t n = hi; n >= lo; --n)
                if (mark_[n]) { mark_[n] = 0; touched_.push_back(n); }
        } else {
            std::sort(touched_.begin(), touched_.end(), [](int32_t a, int32_t b) { return a > b; });
            touched_.erase(std::unique(touched_.begin(), touched_.end()), touched_.end());
        }
    }

    // operand kind of a leaf (and its immediate)
    int leaf_opnd(int32_t n, uint32_t* imm) const {
        const DagNode& x = N(n);
        if (x.op == T_X) return kOpX;
        if (x.op == T_Y) return kOpY;
        *imm = x.imm;
        return kOpC;
    }

    // operand available without any code: a leaf or a node held in a slot
    // (slot returned through *slot), else -1
    int free_opnd(int32_t n, uint32_t* imm, int* slot) const {
        if (is_leaf(N(n).op)) return leaf_opnd(n, imm);
        if (where_[n] >= 0) { *slot = where_[n]; return kOpS; }
        return -1;
    }

    // A free slot; a kept node may not go beyond the cap (-1 then).
    int alloc_slot(bool kept) {
        const int limit = kept ? kept_cap_ : (int)busy_.size() + 1;
        for (int j = 0; j < limit; ++j) {
            if (j == (int)busy_.size()) busy_.push_back(false);
            if (!busy_[j]) {
                busy_[j] = true;
                slot_high = std::max(slot_high, j + 1);
                return j;
            }
        }
        return -1;
    }
    void free_slot(int j) {
        if (j >= 0) busy_[j] = false;
    }

    // consumes one use of n; frees its slot after the last one
    void use(int32_t n) {
        if (is_leaf(N(n).op)) return;
        if (--uses_[n] == 0 && where_[n] >= 0) {
            free_slot(where_[n]);
            where_[n] = -1;
        }
    }

    // Leaves the value of n in A (no use is consumed here).
    void to_acc(int32_t n) {
        uint32_t imm = 0;
        if (is_leaf(N(n).op)) {
            int o = leaf_opnd(n, &imm);
            emit(F_LD, 0, o, 0, 0, imm);
            return;
        }
        if (where_[n] >= 0) {
            emit(F_LD, 0, kOpS, 0, where_[n], 0);
            return;
        }
        if (is_cached(n)) {
            emit(F_CLD, 0, 0, 0, cv_->cached[n], 0);
        } else if (is_col(n)) {
            emit(F_COL, 0, 0, 0, (*col_)[n], 0);
        } else if (is_row(n)) {
            emit(F_ROW, 0, 0, 0, (*row_)[n], 0);
        } else {
            compute(n);
            // no x below n: the same value at all K points of a thread (they
            // share a row); the instruction that computed n says so
            if (!(N(n).vars & 1)) out_.back().uni = 1;
            if (cv_ && cv_->insert[n] >= 0 && !stored_[n]) {
                emit(F_CST, 0, 0, 0, cv_->insert[n], 0);
                stored_[n] = 1;
                stored_log_.push_back(n);
                stored_all_.push_back(n);
            }
        }
        // a kept node is held for the uses that remain after the current one
        if (keep_[n] && uses_[n] > 1) {
            int j = alloc_slot(true);
            if (j >= 0) {
                emit(F_ST, 0, 0, 0, j, 0);
                where_[n] = j;
            } else {
                // no slot under the cap: the plan is redone with n demoted;
                // until then it is parked in a temporary slot so this run
                // stays consistent
                refused.push_back(n);
                j = alloc_slot(false);
                emit(F_ST, 0, 0, 0, j, 0);
                where_[n] = j;
            }
        }
    }

    // Exactly commutative in binary32 for this operator set: a + b == b + a
    // and a * b == b * a bitwise; fminf / fmaxf return the same value in
    // either order (a NaN operand yields the other operand; equal zeros
    // compare equal).
    static bool commutative(int fn) {
        return fn == T_ADD || fn == T_MUL || fn == T_MIN || fn == T_MAX || fn == T_MDIST;
    }

    // A = fn(o, A)
    void emit_rev(int fn, int o, int slot, uint32_t imm) {
        if (commutative(fn)) emit(F_AO, fn, o, 0, slot, imm);
        else emit(F_OA, fn, o, 0, slot, imm);
    }

    // Leaves n's value in a slot: the slot it is held in, or a temporary one
    // (*temp = true) after computing it.
    int hold(int32_t n, bool* temp) {
        *temp = false;
        if (!is_leaf(N(n).op) && where_[n] >= 0) return where_[n];
        to_acc(n);
        if (!is_leaf(N(n).op) && where_[n] >= 0) return where_[n];   // kept by to_acc
        int j = alloc_slot(false);
        emit(F_ST, 0, 0, 0, j, 0);
        *temp = true;
        return j;
    }

    // Computes internal node n (not held anywhere) into A.
    void compute(int32_t n) {
        const DagNode& x = N(n);
        int fn = x.op;
        uint32_t imm = 0;
        if (arity(fn) == 3) {   // if(c, a, b): c and a in slots, b in A, then one select
            bool tc = false, ta = false;
            int sc = hold(x.kid[0], &tc);
            int sa = hold(x.kid[1], &ta);
            to_acc(x.kid[2]);
            emit(F_SEL, fn, kOpS, kOpS, sc, (uint32_t)sa);
            if (tc) free_slot(sc);
            if (ta) free_slot(sa);
            use(x.kid[0]);
            use(x.kid[1]);
            use(x.kid[2]);
            return;
        }
        if (arity(fn) == 1) {
            int32_t c = x.kid[0];
            if (is_leaf(N(c).op)) {
                int o = leaf_opnd(c, &imm);
                emit(F_UT, fn, o, 0, 0, imm);
            } else {
                to_acc(c);
                use(c);
                emit(F_UA, fn, 0, 0, 0, 0);
            }
            return;
        }
        int32_t l = x.kid[0], r = x.kid[1];
        uint32_t il = 0, ir = 0;
        int sl = -1, sr = -1;
        int ol = free_opnd(l, &il, &sl), orr = free_opnd(r, &ir, &sr);
        if (ol >= 0 && orr >= 0) {
            bool ll = is_leaf(N(l).op), rl = is_leaf(N(r).op);
            if (ll && rl && !(ol == kOpC && orr == kOpC)) {
                emit(F_TT, fn, ol, orr, 0, ol == kOpC ? il : ir);
            } else {
                emit(F_LD, 0, ol, 0, sl, il);
                emit(F_AO, fn, orr, 0, sr, ir);
            }
            use(l);
            use(r);
            return;
        }
        if (ol >= 0) {            // right needs code
            to_acc(r);
            emit_rev(fn, ol, sl, il);
            use(r);
            use(l);
            return;
        }
        if (orr >= 0) {           // left needs code
            to_acc(l);
            emit(F_AO, fn, orr, 0, sr, ir);
            use(l);
            use(r);
            return;
        }
        // both operands need code: the one needing more slots goes first
        bool left_first = N(l).su >= N(r).su;
        int32_t first = left_first ? l : r, second = left_first ? r : l;
        to_acc(first);
        uint32_t is = 0;
        int ss = -1;
        int os = free_opnd(second, &is, &ss);
        if (os >= 0) {            // became available while computing `first`
            if (left_first) emit(F_AO, fn, os, 0, ss, is);
            else emit_rev(fn, os, ss, is);
            use(first);
            use(second);
            return;
        }
        // park `first` in a slot while `second` is computed
        int temp = -1;
        int w = where_[first];
        if (w < 0) {
            temp = alloc_slot(false);
            emit(F_ST, 0, 0, 0, temp, 0);
            w = temp;
        }
        to_acc(second);
        if (left_first) emit_rev(fn, kOpS, w, 0);      // A = fn(first, A)
        else emit(F_AO, fn, kOpS, 0, w, 0);            // A = fn(A, first)
        if (temp >= 0) free_slot(temp);
        use(first);
        use(second);
    }
};

}  // namespace

Ins encode(const IrIns& in) {
    uint32_t opc = 0, y = 0;
    // the y word: slot of an S operand, else the immediate of a C operand, else aux
    auto opnd_word = [&](int o) { return o == kOpS ? (uint32_t)in.aux : in.imm; };
    switch (in.form) {
    case F_END: opc = OPC_END; break;
    case F_AO: opc = OPC_AO + bin_index(in.fn) * kNOpnd + in.o1; y = opnd_word(in.o1); break;
    case F_OA: opc = OPC_OA + ord_index(in.fn) * kNOpnd + in.o1; y = opnd_word(in.o1); break;
    case F_TT: opc = OPC_TT + bin_index(in.fn) * 9 + in.o1 * 3 + in.o2; y = in.imm; break;
    case F_UA: opc = OPC_UA + un_index(in.fn); break;
    case F_UT: opc = OPC_UT + un_index(in.fn) * 3 + in.o1; y = in.imm; break;
    case F_LD: opc = OPC_LD + in.o1; y = opnd_word(in.o1); break;
    case F_ST: opc = OPC_ST; y = (uint32_t)in.aux; break;
    case F_ROOT: opc = OPC_ROOT; y = (uint32_t)in.aux; break;
    case F_CST: opc = OPC_CST; y = (uint32_t)in.aux; break;
    case F_CLD: opc = OPC_CLD; y = (uint32_t)in.aux; break;
    case F_SEL: opc = OPC_SEL; y = (uint32_t)in.aux | (in.imm << 16); break;
    case F_COL: opc = OPC_COL; y = (uint32_t)in.aux; break;
    case F_ROW: opc = OPC_ROW; y = (uint32_t)in.aux; break;
    default: opc = OPC_END; break;
    }
    Ins e;
    e.x = opc | (in.uni ? kUniformBit : 0u);
    e.y = y;
    return e;
}

int64_t queue_local_items(int64_t n_items, int n_queues) {
    const int64_t Q = std::max(1, n_queues);
    if (n_items < 8 * Q) return 0;
    return n_items * 3 / 4 / Q * Q;
}

PlanShape default_shape(const PopIR& pop, int64_t N, int sms) {
    PlanShape s;
    s.N = N;
    s.threads = 128;
    // (measured on GB300: K = 8 is the fastest from 256 x 256 points up)
    s.K = N >= (1 << 16) ? 8 : N >= (1 << 14) ? 4 : N >= (1 << 12) ? 2 : 1;
    // Enough (group, tile) work items for ~64 per SM: the atomic queue then
    // balances uneven groups, and smaller groups cost nothing extra.
    int64_t tile = (int64_t)s.K * s.threads;
    int64_t n_tiles = (N + tile - 1) / tile;
    int64_t want = (int64_t)std::max(sms, 1) * 64;
    int64_t T = (int64_t)pop.roots.size();
    int64_t g = (want + n_tiles - 1) / n_tiles;
    // four times as many items where the groups still hold six trees or
    // more (measured on GB300: faster there, slower with fewer trees a group)
    const int64_t g4 = (4 * want + n_tiles - 1) / n_tiles;
    if (T >= 6 * g4) g = g4;
    s.n_groups = (int)std::max<int64_t>(1, std::min(g, std::max<int64_t>(T, 1)));
    return s;
}

std::vector<int32_t> evaluated_nodes(const PopIR& pop, const CacheView& cv) {
    std::vector<uint8_t> seen(pop.dag.size(), 0);
    std::vector<int32_t> out, stack;
    for (int32_t r : pop.roots) {
        stack.assign(1, r);
        while (!stack.empty()) {
            int32_t n = stack.back();
            stack.pop_back();
            const DagNode& d = pop.dag.nodes[n];
            if (seen[n] || is_leaf(d.op)) continue;
            seen[n] = 1;
            if (cv.active() && cv.cached[n] >= 0) continue;
            out.push_back(n);
            for (int c = 0; c < kMaxKids; ++c)
                if (d.kid[c] >= 0) stack.push_back(d.kid[c]);
        }
    }
    return out;
}

namespace {
// What planning reads of a population: its DAG, the roots of its trees and
// their costs (a population, or the subtrees that become column tables).
struct PlanPop {
    const Dag& dag;
    const std::vector<int32_t>& roots;
    const std::vector<float>& tree_cost;
    int64_t tree_nodes;
};
}  // namespace

// One group's bytecode (appended to gen's output), with the kept-slot cap
// that the group's temporaries leave of `budget`.  Returns the slots used.
static int plan_group(GroupGen& gen, IrVec& ir, const PlanPop& pop, const std::vector<int32_t>& trees,
                      int budget) {
    // kept nodes get what the group's temporaries leave of the budget (a
    // tree's evaluation parks up to its Sethi-Ullman number of values)
    int su = 0;
    for (int32_t t : trees) su = std::max(su, pop.dag.nodes[pop.roots[t]].su);
    gen.set_kept_cap(std::max(2, budget - su));
    // A kept node that found no slot under the cap is demoted to
    // re-evaluation and the group is planned again.  Demotion only
    // shrinks the kept set, so this terminates.
    std::vector<int32_t> forbid;
    const size_t mark = ir.size();
    for (int iter = 0;; ++iter) {
        gen.run(trees, pop.roots, forbid);
        if (gen.refused.empty() || iter >= 32) break;
        forbid.insert(forbid.end(), gen.refused.begin(), gen.refused.end());
        gen.rollback();
        ir.resize(mark);
    }
    return gen.slot_high;
}

// Subtrees with cost >= this (a binary32 add = 1) and x but no y below them
// become column tables: a table load costs about one add per point.
constexpr float kColMinCost = 4.f;
constexpr size_t kColMaxEntries = 16384;

static void build_plan_impl(const PlanPop& pop, const PlanShape& shape, HostPlan& plan, const CacheView* cv,
                            const ParallelFor* par, bool columns, bool table_plan);

// Encodes groups [0, n) of `ir` (group g at [off[g], off[g + 1])) onto
// `code`, appending each group's end offset (code.size() after it) to
// `code_off`.  A store followed by the start of a new subexpression, or by a
// table load, is one word.  A table load's word holds the offset of its entry
// (entry * the table's stride).  Roots are numbered in batches of
// kRootBatch, each batch closed by a flush word and its trees (see
// OPC_FLUSH).  Returns whether the interpreter variant with the rest of
// Table 1 is needed.
static bool encode_groups(const IrVec& ir, const int64_t* off, int n, int64_t col_stride, int64_t row_stride,
                          CodeVec& code, std::vector<int64_t>& code_off) {
    bool ext = false;
    auto enc = [&](const IrIns& in) {
        Ins e = encode(in);
        if (in.form == F_COL) e.y = (uint32_t)((int64_t)in.aux * col_stride);
        if (in.form == F_ROW) e.y = (uint32_t)((int64_t)in.aux * row_stride);
        return e;
    };
    int pending = 0;
    uint32_t batch[kRootBatch];
    auto flush = [&]() {
        if (!pending) return;
        code.push_back(Ins{(uint32_t)OPC_FLUSH, (uint32_t)pending});
        for (int i = 0; i < pending; i += 2) code.push_back(Ins{batch[i], i + 1 < pending ? batch[i + 1] : 0u});
        pending = 0;
    };
    for (int g = 0; g < n; ++g) {
        for (int64_t i = off[g]; i < off[g + 1]; ++i) {
            const IrIns& in = ir[i];
            if (in.form == F_ROOT) {
                Ins e = enc(in);
                e.x |= (uint32_t)pending << kStoreSlotShift;
                code.push_back(e);
                batch[pending++] = (uint32_t)in.aux;
                if (pending == kRootBatch) flush();
                continue;
            }
            if (in.form == F_END) flush();
            const bool form_fn = in.form == F_AO || in.form == F_OA || in.form == F_TT || in.form == F_UA ||
                                 in.form == F_UT;
            if (in.form == F_SEL || (form_fn && in.fn >= T_TAN)) ext = true;
            if (in.form == F_ST && i + 1 < off[g + 1] && in.aux >= 0 && in.aux < (1 << 15)) {
                const IrIns& nx = ir[i + 1];
                int fused = -1;
                if (nx.form == F_TT && bin_index(nx.fn) >= 0 && bin_index(nx.fn) < kNHotBin)
                    fused = OPC_STT + bin_index(nx.fn) * 9 + nx.o1 * 3 + nx.o2;
                else if (nx.form == F_UT && un_index(nx.fn) >= 0 && un_index(nx.fn) < kNHotUn)
                    fused = OPC_SUT + un_index(nx.fn) * 3 + nx.o1;
                else if (nx.form == F_COL)
                    fused = OPC_STC;
                else if (nx.form == F_ROW)
                    fused = OPC_STR;
                if (fused >= 0) {
                    Ins e = enc(nx);
                    e.x = (uint32_t)fused | (e.x & kUniformBit) | ((uint32_t)in.aux << kStoreSlotShift);
                    code.push_back(e);
                    ++i;
                    continue;
                }
            }
            code.push_back(enc(in));
        }
        flush();   // (a group always ends in END; kept for a group that would not)
        code_off.push_back((int64_t)code.size());
    }
    return ext;
}

void build_plan(const PopIR& pop, const PlanShape& shape, HostPlan& plan, const CacheView* cv,
                const ParallelFor* par, bool columns) {
    build_plan_impl(PlanPop{pop.dag, pop.roots, pop.tree_cost, pop.tree_nodes}, shape, plan, cv, par, columns,
                    false);
}

// table_plan: the plan of column or row tables (their subtrees in id order:
// the ordering pass would cost more than it saves on these small launches).
static void build_plan_impl(const PlanPop& pop, const PlanShape& shape, HostPlan& plan, const CacheView* cv,
                            const ParallelFor* par, bool columns, bool table_plan) {
    plan = HostPlan();
    plan.shape = shape;
    const int64_t T = (int64_t)pop.roots.size();
    const int G = (int)std::max<int64_t>(1, std::min<int64_t>(shape.n_groups, std::max<int64_t>(T, 1)));
    plan.shape.n_groups = G;
    plan.n_tiles = (int)((plan_chunks(shape) + shape.threads - 1) / shape.threads);

    // Tree order: trees that share a subtree are placed next to each other
    // (sorted by their most expensive subtree that another tree also uses),
    // then the order is cut into G contiguous groups of balanced cost.
    // distinct internal nodes of each tree (flat, tree t at [tree_at[t], tree_at[t+1]))
    std::vector<int32_t> order(T);
    std::iota(order.begin(), order.end(), 0);
    if (!table_plan) {
        // distinct internal nodes of each tree (contiguous chunks of trees
        // on the workers), then whether two trees or more use each node: a
        // node seen by two trees of one chunk, or by two chunks
        const bool many = par && *par && T >= 512;
        const int C = many ? (int)std::min<int64_t>(16, T / 256) : 1;
        const size_t nn = pop.dag.size();
        std::vector<std::vector<int32_t>> nodes_of(C), at_of(C), seen_of(C), dup_of(C);
        auto walk = [&](int c) {
            const int64_t t0 = T * c / C, t1 = T * (c + 1) / C;
            std::vector<int32_t>& seen = seen_of[c];   // last tree of the chunk using the node
            seen.assign(nn, -1);
            std::vector<int32_t> stack;
            std::vector<int32_t>& tree_nodes = nodes_of[c];
            std::vector<int32_t>& tree_at = at_of[c];
            for (int64_t t = t0; t < t1; ++t) {
                tree_at.push_back((int32_t)tree_nodes.size());
                stack.assign(1, pop.roots[t]);
                while (!stack.empty()) {
                    int32_t n = stack.back();
                    stack.pop_back();
                    if (seen[n] == (int32_t)t || is_leaf(pop.dag.nodes[n].op)) continue;
                    if (seen[n] >= 0) dup_of[c].push_back(n);
                    seen[n] = (int32_t)t;
                    tree_nodes.push_back(n);
                    for (int k = 0; k < kMaxKids; ++k)
                        if (pop.dag.nodes[n].kid[k] >= 0) stack.push_back(pop.dag.nodes[n].kid[k]);
                }
            }
            tree_at.push_back((int32_t)tree_nodes.size());
        };
        std::vector<uint8_t> multi(nn, 0);
        const auto merge = [&](size_t n0, size_t n1) {
            for (size_t n = n0; n < n1; ++n) {
                int k = 0;
                for (int c = 0; c < C && k < 2; ++c) k += seen_of[c][n] >= 0;
                if (k >= 2) multi[n] = 1;
            }
        };
        // the costliest node of each tree that another tree also uses
        std::vector<int32_t> key(T, -1);
        auto keys = [&](int c) {
            const int64_t t0 = T * c / C, t1 = T * (c + 1) / C;
            for (int64_t t = t0; t < t1; ++t) {
                float key_cost = 0.f;
                for (int32_t i = at_of[c][t - t0]; i < at_of[c][t - t0 + 1]; ++i) {
                    const int32_t n = nodes_of[c][i];
                    const float cost = pop.dag.nodes[n].cost;
                    if (multi[n] && cost > key_cost) { key_cost = cost; key[t] = n; }
                }
            }
        };
        if (C > 1) {
            (*par)(C, walk);
            const int R = 16;
            (*par)(R, [&](int r) { merge(nn * r / R, nn * (r + 1) / R); });
            (*par)(C, [&](int c) {
                for (int32_t n : dup_of[c]) __atomic_store_n(&multi[n], (uint8_t)1, __ATOMIC_RELAXED);
            });
            (*par)(C, keys);
        } else {
            walk(0);
            for (int32_t n : dup_of[0]) multi[n] = 1;
            keys(0);
        }
        std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
            if (key[a] != key[b]) return key[a] > key[b];
            return a < b;
        });
    }
    double total = 0;
    for (int64_t t = 0; t < T; ++t) total += pop.tree_cost[t] + 1.0;
    std::vector<std::vector<int32_t>> groups(G);
    plan.group_cost.assign(G, 0.0);
    {
        double acc = 0;
        int g = 0;
        for (int32_t t : order) {
            double c = pop.tree_cost[t] + 1.0;
            // move on when this group reached its share (keep at least one tree per group)
            if (g < G - 1 && !groups[g].empty() && acc + 0.5 * c > total * (g + 1) / G) ++g;
            groups[g].push_back(t);
            plan.group_cost[g] += c;
            acc += c;
        }
    }

    const int64_t W = shape.W > 0 ? shape.W : shape.N;
    const int64_t H = W > 0 ? shape.N / W : 0;
    const bool tables = columns && W > 1 && H > 1 && !table_plan;   // (a table's plan has none)
    // Column and row tables (grids of at least two rows and two columns): the
    // largest costly subtrees with x and no y below them (one value per
    // column) and with no x below them (one value per row), i.e. those used
    // by a node evaluated in this plan, or tree roots.  The tables' own plans
    // are phenotype launches on one row of W points and on one column of H
    // points.
    std::vector<int32_t> col, row;
    std::vector<std::function<void()>> table_builds;   // run beside the groups' planning
    if (tables) {
        const size_t nn = pop.dag.size();
        const bool cview = cv && cv->active();
        // a cache load or store at or below a node (such a subtree is
        // evaluated in this plan): one pass in id order, operands first
        std::vector<uint8_t> blocked;
        if (cview) {
            blocked.assign(nn, 0);
            for (size_t n = 0; n < nn; ++n) {
                const DagNode& d = pop.dag.nodes[n];
                bool b = cv->cached[n] >= 0 || cv->insert[n] >= 0;
                for (int c = 0; c < kMaxKids; ++c)
                    if (d.kid[c] >= 0) b = b || blocked[d.kid[c]];
                blocked[n] = b;
            }
        }
        // 1: may be a column table's subtree (x and no y below it), 2: a row
        // table's (no x below it), 0: neither
        const auto elig = [&](size_t n) -> int {
            const DagNode& d = pop.dag.nodes[n];
            if (is_leaf(d.op) || d.cost < kColMinCost || (cview && blocked[n])) return 0;
            return d.vars == 1 ? 1 : (d.vars & 1) ? 0 : 2;
        };
        std::vector<uint8_t> cneed(nn, 0), rneed(nn, 0);
        for (int32_t r : pop.roots) {
            const int e = elig(r);
            cneed[r] = e == 1;
            rneed[r] = e == 2;
        }
        // the eligible operands of nodes that are not inside a table's
        // subtree (nor one); the marks are idempotent stores, so node ranges
        // run on the workers
        const auto mark = [&](size_t n0, size_t n1) {
            for (size_t n = n0; n < n1; ++n) {
                if (elig(n)) continue;
                const DagNode& d = pop.dag.nodes[n];
                for (int c = 0; c < kMaxKids; ++c) {
                    if (d.kid[c] < 0) continue;
                    const int e = elig(d.kid[c]);
                    if (e) __atomic_store_n(&(e == 1 ? cneed : rneed)[d.kid[c]], (uint8_t)1, __ATOMIC_RELAXED);
                }
            }
        };
        if (par && *par && nn >= (1u << 16)) {
            const int C = 16;
            (*par)(C, [&](int c) { mark(nn * c / C, nn * (c + 1) / C); });
        } else {
            mark(0, nn);
        }
        auto make_tables = [&](const std::vector<uint8_t>& need, std::vector<int32_t>& view,
                               std::vector<int32_t>& roots, std::shared_ptr<HostPlan>& tplan, int64_t& stride,
                               int64_t n_points, int64_t row_len) {
            for (size_t n = 0; n < nn; ++n)
                if (need[n]) roots.push_back((int32_t)n);
            const int64_t st = (n_points + 15) / 16 * 16;
            // (an entry's offset, entry * stride, is a 32-bit bytecode word)
            if (roots.empty() || roots.size() > kColMaxEntries || (int64_t)roots.size() * st > (int64_t)UINT32_MAX) {
                roots.clear();
                return;
            }
            view.assign(nn, -1);
            for (size_t e = 0; e < roots.size(); ++e) view[roots[e]] = (int32_t)e;
            stride = st;
            std::vector<float> costs;
            for (int32_t r : roots) costs.push_back(pop.dag.nodes[r].cost);
            PlanShape ts;
            ts.N = n_points;
            ts.W = row_len;
            ts.threads = 128;
            // one row: K points of it per thread; one column: a point per thread
            ts.K = row_len == 1 ? 1 : n_points >= (1 << 14) ? 4 : n_points >= (1 << 12) ? 2 : 1;
            ts.dedup = shape.dedup;
            // a small launch: about two items per SM, and at most 8 subtrees
            // a group (each group is a planner pass on the host; many tables
            // are planned on the workers)
            const int64_t tiles = (n_points + ts.K * ts.threads - 1) / (ts.K * ts.threads);
            const int64_t R = (int64_t)roots.size();
            ts.n_groups = (int)std::max<int64_t>(
                1, std::min<int64_t>(R, std::max<int64_t>((152 * 2 + tiles - 1) / tiles, (R + 7) / 8)));
            tplan = std::make_shared<HostPlan>();
            HostPlan* tp = tplan.get();
            const bool big = R >= 256;
            table_builds.push_back([&pop, &roots, costs, ts, tp, par, big]() {
                build_plan_impl(PlanPop{pop.dag, roots, costs, 0}, ts, *tp, nullptr, big ? par : nullptr, false, true);
            });
        };
        make_tables(cneed, col, plan.col_roots, plan.col_plan, plan.col_stride, W, W);
        make_tables(rneed, row, plan.row_roots, plan.row_plan, plan.row_stride, H, 1);
    }
    const std::vector<int32_t>* colp = col.empty() ? nullptr : &col;
    const std::vector<int32_t>* rowp = row.empty() ? nullptr : &row;

    // Slot cap for kept nodes: keep a CTA's dynamic shared memory (target
    // values + slots) within the SM's share for the interpreter's resident
    // CTAs at this K.  Temporaries may exceed it (a tree needs as many as its
    // Sethi-Ullman number).
    const int slot_bytes = shape.K * shape.threads * 4;
    // (less the target values and the root-sum area: kRootBatch floats per thread)
    const int budget =
        std::max(4, (smem_budget_per_cta(shape.K) - kRootBatch * 4 * shape.threads) / slot_bytes - 1);
    plan.group_off.push_back(0);
    if (par && *par && G > 1 && !(cv && cv->active())) {
        // contiguous runs of groups, one planner (and its per-node arrays)
        // each, and the tables' plans as tasks of their own
        const int P = std::min(G, 32);
        const int NT = (int)table_builds.size();
        // each run is planned and encoded on its own; the runs are then
        // placed back to back (offsets shifted)
        std::vector<IrVec> part(P);
        std::vector<std::vector<int64_t>> ends(P), cends(P);
        std::vector<CodeVec> pcode(P);
        std::vector<int> slots(P, 0);
        std::vector<uint8_t> pext(P, 0);
        (*par)(P + NT, [&](int t) {
            if (t < NT) {
                table_builds[t]();
                return;
            }
            t -= NT;
            const int g0 = (int)((int64_t)G * t / P), g1 = (int)((int64_t)G * (t + 1) / P);
            // room for about the run's instructions, so that the output is
            // not moved as it grows: at most two for each of its trees'
            // tokens, its share of the population's tokens taken as its
            // share of the cost
            double est = 0;
            for (int g = g0; g < g1; ++g) est += plan.group_cost[g];
            part[t].reserve((size_t)(2.0 * (double)pop.tree_nodes * est / std::max(total, 1.0) + 64.0));
            GroupGen gen(pop.dag, part[t], shape.dedup, budget, nullptr, colp, rowp);
            ends[t].push_back(0);
            for (int g = g0; g < g1; ++g) {
                slots[t] = std::max(slots[t], plan_group(gen, part[t], pop, groups[g], budget));
                ends[t].push_back((int64_t)part[t].size());
            }
            pcode[t].reserve(part[t].size());
            pext[t] = encode_groups(part[t], ends[t].data(), g1 - g0, plan.col_stride, plan.row_stride, pcode[t],
                                    cends[t]);
        });
        // the runs' places, then their copies on the workers
        std::vector<int64_t> base(P + 1, 0), cbase(P + 1, 0);
        for (int t = 0; t < P; ++t) {
            base[t + 1] = base[t] + (int64_t)part[t].size();
            cbase[t + 1] = cbase[t] + (int64_t)pcode[t].size();
        }
        plan.ir.resize((size_t)base[P]);
        plan.code.reserve((size_t)cbase[P] + 1);
        plan.code.resize((size_t)cbase[P]);
        (*par)(P, [&](int t) {
            std::copy(part[t].begin(), part[t].end(), plan.ir.begin() + base[t]);
            std::copy(pcode[t].begin(), pcode[t].end(), plan.code.begin() + cbase[t]);
        });
        plan.code_off.assign(1, 0);
        for (int t = 0; t < P; ++t) {
            plan.n_slots = std::max(plan.n_slots, slots[t]);
            plan.ext = plan.ext || pext[t];
            for (size_t i = 1; i < ends[t].size(); ++i) plan.group_off.push_back(base[t] + ends[t][i]);
            for (int64_t e : cends[t]) plan.code_off.push_back(cbase[t] + e);
        }
    } else {
        for (auto& b : table_builds) b();
        GroupGen gen(pop.dag, plan.ir, shape.dedup, budget, cv, colp, rowp);
        for (int g = 0; g < G; ++g) {
            plan.n_slots = std::max(plan.n_slots, plan_group(gen, plan.ir, pop, groups[g], budget));
            plan.group_off.push_back((int64_t)plan.ir.size());
        }
        plan.code.reserve(plan.ir.size() + 1);
        plan.code_off.assign(1, 0);
        plan.ext = encode_groups(plan.ir, plan.group_off.data(), G, plan.col_stride, plan.row_stride, plan.code,
                                 plan.code_off);
    }
    plan.group_order.resize(G);
    std::iota(plan.group_order.begin(), plan.group_order.end(), 0);
    std::stable_sort(plan.group_order.begin(), plan.group_order.end(),
                     [&](int32_t a, int32_t b) { return plan.group_cost[a] > plan.group_cost[b]; });
    plan.n_items = (int64_t)G * plan.n_tiles;
    plan.code.push_back(encode(IrIns{F_END, 0, 0, 0, 0, 0}));
}

}  // namespace tgp

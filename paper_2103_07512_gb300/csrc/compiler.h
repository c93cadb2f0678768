// compiler.h -- host side of the hot path: token decode and validation,
// hash-consing into the population DAG, and bytecode generation.
#pragma once
#include <cstdint>
#include <functional>
#include <memory>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "tgp_ir.h"

namespace tgp {

// One unique node of the population DAG.  Identity is structural: the key
// (op, kid0, kid1, imm bits) *is* the node, so two equal subtrees always map
// to the same id (Handley's DAG, Sec. 2 of TensorGP).
struct DagNode {
    int16_t op;
    uint8_t vars;       // bit 0: x is the node or below it; bit 1: y likewise
    uint8_t spare_;
    int32_t kid[kMaxKids];   // operands in order, -1 when absent
    uint32_t imm;       // binary32 bits of a CONST
    int32_t su;         // register slots needed to evaluate it (Sethi-Ullman)
    int32_t depth;      // root alone = 0
    float cost;         // issue cost of evaluating it as a tree, per point
};

// Node arrays: an allocator that leaves a new element of a trivial type
// uninitialised, so that sizing an array that is filled right after (by
// several workers) does not first zero it on one thread.
template <class T>
struct NoInitAlloc : std::allocator<T> {
    template <class U>
    struct rebind {
        using other = NoInitAlloc<U>;
    };
    NoInitAlloc() = default;
    template <class U>
    NoInitAlloc(const NoInitAlloc<U>&) noexcept {}
    template <class U>
    void construct(U* p) noexcept(std::is_nothrow_default_constructible<U>::value) {
        ::new ((void*)p) U;
    }
    template <class U, class... A>
    void construct(U* p, A&&... a) {
        ::new ((void*)p) U(std::forward<A>(a)...);
    }
};
using NodeVec = std::vector<DagNode, NoInitAlloc<DagNode>>;
using IrVec = std::vector<IrIns, NoInitAlloc<IrIns>>;
using CodeVec = std::vector<Ins, NoInitAlloc<Ins>>;

class Dag {
public:
    NodeVec nodes;
    int32_t intern(int op, int32_t k0, int32_t k1, uint32_t imm, int32_t k2 = -1);
    size_t size() const { return nodes.size(); }
    // Room for n nodes without growing the node array or the hash table.
    void reserve(size_t n);
    // Takes `v` as the node array (distinct keys, operands before their
    // users); the hash index over it is rebuilt by the next intern.
    void assign_nodes(NodeVec&& v);

private:
    std::vector<int32_t> table_;   // open addressing, -1 = empty
    size_t mask_ = 0;
    size_t used_ = 0;
    void rehash(size_t cap);
};

inline bool is_leaf(int op) { return op == T_X || op == T_Y || op == T_CONST; }
int arity(int op);       // -1 for an unknown opcode
float op_cost(int op);   // planning estimate of the issue cost per point

struct PopIR {
    Dag dag;
    std::vector<int32_t> roots;       // DAG id of each tree
    std::vector<int32_t> tree_size;   // tokens per tree
    std::vector<float> tree_cost;     // cost of each tree evaluated as a tree
    int64_t tree_nodes = 0;
};

// Validates and hash-conses a token population.  Returns 0, or -2 (tokens) /
// -1 (argument) with a message in err.  With `simplify`, every node goes
// through intern_simplified (limits apply to the trees as given).
// With `par` (and a large population), chunks of trees are parsed
// concurrently; the result equals a serial parse (same nodes, same ids).
using ParallelFor = std::function<void(int n, const std::function<void(int)>& body)>;
int parse_population(const int32_t* ops, const float* imm, int64_t n_imm, const int64_t* tree_off,
                     int32_t n_trees, int32_t order, PopIR& out, std::string& err, bool simplify = true,
                     const ParallelFor* par = nullptr);

// Hash-conses one node after exact algebraic simplification (constant
// folding, identities, canonical operand order; see compiler.cpp).  The
// operands must already be nodes of `dag`.
int32_t intern_simplified(Dag& dag, int op, int32_t k0, int32_t k1, uint32_t imm, int32_t k2 = -1);

// Appends the trees of `src` to `dst`, hash-consing src's nodes into dst's
// DAG (subtrees common to both are shared).
void append_population(PopIR& dst, const PopIR& src);

// Shape of one launch plan.
struct PlanShape {
    int64_t N = 0;       // grid points
    int64_t W = 0;       // grid width (row length); 0: the N points form one row
    int K = 8;           // points per thread
    int threads = 128;   // threads per CTA
    int n_groups = 1;    // tree groups
    bool dedup = true;   // hold shared subtrees (false: recompute at each use)
    bool operator<(const PlanShape& o) const {
        if (dedup != o.dedup) return dedup < o.dedup;
        if (N != o.N) return N < o.N;
        if (W != o.W) return W < o.W;
        if (K != o.K) return K < o.K;
        if (threads != o.threads) return threads < o.threads;
        return n_groups < o.n_groups;
    }
};

// Work units of a launch: every row of the grid is cut into ceil(W / K)
// chunks of K consecutive points (the last one ragged); one thread per chunk.
inline int64_t plan_chunks(const PlanShape& s) {
    const int64_t w = s.W > 0 ? s.W : s.N;
    const int64_t rows = w > 0 ? s.N / w : 0;
    return rows * ((w + s.K - 1) / s.K);
}

struct HostPlan {
    PlanShape shape;
    IrVec ir;                           // decoded, all groups back to back
    CodeVec code;                       // encoded, plus one trailing END
    std::vector<int64_t> group_off;     // [n_groups + 1] offsets into ir
    std::vector<int64_t> code_off;      // [n_groups + 1] offsets into code (fused pairs are one word)
    std::vector<int32_t> group_order;   // groups by descending estimated cost
    std::vector<double> group_cost;
    int n_slots = 0;                    // shared-memory value slots per thread
    bool ext = false;                   // uses operators beyond the benchmark function set
    int n_tiles = 0;
    int64_t n_items = 0;
    // Column tables: subtrees with x but no y below them have one value per
    // grid column.  They are evaluated once on a one-row grid by col_plan (a
    // phenotype launch into a table of col_roots.size() entries of
    // col_stride floats each) before the launch, which loads them (F_COL).
    std::vector<int32_t> col_roots;
    std::shared_ptr<HostPlan> col_plan;
    int64_t col_stride = 0;
    // Row tables, likewise: subtrees with no x below them have one value per
    // grid row, evaluated on one column of H points (F_ROW loads them).
    std::vector<int32_t> row_roots;
    std::shared_ptr<HostPlan> row_plan;
    int64_t row_stride = 0;
};

// Default shape for a grid of N points on a device with `sms` SMs.
PlanShape default_shape(const PopIR& pop, int64_t N, int sms);

// Cross-call subtree cache as the planner sees it (indexed by the
// population's DAG node ids; empty vectors = no cache).
//   cached[n] >= 0: node n's values for every point are in cache entry
//                   cached[n]; it is loaded (F_CLD) and its subtree is not
//                   evaluated.
//   insert[n] >= 0: after node n is first evaluated, its values are stored
//                   into cache entry insert[n] (F_CST).
// Entry numbers index the launch's table of entry pointers.
struct CacheView {
    std::vector<int32_t> cached;
    std::vector<int32_t> insert;
    bool active() const { return !cached.empty(); }
};

// Internal nodes a plan evaluates (reachable from the roots without passing
// through a cached node), for choosing insertions.
std::vector<int32_t> evaluated_nodes(const PopIR& pop, const CacheView& cv);

// Partitions the trees into shape.n_groups groups and emits their bytecode.
// A ParallelFor runs body(i) for every i in [0, n), possibly concurrently,
// and returns when all calls have returned.

// With `par`, the tree groups are planned concurrently (each group's plan
// depends on its own trees only, so the result is the same); a cache view
// keeps the planning serial (a node is stored by the first group that
// evaluates it).
// With `columns` (on a grid of at least two rows and two columns), the costly
// subtrees that have x but no y below them become column tables, and those
// with no x below them row tables (none holding a node of the cache view).
void build_plan(const PopIR& pop, const PlanShape& shape, HostPlan& plan, const CacheView* cv = nullptr,
                const ParallelFor* par = nullptr, bool columns = false);

Ins encode(const IrIns& in);

// Items of a launch that go to the per-SM chunks of its work queues (three
// quarters of them, a multiple of n_queues; none for launches of fewer than
// 8 items per queue); the rest go to the global queue.
int64_t queue_local_items(int64_t n_items, int n_queues);

// The node of one token with operands k (as the parser makes it: clip is
// lowered to max(min(z, x), y); simplified when `simplify`).
int32_t make_node(Dag& dag, int op, const int32_t (&k)[kMaxKids], uint32_t bits, bool simplify);

// Drops DAG nodes no tree reaches, keeping ids in topological order.
void compact(PopIR& pop);

}  // namespace tgp

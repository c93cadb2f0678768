// tgp_ir.h -- bytecode of the fused population interpreter.
//
// The host compiler turns the population DAG into one linear instruction
// stream per tree group.  The device interpreter keeps K points per thread:
//   A[K]       accumulator, in registers (the result of every instruction
//              but ST)
//   X[K],Y[K]  grid coordinates, in registers
//   S[j][K]    value slots j = 0..n_slots-1 in shared memory: shared DAG
//              nodes that are evaluated once and reused, and left operands
//              parked while the right one is computed.  A slot is named by a
//              run-time index in the instruction, so one switch case serves
//              every slot.
// Terminals never get an instruction of their own: they are operands of the
// instruction that consumes them.  Every case is specialised on its operand
// kinds (x, y, immediate, slot), so no register is indexed at run time.
#pragma once
#include <stdint.h>

#ifndef __CUDACC__
#define __host__
#define __device__
#endif

namespace tgp {

// Token opcodes (same numbering as the public header).
enum TokOp : int {
    T_X = 0, T_Y = 1, T_CONST = 2, T_ADD = 3, T_SUB = 4, T_MUL = 5, T_DIV = 6,
    T_SIN = 7, T_COS = 8, T_NEG = 9, T_ABS = 10, T_MIN = 11, T_MAX = 12,
    T_TAN = 13, T_EXP = 14, T_LOG = 15, T_POW = 16, T_MDIST = 17, T_SQRT = 18,
    T_SIGN = 19, T_CLIP = 20, T_MOD = 21, T_FRAC = 22, T_IF = 23, T_NOPS = 24
};
constexpr int kMaxKids = 3;   // clip and if take three operands

// Operand kinds.
constexpr int kOpX = 0, kOpY = 1, kOpC = 2, kOpS = 3;
constexpr int kNOpnd = 4;

// Instruction forms (decoded IR).  `aux` is the slot of an S operand, the
// slot written by ST, or the tree of ROOT; `imm` the immediate of a C operand.
enum Form : int {
    F_END = 0,
    F_AO,     // A = fn(A, o1)        fn binary; o1 in {x, y, imm, slot}
    F_OA,     // A = fn(o1, A)        fn in {sub, div}; o1 in {x, y, imm, slot}
    F_TT,     // A = fn(o1, o2)       fn binary; o1, o2 in {x, y, imm}, not both imm
    F_UA,     // A = fn(A)            fn unary
    F_UT,     // A = fn(o1)           fn unary; o1 in {x, y, imm}
    F_LD,     // A = o1               o1 in {x, y, imm, slot}
    F_ST,     // slot aux = A
    F_ROOT,   // tree aux is complete in A: fitness partial or phenotype store
    F_CST,    // cache entry aux = A (HBM)
    F_CLD,    // A = cache entry aux (HBM)
    F_SEL,    // A = slot aux != 0 ? slot imm : A    (if; both operands in slots)
    F_COL,    // A = column-table entry aux at the thread's columns (a subtree with no y below)
    F_ROW,    // A = row-table entry aux at the thread's row (a subtree with no x below)
    F_NFORMS
};

// binary function index 0..8, reversed-operand index 0..3, unary 0..9
constexpr int kNBin = 9, kNOrd = 4, kNUn = 10;
__host__ __device__ constexpr int bin_index(int tok) {
    return tok == T_ADD ? 0 : tok == T_SUB ? 1 : tok == T_MUL ? 2 : tok == T_DIV ? 3
         : tok == T_MIN ? 4 : tok == T_MAX ? 5 : tok == T_POW ? 6 : tok == T_MDIST ? 7
         : tok == T_MOD ? 8 : -1;
}
__host__ __device__ constexpr int ord_index(int tok) {   // F_OA functions (not commutative)
    return tok == T_SUB ? 0 : tok == T_DIV ? 1 : tok == T_POW ? 2 : tok == T_MOD ? 3 : -1;
}
__host__ __device__ constexpr int un_index(int tok) {
    return tok == T_SIN ? 0 : tok == T_COS ? 1 : tok == T_NEG ? 2 : tok == T_ABS ? 3
         : tok == T_TAN ? 4 : tok == T_EXP ? 5 : tok == T_LOG ? 6 : tok == T_SQRT ? 7
         : tok == T_SIGN ? 8 : tok == T_FRAC ? 9 : -1;
}

// Encoded opcode layout (dense, so the device switch becomes a jump table).
constexpr int OPC_END = 0;
constexpr int OPC_AO = 1;                                  // + bin * 4 + o1
constexpr int OPC_OA = OPC_AO + kNBin * kNOpnd;            // + ord * 4 + o1
constexpr int OPC_TT = OPC_OA + kNOrd * kNOpnd;            // + bin * 9 + o1 * 3 + o2
constexpr int OPC_UA = OPC_TT + kNBin * 9;                 // + un
constexpr int OPC_UT = OPC_UA + kNUn;                      // + un * 3 + o1
constexpr int OPC_LD = OPC_UT + kNUn * 3;                  // + o1
constexpr int OPC_ST = OPC_LD + kNOpnd;
constexpr int OPC_ROOT = OPC_ST + 1;
constexpr int OPC_CST = OPC_ROOT + 1;
constexpr int OPC_CLD = OPC_CST + 1;
constexpr int OPC_SEL = OPC_CLD + 1;
constexpr int OPC_COUNT = OPC_SEL + 1;
// Fused "store, then start a new subexpression": slot x >> 16 = A, then the
// F_TT of one of the first kNHotBin binary functions (+ bin * 9 + o1 * 3 + o2)
// or the F_UT of one of the first kNHotUn unary ones (+ un * 3 + o1).  A
// subexpression that follows a store almost always starts from terminals.
constexpr int kNHotBin = 6;    // add sub mul div min max
constexpr int kNHotUn = 4;     // sin cos neg abs
constexpr int OPC_STT = OPC_COUNT;
constexpr int OPC_SUT = OPC_STT + kNHotBin * 9;
constexpr int OPC_FUSED_END = OPC_SUT + kNHotUn * 3;
// The dispatch takes the low byte of x; every one of its 256 entries is a
// valid target (codes without a form leave the loop).
constexpr int kDispatchMask = 255;
constexpr int kStoreSlotShift = 16;
// F_COL: A = the thread's K values of a column table entry; y = the entry's
// first float in the table (entry index * the table's stride).
constexpr int OPC_COL = OPC_FUSED_END;
static_assert(OPC_COL < kDispatchMask + 1, "opcodes must fit the dispatch byte");
// Codes with which the dispatch loop leaves for sin / cos of a value that all
// of a thread's points share (y, an immediate), held in A[0]; never in bytecode.
constexpr int kExitSinUniform = 250;
constexpr int kExitCosUniform = 251;
// Set in an opcode word (above the dispatch byte) when the instruction
// computes a value with no x below it, which is the same at all of a
// thread's points (they share a row): a division or a library call is then
// evaluated once for the K points.
constexpr uint32_t kUniformBit = 0x100;
static_assert(OPC_COL < kExitSinUniform, "exit codes must not be opcodes");
// F_ROW: A = the row table entry's value at the thread's row; y as F_COL.
constexpr int OPC_ROW = 252;
static_assert(OPC_ROW > kExitCosUniform && OPC_ROW <= kDispatchMask, "F_ROW code");
// Fused "store, then load a table entry": slot x >> 16 = A, then F_COL / F_ROW.
constexpr int OPC_STC = 253;
constexpr int OPC_STR = 254;
static_assert(OPC_STR <= kDispatchMask, "fused table codes");
// Tree roots of a fitness launch.  A root word (OPC_ROOT, y = the tree) also
// carries in x >> kStoreSlotShift its place j (0 .. kRootBatch - 1) in the
// group's current batch of roots: the thread's sum of squared residuals of
// the tree at its K points goes to element j of its root-sum area in shared
// memory.  After every kRootBatch roots of a group, and before its END when
// some are pending, a flush word (OPC_FLUSH, y = n, the batch's roots) is
// followed by ceil(n / 2) data words holding the batch's trees (x, y: two
// trees each; never dispatched): the flush adds each root's sums over the
// lanes of each warp and stores one partial per (tree, tile, warp).
constexpr int OPC_FLUSH = 255;
constexpr int kRootBatch = 4;

// One encoded instruction: x = opcode (low byte; a fused store's slot in the
// high half), y = immediate bits, slot, or aux.
struct Ins {
    uint32_t x;
    uint32_t y;
};

// Decoded instruction (host side; also what tgp_debug_plan reports).
struct IrIns {
    int32_t form, fn, o1, o2;
    int32_t aux;
    uint32_t imm;   // binary32 bits of the immediate operand
    int32_t uni;   // computes a value with no x below it: the same at all of a thread's points
};

// Resident CTAs per SM the interpreter is built for, by points per thread K
// (the kernel's launch bounds; the planner keeps a CTA's shared memory within
// the SM's share for this many CTAs).
#ifndef TGP_MINB16
#define TGP_MINB16 4
#endif
#ifndef TGP_MINB8
#define TGP_MINB8 7
#endif
#ifndef TGP_MINB4
#define TGP_MINB4 10
#endif
#ifndef TGP_MINB2
#define TGP_MINB2 10
#endif
__host__ __device__ constexpr int target_ctas_per_sm(int K) {
    return K >= 16 ? TGP_MINB16 : K >= 8 ? TGP_MINB8 : K >= 4 ? TGP_MINB4 : TGP_MINB2;
}
// Dynamic shared memory one CTA may use at that occupancy: 228 KB per SM, of
// which 1 KB per CTA is reserved by the hardware, less the kernel's static
// shared memory.
__host__ __device__ constexpr int smem_budget_per_cta(int K) {
    return 228 * 1024 / target_ctas_per_sm(K) - 1024 - 64;
}

// Fitness: a thread's sum of squared residuals of a tree (its K points) that
// reaches 2^120 (or is not finite) is recomputed from the residuals scaled by
// 2^-80, so that no square overflows; a warp with such a thread sums in
// units of 2^-160 and stores its partial negated: its value is then
// -partial * 2^160.
constexpr float kSumBig = 0x1p120f;
constexpr float kResidualScale = 0x1p-80f;

// Work queues of one launch: the first local_items items are cut into one
// contiguous chunk per SM (at most kMaxQueues), so that the CTAs of an SM
// take consecutive items (the same tree group, so the same bytecode, which
// then stays in that SM's L1); the rest are handed out by one global queue
// (dynamic balance at the end).  A chunk that no SM took (SM ids beyond the
// queue count) is drained last by any CTA.
constexpr int kMaxQueues = 256;
constexpr int kQueueWords = kMaxQueues + 1;   // chunk heads, then the global head

// One domain of a launch that fuses several (fitness only): its items are
// [item0, next segment's item0); its own program, grid, target, partial sums
// and tables.
struct SegParams {
    const Ins* code;
    const int64_t* group_off;
    const int32_t* item_group;
    int64_t item0;
    int32_t n_tiles;
    int32_t W, H;
    int32_t row0, H_grid;       // a band of rows of a larger grid (see EvalParams)
    float xlo, xhi, ylo, yhi;
    const float* target;        // [N] or nullptr for the inline Pagie polynomial
    const float* pagie_x;       // Pagie: x^4/(1+x^4) per column (see EvalParams)
    float* partial;             // [its trees][n_tiles][warps]
    const float* coltab;        // its column and row tables (see EvalParams)
    const float* rowtab;
};

// Parameters of one interpreter launch.
struct EvalParams {
    const Ins* code;            // all groups back to back
    const int64_t* group_off;   // [n_groups + 1] instruction offsets
    const int32_t* item_group;  // [n_groups] groups in descending cost order
    int64_t n_items;            // n_groups * n_tiles
    int32_t n_tiles;
    int32_t warps_per_tile;
    int64_t N;                  // points
    int32_t W, H;               // the launch's points: H rows of W
    int32_t row0, H_grid;       // its rows are rows row0 .. row0 + H - 1 of an H_grid-row grid on
                                // [ylo, yhi] (y = ylo + (row0 + row) * ((yhi - ylo) / (H_grid - 1)))
    float xlo, xhi, ylo, yhi;
    const float* target;        // [N] or nullptr for the inline Pagie polynomial
    const float* pagie_x;       // Pagie: its x part x^4/(1+x^4) at every column, padded to a
                                // multiple of 16 (the y part is formed per thread), or nullptr
    float* partial;             // [n_trees][n_tiles][warps] fitness partial sums (negated: scaled, see kSumBig)
    float* out;                 // [n_trees][N] phenotypes (phenotype launches)
    float* const* cache;        // cache entry pointers (F_CST / F_CLD), or nullptr
    int32_t* counter;           // [kQueueWords] work-queue heads, zero before the launch
    int32_t n_queues;           // chunk q holds items [q L / n_queues, (q+1) L / n_queues)
    int64_t local_items;        // L: items in the per-SM chunks; [L, n_items) in the global queue
    int32_t n_slots;            // shared-memory value slots per thread
    int32_t max_items_per_cta;  // bound on the work-queue loop
    int32_t trig_rad;           // sin/cos/tan in radians (interpreter variant with the rest of Table 1 only)
    const float* coltab;        // column tables (F_COL words hold the offset of their entry), or nullptr
    const float* rowtab;        // row tables (F_ROW words likewise), or nullptr
    int64_t out_stride;         // floats between the phenotype rows of two trees (N, or a table's stride)
    const SegParams* segs;      // a launch fusing several domains: [n_segs] segments, or nullptr
    int32_t n_segs;             // (the fields above from code to rowtab are then unused)
};

struct FinalizeParams {
    const float* partial;       // [n_trees][per_tree] (negated: in units of 2^-160)
    int64_t per_tree;           // n_tiles * warps
    int32_t n_trees;
    double n_points;            // N
    double* rmse;               // [n_trees]
    int32_t sse;                // nonzero: write the sums of squared residuals, not the RMSE
};

}  // namespace tgp

// tgp_ir.h -- bytecode of the fused population interpreter.
//
// The host compiler turns the population DAG into one linear instruction
// stream per tree group.  The device interpreter keeps K points per thread
// and holds every value in registers:
//   A[K]       accumulator (every instruction but ST/SPILL/FILL writes it)
//   R[j][K]    register slots j = 0..M-1 (shared DAG nodes, pending operands)
//   F[K]       fill buffer, loaded from a shared-memory spill slot
//   X[K],Y[K]  grid coordinates, T[K] the target values
// Terminals never get an instruction of their own: they are operands of the
// instruction that consumes them.  Because the switch case of every form is
// specialised on its operand registers, no register is ever indexed at run
// time.
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
    T_SIN = 7, T_COS = 8, T_NEG = 9, T_ABS = 10, T_MIN = 11, T_MAX = 12, T_NOPS = 13
};

constexpr int kNReg = 6;                 // register slots M
constexpr int kOpX = 0, kOpY = 1, kOpC = 2, kOpR0 = 3, kOpF = 3 + kNReg;
constexpr int kNOpnd = 4 + kNReg;        // x, y, imm, R0..R(M-1), F

// Instruction forms (decoded IR).
enum Form : int {
    F_END = 0,
    F_AO,     // A = fn(A, o1)                 fn binary, o1 any operand
    F_OA,     // A = fn(o1, A)                 fn in {sub, div, min, max}
    F_TT,     // A = fn(o1, o2)                o1, o2 in {x, y, imm}, not both imm
    F_UA,     // A = fn(A)                     fn unary
    F_UT,     // A = fn(o1)                    o1 in {x, y, imm}
    F_LD,     // A = o1                        o1 any operand
    F_ST,     // R[o1 - kOpR0] = A
    F_SPILL,  // smem[aux] = A
    F_FILL,   // F = smem[aux]
    F_ROOT,   // tree aux is complete in A: fitness partial or phenotype store
    F_CST,    // cache entry aux = A (HBM)
    F_CLD,    // A = cache entry aux (HBM)
    F_NFORMS
};

// binary function index 0..5 and unary 0..3
constexpr int kNBin = 6, kNUn = 4, kNOrd = 4;   // kNOrd: binaries needing the F_OA form
__host__ __device__ constexpr int bin_index(int tok) {
    return tok == T_ADD ? 0 : tok == T_SUB ? 1 : tok == T_MUL ? 2 : tok == T_DIV ? 3
         : tok == T_MIN ? 4 : tok == T_MAX ? 5 : -1;
}
__host__ __device__ constexpr int ord_index(int tok) {   // F_OA functions
    return tok == T_SUB ? 0 : tok == T_DIV ? 1 : tok == T_MIN ? 2 : tok == T_MAX ? 3 : -1;
}
__host__ __device__ constexpr int un_index(int tok) {
    return tok == T_SIN ? 0 : tok == T_COS ? 1 : tok == T_NEG ? 2 : tok == T_ABS ? 3 : -1;
}

// Encoded opcode layout (dense, so the device switch becomes a jump table).
constexpr int OPC_END = 0;
constexpr int OPC_AO = 1;                                  // + bin * kNOpnd + o1
constexpr int OPC_OA = OPC_AO + kNBin * kNOpnd;            // + ord * kNOpnd + o1
constexpr int OPC_TT = OPC_OA + kNOrd * kNOpnd;            // + bin * 9 + o1 * 3 + o2
constexpr int OPC_UA = OPC_TT + kNBin * 9;                 // + un
constexpr int OPC_UT = OPC_UA + kNUn;                      // + un * 3 + o1
constexpr int OPC_LD = OPC_UT + kNUn * 3;                  // + o1
constexpr int OPC_ST = OPC_LD + kNOpnd;                    // + j
constexpr int OPC_SPILL = OPC_ST + kNReg;
constexpr int OPC_FILL = OPC_SPILL + 1;
constexpr int OPC_ROOT = OPC_FILL + 1;
constexpr int OPC_CST = OPC_ROOT + 1;
constexpr int OPC_CLD = OPC_CST + 1;
constexpr int OPC_COUNT = OPC_CLD + 1;

// One encoded instruction: x = opcode | (aux16 << 16), y = imm bits or aux32.
struct Ins {
    uint32_t x;
    uint32_t y;
};

// Decoded instruction (host side; also what tgp_debug_plan reports).
struct IrIns {
    int32_t form, fn, o1, o2;
    int32_t aux;
    uint32_t imm;   // binary32 bits of the immediate operand
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
    int32_t W, H;
    float xlo, xhi, ylo, yhi;
    const float* target;        // [N] or nullptr for the inline Pagie polynomial
    float* partial;             // [n_trees][n_tiles][warps] fitness partial sums
    float* out;                 // [n_trees][N] phenotypes (phenotype launches)
    float* const* cache;        // cache entry pointers (F_CST / F_CLD), or nullptr
    int32_t* counter;           // work-queue head, zero before the launch
    int32_t spill_slots;        // shared-memory spill slots per thread
    int32_t max_items_per_cta;  // bound on the work-queue loop
};

struct FinalizeParams {
    const float* partial;       // [n_trees][per_tree]
    int64_t per_tree;           // n_tiles * warps
    int32_t n_trees;
    double n_points;            // N
    double* rmse;               // [n_trees]
};

}  // namespace tgp

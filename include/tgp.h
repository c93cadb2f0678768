/*
 * tgp.h -- C ABI of libtgp: GPU evaluation of a population of GP expression
 * trees over every point of a regular 2-D grid, with structurally identical
 * subtrees deduplicated into a population DAG, reduced to per-tree RMSE.
 *
 * Method: TensorGP (Baeta, Correia, Martins, Machado; arXiv 2103.07512).
 *   - tensor phenotype: each individual evaluates to a tensor over the whole
 *     fixed domain of fitness cases (Sec. 3.1);
 *   - caching of intermediate subtree results and a population DAG that does
 *     not duplicate identical subtrees (Sec. 2, Handley; Sec. 3.1);
 *   - fixed-size cache with update and flush (Sec. 2, Keijzer);
 *   - operators and protections of Table 1, trigonometry on pi*x (Sec. 3.2);
 *   - Pagie target, Eq. 1; RMSE fitness (Sec. 4.1, Table 2).
 *
 * Conventions for every entry point:
 *   - Return value: TGP_OK (0) or a negative tgp_status.  Nothing aborts or
 *     exits the process.  tgp_last_error() gives a message for the calling
 *     thread's most recent failure.
 *   - Ownership: the caller owns every pointer it passes; arrays are read (or
 *     copied) during the call unless stated otherwise.  The library owns the
 *     objects behind handles until the matching release call.
 *   - Streams: `stream` is a cudaStream_t (e.g. torch.cuda.Stream.cuda_stream)
 *     or NULL for the legacy default stream.  Device work is enqueued on it.
 *   - Thread safety: calls on one context may come from several threads; host
 *     state is serialised by a per-context lock.  Two concurrent evaluations of
 *     the same (population, domain) pair on different streams are not allowed
 *     (they share device scratch); distinct pairs may overlap freely.
 *   - Device memory: allocated by the library on the context's device with
 *     cudaMalloc; TGP_E_NOMEM when an allocation fails.
 */
#ifndef TGP_H
#define TGP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tgp_ctx tgp_ctx;
typedef int64_t tgp_handle;

typedef enum tgp_status {
    TGP_OK = 0,
    TGP_E_INVALID = -1,       /* bad argument or handle */
    TGP_E_TOKENS = -2,        /* malformed token stream (arity, opcode, imm, limits) */
    TGP_E_NOMEM = -3,         /* host or device allocation failed */
    TGP_E_BUDGET = -4,        /* request does not fit the context's HBM budget */
    TGP_E_CUDA = -5,          /* a CUDA runtime call failed (message has the name) */
    TGP_E_TIMEOUT = -6,       /* a bounded wait ran out */
    TGP_E_DEVICE_CHECK = -7,  /* a device-side check recorded a violation */
    TGP_E_BUSY = -8           /* object in use (e.g. releasing a pinned cache entry) */
} tgp_status;

/* Token order of a population (Sec. 3.1: genotype as an expression tree). */
enum { TGP_PREFIX = 0, TGP_POSTFIX = 1 };

/* Target of the fitness (Sec. 4.1). */
enum {
    TGP_TARGET_PAGIE = 0,   /* Eq. 1, computed inline from the coordinates */
    TGP_TARGET_TENSOR = 1,  /* float[H*W], host or device pointer */
    TGP_TARGET_TOKENS = 2   /* one expression tree (tgp_target_tokens*) evaluated on the grid */
};

/* Opcodes of the token stream: the terminals and the mathematical and
 * conditional operators of Table 1.  Arity: X, Y, CONST 0; SIN, COS, NEG, ABS,
 * TAN, EXP, LOG, SQRT, SIGN, FRAC 1; ADD, SUB, MUL, DIV, MIN, MAX, POW, MDIST,
 * MOD 2; CLIP, IF 3.  CONST takes the next value of `imm`.  Readings where
 * Table 1 is silent: mod is the floored remainder (sign of the divisor);
 * log(0) = -inf; tan at an odd multiple of 1/2 is +-inf; if treats NaN as
 * true. */
enum {
    TGP_OP_X = 0, TGP_OP_Y = 1, TGP_OP_CONST = 2,
    TGP_OP_ADD = 3,  /* a + b                                  (Table 1, add)  */
    TGP_OP_SUB = 4,  /* a - b                                  (Table 1, sub)  */
    TGP_OP_MUL = 5,  /* a * b                                  (Table 1, mult) */
    TGP_OP_DIV = 6,  /* a / b, 0 when b == 0                   (Table 1, div)  */
    TGP_OP_SIN = 7,  /* sin(pi * a)                            (Sec. 3.2)      */
    TGP_OP_COS = 8,  /* cos(pi * a)                            (Sec. 3.2)      */
    TGP_OP_NEG = 9,  /* -a                                     (Table 1, neg)  */
    TGP_OP_ABS = 10, /* |a|                                    (Table 1, abs)  */
    TGP_OP_MIN = 11, /* fminf(a, b)                            (Table 1, min)  */
    TGP_OP_MAX = 12, /* fmaxf(a, b)                            (Table 1, max)  */
    TGP_OP_TAN = 13, /* tan(pi * a) = sin(pi a) / cos(pi a)    (Table 1, Sec. 3.2) */
    TGP_OP_EXP = 14, /* e^a                                    (Table 1, exp)  */
    TGP_OP_LOG = 15, /* log(a), -1 when a < 0                  (Table 1, log)  */
    TGP_OP_POW = 16, /* a^b, 0 when a = b = 0                  (Table 1, pow)  */
    TGP_OP_MDIST = 17, /* (a + b) / 2                          (Table 1, mdist) */
    TGP_OP_SQRT = 18, /* sqrt(a), 0 when a < 0                 (Table 1, sqrt) */
    TGP_OP_SIGN = 19, /* -1, 0 or 1 (NaN stays NaN)            (Table 1, sign) */
    TGP_OP_CLIP = 20, /* clip(x, y, z) = max(min(z, x), y)     (Table 1, clip; arity 3) */
    TGP_OP_MOD = 21, /* a - b floor(a / b), NaN when b = 0     (Table 1, mod)  */
    TGP_OP_FRAC = 22, /* a - floor(a)                          (Table 1, frac) */
    TGP_OP_IF = 23,  /* if(c, a, b): a where c != 0, else b    (Table 1, if; arity 3) */
    TGP_N_OPS = 24
};

/* Limits checked by tgp_compile_population (TGP_E_TOKENS beyond them). */
#define TGP_MAX_DEPTH 1024              /* root alone has depth 0 */
#define TGP_MAX_TREE_TOKENS (1 << 24)
#define TGP_MAX_TREES (1 << 24)

/* tgp_config.flags */
#define TGP_F_HOST_ONLY 1     /* no device: compile and inspect plans only (for
                                 machines without a GPU); device calls fail with
                                 TGP_E_INVALID (a domain with the Pagie target,
                                 which holds no device memory, may be loaded for
                                 tgp_plan_work).  Plans assume 152 SMs. */
#define TGP_F_NO_DEDUP 2      /* evaluate every tree as a tree: a shared subtree
                                 is recomputed at each use instead of being held
                                 (the uncached reference; results are bitwise
                                 equal to the deduplicated evaluation) */
#define TGP_F_TIME_KERNELS 4  /* record CUDA events around every interpreter
                                 launch on its stream; tgp_stats_get reports the
                                 summed kernel time */
#define TGP_F_NO_SIMPLIFY 8   /* compile trees as given.  By default nodes are
                                 simplified while hash-consing (algebraic
                                 simplification ahead of caching: Sec. 2, Wong
                                 and Zhang; Sec. 5): constant folding
                                 of the exactly reproducible operators, the
                                 identities neg(neg a) = a, abs(neg a) = abs a,
                                 abs(abs a) = abs a, a*1 = a, a/1 = a, a/0 = 0,
                                 a+(-0) = a, a-(+0) = a, (-0)-a = -a,
                                 min(a,a) = max(a,a) = a, and one operand order
                                 for add and mul.  Each is exact in binary32, so
                                 results are bitwise those of the trees as given
                                 (a NaN may differ in sign or payload). */
#define TGP_F_NO_COLUMNS 32   /* evaluate every subtree at every point.  By default a
                                 costly subtree with x but no y below it (its value
                                 depends on the grid column only) is evaluated once
                                 per column, in a phenotype launch on one row of W
                                 points before the launch that loads it, and one
                                 with no x below it once per row (one column of H
                                 points); results are bitwise the same (the same
                                 arithmetic on the same binary32 coordinates).
                                 With the cross-call cache, subtrees that hold a
                                 cache load or store are not tabled;
                                 tgp_fitness_noalloc uses no tables. */
#define TGP_F_TRIG_RADIANS 16 /* sin, cos and tan take their argument in radians
                                 (the footnote of Table 1) instead of multiplied
                                 by pi (Sec. 3.2, the default): CUDA's binary32
                                 sinf, cosf and tanf (within 2, 2 and 4 ulp) */

/* Context configuration.  Zero-initialise, then set what you need. */
typedef struct tgp_config {
    int32_t device;              /* CUDA device ordinal */
    int32_t flags;               /* TGP_F_* */
    int64_t cache_budget_bytes;  /* HBM budget of the cross-call subtree cache; 0 disables it.
                                    With a budget, a subtree of at least cache_min_cost that a
                                    call evaluates on a domain for the second time is stored (one
                                    float per point; 64 stores per call at most) and later calls,
                                    of any population, load it instead of evaluating it (Sec. 2,
                                    Handley).  Over budget, entries the calling population does
                                    not reference are flushed, lowest cost (discounted by the calls
                                    since their last use) first, and their memory is reused (Sec.
                                    2, Keijzer).  Results are bitwise those without the cache. */
    int32_t points_per_thread;   /* 0 = automatic (autotuned); else 1, 2, 4, 8 or 16 */
    int32_t threads_per_block;   /* 0 = automatic; else 32, 64 or 128 */
    int32_t n_groups;            /* 0 = automatic; else trees are split into this many groups */
    int32_t cache_min_cost;      /* subtrees cheaper than this (per point, a binary32 add = 1) are
                                    never stored in the cache; 0 = 48.  With column and row tables,
                                    a subtree with no x or no y below it is never stored and counts
                                    as one add in the cost of the subtrees above it. */
    int32_t plan_threads;        /* host threads that plan a population's tree groups
                                    concurrently (the calling thread included); 0 = up to 16
                                    (at most the host's hardware threads), 1 = serial.  The
                                    bytecode does not depend on it. */
    int32_t cache_ids_max;       /* with the cache on, cache entries are keyed by a context-wide
                                    DAG of every subtree adopted so far (exact structural
                                    identity).  Past this many nodes, and past twice what the
                                    live populations held at its last rebuild, that DAG is
                                    rebuilt from the live populations and the cache flushed:
                                    host memory stays bounded in a long-running process.
                                    0 = 2^23 (about 400 MB). */
    int32_t reserved[2];
} tgp_config;

/* A target given as one expression tree (TGP_TARGET_TOKENS). */
typedef struct tgp_target_tokens {
    const int32_t* ops;   /* opcodes of one tree */
    const float* imm;     /* one value per CONST token, in stream order */
    int64_t n_ops;
    int64_t n_imm;
    int32_t order;        /* TGP_PREFIX or TGP_POSTFIX */
} tgp_target_tokens;

/* Counters, reset by tgp_create only. */
typedef struct tgp_stats {
    int64_t tree_nodes;       /* sum of tree sizes of the last compiled population */
    int64_t dag_nodes;        /* unique nodes of its population DAG (terminals included) */
    int64_t dag_internal;     /* unique function nodes */
    int64_t code_instrs;      /* bytecode instructions of the last plan used */
    int64_t n_groups;         /* tree groups of the last plan */
    int64_t n_items;          /* (group, tile) work items of the last launch */
    int32_t points_per_thread, threads_per_block;
    int32_t slots;            /* shared-memory value slots per thread of the last plan */
    int32_t reserved0;
    int64_t cache_entries;    /* live cache entries */
    int64_t cache_bytes;      /* HBM held by live cache entries */
    int64_t cache_hits;       /* subtree loads served from the cache */
    int64_t cache_inserts;
    int64_t cache_evictions;
    int64_t launches;         /* kernels launched by the library so far (a graph replay counts
                                 the kernels it holds) */
    double eval_ms_sum;       /* TGP_F_TIME_KERNELS: summed interpreter kernel time */
    int64_t eval_timed;       /* TGP_F_TIME_KERNELS: launches summed in eval_ms_sum */
    int64_t cache_reserved;   /* HBM reserved for the cache (slabs carved into entries; at most
                                 the budget, freed with the context) */
    int64_t cache_id_nodes;   /* nodes of the context-wide DAG that keys the cache */
    int64_t cache_id_rebuilds;   /* its rebuilds (each a full flush of the cache) */
    int64_t reserved[3];
} tgp_stats;

/* Creates a context on cfg->device (cfg may be NULL: device 0, defaults). */
int tgp_create(tgp_ctx** out, const tgp_config* cfg);

/* Frees the context and everything it owns (domains, populations, cache). */
int tgp_destroy(tgp_ctx* ctx);

/* Message of the calling thread's last failed call ("" if none).  The string
 * stays valid until the next call on this thread. */
const char* tgp_last_error(const tgp_ctx* ctx);

/*
 * Loads a domain: a W x H grid of fitness cases (Sec. 3.1; Table 2 uses square
 * grids of 2^(2n) points) and the target.  Points are an inclusive linspace:
 * x = xlo + col*((xhi-xlo)/(W-1)), y = ylo + row*((yhi-ylo)/(H-1)) in binary32
 * (x = xlo when W == 1), flat index p = row*W + col.  Coordinates are never
 * stored: kernels form them from the thread index.
 *   target_kind TGP_TARGET_PAGIE: target must be NULL.
 *   TGP_TARGET_TENSOR: target is float[H*W] in host or device memory (copied).
 *   TGP_TARGET_TOKENS: target is a tgp_target_tokens*; the tree is evaluated
 *     once on the device into the domain's target tensor.
 * W, H >= 1 and W*H <= 2^31 - 1.
 */
int tgp_load_domain(tgp_ctx* ctx, int32_t W, int32_t H, float xlo, float xhi, float ylo, float yhi,
                    int32_t target_kind, const void* target, tgp_handle* domain_out);

/*
 * Loads rows row0 .. row0 + n_rows - 1 of the W x H grid of tgp_load_domain
 * as a domain of W x n_rows points: the points, their flat order within the
 * band and their binary32 coordinates are exactly those of the full grid's
 * rows (y = ylo + row*((yhi-ylo)/(H-1)) with the full grid's row index and H).
 * For fitness sharded by rows over several GPUs (the fitness cases of
 * Sec. 3.1 split into contiguous bands, one per process; see
 * tgp_fitness_sse_dev).  A TGP_TARGET_TENSOR target holds the band's
 * n_rows*W values; a token target is evaluated on the band's points.
 * Errors: TGP_E_INVALID unless 0 <= row0, n_rows >= 1, row0 + n_rows <= H.
 */
int tgp_load_domain_rows(tgp_ctx* ctx, int32_t W, int32_t H, float xlo, float xhi, float ylo, float yhi,
                         int32_t row0, int32_t n_rows, int32_t target_kind, const void* target,
                         tgp_handle* domain_out);

/* Releases a domain and the device memory it holds. */
int tgp_release_domain(tgp_ctx* ctx, tgp_handle domain);

/*
 * Compiles a population from token arrays (host memory, copied):
 *   ops[tree_off[t] .. tree_off[t+1]) is tree t, in `order`;
 *   imm holds one binary32 value per CONST token of the whole stream, in
 *   stream order (n_imm values); every value must be finite.
 * Host work only: validation, hash-consing of identical subtrees into the
 * population DAG (Sec. 2: Handley's DAG), and per-tree statistics.  Bytecode
 * for a given grid size is planned and uploaded lazily by the first
 * tgp_evaluate / tgp_fitness on a domain of that size.
 * Errors: TGP_E_TOKENS with a message naming the tree and token.
 */
int tgp_compile_population(tgp_ctx* ctx, const int32_t* ops, const float* imm, int64_t n_imm,
                           const int64_t* tree_off, int32_t n_trees, int32_t order,
                           tgp_handle* pop_out);

/* Releases a population, its plans and device buffers. */
int tgp_release_population(tgp_ctx* ctx, tgp_handle pop);

/*
 * Tensor phenotypes (Sec. 3.1): writes out_dev[t*H*W + p] = value of tree t at
 * point p, binary32, for every tree and point.  out_dev is a device pointer
 * to n_trees*H*W floats owned by the caller.  Asynchronous on `stream`.
 */
int tgp_evaluate(tgp_ctx* ctx, tgp_handle pop, tgp_handle domain, void* stream, float* out_dev);

/*
 * RMSE fitness of every tree against the domain's target (Sec. 4.1):
 *   rmse[t] = sqrt( sum_p (f_t(p) - target(p))^2 / (H*W) ),
 * +inf when the sum is not finite.  Residuals are formed and squared in
 * binary32 and summed in binary32 over a warp's points (a thread's K points,
 * then a butterfly over the 32 threads: at most 512 squares, relative error
 * below 2^-19); a sum that would overflow binary32 is formed from
 * residuals scaled by 2^-80.  The per-warp partials are added in binary64 in
 * a fixed order, so results are bitwise reproducible, and finite whenever
 * every element is.
 * rmse_host: host array of n_trees doubles.  blocking != 0: returns after the
 * values are in rmse_host.  blocking == 0: the copy is enqueued on `stream`
 * and rmse_host is valid once the stream has synchronised (pass pinned memory
 * for a truly asynchronous copy).
 */
int tgp_fitness(tgp_ctx* ctx, tgp_handle pop, tgp_handle domain, void* stream,
                double* rmse_host, int32_t blocking);

/* As tgp_fitness, but writes the n_trees doubles to device memory rmse_dev
 * and never synchronises (suitable for CUDA graph capture). */
int tgp_fitness_dev(tgp_ctx* ctx, tgp_handle pop, tgp_handle domain, void* stream, double* rmse_dev);

/*
 * The sums under the square root of tgp_fitness_dev: writes
 * sse_dev[t] = sum over the domain's points of (f_t(p) - target(p))^2, formed
 * and added exactly as for the RMSE (same partials, same fixed binary64
 * order), +inf when not finite.  sse_dev: device array of n_trees doubles.
 * Asynchronous on `stream`; never synchronises.  With a grid split by rows
 * (tgp_load_domain_rows), each GPU computes its band's sums; the RMSE of
 * Sec. 4.1 over the whole grid is sqrt((sum of the bands' values) / (W*H)).
 */
int tgp_fitness_sse_dev(tgp_ctx* ctx, tgp_handle pop, tgp_handle domain, void* stream, double* sse_dev);

/*
 * tgp_fitness_noalloc -- the fitness of tgp_fitness_dev, computed without
 * allocating any device memory.  (This entry point has no counterpart in the
 * paper; it serves callers of this library.)
 *
 * For callers that cannot call cudaMalloc: a host that has already reserved
 * the device's memory for its own pool, code that must not risk the implicit
 * device synchronisation an allocation or free may cause, or code that must
 * not touch the allocator after start-up.  The plan's bytecode, the work-queue
 * head and the per-tile partial sums live in one fixed device array of
 * TGP_NOALLOC_SCRATCH_BYTES (8 MiB) that is part of the library image: every
 * GPU that loads the library holds it until the process exits.
 *   - The caller passes the inputs (a compiled population and a loaded
 *     domain; a Pagie domain holds no device memory, a tensor or token target
 *     was allocated when the domain was loaded) and the output: rmse_dev, a
 *     device array of n_trees doubles.  Asynchronous on `stream`.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - Rejects, with TGP_E_INVALID and a message giving the bytes needed, a
 *     population whose bytecode plus partial sums (n_trees * tiles * warps
 *     floats) exceed the array.
 *   - Plans without the column and row tables of tgp_fitness_dev (they would
 *     need device memory of their own); the values, and so the results, are
 *     bitwise the same, the launch does the tabled work at every point.
 *   - All calls share the one array and it keeps the previous call's
 *     contents (the queue heads are cleared on every call); calls whose device
 *     work overlaps -- on different streams or from different threads without
 *     ordering -- race on it and give wrong results.
 * Allocates no device memory and calls no allocating library routine.
 */
#define TGP_NOALLOC_SCRATCH_BYTES (8 << 20)
int tgp_fitness_noalloc(tgp_ctx* ctx, tgp_handle pop, tgp_handle domain, void* stream, double* rmse_dev);

/*
 * The fitness of tgp_fitness_dev, launched as a CUDA graph.  The first call
 * for a (population, domain, rmse_dev) triple plans and uploads the
 * population, synchronises `stream`, captures the launch sequence (queue
 * reset, interpreter, finalize) and instantiates it; later calls replay the
 * graph (one cudaGraphLaunch).  The graph is freed with the population.  The
 * first call must not itself be made during a stream capture.  `stream` must
 * be a created stream (NULL and the per-thread default stream cannot be
 * captured: TGP_E_INVALID).
 */
int tgp_fitness_graph(tgp_ctx* ctx, tgp_handle pop, tgp_handle domain, void* stream, double* rmse_dev);

/*
 * Autotuner: times candidate launch shapes (points per thread K in {2,4,8,16},
 * 128 threads per block, and 64 for K in {4,8}; tree groups for ~16/64/256/512
 * work items per SM) on this population and
 * domain, with CUDA events on `stream` (synchronous), and records the fastest
 * for the (grid size, tree-count bucket, node-count bucket) of the
 * population.  Later plans of any population in the same bucket use it
 * unless the context's configuration forces a shape.  Outputs (may be NULL):
 * the chosen K, group count and its kernel time in milliseconds (the chosen
 * threads per block is in tgp_stats after the next launch).
 */
int tgp_autotune(tgp_ctx* ctx, tgp_handle pop, tgp_handle domain, void* stream, int32_t* K_out,
                 int32_t* groups_out, double* ms_out);

/* Copies the context's counters.  With TGP_F_TIME_KERNELS it first waits for
 * the timing events of launches not yet summed. */
int tgp_stats_get(tgp_ctx* ctx, tgp_stats* out);

/*
 * Host-only inspection of the bytecode plan the library would run for a grid
 * of n_points points in one row (used by CPU tests of the compiler; no device
 * needed; a one-row grid has no column tables).
 * Fills up to `cap` decoded instructions into ins_out[i*6 .. i*6+5] as
 * (form, fn, operand1, operand2, aux, imm_bits) and the group boundaries
 * into group_off_out[0..n_groups] (cap_groups entries at most).
 * *n_ins and *n_groups receive the full sizes.  Forms and operand numbering
 * are listed in tgp_debug_layout.
 */
int tgp_debug_plan(tgp_ctx* ctx, tgp_handle pop, int64_t n_points,
                   int32_t* ins_out, int64_t cap, int64_t* n_ins,
                   int64_t* group_off_out, int64_t cap_groups, int32_t* n_groups);

/* Layout constants of the decoded bytecode: out[0] = number of operand
 * kinds (0 = x, 1 = y, 2 = immediate, 3 = value slot named by aux);
 * out[1] = number of forms. */
int tgp_debug_layout(int32_t* out, int32_t n);

/*
 * Measures, with a straight-line kernel per operator, the issue cost of each
 * opcode relative to one binary32 add (cost[TGP_OP_ADD] == 1; terminals 0).
 * cost_out: host array of TGP_N_OPS doubles.  Synchronous; for roofline
 * accounting only.
 */
int tgp_calibrate_op_costs(tgp_ctx* ctx, double* cost_out);

/*
 * The binary32 issue peak of the device, measured: the rate, in lane
 * operations per second, of a straight-line kernel of independent binary32
 * add chains on every SM (the unit tgp_calibrate_op_costs expresses costs in),
 * and of the same with fused multiply-adds.  Synchronous; for roofline
 * accounting only.
 */
int tgp_calibrate_peak(tgp_ctx* ctx, double* add_lane_ops_per_s, double* fma_lane_ops_per_s);

/*
 * The work the fitness launches of `pop` on `domain` evaluate, as planned
 * (host side; builds the plan if the population has none for the domain's
 * grid): work_out[op] = evaluations of operator op (TGP_OP_*), summed over
 * the launch's points for instructions evaluated at every point, over its
 * threads for values with no x below them (evaluated once per thread), and
 * over the W (H) points of the column (row) table launches;
 * work_out[TGP_N_OPS] = residuals formed at tree roots (one per tree and
 * point: a subtract, a multiply and an add each).  Shared subtrees count once
 * per evaluation the plan makes of them, loads from tables or the cache not
 * at all.  work_out: host array of TGP_N_OPS + 1 doubles.  The plan ignores
 * the subtree cache (the plan of a cache-free context).
 */
int tgp_plan_work(tgp_ctx* ctx, tgp_handle pop, tgp_handle domain, double* work_out);

/* ------------------------------------------------------------------------
 * Generational step on the host (TensorGP, Sec. 3 and Table 2).
 *
 * tgp_evolve builds the next generation of `pop` from its trees' RMSE values
 * and registers it as a new population (`pop` stays valid; release it when
 * done).  Variation works on the population DAG itself: crossover and
 * mutation rebuild only the nodes on the path from the replaced subtree to
 * the root, and every unchanged subtree keeps its structural identity, so the
 * next generation needs no token re-parse and subtrees already in the
 * context's cache stay cached.
 *
 *   selection: tournament of `tournament` trees drawn with replacement; the
 *     lowest RMSE wins (NaN and +inf rank last; ties go to the lower index);
 *   elitism: the `elitism` best trees (stable order of RMSE) are copied first;
 *   then, per offspring, with probability p_crossover a subtree crossover (a
 *     uniformly chosen node occurrence of the first parent, in preorder, is
 *     replaced by a uniformly chosen subtree of a second tournament winner),
 *     else with probability p_mutation a subtree mutation (the chosen node is
 *     replaced by a grow tree of depth 0..mutation_depth over `functions`,
 *     terminals x, y and constants uniform in [const_lo, const_hi)), else a
 *     copy; an offspring deeper than max_depth (measured on the stored tree,
 *     clip being stored as max(min(z, x), y)), or larger than 2^24 tokens
 *     once its shared subtrees are written out, is replaced by its first
 *     parent.
 *
 * Zero fields take the defaults: tournament 3, p_crossover 0.9, p_mutation
 * 0.1, elitism 1, max_depth 12 (at most 1024), mutation_depth 4 (a negative
 * probability or elitism means none),
 * functions {add, sub, mult, div, sin, cos, neg, abs, min, max}, constants in
 * [-1, 1).  The random stream is splitmix64 from `seed`: the same population,
 * RMSE values and configuration give the same next generation.  With the
 * context's simplification on, rebuilt nodes are simplified exactly as
 * tgp_compile_population would.  Works on host-only contexts.
 *
 * rmse: host array with one value per tree of `pop`.
 */
typedef struct tgp_evolve_config {
    int32_t tournament;
    float p_crossover;
    float p_mutation;
    int32_t elitism;
    int32_t max_depth;
    int32_t mutation_depth;
    const int32_t* functions;   /* opcodes of arity >= 1, NULL for the default set */
    int32_t n_functions;
    float const_lo, const_hi;
    uint64_t seed;
    int64_t reserved[4];
} tgp_evolve_config;

int tgp_evolve(tgp_ctx* ctx, tgp_handle pop, const double* rmse, const tgp_evolve_config* cfg,
               tgp_handle* next_pop);

/*
 * Writes the trees of a population as prefix-order tokens (the format of
 * tgp_compile_population with order TGP_PREFIX): ops[cap_ops], imm[cap_imm]
 * (one binary32 per CONST, in token order) and tree_off[cap_off] (n_trees + 1
 * offsets).  Trees are written as stored, i.e. after the context's
 * simplification and with clip(x, y, z) as its definition max(min(z, x), y).  *n_ops, *n_imm and *n_trees (each may be NULL) receive
 * the sizes; pass NULL arrays to query them.  TGP_E_INVALID when an array is
 * too small (nothing beyond its capacity is written).
 */
int tgp_population_tokens(tgp_ctx* ctx, tgp_handle pop, int32_t* ops, int64_t cap_ops, float* imm, int64_t cap_imm,
                          int64_t* tree_off, int64_t cap_off, int64_t* n_ops, int64_t* n_imm, int32_t* n_trees);

/* ------------------------------------------------------------------------
 * Serving: evaluation jobs that arrive over time.
 *
 * A server owns a worker thread on a context.  tgp_server_submit copies and
 * validates a job (tokens, grid, target) in the caller's thread and queues
 * it; the worker admits queued jobs in arrival order when a launch slot (one
 * CUDA stream) is free and the job's device memory fits the HBM budget.  One
 * launch takes the head of the queue, every queued job on the same domain
 * (same grid and target; their trees become one population), and queued jobs
 * on other domains whose launch shape is the head's (points per thread and
 * threads per block, as tgp_fitness_dev would choose them) -- one interpreter
 * launch over all their domains (up to 64), each domain's items carrying its
 * own grid, target and program.  This is continuous batching at launch
 * granularity: jobs that arrive while others run join the next launch, and
 * launches on different slots overlap on the device.  Domains stay resident on the
 * device between jobs (least recently used ones not in use are released when
 * the budget needs room), and so does the context's subtree cache (the
 * context's cache_budget_bytes).  A job's RMSE values do not depend on which
 * other jobs share its launch.
 * ------------------------------------------------------------------------ */
typedef struct tgp_server tgp_server;

typedef struct tgp_server_config {
    int32_t streams;           /* launch slots (CUDA streams), 1..16; 0 = 4 */
    int32_t max_batch_trees;   /* trees fused into one launch at most; 0 = 4096 (a larger job runs alone) */
    int64_t hbm_budget_bytes;  /* device memory for resident domains and admitted launches;
                                  0 = 80% of the free memory at creation */
    int64_t reserved[6];
} tgp_server_config;

/* One evaluation job: a population (as for tgp_compile_population) scored on
 * a grid (as for tgp_load_domain) against the Pagie target or one target
 * tree.  Every pointer is read during tgp_server_submit only. */
typedef struct tgp_job {
    const int32_t* ops;
    const float* imm;
    int64_t n_imm;
    const int64_t* tree_off;
    int32_t n_trees;
    int32_t order;
    int32_t W, H;
    float xlo, xhi, ylo, yhi;
    int32_t target_kind;                     /* TGP_TARGET_PAGIE or TGP_TARGET_TOKENS */
    const tgp_target_tokens* target_tokens;  /* TGP_TARGET_TOKENS only */
} tgp_job;

/* Timeline of a finished job, nanoseconds of a monotonic host clock. */
typedef struct tgp_job_info {
    int64_t submit_ns;   /* tgp_server_submit was entered (the job's arrival) */
    int64_t launch_ns;   /* its launch was enqueued */
    int64_t done_ns;     /* its RMSE values were in host memory */
    int64_t batch;       /* launch sequence number */
    int32_t batch_jobs;  /* jobs fused into that launch */
    int32_t status;      /* TGP_OK or the error of its launch */
    int64_t reserved[4];
} tgp_job_info;

typedef struct tgp_server_stats {
    int64_t submitted, completed, failed;
    int64_t batches;             /* launches */
    int64_t max_batch_jobs;
    int64_t max_in_flight;       /* most launches on the device at once */
    int64_t domains_resident;
    int64_t domains_loaded, domains_released;
    int64_t bytes_in_use;        /* resident domains + launches in flight */
    int64_t max_bytes_in_use;
    int64_t hbm_budget_bytes;
    int64_t queued;              /* jobs waiting for admission */
    int64_t worker_busy_ns;      /* host time the worker spent preparing and enqueueing launches */
    int64_t domain_load_ns;      /* part of it spent loading domains */
    int64_t max_batch_domains;   /* most domains fused into one launch */
    int64_t adopt_ns;            /* part of it registering the launches' populations with the
                                    context (their context-wide ids when the cache is on) */
    int64_t fitness_ns;          /* part of it in the fitness calls (cache view, plan, upload,
                                    launches) */
} tgp_server_stats;

/* Starts a server on ctx (a device context; the server uses it from its
 * worker thread and the caller may keep using it).  cfg may be NULL. */
int tgp_server_create(tgp_ctx* ctx, const tgp_server_config* cfg, tgp_server** out);

/* Finishes every job already submitted, then stops the worker and frees the
 * server (results not collected are dropped). */
int tgp_server_destroy(tgp_server* srv);

/* Validates and queues a job; *job_id receives its id.  TGP_E_TOKENS /
 * TGP_E_INVALID for a malformed job (nothing queued); TGP_E_BUDGET when the
 * job alone cannot fit the HBM budget. */
int tgp_server_submit(tgp_server* srv, const tgp_job* job, int64_t* job_id);

/* Waits up to timeout_us microseconds (< 0: no limit, 0: poll) for a job.
 * Done: copies its n_trees RMSE values (as tgp_fitness) into rmse_host and
 * its timeline into info (either may be NULL), forgets the job and returns
 * the job's status.  Not done in time: TGP_E_TIMEOUT, the job stays.  An
 * unknown or already collected id: TGP_E_INVALID. */
int tgp_server_wait(tgp_server* srv, int64_t job_id, int64_t timeout_us, double* rmse_host,
                    tgp_job_info* info);

int tgp_server_stats_get(tgp_server* srv, tgp_server_stats* out);

#ifdef __cplusplus
}
#endif

#endif /* TGP_H */

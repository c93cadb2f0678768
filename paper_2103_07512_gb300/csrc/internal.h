// internal.h -- what the context exposes to other translation units of the
// library (not part of the public C ABI).
#pragma once
#include <memory>
#include <mutex>
#include <vector>

#include "../../include/tgp.h"
#include "compiler.h"

namespace tgp {
namespace internal {

// A population and a domain, read under the context lock.
struct View {
    const PopIR* ir = nullptr;
    int32_t W = 0, H = 0;
    int32_t row0 = 0, H_grid = 0;    // a band of rows of a larger grid (tgp_load_domain_rows)
    float xlo = 0, xhi = 0, ylo = 0, yhi = 0;
    const float* target = nullptr;   // device target tensor, nullptr for Pagie
    const float* pagie_x = nullptr;  // Pagie: the x part per column (nullptr: formed inline)
    PlanShape shape;                 // the shape tgp_fitness would use
    int sms = 0;
    int device = 0;
    bool trig_radians = false;       // TGP_F_TRIG_RADIANS
    const ParallelFor* par = nullptr;   // the context's planning workers
};

// Locks the context into `lk`, makes its device current and fills `v`.
int view(tgp_ctx* ctx, tgp_handle pop, tgp_handle domain, std::unique_lock<std::mutex>& lk, View* v);

// tgp_load_domain_rows on `stream` (n_rows < 0: all rows from row0).  sync:
// returns after a target tree has been evaluated (as tgp_load_domain does);
// otherwise the evaluation is left in flight and every later use of the
// domain, on any stream, waits for it.
int load_domain(tgp_ctx* ctx, int32_t W, int32_t H, float xlo, float xhi, float ylo, float yhi, int32_t target_kind,
                const void* target, void* stream, bool sync, tgp_handle* domain_out, int32_t row0 = 0,
                int32_t n_rows = -1);

// A copy of a population's IR (its DAG and roots).
int population_copy(tgp_ctx* ctx, tgp_handle pop, PopIR* out);

// Whether the context simplifies populations while compiling them.
bool context_simplifies(const tgp_ctx* ctx);

// The context's CUDA device; TGP_E_INVALID for a host-only context.
int context_device(tgp_ctx* ctx, int* device);

// A host plan built ahead of the launch, for the shape the context would
// choose for its population on N points.
struct PrePlan {
    PlanShape shape;
    HostPlan plan;
};

// Builds the plan of `ir` on a grid of N points in rows of W without holding
// the context lock (only the shape choice takes it), so that callers may plan
// in their own threads.
int preplan(tgp_ctx* ctx, const PopIR& ir, int64_t N, int64_t W, std::shared_ptr<PrePlan>* out);

// Registers a population built on the host (e.g. several jobs' trees merged
// with append_population) as if it had been compiled from tokens.  `pre`, if
// given, is used by the first launch whose shape matches it.
int adopt_population(tgp_ctx* ctx, PopIR&& ir, tgp_handle* out, std::shared_ptr<PrePlan> pre = nullptr);

// Gives an existing population new trees, keeping its device buffers for the
// next plans (no allocation or free when they are large enough).  The
// population's previous launches must have completed.
int replace_population(tgp_ctx* ctx, tgp_handle pop, PopIR&& ir, std::shared_ptr<PrePlan> pre = nullptr);

// Device bytes one fitness launch of `ir` on N points in rows of W needs
// beyond its domain (partial sums, bytecode, results).
int64_t estimate_bytes(tgp_ctx* ctx, const PopIR& ir, int64_t N, int64_t W);

// One population on one domain in a fused launch: its RMSE values go to
// rmse_dev (n_trees doubles of device memory).
struct FusedSegment {
    tgp_handle pop = 0;
    tgp_handle domain = 0;
    double* rmse_dev = nullptr;
};

// The fitness of several populations, each on its own domain, as tgp_fitness_dev
// would compute them, in one interpreter launch on `stream` (preceded by the
// domains' table launches, followed by one finalize per segment).  Every
// population must plan to the same points per thread and threads per block
// on its domain; results are then bitwise those of separate calls.
// segs_dev: device memory for segs.size() SegParams; counter_dev: kQueueWords
// int32 of device memory (both the caller's, not used by concurrent launches).
int fitness_fused(tgp_ctx* ctx, const std::vector<FusedSegment>& segs, void* stream, SegParams* segs_dev,
                  int32_t* counter_dev);

// The launch shape (points per thread, threads per block) tgp_fitness_dev
// would use for `pop` on `domain`.
int launch_shape(tgp_ctx* ctx, tgp_handle pop, tgp_handle domain, int* K, int* threads);

// Records the calling thread's error message; returns `code`.
int set_error(int code, const char* fmt, ...);

}  // namespace internal
}  // namespace tgp

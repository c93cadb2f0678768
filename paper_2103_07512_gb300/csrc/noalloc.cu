// noalloc.cu -- tgp_fitness_noalloc: the fitness path without any device
// allocation.
//
// Some callers cannot call cudaMalloc: a host application that hands the
// library a device whose memory it has already reserved in full for its own
// pool, code that runs where an allocation could implicitly synchronise the
// device (cudaMalloc / cudaFree may wait for all work in flight), or a caller
// that must not touch the allocator once it has started.  For them this entry
// point keeps everything the fitness kernels need beyond their inputs and
// outputs -- the bytecode of the plan, the work-queue heads and the per-warp
// partial sums -- in one fixed array of device memory that is part of the
// library image: every GPU that loads the library holds it until the process
// exits, and no call allocates device memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/tgp.h"
#include "compiler.h"
#include "internal.h"
#include "kernels.h"

namespace tgp {
namespace {

// The fixed scratch (TGP_NOALLOC_SCRATCH_BYTES, 8 MiB).  In host code its name
// is only a host-side stand-in: kernels are given the device address that
// cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) unsigned char g_scratch[TGP_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_scratch on `device` (which must be current).  Looked up
// once per device, on the first call there.
int scratch_address(int device, unsigned char** out) {
    if (device < 0 || device >= kMaxDevices)
        return internal::set_error(TGP_E_INVALID, "device %d out of range for the fixed scratch", device);
    std::lock_guard<std::mutex> g(g_addr_mu);
    if (!g_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess)
            return internal::set_error(TGP_E_CUDA, "cudaGetSymbolAddress of the fixed scratch failed: %s",
                                       cudaGetErrorString(e));
        g_addr[device] = p;
    }
    *out = static_cast<unsigned char*>(g_addr[device]);
    return TGP_OK;
}

size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

}  // namespace
}  // namespace tgp

using namespace tgp;

extern "C" int tgp_fitness_noalloc(tgp_ctx* ctx, tgp_handle pop, tgp_handle domain, void* stream,
                                   double* rmse_dev) {
    if (!ctx || !rmse_dev) return internal::set_error(TGP_E_INVALID, "ctx / rmse_dev is NULL");
    std::unique_lock<std::mutex> lk;
    internal::View v;
    int rc = internal::view(ctx, pop, domain, lk, &v);
    if (rc) return rc;
    const int64_t T = (int64_t)v.ir->roots.size();
    if (T == 0) return TGP_OK;

    // host-side plan (host memory only)
    HostPlan hp;
    build_plan(*v.ir, v.shape, hp, nullptr, v.par);
    const int warps = hp.shape.threads / 32;
    const size_t n_partial = (size_t)T * hp.n_tiles * warps;
    const size_t off_counter = 0;
    const int Q = std::max(1, std::min(v.sms, kMaxQueues));   // work queues, one per SM
    const size_t off_code = align256(kQueueWords * sizeof(int32_t));
    const size_t off_goff = off_code + align256(hp.code.size() * sizeof(Ins));
    const size_t off_gord = off_goff + align256(hp.code_off.size() * sizeof(int64_t));
    const size_t off_part = off_gord + align256(hp.group_order.size() * sizeof(int32_t));
    const size_t need = off_part + n_partial * sizeof(float);
    if (need > (size_t)TGP_NOALLOC_SCRATCH_BYTES)
        return internal::set_error(TGP_E_INVALID,
                                   "population needs %zu bytes of scratch for %lld trees on %lld points; "
                                   "the fixed scratch of tgp_fitness_noalloc holds %d bytes",
                                   need, (long long)T, (long long)hp.shape.N, (int)TGP_NOALLOC_SCRATCH_BYTES);

    unsigned char* base = nullptr;
    rc = scratch_address(v.device, &base);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    int32_t* counter = reinterpret_cast<int32_t*>(base + off_counter);
    Ins* code = reinterpret_cast<Ins*>(base + off_code);
    int64_t* goff = reinterpret_cast<int64_t*>(base + off_goff);
    int32_t* gord = reinterpret_cast<int32_t*>(base + off_gord);
    float* partial = reinterpret_cast<float*>(base + off_part);

#define NA_TRY(call)                                                                              \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return internal::set_error(TGP_E_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

    // The array keeps the previous call's contents: the queue heads must start
    // at zero; code and offsets are overwritten; every partial the finalize
    // reads is written by this launch.  Copies from pageable host memory
    // return once staged, so the host plan may go out of scope afterwards.
    NA_TRY(cudaMemsetAsync(counter, 0, kQueueWords * sizeof(int32_t), s));
    NA_TRY(cudaMemcpyAsync(code, hp.code.data(), hp.code.size() * sizeof(Ins), cudaMemcpyHostToDevice, s));
    NA_TRY(cudaMemcpyAsync(goff, hp.code_off.data(), hp.code_off.size() * sizeof(int64_t),
                           cudaMemcpyHostToDevice, s));
    NA_TRY(cudaMemcpyAsync(gord, hp.group_order.data(), hp.group_order.size() * sizeof(int32_t),
                           cudaMemcpyHostToDevice, s));

    const size_t smem = eval_smem_bytes(hp.shape.K, hp.shape.threads, hp.n_slots);
    int bps = 0;
    NA_TRY(eval_occupancy(hp.shape.K, false, hp.ext || v.trig_radians, hp.shape.threads, smem, &bps));
    if (bps <= 0) return internal::set_error(TGP_E_INVALID, "interpreter cannot be resident with this plan");
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(hp.n_items, (int64_t)bps * std::max(v.sms, 1)));

    EvalParams p{};
    p.code = code;
    p.group_off = goff;
    p.item_group = gord;
    p.n_items = hp.n_items;
    p.n_tiles = hp.n_tiles;
    p.warps_per_tile = warps;
    p.N = (int64_t)v.W * v.H;
    p.W = v.W;
    p.H = v.H;
    p.row0 = v.row0;
    p.H_grid = v.H_grid;
    p.xlo = v.xlo;
    p.xhi = v.xhi;
    p.ylo = v.ylo;
    p.yhi = v.yhi;
    p.target = v.target;
    p.pagie_x = v.pagie_x;
    p.partial = partial;
    p.out = nullptr;
    p.cache = nullptr;
    p.counter = counter;
    p.n_queues = Q;
    p.local_items = queue_local_items(hp.n_items, Q);
    p.n_slots = hp.n_slots;
    p.max_items_per_cta = (int32_t)std::min<int64_t>(hp.n_items, INT32_MAX);
    p.trig_rad = v.trig_radians ? 1 : 0;
    p.out_stride = p.N;
    NA_TRY(launch_eval(p, hp.shape.K, false, hp.ext || v.trig_radians, grid, hp.shape.threads, smem, s));

    FinalizeParams f{};
    f.partial = partial;
    f.per_tree = (int64_t)hp.n_tiles * warps;
    f.n_trees = (int32_t)T;
    f.n_points = (double)p.N;
    f.rmse = rmse_dev;
    NA_TRY(launch_finalize(f, s));
#undef NA_TRY
    return TGP_OK;
}

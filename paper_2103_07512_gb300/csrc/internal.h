// internal.h -- what the context exposes to other translation units of the
// library (not part of the public C ABI).
#pragma once
#include <mutex>

#include "../../include/tgp.h"
#include "compiler.h"

namespace tgp {
namespace internal {

// A population and a domain, read under the context lock.
struct View {
    const PopIR* ir = nullptr;
    int32_t W = 0, H = 0;
    float xlo = 0, xhi = 0, ylo = 0, yhi = 0;
    const float* target = nullptr;   // device target tensor, nullptr for Pagie
    PlanShape shape;                 // the shape tgp_fitness would use
    int sms = 0;
    int device = 0;
};

// Locks the context into `lk`, makes its device current and fills `v`.
int view(tgp_ctx* ctx, tgp_handle pop, tgp_handle domain, std::unique_lock<std::mutex>& lk, View* v);

// Records the calling thread's error message; returns `code`.
int set_error(int code, const char* fmt, ...);

}  // namespace internal
}  // namespace tgp

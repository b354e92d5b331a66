// runtime.cu -- host-side services shared by the library: device allocation (with the
// fault injection used by the tests) and NVTX trace ranges.
#include <atomic>

#include <nvtx3/nvToolsExt.h>

#include "lbm_internal.h"

namespace lbm {
namespace {
// allocations left before injected failures start; negative: no injection
std::atomic<long long> g_alloc_budget{-1};
}  // namespace

void set_alloc_budget(long long n) { g_alloc_budget.store(n < 0 ? -1 : n); }

cudaError_t dev_alloc(void **p, size_t bytes)
{
    long long b = g_alloc_budget.load();
    while (b >= 0) {
        if (b == 0) {
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
        if (g_alloc_budget.compare_exchange_weak(b, b - 1)) break;
    }
    return cudaMalloc(p, bytes);
}

TraceRange::TraceRange(const char *name) { nvtxRangePushA(name); }
TraceRange::~TraceRange() { nvtxRangePop(); }

}  // namespace lbm

extern "C" void lbm_debug_fail_alloc_after(int64_t n) { lbm::set_alloc_budget((long long)n); }

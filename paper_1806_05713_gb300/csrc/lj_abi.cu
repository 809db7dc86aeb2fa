// lj_abi.cu -- status codes, error text and shared host-side checks of the
// C ABI declared in lj_gb300.h.
#include <atomic>
#include <cmath>
#include <cstdio>

#include "lj_internal.cuh"

namespace lj {

namespace {
thread_local char g_cuda_error[256] = "no CUDA error";
std::atomic<unsigned long long> g_launches{0};
}

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void record_cuda_error(cudaError_t err, const char *where)
{
    std::snprintf(g_cuda_error, sizeof(g_cuda_error), "%s: %s (%d) in %s", cudaGetErrorName(err),
                  cudaGetErrorString(err), static_cast<int>(err), where ? where : "?");
}

int check_box(const double box[3], double r_search)
{
    if (!box) return LJ_ERR_ARG;
    for (int a = 0; a < 3; ++a) {
        if (!std::isfinite(box[a]) || !(box[a] > 0.0)) return LJ_ERR_BOX;
        if (box[a] < 2.0 * r_search) return LJ_ERR_BOX;
    }
    return LJ_OK;
}

}  // namespace lj

extern "C" const char *lj_status_string(int status)
{
    switch (status) {
        case LJ_OK: return "LJ_OK: success";
        case LJ_ERR_ARG: return "LJ_ERR_ARG: invalid argument";
        case LJ_ERR_BOX: return "LJ_ERR_BOX: a box side is shorter than twice the search length";
        case LJ_ERR_RANGE: return "LJ_ERR_RANGE: a position is outside [0, L) or not finite";
        case LJ_ERR_CAPACITY: return "LJ_ERR_CAPACITY: output or workspace too small";
        case LJ_ERR_CUDA: return "LJ_ERR_CUDA: a CUDA runtime call failed";
        case LJ_ERR_DEVICE: return "LJ_ERR_DEVICE: no usable sm_103 device";
        default: return "unknown LJ status";
    }
}

extern "C" const char *lj_last_cuda_error(void) { return lj::g_cuda_error; }

extern "C" int lj_version(void) { return 1 * 10000 + 0 * 100 + 0; }

extern "C" unsigned long long lj_kernel_launch_count(void)
{
    return lj::g_launches.load(std::memory_order_relaxed);
}

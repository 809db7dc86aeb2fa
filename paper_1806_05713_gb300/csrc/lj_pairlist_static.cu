// lj_pairlist_static.cu -- a variant of lj_build_pairlist that allocates
// nothing, for callers that cannot call cudaMalloc.
//
// Some callers cannot allocate device memory at all: code running inside a
// framework that owns every allocation, a host thread that must not touch
// the allocator while a stream is being captured or replayed, or a plugin
// whose host never gives it a workspace.  lj_build_pairlist needs a scratch
// buffer (cell counts and starts, the atoms in cell order, row counts, scan
// partial sums).  This entry point takes that scratch from one array of
// fixed size in the library's own device memory instead of from the caller.
//
// The array is a file-scope __device__ object, so every GPU that loads the
// library holds it until the process exits.  Host code cannot use its name
// as a device address (in host code the name denotes a host-side shadow), so
// the first call on each device looks the address up with
// cudaGetSymbolAddress, with that device current, and caches it.  That first
// call should therefore come before any stream capture.  All calls share the
// one array: calls whose GPU work overlaps (on different streams or host
// threads) race on it and must be serialised by the caller: the array stays
// in use until the call's work on its stream has completed, which is after
// the call returns (the last kernels still read it), so order a second call
// after the first through that stream or an event, not by host order alone.
// Everything the builder needs zeroed is cleared at the start of each call.
// The builder is handed exactly the two-walk workspace (count, scan, fill),
// so this entry point never takes the one-walk path with its row slabs and
// never creates or uses a side stream: every operation it enqueues goes on
// the caller's stream.
#include <mutex>

#include "lj_internal.cuh"

namespace lj {
int build_pairlist_impl(const double *q4, int64_t n, const double box[3], double rs, int half,
                        int32_t *row_ptr, int32_t *col, int64_t cap, void *ws, size_t ws_bytes,
                        int64_t *nnz_out, int64_t *max_row_out, cudaStream_t st);
size_t pairlist_workspace_bytes_min_impl(int64_t n, const double box[3], double rs);
}  // namespace lj

static __device__ __align__(256) unsigned char lj_static_scratch[LJ_STATIC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void *g_static_addr[kMaxDevices] = {};
}  // namespace

extern "C" int lj_build_pairlist_static(const double *q4_dev, int64_t n, const double box[3],
                                        double r_search, int half, int32_t *row_ptr_dev,
                                        int32_t *col_dev, int64_t col_capacity, int64_t *nnz_out,
                                        int64_t *max_row_out, void *stream)
{
    if (nnz_out) *nnz_out = 0;
    if (max_row_out) *max_row_out = 0;
    if (n < 0 || !box || !nnz_out) return LJ_ERR_ARG;
    if (n > LJ_STATIC_MAX_ATOMS) return LJ_ERR_CAPACITY;
    // the builder's two-walk path (no row slabs) fits the static scratch
    const size_t need = lj::pairlist_workspace_bytes_min_impl(n, box, r_search);
    if (need > LJ_STATIC_SCRATCH_BYTES) return LJ_ERR_CAPACITY;
    int dev = 0;
    LJ_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return LJ_ERR_DEVICE;
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_static_mu);
        if (!g_static_addr[dev]) {
            void *p = nullptr;
            LJ_TRY_CUDA(cudaGetSymbolAddress(&p, lj_static_scratch));
            g_static_addr[dev] = p;
        }
        scratch = g_static_addr[dev];
    }
    // `need` bytes (not the whole array): the builder then takes its two-walk
    // path, which has no row slabs and no side stream.
    return lj::build_pairlist_impl(q4_dev, n, box, r_search, half, row_ptr_dev, col_dev,
                                   col_capacity, scratch, need, nnz_out, max_row_out,
                                   static_cast<cudaStream_t>(stream));
}

// lj_batched.cu -- many independent LJ systems of uneven size in one
// persistent launch, and the autotuners.
//
// Each system is its own instance of the paper's method (Algorithm 3 over
// its own sorted list, Algorithm 1 per pair); a GPU kernel per system would
// leave most of the 152 SMs idle for the small ones and pay one launch
// each.  Here the rows of all systems are cut into work items of at most
// rows_per_item rows of one system; a grid of as many blocks as fit on the
// GPU at once pulls items from a counter (one atomic per item per warp)
// until none is left, with the items ordered longest first.  Per-system
// constants (box, cutoff, dt, eps, sigma, list kind, array offsets) live in
// a device plan written once by lj_batch_init, so a call enqueues only a
// memset and kernels -- no host synchronisation, no allocation -- and can be
// captured in a CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "lj_dfloat.cuh"
#include "lj_fixed.cuh"
#include "lj_rows.cuh"

namespace lj {
namespace {

constexpr int kBatchThreads = 256;

struct SysDev {
    long long atom_off, row_off, entry_off;
    int n, half, cubic, fixed;
    Fp64Params fp;
    FixParams fx;
    MixedParams mp;
    DfParams dp;
};

// Arithmetic form of a batched launch (lj_batch.precision).
enum Form { kFp64 = LJ_FP64, kMixed = LJ_MIXED, kDfloat = LJ_DFLOAT };

struct Item {
    int sys;
    int row_begin;
    int row_end;
    int pad;
};

struct PlanView {
    SysDev *sys;
    Item *items;
};

PlanView plan_view(void *base, int nsys)
{
    Carver c(base);
    PlanView v;
    v.sys = c.take<SysDev>(size_t(nsys));
    v.items = c.take<Item>(0);
    return v;
}

size_t plan_bytes_for(int nsys, long long nitems)
{
    Carver c(nullptr);
    c.take<SysDev>(size_t(nsys));
    c.take<Item>(size_t(nitems));
    return c.used + 256;
}

long long count_items(const lj_system *systems, int nsys, int rpi)
{
    long long items = 0;
    for (int s = 0; s < nsys; ++s) items += (systems[s].n + rpi - 1) / rpi;
    return items;
}

// Per-atom fixed-point positions of every system (MIXED form): one block
// per work item, one thread per row of the item.
__global__ void batched_prepass_kernel(const SysDev *__restrict__ sys, const Item *__restrict__ items,
                                       const double *__restrict__ q4, uint4 *__restrict__ rel)
{
    const Item it = items[blockIdx.x];
    const SysDev &S = sys[it.sys];
    for (int r = it.row_begin + threadIdx.x; r < it.row_end; r += blockDim.x) {
        const long long a = S.atom_off + r;
        double x[3];
        load_xyz(q4, a, x[0], x[1], x[2]);
        rel[a] = make_uint4(__double2uint_rz(x[0] * S.mp.to_fixed[0]),
                            __double2uint_rz(x[1] * S.mp.to_fixed[1]),
                            __double2uint_rz(x[2] * S.mp.to_fixed[2]), 0u);
    }
}

// Double-float records of every system (DFLOAT form), as dfloat_prepass_kernel.
__global__ void batched_df_prepass_kernel(const SysDev *__restrict__ sys, const Item *__restrict__ items,
                                          const double *__restrict__ q4, DfRec *__restrict__ rec)
{
    const Item it = items[blockIdx.x];
    const SysDev &S = sys[it.sys];
    for (int r = it.row_begin + threadIdx.x; r < it.row_end; r += blockDim.x) {
        const long long a = S.atom_off + r;
        double x[3];
        load_xyz(q4, a, x[0], x[1], x[2]);
        rec[a] = make_rec(x, S.dp);
    }
}

// 64-bit fixed-point positions of every system (FP64 form).
__global__ void batched_fixed_prepass_kernel(const SysDev *__restrict__ sys,
                                             const Item *__restrict__ items,
                                             const double *__restrict__ q4, longlong4 *__restrict__ X)
{
    const Item it = items[blockIdx.x];
    const SysDev &S = sys[it.sys];
    for (int r = it.row_begin + threadIdx.x; r < it.row_end; r += blockDim.x) {
        const long long a = S.atom_off + r;
        double x, y, z;
        load_xyz(q4, a, x, y, z);
        X[a] = make_longlong4(__double2ll_rn(x * S.fx.scale), __double2ll_rn(y * S.fx.scale),
                              __double2ll_rn(z * S.fx.scale), 0);
    }
}

// rel: MIXED fixed-point positions; rec: DFLOAT records; X: FP64 fixed-point
// positions (each indexed by the batch-wide atom number).
// CUBIC (DFLOAT only): every system of the batch has a cubic box; otherwise
// the displacement is scaled per axis (by 1 on the cubic systems).
// FP64, lj_batch.tpi = LJ_SCHED_STREAM: the warp cuts the entries of its work
// item's rows into one chunk per lane (fp64_fixed_stream).  Four 256-thread
// blocks per SM (64 registers) run it 2-3 % faster than three (80).
__global__ void __launch_bounds__(kBatchThreads, 4)
batched_stream_kernel(const SysDev *__restrict__ sys, const Item *__restrict__ items,
                      long long nitems, const double *__restrict__ q4,
                      const longlong4 *__restrict__ X, double *__restrict__ p4,
                      const int *__restrict__ row_ptr, const int *__restrict__ col,
                      unsigned long long *__restrict__ counter)
{
    const int lane = threadIdx.x & 31;
    while (true) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(counter, 1ull);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= static_cast<unsigned long long>(nitems)) break;
        const Item I = items[it];
        const SysDev &S = sys[I.sys];
        const double *sq = q4 + 4 * S.atom_off;
        double *sp = p4 + 4 * S.atom_off;
        const int *srp = row_ptr + S.row_off;
        const int *scol = col + S.entry_off;
        const Fp64Params &P = S.fp;
        if (S.fixed) {
            const longlong4 *sX = X + S.atom_off;
            if (S.half)
                fp64_fixed_stream<true>(sq, sX, sp, srp, scol, I.row_begin, I.row_end, P, S.fx);
            else
                fp64_fixed_stream<false>(sq, sX, sp, srp, scol, I.row_begin, I.row_end, P, S.fx);
        } else {  // a box wider than 1024 r_c: image-selected rows, 8 lanes each
            for (int r0 = I.row_begin; r0 < I.row_end; r0 += 4) {
                const int r = r0 + lane / 8;
                if (r < I.row_end) {
                    if (S.half)
                        fp64_row<8, true, 1, true>(sq, sp, srp, scol, r, P, group_mask<8>());
                    else
                        fp64_row<8, false, 1, true>(sq, sp, srp, scol, r, P, group_mask<8>());
                }
            }
        }
    }
}

template <int TPI, int FORM, bool CUBIC>
__global__ void __launch_bounds__(kBatchThreads)
batched_force_kernel(const SysDev *__restrict__ sys, const Item *__restrict__ items,
                     long long nitems, const double *__restrict__ q4, const uint4 *__restrict__ rel,
                     const DfRec *__restrict__ rec, const longlong4 *__restrict__ X,
                     double *__restrict__ p4,
                     const int *__restrict__ row_ptr, const int *__restrict__ col,
                     unsigned long long *__restrict__ counter)
{
    const int lane = threadIdx.x & 31;
    const unsigned gm = group_mask<TPI>();
    constexpr int kGroups = 32 / TPI;
    while (true) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(counter, 1ull);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= static_cast<unsigned long long>(nitems)) break;
        const Item I = items[it];
        const SysDev &S = sys[I.sys];
        const double *sq = q4 + 4 * S.atom_off;
        double *sp = p4 + 4 * S.atom_off;
        const int *srp = row_ptr + S.row_off;
        const int *scol = col + S.entry_off;
        const bool half = S.half != 0;
        for (int r0 = I.row_begin; r0 < I.row_end; r0 += kGroups) {
            const int r = r0 + lane / TPI;
            if (r < I.row_end) {  // uniform within a group
                if (FORM == kDfloat) {
                    const DfRec *srec = rec + S.atom_off;
                    const DfParams &P = S.dp;  // fields read where used
                    if (half)
                        dfloat_row2<TPI, true, CUBIC>(sq, srec, sp, srp, scol, r, P, gm);
                    else
                        dfloat_row2<TPI, false, CUBIC>(sq, srec, sp, srp, scol, r, P, gm);
                } else if (FORM == kMixed) {
                    const uint4 *srel = rel + S.atom_off;
                    const MixedParams &P = S.mp;
                    if (half)
                        mixed_row_pf<TPI, true, 1>(sq, srel, sp, srp, scol, r, P);
                    else
                        mixed_row_pf<TPI, false, 1>(sq, srel, sp, srp, scol, r, P);
                } else {
                    const longlong4 *sX = X + S.atom_off;
                    const Fp64Params &P = S.fp;
                    const FixParams &F = S.fx;
                    if (S.fixed) {
                        if (half)
                            fp64_fixed_row<TPI, true>(sq, sX, sp, srp, scol, r, P, F, gm);
                        else
                            fp64_fixed_row<TPI, false>(sq, sX, sp, srp, scol, r, P, F, gm);
                    } else {  // a box wider than 1024 r_c
                        if (half)
                            fp64_row<TPI, true, 1, true>(sq, sp, srp, scol, r, P, gm);
                        else
                            fp64_row<TPI, false, 1, true>(sq, sp, srp, scol, r, P, gm);
                    }
                }
            }
        }
    }
}

template <int FORM, bool CUBIC>
int launch_batched(const lj_batch *b, const PlanView &v, const double *q4, const uint4 *rel,
                   const DfRec *rec, const longlong4 *X, double *p4, const int *rp, const int *col,
                   unsigned long long *counter, cudaStream_t st)
{
    const long long ni = b->nitems;
    const int grid = b->blocks;
#define LJ_BATCH_CASE(T)                                                                        \
    case T:                                                                                     \
        batched_force_kernel<T, FORM, CUBIC><<<grid, kBatchThreads, 0, st>>>(v.sys, v.items, ni, q4, \
                                                               rel, rec, X, p4, rp, col, counter); \
        break;
    if (b->tpi == LJ_SCHED_STREAM) {
        if constexpr (FORM == kFp64) {
            batched_stream_kernel<<<grid, kBatchThreads, 0, st>>>(v.sys, v.items, ni, q4, X, p4,
                                                                   rp, col, counter);
            LJ_TRY_LAUNCH("batched_stream_kernel");
            return LJ_OK;
        }
        return LJ_ERR_ARG;
    }
    switch (b->tpi) {
        LJ_BATCH_CASE(1)
        LJ_BATCH_CASE(2)
        LJ_BATCH_CASE(4)
        LJ_BATCH_CASE(8)
        LJ_BATCH_CASE(16)
        LJ_BATCH_CASE(32)
        default: return LJ_ERR_ARG;
    }
#undef LJ_BATCH_CASE
    LJ_TRY_LAUNCH("batched_force_kernel");
    return LJ_OK;
}

template <int FORM, bool CUBIC>
int persistent_blocks(int tpi)
{
    int per_sm = 0;
    cudaError_t e = cudaErrorInvalidValue;
#define LJ_OCC(T)                                                                                 \
    case T:                                                                                       \
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_force_kernel<T, FORM, CUBIC>, \
                                                          kBatchThreads, 0);                      \
        break;
    if (tpi == LJ_SCHED_STREAM) {
        if constexpr (FORM == kFp64)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_stream_kernel,
                                                               kBatchThreads, 0);
    }
    switch (tpi) {
        LJ_OCC(1)
        LJ_OCC(2)
        LJ_OCC(4)
        LJ_OCC(8)
        LJ_OCC(16)
        LJ_OCC(32)
        default: break;
    }
#undef LJ_OCC
    if (e != cudaSuccess || per_sm < 1) per_sm = 4;
    return per_sm * num_sms();
}

bool valid_tpi(int t, int precision)
{
    if (t == LJ_SCHED_STREAM) return precision == LJ_FP64;
    if (precision == LJ_DFLOAT) return t == 4 || t == 8 || t == 16;
    return t == 1 || t == 2 || t == 4 || t == 8 || t == 16 || t == 32;
}

}  // namespace

int check_force_args(const double *q4, const double *p4, int64_t n, const int32_t *row_ptr,
                     const int32_t *col, int64_t nnz, double r_cut, const double box[3], double eps,
                     double sigma, double dt);

}  // namespace lj

extern "C" size_t lj_batch_plan_bytes(const lj_system *systems, int nsys, int rows_per_item)
{
    if (!systems || nsys <= 0 || rows_per_item < 1) return 0;
    return lj::plan_bytes_for(nsys, lj::count_items(systems, nsys, rows_per_item));
}

extern "C" int lj_batch_init(lj_batch *batch, const lj_system *systems, int nsys, double dt,
                             int precision, int tpi, int rows_per_item, void *plan_dev,
                             size_t plan_bytes, void *stream)
{
    using namespace lj;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!batch || !systems || nsys <= 0 || rows_per_item < 1 || !plan_dev) return LJ_ERR_ARG;
    if (precision != LJ_FP64 && precision != LJ_MIXED && precision != LJ_DFLOAT) return LJ_ERR_ARG;
    if (!valid_tpi(tpi, precision)) return LJ_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(plan_dev) & 255u) return LJ_ERR_ARG;
    long long total_atoms = 0;
    std::vector<SysDev> host_sys(static_cast<size_t>(nsys));
    for (int s = 0; s < nsys; ++s) {
        const lj_system &y = systems[s];
        if (y.n < 0 || y.nnz < 0 || y.atom_offset < 0 || y.row_offset < 0 || y.entry_offset < 0)
            return LJ_ERR_ARG;
        if (y.n >= (int64_t(1) << 31) - 1) return LJ_ERR_CAPACITY;
        if (tpi == LJ_SCHED_STREAM && y.nnz > kStreamMaxEntries) return LJ_ERR_CAPACITY;
        const double *fake = reinterpret_cast<const double *>(256);
        const int32_t *fakei = reinterpret_cast<const int32_t *>(256);
        const int rc = check_force_args(fake, fake, y.n, fakei, fakei, y.nnz, y.r_cut, y.box, y.eps,
                                        y.sigma, dt);
        if (rc != LJ_OK) return rc;
        SysDev &d = host_sys[size_t(s)];
        d.atom_off = y.atom_offset;
        d.row_off = y.row_offset;
        d.entry_off = y.entry_offset;
        d.n = static_cast<int>(y.n);
        d.half = y.half ? 1 : 0;
        d.fp = make_fp64_params(y.box, dt, y.r_cut, y.eps, y.sigma);
        d.fx = make_fix_params(y.box);
        d.fixed = fixed_point_ok(y.box, y.r_cut) ? 1 : 0;
        d.mp = make_mixed_params(y.box, dt, y.r_cut, y.eps, y.sigma);
        d.dp = make_dfloat_params(y.box, dt, y.r_cut, y.eps, y.sigma);
        d.cubic = y.box[1] == y.box[0] && y.box[2] == y.box[0];
        if (precision == LJ_DFLOAT && (d.dp.k_exp < -700 || d.dp.k_exp > 700)) return LJ_ERR_ARG;
        total_atoms = std::max<long long>(total_atoms, y.atom_offset + y.n);
    }
    // Work items, longest (estimated entries) first.
    struct HostItem {
        Item it;
        double cost;
    };
    std::vector<HostItem> items;
    items.reserve(size_t(count_items(systems, nsys, rows_per_item)));
    for (int s = 0; s < nsys; ++s) {
        const double per_row = systems[s].n > 0 ? double(systems[s].nnz) / double(systems[s].n) : 0.0;
        for (long long r = 0; r < systems[s].n; r += rows_per_item) {
            const int e = static_cast<int>(std::min<long long>(systems[s].n, r + rows_per_item));
            items.push_back({{s, static_cast<int>(r), e, 0}, per_row * double(e - r)});
        }
    }
    std::stable_sort(items.begin(), items.end(),
                     [](const HostItem &a, const HostItem &b) { return a.cost > b.cost; });
    const size_t need = plan_bytes_for(nsys, static_cast<long long>(items.size()));
    if (plan_bytes < need) return LJ_ERR_CAPACITY;
    std::vector<char> host(need, 0);
    PlanView hv = plan_view(host.data(), nsys);
    std::memcpy(hv.sys, host_sys.data(), sizeof(SysDev) * host_sys.size());
    for (size_t k = 0; k < items.size(); ++k) hv.items[k] = items[k].it;
    LJ_TRY_CUDA(cudaMemcpyAsync(plan_dev, host.data(), need, cudaMemcpyHostToDevice, st));
    LJ_TRY_CUDA(cudaStreamSynchronize(st));
    batch->plan_dev = plan_dev;
    batch->plan_bytes = plan_bytes;
    batch->nitems = static_cast<int64_t>(items.size());
    batch->total_atoms = total_atoms;
    batch->dt = dt;
    batch->nsys = nsys;
    batch->precision = precision;
    batch->tpi = tpi;
    batch->rows_per_item = rows_per_item;
    bool all_cubic = true;
    for (int s = 0; s < nsys; ++s) all_cubic = all_cubic && host_sys[size_t(s)].cubic;
    batch->flags = all_cubic ? 1 : 0;
    batch->blocks = precision == LJ_MIXED    ? persistent_blocks<kMixed, true>(tpi)
                    : precision == LJ_DFLOAT ? (all_cubic ? persistent_blocks<kDfloat, true>(tpi)
                                                          : persistent_blocks<kDfloat, false>(tpi))
                                             : persistent_blocks<kFp64, true>(tpi);
    return LJ_OK;
}

extern "C" size_t lj_force_batched_workspace_bytes(const lj_batch *batch)
{
    if (!batch) return 0;
    size_t bytes = 256;
    if (batch->precision == LJ_MIXED) bytes += size_t(batch->total_atoms) * sizeof(uint4) + 256;
    if (batch->precision == LJ_DFLOAT) bytes += size_t(batch->total_atoms) * sizeof(lj::DfRec) + 256;
    if (batch->precision == LJ_FP64) bytes += size_t(batch->total_atoms) * sizeof(longlong4) + 256;
    return bytes;
}

extern "C" int lj_force_batched(const lj_batch *batch, const double *q4_dev, double *p4_dev,
                                const int32_t *row_ptr_dev, const int32_t *col_dev,
                                void *workspace_dev, size_t workspace_bytes, void *stream)
{
    using namespace lj;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!batch || !batch->plan_dev || !q4_dev || !p4_dev || !row_ptr_dev) return LJ_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(q4_dev) | reinterpret_cast<uintptr_t>(p4_dev)) & 31u)
        return LJ_ERR_ARG;
    if (!workspace_dev || workspace_bytes < lj_force_batched_workspace_bytes(batch))
        return LJ_ERR_CAPACITY;
    if (batch->nitems == 0) return LJ_OK;
    const PlanView v = plan_view(batch->plan_dev, batch->nsys);
    Carver c(workspace_dev);
    unsigned long long *counter = c.take<unsigned long long>(1);
    LJ_TRY_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st));
    if (batch->precision == LJ_MIXED) {
        uint4 *rel = c.take<uint4>(size_t(batch->total_atoms));
        batched_prepass_kernel<<<unsigned(batch->nitems), 128, 0, st>>>(v.sys, v.items, q4_dev, rel);
        LJ_TRY_LAUNCH("batched_prepass_kernel");
        return launch_batched<kMixed, true>(batch, v, q4_dev, rel, nullptr, nullptr, p4_dev,
                                            row_ptr_dev, col_dev, counter, st);
    }
    if (batch->precision == LJ_DFLOAT) {
        DfRec *rec = c.take<DfRec>(size_t(batch->total_atoms));
        batched_df_prepass_kernel<<<unsigned(batch->nitems), 128, 0, st>>>(v.sys, v.items, q4_dev, rec);
        LJ_TRY_LAUNCH("batched_df_prepass_kernel");
        if (batch->flags & 1)
            return launch_batched<kDfloat, true>(batch, v, q4_dev, nullptr, rec, nullptr, p4_dev,
                                                 row_ptr_dev, col_dev, counter, st);
        return launch_batched<kDfloat, false>(batch, v, q4_dev, nullptr, rec, nullptr, p4_dev,
                                              row_ptr_dev, col_dev, counter, st);
    }
    longlong4 *X = c.take<longlong4>(size_t(batch->total_atoms));
    batched_fixed_prepass_kernel<<<unsigned(batch->nitems), 128, 0, st>>>(v.sys, v.items, q4_dev, X);
    LJ_TRY_LAUNCH("batched_fixed_prepass_kernel");
    return launch_batched<kFp64, true>(batch, v, q4_dev, nullptr, nullptr, X, p4_dev, row_ptr_dev,
                                       col_dev, counter, st);
}

// ---------------------------------------------------------------------------
// Autotuners
// ---------------------------------------------------------------------------

namespace {

struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    ~EventPair()
    {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

template <class F>
int time_median(F launch, int reps, cudaStream_t st, float *ms_out)
{
    EventPair ev;
    LJ_TRY_CUDA(cudaEventCreate(&ev.a));
    LJ_TRY_CUDA(cudaEventCreate(&ev.b));
    int rc = launch();  // warm-up
    if (rc != LJ_OK) return rc;
    std::vector<float> t;
    for (int r = 0; r < std::max(1, reps); ++r) {
        LJ_TRY_CUDA(cudaEventRecord(ev.a, st));
        rc = launch();
        if (rc != LJ_OK) return rc;
        LJ_TRY_CUDA(cudaEventRecord(ev.b, st));
        LJ_TRY_CUDA(cudaEventSynchronize(ev.b));
        float ms = 0.f;
        LJ_TRY_CUDA(cudaEventElapsedTime(&ms, ev.a, ev.b));
        t.push_back(ms);
    }
    std::sort(t.begin(), t.end());
    *ms_out = t[t.size() / 2];
    return LJ_OK;
}

}  // namespace

extern "C" int lj_autotune_force(const double *q4_dev, double *p4_scratch_dev, int64_t n,
                                 const int32_t *row_ptr_dev, const int32_t *col_dev, int64_t nnz,
                                 int half, double dt, double r_cut, const double box[3], double eps,
                                 double sigma, int precision, const int *tpis, int n_tpi, int reps,
                                 void *workspace_dev, size_t workspace_bytes, int *best_tpi,
                                 float *best_ms, float *ms_out, void *stream)
{
    using namespace lj;
    if (!tpis || n_tpi <= 0 || !best_tpi || !best_ms) return LJ_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    *best_tpi = 0;
    *best_ms = INFINITY;
    for (int c = 0; c < n_tpi; ++c) {
        float ms = INFINITY;
        const int t = tpis[c];
        int rc = time_median(
            [&]() {
                return lj_force(q4_dev, p4_scratch_dev, n, row_ptr_dev, col_dev, nnz, half, dt,
                                r_cut, box, eps, sigma, precision, t, workspace_dev, workspace_bytes,
                                stream);
            },
            reps, st, &ms);
        if (rc == LJ_ERR_ARG) ms = INFINITY;  // schedule not offered for this precision
        else if (rc != LJ_OK) return rc;
        if (ms_out) ms_out[c] = ms;
        if (ms < *best_ms) {
            *best_ms = ms;
            *best_tpi = t;
        }
    }
    return *best_tpi ? LJ_OK : LJ_ERR_ARG;
}

extern "C" int lj_autotune_batched(const lj_system *systems, int nsys, double dt, int precision,
                                   const int *tpis, int n_tpi, const int *rows_per_item, int n_rpi,
                                   const double *q4_dev, double *p4_scratch_dev,
                                   const int32_t *row_ptr_dev, const int32_t *col_dev,
                                   void *plan_dev, size_t plan_bytes, void *workspace_dev,
                                   size_t workspace_bytes, int reps, int *best_tpi,
                                   int *best_rows_per_item, float *best_ms, void *stream)
{
    using namespace lj;
    if (!tpis || n_tpi <= 0 || !rows_per_item || n_rpi <= 0 || !best_tpi || !best_rows_per_item ||
        !best_ms)
        return LJ_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    *best_tpi = 0;
    *best_rows_per_item = 0;
    *best_ms = INFINITY;
    for (int a = 0; a < n_tpi; ++a) {
        if (!valid_tpi(tpis[a], precision)) continue;  // not offered for this form
        for (int b = 0; b < n_rpi; ++b) {
            lj_batch batch{};
            int rc = lj_batch_init(&batch, systems, nsys, dt, precision, tpis[a], rows_per_item[b],
                                   plan_dev, plan_bytes, stream);
            if (rc != LJ_OK) return rc;
            float ms = INFINITY;
            rc = time_median(
                [&]() {
                    return lj_force_batched(&batch, q4_dev, p4_scratch_dev, row_ptr_dev, col_dev,
                                            workspace_dev, workspace_bytes, stream);
                },
                reps, st, &ms);
            if (rc != LJ_OK) return rc;
            if (ms < *best_ms) {
                *best_ms = ms;
                *best_tpi = tpis[a];
                *best_rows_per_item = rows_per_item[b];
            }
        }
    }
    return *best_tpi ? LJ_OK : LJ_ERR_ARG;
}

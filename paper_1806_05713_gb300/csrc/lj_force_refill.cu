// lj_force_refill.cu -- FP64 "group-refill" schedule of the LJ momentum
// update.
//
// Same arithmetic as fp64_row (Algorithm 1 inside the sorted-list loop of
// Algorithm 3).  On GB300 an FP64 instruction occupies the FP64 pipe for its
// full issue slot whatever the number of active lanes, so a warp whose
// groups walk rows of different length (a half list in random order has rows
// of 0 to ~140 entries) keeps paying for the groups that have finished.
// Here each group of TPI lanes takes the next row as soon as its own ends:
// the warp takes chunks of rows from a global counter and hands them to its
// groups, so every group is busy on every iteration until the rows run out
// (the lane-counter / remainder-loop idea of the paper's Algorithm 4,
// applied across rows).  A finished row adds its partial sums to p_i with
// FP64 atomics in L2 (one per lane and component), so no FP64 reduction
// runs on the pipe.  U = 2 carries two entries per lane and iteration (the
// paper's software pipelining).  The grid is persistent and sized so that
// each group sees several rows.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "lj_fixed.cuh"
#include "lj_rows.cuh"

namespace lj {
namespace {

constexpr int kRefillThreads = 256;
constexpr int kRowsPerGroupTarget = 8;

template <int TPI, bool HALF, int U>
__global__ void __launch_bounds__(kRefillThreads)
force_refill_kernel(const double *__restrict__ q4, double *__restrict__ p4, int n,
                    const int *__restrict__ row_ptr, const int *__restrict__ col, Fp64Params P,
                    unsigned *__restrict__ counter)
{
    constexpr int G = 32 / TPI;          // groups per warp
    constexpr int kChunk = 4 * G;        // rows per counter fetch
    const int lane = threadIdx.x & 31;
    const int sub = lane & (TPI - 1);
    const int leader = lane & ~(TPI - 1);
    const unsigned below_leader = (1u << leader) - 1u;
    int chunk_next = 0, chunk_end = 0;   // warp-uniform
    bool exhausted = false;              // warp-uniform
    int row = -1, k = 0, ke = 0;         // group-uniform
    double xi = 0.0, yi = 0.0, zi = 0.0, ax = 0.0, ay = 0.0, az = 0.0;
    while (true) {
        bool need = k >= ke;
        if (need && row >= 0) {
            double *pi = p4 + 4 * static_cast<int64_t>(row);
            if (HALF || TPI == 1) {
                atomicAdd(pi + 0, ax);
                atomicAdd(pi + 1, ay);
                atomicAdd(pi + 2, az);
            } else {
                ax = group_sum<TPI>(ax);
                ay = group_sum<TPI>(ay);
                az = group_sum<TPI>(az);
                if (sub == 0) {
                    atomicAdd(pi + 0, ax);
                    atomicAdd(pi + 1, ay);
                    atomicAdd(pi + 2, az);
                }
            }
            row = -1;
        }
        unsigned want = __ballot_sync(0xffffffffu, need && sub == 0);
        while (want && !exhausted) {
            if (chunk_next >= chunk_end) {
                unsigned c = 0;
                if (lane == 0) c = atomicAdd(counter, static_cast<unsigned>(kChunk));
                c = __shfl_sync(0xffffffffu, c, 0);
                if (c >= static_cast<unsigned>(n)) {
                    exhausted = true;
                    break;
                }
                chunk_next = static_cast<int>(c);
                chunk_end = min(n, chunk_next + kChunk);
            }
            const int avail = chunk_end - chunk_next;
            const int rank = __popc(want & below_leader);
            if (need && rank < avail) {
                row = chunk_next + rank;
                k = row_ptr[row];
                ke = row_ptr[row + 1];
                load_q4_256(q4, row, xi, yi, zi);
                ax = ay = az = 0.0;
                need = false;
            }
            chunk_next += min(avail, __popc(want));
            want = __ballot_sync(0xffffffffu, need && sub == 0);
        }
        if (!__any_sync(0xffffffffu, k < ke)) {
            if (exhausted) break;
            continue;  // only empty rows were handed out: hand them in, refill
        }
        // One iteration of the row walk for every group (fp64_row's body).
        int j[U];
        bool valid[U], in[U], near[U];
        double dx[U], dy[U], dz[U], r2[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int kk = k + sub + u * TPI;
            valid[u] = kk < ke;
            j[u] = valid[u] ? col[kk] : (row >= 0 ? row : 0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            double xj, yj, zj;
            load_q4_256(q4, j[u], xj, yj, zj);
            dx[u] = xj - xi;
            dy[u] = yj - yi;
            dz[u] = zj - zi;
        }
        bool anynear = false, anyin = false;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            min_image3(dx[u], dy[u], dz[u], P.L, P.half_bits);
            r2[u] = fma(dz[u], dz[u], fma(dy[u], dy[u], dx[u] * dx[u]));
            const long long rb = __double_as_longlong(r2[u]);
            in[u] = valid[u] && rb < P.rc2_bits;
            near[u] = valid[u] && static_cast<unsigned long long>(rb - P.rc2_bits + 64) < 128ull;
            anynear |= near[u];
        }
        if (__any_sync(0xffffffffu, anynear)) {
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (near[u]) in[u] = exact_in_cutoff(dx[u], dy[u], dz[u], P.rc2);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (!valid[u]) r2[u] = 1.0;
            anyin |= in[u];
        }
        if (__any_sync(0xffffffffu, anyin)) {
            double fn[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const double w = rcp_fp64(r2[u]);
                const double w2 = w * w;
                const double w4 = w2 * w2;
                const double w3 = w2 * w;
                fn[u] = w4 * fma(P.B, w3, -P.A);  // -df: p_i -= fn d, p_j += fn d
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (in[u]) {
                    if (HALF) {
                        const double fx = fn[u] * dx[u], fy = fn[u] * dy[u], fz = fn[u] * dz[u];
                        atomicAdd(p4 + 4 * static_cast<int64_t>(j[u]) + 0, fx);
                        atomicAdd(p4 + 4 * static_cast<int64_t>(j[u]) + 1, fy);
                        atomicAdd(p4 + 4 * static_cast<int64_t>(j[u]) + 2, fz);
                        ax -= fx;
                        ay -= fy;
                        az -= fz;
                    } else {
                        ax = fma(-fn[u], dx[u], ax);
                        ay = fma(-fn[u], dy[u], ay);
                        az = fma(-fn[u], dz[u], az);
                    }
                }
            }
        }
        if (k < ke) k += TPI * U;
    }
}

// The group-refill walk with the exact fixed-point displacement of
// LJ_SCHED_FIXED (LJ_SCHED_FIXED | LJ_SCHED_REFILL | t): a group's row
// switch costs integer loads only (no FP64 set-up), so refilling the groups
// of a warp as their rows end takes the rows' unequal lengths off the FP64
// pipe.  p_i is handed to L2 per lane and component with FP64 atomics for
// both list kinds (so a full list's rounding order varies between calls).
template <int TPI>
__global__ void __launch_bounds__(kRefillThreads)
force_fixed_refill_kernel(const double *__restrict__ q4, const longlong4 *__restrict__ X,
                          double *__restrict__ p4, int n, const int *__restrict__ row_ptr,
                          const int *__restrict__ col, Fp64Params P, FixParams F, int half,
                          unsigned *__restrict__ counter)
{
    constexpr int G = 32 / TPI;
    constexpr int kChunk = 4 * G;
    const int lane = threadIdx.x & 31;
    const int sub = lane & (TPI - 1);
    const int leader = lane & ~(TPI - 1);
    const unsigned below_leader = (1u << leader) - 1u;
    int chunk_next = 0, chunk_end = 0;   // warp-uniform
    bool exhausted = false;              // warp-uniform
    int row = -1, k = 0, ke = 0;         // group-uniform
    long long xi = 0, yi = 0, zi = 0;
    double ax = 0.0, ay = 0.0, az = 0.0;
    while (true) {
        bool need = k >= ke;
        if (need && row >= 0) {
            double *pi = p4 + 4 * static_cast<int64_t>(row);
            atomicAdd(pi + 0, ax);
            atomicAdd(pi + 1, ay);
            atomicAdd(pi + 2, az);
            row = -1;
        }
        unsigned want = __ballot_sync(0xffffffffu, need && sub == 0);
        while (want && !exhausted) {
            if (chunk_next >= chunk_end) {
                unsigned c = 0;
                if (lane == 0) c = atomicAdd(counter, static_cast<unsigned>(kChunk));
                c = __shfl_sync(0xffffffffu, c, 0);
                if (c >= static_cast<unsigned>(n)) {
                    exhausted = true;
                    break;
                }
                chunk_next = static_cast<int>(c);
                chunk_end = min(n, chunk_next + kChunk);
            }
            const int avail = chunk_end - chunk_next;
            const int rank = __popc(want & below_leader);
            if (need && rank < avail) {
                row = chunk_next + rank;
                k = row_ptr[row];
                ke = row_ptr[row + 1];
                load_fixed(X, row, xi, yi, zi);
                ax = ay = az = 0.0;
                need = false;
            }
            chunk_next += min(avail, __popc(want));
            want = __ballot_sync(0xffffffffu, need && sub == 0);
        }
        if (!__any_sync(0xffffffffu, k < ke)) {
            if (exhausted) break;
            continue;  // only empty rows were handed out: hand them in, refill
        }
        const int kk = k + sub;
        const bool valid = kk < ke;
        const int j = valid ? col[kk] : (row >= 0 ? row : 0);
        long long xj, yj, zj;
        load_fixed(X, j, xj, yj, zj);
        double dx, dy, dz, r2;
        const bool in = fixed_entry(q4, xi, yi, zi, xj, yj, zj, valid, row >= 0 ? row : 0, j, P, F,
                                    0xffffffffu, dx, dy, dz, r2);
        if (__any_sync(0xffffffffu, in)) {
            const double w = rcp_fp64_fixed(in ? r2 : 1.0, 0xffffffffu);
            const double w2 = w * w;
            const double w4 = w2 * w2;
            const double w3 = w2 * w;
            const double fn = w4 * fma(P.B, w3, -P.A);  // -df: p_i -= fn d, p_j += fn d
            if (in) {
                if (half) {
                    const double fx = fn * dx, fy = fn * dy, fz = fn * dz;
                    double *pj = p4 + 4 * static_cast<int64_t>(j);
                    atomicAdd(pj + 0, fx);
                    atomicAdd(pj + 1, fy);
                    atomicAdd(pj + 2, fz);
                    ax -= fx;
                    ay -= fy;
                    az -= fz;
                } else {
                    ax = fma(-fn, dx, ax);
                    ay = fma(-fn, dy, ay);
                    az = fma(-fn, dz, az);
                }
            }
        }
        if (k < ke) k += TPI;
    }
}

template <int TPI>
int launch_fixed_refill(const double *q4, const longlong4 *X, double *p4, int n, const int *rp,
                        const int *col, int half, const Fp64Params &P, const FixParams &F,
                        unsigned *counter, cudaStream_t st)
{
    static int max_blocks = 0;
    if (max_blocks == 0) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, force_fixed_refill_kernel<TPI>,
                                                          kRefillThreads, 0) != cudaSuccess ||
            per_sm < 1)
            per_sm = 2;
        max_blocks = per_sm * num_sms();
    }
    constexpr int G = 32 / TPI;
    constexpr int warps_per_block = kRefillThreads / 32;
    const long long want_warps = std::max<long long>(1, n / (G * kRowsPerGroupTarget));
    int blocks = static_cast<int>((want_warps + warps_per_block - 1) / warps_per_block);
    blocks = std::max(std::min(blocks, max_blocks), std::min(max_blocks, 2 * num_sms()));
    force_fixed_refill_kernel<TPI><<<blocks, kRefillThreads, 0, st>>>(q4, X, p4, n, rp, col, P, F,
                                                                      half, counter);
    LJ_TRY_LAUNCH("force_fixed_refill_kernel");
    return LJ_OK;
}

template <int TPI, bool HALF, int U>
int launch_refill(const double *q4, double *p4, int n, const int *rp, const int *col,
                  const Fp64Params &P, unsigned *counter, cudaStream_t st)
{
    static int max_blocks = 0;
    if (max_blocks == 0) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, force_refill_kernel<TPI, HALF, U>,
                                                          kRefillThreads, 0) != cudaSuccess ||
            per_sm < 1)
            per_sm = 2;
        max_blocks = per_sm * num_sms();
    }
    constexpr int G = 32 / TPI;
    constexpr int warps_per_block = kRefillThreads / 32;
    // Enough warps to fill the GPU, few enough that each group sees several rows.
    const long long want_warps = std::max<long long>(1, n / (G * kRowsPerGroupTarget));
    int blocks = static_cast<int>((want_warps + warps_per_block - 1) / warps_per_block);
    blocks = std::max(std::min(blocks, max_blocks), std::min(max_blocks, 2 * num_sms()));
    force_refill_kernel<TPI, HALF, U><<<blocks, kRefillThreads, 0, st>>>(q4, p4, n, rp, col, P, counter);
    LJ_TRY_LAUNCH("force_refill_kernel");
    return LJ_OK;
}

}  // namespace

size_t force_refill_workspace_bytes() { return 256; }

// sched: LJ_SCHED_FIXED | LJ_SCHED_REFILL | tpi (tpi 4 or 8); X: the
// fixed-point positions (already written by the caller's pre-pass).
int force_fixed_refill_fp64(const double *q4, const longlong4 *X, double *p4, int n,
                            const int *row_ptr, const int *col, int half, const double box[3],
                            double dt, double rc, double eps, double sigma, int sched, void *ws,
                            size_t ws_bytes, cudaStream_t st)
{
    if (!ws || ws_bytes < force_refill_workspace_bytes()) return LJ_ERR_CAPACITY;
    const Fp64Params P = make_fp64_params(box, dt, rc, eps, sigma);
    const FixParams F = make_fix_params(box);
    unsigned *counter = static_cast<unsigned *>(ws);
    LJ_TRY_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned), st));
    switch (sched & 63) {
        case 4: return launch_fixed_refill<4>(q4, X, p4, n, row_ptr, col, half, P, F, counter, st);
        case 8: return launch_fixed_refill<8>(q4, X, p4, n, row_ptr, col, half, P, F, counter, st);
        default: return LJ_ERR_ARG;
    }
}

// sched: LJ_SCHED_REFILL | tpi (tpi 0 or 1: one lane per row), optionally
// | LJ_SCHED_SWP2 for two entries per lane and iteration.
int force_refill_fp64(const double *q4, double *p4, int n, const int *row_ptr, const int *col,
                      int half, const double box[3], double dt, double rc, double eps,
                      double sigma, int sched, void *ws, size_t ws_bytes, cudaStream_t st)
{
    if (!ws || ws_bytes < force_refill_workspace_bytes()) return LJ_ERR_CAPACITY;
    const Fp64Params P = make_fp64_params(box, dt, rc, eps, sigma);
    unsigned *counter = static_cast<unsigned *>(ws);
    LJ_TRY_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned), st));
    const bool swp = (sched & LJ_SCHED_SWP2) != 0;
    const int tpi = sched & 63;
#define LJ_REFILL(T, U)                                                                          \
    return half ? launch_refill<T, true, U>(q4, p4, n, row_ptr, col, P, counter, st)            \
                : launch_refill<T, false, U>(q4, p4, n, row_ptr, col, P, counter, st)
    switch (tpi) {
        case 0:
        case 1:
            if (swp) LJ_REFILL(1, 2);
            LJ_REFILL(1, 1);
        case 4:
            if (swp) LJ_REFILL(4, 2);
            LJ_REFILL(4, 1);
        case 8:
            if (swp) LJ_REFILL(8, 2);
            LJ_REFILL(8, 1);
        default:
            return LJ_ERR_ARG;
    }
#undef LJ_REFILL
}

}  // namespace lj

// lj_force_queue.cu -- FP64 "lane-queue" schedule of the LJ momentum update.
//
// Same arithmetic as fp64_row (Algorithm 1 inside the sorted-list loop of
// Algorithm 3).  GB300's FP64 pipe spends a full issue slot on every FP64
// warp instruction however many lanes are active, so idle lanes cost as
// much as busy ones.  This schedule splits the pair work the way the
// paper's software pipelining splits its loop body (section "Software
// Pipelining": A load q_j, B distance, C force, D store), into two phases
// that each run with every lane busy:
//
//   screen  every lane takes the next entry of its own share of its group's
//           row, forms d = q_j - q_i (minimum image) and r^2, and pushes the
//           pairs inside r_c onto its own FIFO queue in shared memory
//           (margin pairs, about a seventh of the list, stop here);
//   force   when every lane that still has work holds a queued pair, each
//           lane pops one and computes u = 1/r^2, df and df d, sends -df d
//           to p_j (half list) and adds df d to its register sum for p_i.
//
// A lane's queue holds pairs of its rows in order; when the popped pair
// belongs to a new row the lane hands the old row's sum to p_i with FP64
// atomics in L2 (no FP64 reduction on the pipe).  Groups of TPI lanes take
// rows from a per-warp chunk that warps refill from a global counter, as in
// the group-refill schedule, so lanes do not wait for longer rows.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "lj_rows.cuh"

namespace lj {
namespace {

constexpr int kQueueThreads = 256;
constexpr int kRowsPerGroupTarget = 4;

template <int D>
struct QueueSmem {
    double dx[D][kQueueThreads];
    double dy[D][kQueueThreads];
    double dz[D][kQueueThreads];
    double r2[D][kQueueThreads];
    int j[D][kQueueThreads];
    int row[D][kQueueThreads];
};

template <int TPI, bool HALF, int D>
__global__ void __launch_bounds__(kQueueThreads)
force_queue_kernel(const double *__restrict__ q4, double *__restrict__ p4, int n,
                   const int *__restrict__ row_ptr, const int *__restrict__ col, Fp64Params P,
                   unsigned *__restrict__ counter)
{
    __shared__ QueueSmem<D> Q;
    constexpr int G = 32 / TPI;
    constexpr int kChunk = 4 * G;
    const int t = threadIdx.x;
    const int lane = t & 31;
    const int sub = lane & (TPI - 1);
    const int leader = lane & ~(TPI - 1);
    const unsigned below_leader = (1u << leader) - 1u;
    const unsigned gmask = TPI == 32 ? 0xffffffffu : (((1u << TPI) - 1u) << leader);
    int chunk_next = 0, chunk_end = 0;  // warp-uniform
    bool exhausted = false;             // warp-uniform
    int row = -1, k = 0, ke = 0;        // this lane's share of its group's row
    double xi = 0.0, yi = 0.0, zi = 0.0;
    int qh = 0, qn = 0;                 // queue head and length
    int acc_row = -1;
    double ax = 0.0, ay = 0.0, az = 0.0;
    while (true) {
        // Groups whose row is fully screened take a new one.
        bool need = (__ballot_sync(0xffffffffu, k < ke) & gmask) == 0u;  // group-uniform
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
                k = row_ptr[row] + sub;
                ke = row_ptr[row + 1];
                load_q4_256(q4, row, xi, yi, zi);
                need = false;
            }
            chunk_next += min(avail, __popc(want));
            want = __ballot_sync(0xffffffffu, need && sub == 0);
        }
        const bool canA = k < ke && qn < D;
        const bool hasB = qn > 0;
        const unsigned mA = __ballot_sync(0xffffffffu, canA);
        const unsigned mB = __ballot_sync(0xffffffffu, hasB);
        const unsigned mWork = __ballot_sync(0xffffffffu, k < ke || hasB);
        if (mWork == 0u) {
            if (exhausted) break;
            continue;  // rows handed out were empty: take more
        }
        if (mB == mWork || mA == 0u) {
            // ---- force phase: one queued pair per lane ----
            const int s = qh;
            double dx = 0.0, dy = 0.0, dz = 0.0, r2 = 1.0;
            int j = 0, prow = -1;
            if (hasB) {
                dx = Q.dx[s][t];
                dy = Q.dy[s][t];
                dz = Q.dz[s][t];
                r2 = Q.r2[s][t];
                j = Q.j[s][t];
                prow = Q.row[s][t];
            }
            const double w = rcp_fp64(r2);
            const double w2 = w * w;
            const double w4 = w2 * w2;
            const double w3 = w2 * w;
            const double fn = w4 * fma(P.B, w3, -P.A);  // -df: p_i -= fn d, p_j += fn d
            if (hasB) {
                if (prow != acc_row) {
                    if (acc_row >= 0) {
                        double *pi = p4 + 4 * static_cast<int64_t>(acc_row);
                        atomicAdd(pi + 0, ax);
                        atomicAdd(pi + 1, ay);
                        atomicAdd(pi + 2, az);
                    }
                    acc_row = prow;
                    ax = ay = az = 0.0;
                }
                if (HALF) {
                    const double fx = fn * dx, fy = fn * dy, fz = fn * dz;
                    atomicAdd(p4 + 4 * static_cast<int64_t>(j) + 0, fx);
                    atomicAdd(p4 + 4 * static_cast<int64_t>(j) + 1, fy);
                    atomicAdd(p4 + 4 * static_cast<int64_t>(j) + 2, fz);
                    ax -= fx;
                    ay -= fy;
                    az -= fz;
                } else {
                    ax = fma(-fn, dx, ax);
                    ay = fma(-fn, dy, ay);
                    az = fma(-fn, dz, az);
                }
                qh = qh + 1 == D ? 0 : qh + 1;
                --qn;
            }
        } else {
            // ---- screen phase: one entry per lane ----
            const int jj = canA ? col[k] : (row >= 0 ? row : 0);
            double xj, yj, zj;
            load_q4_256(q4, jj, xj, yj, zj);
            double dx = xj - xi, dy = yj - yi, dz = zj - zi;
            min_image3(dx, dy, dz, P.L, P.half_bits);
            const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
            const long long rb = __double_as_longlong(r2);
            bool in = canA && rb < P.rc2_bits;
            const bool near = canA && static_cast<unsigned long long>(rb - P.rc2_bits + 64) < 128ull;
            if (__any_sync(0xffffffffu, near)) {
                if (near) in = exact_in_cutoff(dx, dy, dz, P.rc2);
            }
            if (in) {
                int s = qh + qn;
                s = s >= D ? s - D : s;
                Q.dx[s][t] = dx;
                Q.dy[s][t] = dy;
                Q.dz[s][t] = dz;
                Q.r2[s][t] = r2;
                Q.j[s][t] = jj;
                Q.row[s][t] = row;
                ++qn;
            }
            if (canA) k += TPI;
        }
    }
    if (acc_row >= 0) {
        double *pi = p4 + 4 * static_cast<int64_t>(acc_row);
        atomicAdd(pi + 0, ax);
        atomicAdd(pi + 1, ay);
        atomicAdd(pi + 2, az);
    }
}

template <int TPI, bool HALF, int D>
int launch_queue(const double *q4, double *p4, int n, const int *rp, const int *col,
                 const Fp64Params &P, unsigned *counter, cudaStream_t st)
{
    static int max_blocks = 0;
    if (max_blocks == 0) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, force_queue_kernel<TPI, HALF, D>,
                                                          kQueueThreads, 0) != cudaSuccess ||
            per_sm < 1)
            per_sm = 2;
        max_blocks = per_sm * num_sms();
    }
    constexpr int G = 32 / TPI;
    constexpr int warps_per_block = kQueueThreads / 32;
    const long long want_warps = std::max<long long>(1, n / (G * kRowsPerGroupTarget));
    int blocks = static_cast<int>((want_warps + warps_per_block - 1) / warps_per_block);
    blocks = std::max(std::min(blocks, max_blocks), std::min(max_blocks, 2 * num_sms()));
    force_queue_kernel<TPI, HALF, D><<<blocks, kQueueThreads, 0, st>>>(q4, p4, n, rp, col, P, counter);
    LJ_TRY_LAUNCH("force_queue_kernel");
    return LJ_OK;
}

}  // namespace

// sched: LJ_SCHED_QUEUE | tpi (tpi = 1, 2, 4 or 8).
int force_queue_fp64(const double *q4, double *p4, int n, const int *row_ptr, const int *col,
                     int half, const double box[3], double dt, double rc, double eps, double sigma,
                     int sched, void *ws, size_t ws_bytes, cudaStream_t st)
{
    if (!ws || ws_bytes < 256) return LJ_ERR_CAPACITY;
    const Fp64Params P = make_fp64_params(box, dt, rc, eps, sigma);
    unsigned *counter = static_cast<unsigned *>(ws);
    LJ_TRY_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned), st));
    constexpr int D = 4;
#define LJ_QUEUE(T)                                                                    \
    return half ? launch_queue<T, true, D>(q4, p4, n, row_ptr, col, P, counter, st)   \
                : launch_queue<T, false, D>(q4, p4, n, row_ptr, col, P, counter, st)
    switch (sched & 63) {
        case 0:
        case 1: LJ_QUEUE(1);
        case 2: LJ_QUEUE(2);
        case 4: LJ_QUEUE(4);
        case 8: LJ_QUEUE(8);
        default: return LJ_ERR_ARG;
    }
#undef LJ_QUEUE
}

}  // namespace lj

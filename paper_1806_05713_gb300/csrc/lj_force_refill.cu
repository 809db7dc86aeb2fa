// lj_force_refill.cu -- FP64 "lane-refill" schedule of the LJ momentum update.
//
// Same arithmetic as the FP64 form in lj_force.cu (Algorithm 1 inside the
// sorted-list loop of Algorithm 3), scheduled for a GPU on which FP64
// instructions are the bottleneck.  Each lane owns one row i at a time --
// q_i and the p_i sum stay in registers, as Algorithm 3 keeps the i data in
// registers -- and walks its row one entry per iteration.  A lane whose row
// ends adds its sum to p_i (one FP64 atomic per component, done in L2 and
// not on the FP64 pipe) and immediately takes the next row from its warp's
// chunk of 32 rows; a warp whose chunk is used up takes the next chunk from
// a global counter.  So every lane does useful work on every iteration until
// the rows run out: no lane waits for a longer row of its warp (the
// imbalance the paper's remainder-loop elimination attacks for SIMD), and no
// cross-lane reduction is needed.  The grid is persistent: one launch of
// as many blocks as fit on the GPU at once.
#include <cmath>
#include <cstring>

#include "lj_internal.cuh"

namespace lj {
namespace {

constexpr int kRefillThreads = 256;
constexpr int kChunk = 32;

struct RefillParams {
    double L[3];
    long long half_bits[3];
    long long rc2_bits;
    double rc2;
    double A, B;  // df = u^4 (A - B u^3)
};

__device__ __forceinline__ void gather_q(const double *__restrict__ q4, int j, double &x,
                                         double &y, double &z)
{
    double w;
    asm("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];"
        : "=d"(x), "=d"(y), "=d"(z), "=d"(w)
        : "l"(q4 + 4 * static_cast<int64_t>(j)));
}

template <bool HALF>
__global__ void __launch_bounds__(kRefillThreads)
force_refill_kernel(const double *__restrict__ q4, double *__restrict__ p4, int n,
                    const int *__restrict__ row_ptr, const int *__restrict__ col, RefillParams P,
                    unsigned *__restrict__ counter)
{
    const int lane = threadIdx.x & 31;
    int chunk_next = 0, chunk_end = 0;  // warp-uniform
    bool exhausted = false;             // warp-uniform: no rows left anywhere
    int row = -1, k = 0, ke = 0;
    double xi = 0.0, yi = 0.0, zi = 0.0, ax = 0.0, ay = 0.0, az = 0.0;
    while (true) {
        // Lanes whose row is done hand in their sum and take a new row.
        bool need = k >= ke;
        if (need && row >= 0) {
            double *pi = p4 + 4 * static_cast<int64_t>(row);
            atomicAdd(pi + 0, ax);
            atomicAdd(pi + 1, ay);
            atomicAdd(pi + 2, az);
            row = -1;
        }
        unsigned want = __ballot_sync(0xffffffffu, need);
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
            const int rank = __popc(want & lanemask_lt());
            if (need && rank < avail) {
                row = chunk_next + rank;
                k = row_ptr[row];
                ke = row_ptr[row + 1];
                gather_q(q4, row, xi, yi, zi);
                ax = ay = az = 0.0;
                need = false;
            }
            chunk_next += min(avail, __popc(want));
            want = __ballot_sync(0xffffffffu, need);
        }
        const bool valid = k < ke;
        if (!__any_sync(0xffffffffu, valid)) {
            if (exhausted || !__any_sync(0xffffffffu, need)) break;
            continue;  // every lane got an empty row: hand them in, refill
        }
        const int j = valid ? col[k] : (row >= 0 ? row : 0);
        double xj, yj, zj;
        gather_q(q4, j, xj, yj, zj);
        double dx = xj - xi, dy = yj - yi, dz = zj - zi;
        min_image3(dx, dy, dz, P.L, P.half_bits);
        double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
        const long long rb = __double_as_longlong(r2);
        bool in = valid && rb < P.rc2_bits;
        const bool near = valid && static_cast<unsigned long long>(rb - P.rc2_bits + 64) < 128ull;
        if (__any_sync(0xffffffffu, near)) {
            if (near) {
                const double e2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                                            __dmul_rn(dz, dz));
                in = e2 < P.rc2;
            }
        }
        if (!valid) r2 = 1.0;
        if (__any_sync(0xffffffffu, in)) {
            const double u = rcp_fp64(r2);
            const double u2 = u * u;
            const double u4 = u2 * u2;
            const double u3 = u2 * u;
            const double fn = u4 * fma(P.B, u3, -P.A);  // -df: p_i -= fn d, p_j += fn d
            if (in) {
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
            }
        }
        if (valid) ++k;
    }
}

template <bool HALF>
int grid_for()
{
    static int blocks = 0;
    if (blocks == 0) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, force_refill_kernel<HALF>,
                                                          kRefillThreads, 0) != cudaSuccess ||
            per_sm < 1)
            per_sm = 4;
        blocks = per_sm * num_sms();
    }
    return blocks;
}

}  // namespace

size_t force_refill_workspace_bytes() { return 256; }

int force_refill_fp64(const double *q4, double *p4, int n, const int *row_ptr, const int *col,
                      int half, const double box[3], double dt, double rc, double eps,
                      double sigma, void *ws, size_t ws_bytes, cudaStream_t st)
{
    if (!ws || ws_bytes < force_refill_workspace_bytes()) return LJ_ERR_CAPACITY;
    RefillParams P{};
    for (int a = 0; a < 3; ++a) {
        P.L[a] = box[a];
        const double h = 0.5 * box[a];
        std::memcpy(&P.half_bits[a], &h, sizeof(double));
    }
    P.rc2 = rc * rc;
    std::memcpy(&P.rc2_bits, &P.rc2, sizeof(double));
    const double s2 = sigma * sigma, s6 = s2 * s2 * s2, s12 = s6 * s6;
    P.A = 24.0 * eps * s6 * dt;
    P.B = 48.0 * eps * s12 * dt;
    unsigned *counter = static_cast<unsigned *>(ws);
    LJ_TRY_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned), st));
    const int needed = (n + kChunk - 1) / kChunk;
    if (half) {
        const int grid = std::min(grid_for<true>(), needed);
        force_refill_kernel<true><<<grid, kRefillThreads, 0, st>>>(q4, p4, n, row_ptr, col, P, counter);
    } else {
        const int grid = std::min(grid_for<false>(), needed);
        force_refill_kernel<false><<<grid, kRefillThreads, 0, st>>>(q4, p4, n, row_ptr, col, P, counter);
    }
    LJ_TRY_LAUNCH("force_refill_kernel");
    return LJ_OK;
}

}  // namespace lj

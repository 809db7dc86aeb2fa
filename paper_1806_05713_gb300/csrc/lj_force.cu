// lj_force.cu -- the LJ momentum update over the sorted CSR list
// (Watanabe & Nakagawa, arXiv 1806.05713: Algorithm 1 for one pair inside
// the sorted-list double loop of Algorithm 3).
//
// Schedules ("threads per i", TPI): a group of TPI lanes of one warp owns
// row i, keeps q_i in registers (Algorithm 3 keeps the i data in registers),
// strides over the row's j (the lane-predicated tail replaces the paper's
// remainder-loop elimination, Algorithm 4), and reduces its partial sums
// with warp shuffles.  Within a row no two lanes hold the same j, so the
// p_j updates of a half list need no conflict detection (the paper's CDE);
// across rows they meet other rows' updates, hence FP64 atomics there.
//
// Forms:
//  * FP64: every step in IEEE double precision.  GB300 issues FP64 at a
//    small fraction of its FP32 rate, so the kernels spend FP64 operations
//    only where the value needs them.  The default schedule (LJ_SCHED_FIXED,
//    lj_fixed.cuh) takes the minimum-image displacement and r^2 exactly in
//    integer fixed point and the reciprocal from a double-float seed built
//    on the FP32 pipe plus one FP64 Newton step: 13 FP64 instructions per
//    entry.  The older schedules (fp64_row in lj_rows.cuh) test the minimum
//    image and the cutoff by integer compares of IEEE bit patterns and take
//    the division as an FP32 seed plus one third-order FP64 correction.  In
//    all of them df = u^4 (A - B u^3) with u = 1/r^2 takes five FP64
//    operations after the reciprocal.
//  * MIXED: a pre-pass turns each FP64 position into a 32-bit fixed-point
//    fraction of the box side (X = floor(x 2^32 / L), computed in FP64), so
//    X_j - X_i in wrapping integer arithmetic is the minimum-image
//    displacement exactly, and one conversion and one multiply give it in
//    FP32 to its last bit (absolute FP32 coordinates would lose ~1e-5 at
//    L ~ 100).  The pair arithmetic is FP32, per-lane i-sums are
//    Kahan-compensated FP32, combined across lanes with error-free
//    transformations and added to the FP64 momentum once per row (head and
//    compensation as two FP64 additions in L2); half-list p_j updates are
//    FP64 atomics of exactly converted FP32 values.
//  * DFLOAT (lj_force_dfloat.cu): the pair arithmetic in double-float on
//    the FP32 pipe, held to the FP64 tolerance.
// In every form a pair whose r^2 lies within a proven error band of r_c^2
// is re-decided with the exact FP64 definition, so the set of interacting
// pairs is the same as in double precision.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "lj_fixed.cuh"
#include "lj_rows.cuh"

namespace lj {
namespace {

// ---------------------------------------------------------------------------
// FP64 form
// ---------------------------------------------------------------------------
// order: NULL (rows in index order) or a permutation of the rows (the
// length-sorted order of LJ_SCHED_SORTED).
template <int TPI, bool HALF, int U, bool IMG>
__global__ void __launch_bounds__(256)
force_fp64_kernel(const double *__restrict__ q4, double *__restrict__ p4, int n,
                  const int *__restrict__ row_ptr, const int *__restrict__ col, Fp64Params P,
                  const int *__restrict__ order)
{
    const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / TPI;
    // A group past the last row exits as a whole; the votes and shuffles in
    // the row walk name only the group's own lanes, which iterate together.
    if (gid >= n) return;
    const int i = order ? order[gid] : gid;
    fp64_row<TPI, HALF, U, IMG>(q4, p4, row_ptr, col, i, P, group_mask<TPI>());
}

// FP64 form with the exact fixed-point displacement (LJ_SCHED_FIXED).
// 128-thread blocks (a finer last wave than 256 at the same occupancy,
// about 1 % faster).  At least eight blocks an SM: the row's selects (no
// branch on the magnitude of a displacement) keep more values live, and
// 64 registers hold them without spilling (twelve blocks in 40 registers
// spilled and ran 0.6-0.8 % slower).  (Two entries per lane -- the paper's
// software pipelining on this row -- needed 74 registers and ran 0.298 ms
// against 0.263 at N = 119,164: the occupancy hides the FP64 latency
// better.)
template <int TPI, bool HALF>
__global__ void __launch_bounds__(128, 8)
force_fixed_kernel(const double *__restrict__ q4, const longlong4 *__restrict__ X,
                   double *__restrict__ p4, int n, const int *__restrict__ row_ptr,
                   const int *__restrict__ col, Fp64Params P, FixParams F,
                   const int *__restrict__ order)
{
    const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / TPI;
    if (gid >= n) return;
    const int i = order ? order[gid] : gid;
    fp64_fixed_row<TPI, HALF>(q4, X, p4, row_ptr, col, i, P, F, group_mask<TPI>());
}

// FP64 form, exact fixed-point displacement, R rows per warp walked as one
// stream of entries (LJ_SCHED_STREAM).
template <bool HALF, int R>
__global__ void __launch_bounds__(128, 8)
force_fixed_stream_kernel(const double *__restrict__ q4, const longlong4 *__restrict__ X,
                          double *__restrict__ p4, int n, const int *__restrict__ row_ptr,
                          const int *__restrict__ col, Fp64Params P, FixParams F)
{
    const long long w = (static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    if (w * R >= n) return;
    const int i0 = static_cast<int>(w * R);
    fp64_fixed_stream<HALF>(q4, X, p4, row_ptr, col, i0, min(i0 + R, n), P, F);
}

// MIXED form, 128-thread blocks (a finer last wave: the full list 2-4 %
// faster than with 256).  U = 1: one entry per lane and iteration, its
// gathers one iteration ahead; U = 2 (LJ_SCHED_SWP2): two entries per lane.
template <int TPI, bool HALF, int U>
__global__ void __launch_bounds__(128)
force_mixed_kernel(const double *__restrict__ q4, const uint4 *__restrict__ rel,
                   double *__restrict__ p4, int n, const int *__restrict__ row_ptr,
                   const int *__restrict__ col, MixedParams P, const int *__restrict__ order)
{
    const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / TPI;
    if (gid >= n) return;
    const int i = order ? order[gid] : gid;
    mixed_row_pf<TPI, HALF, U>(q4, rel, p4, row_ptr, col, i, P);
}

// Force and potential energy in one pass (FP64, 8 lanes per row, exact
// fixed-point displacement): each thread keeps its row's pair-energy sum and
// in-cutoff count; a fixed-order block reduction writes one partial per
// block (the final sum is taken by energy_partials_kernel).  FS: the
// force-shifted truncation (fixed-point rows only).
template <bool FS>
__global__ void __launch_bounds__(256)
force_energy_fp64_kernel(const double *__restrict__ q4, const longlong4 *__restrict__ X,
                         double *__restrict__ p4, int n, const int *__restrict__ row_ptr,
                         const int *__restrict__ col, Fp64Params P, FixParams F, int half,
                         double *__restrict__ partial)
{
    constexpr int TPI = 8;
    __shared__ double red_e[8], red_w[8];
    __shared__ long long red_c[8];
    const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / TPI;
    double ev = 0.0, wv = 0.0;
    int cnt = 0;
    if (gid < n) {
        if (FS || X) {
            if (half)
                fp64_fixed_row<TPI, true, true, FS>(q4, X, p4, row_ptr, col, gid, P, F,
                                                    group_mask<TPI>(), &ev, &cnt, &wv);
            else
                fp64_fixed_row<TPI, false, true, FS>(q4, X, p4, row_ptr, col, gid, P, F,
                                                     group_mask<TPI>(), &ev, &cnt, &wv);
        } else {  // a box wider than 1024 r_c: image-selected rows
            if (half)
                fp64_row<TPI, true, 1, true, 0, true>(q4, p4, row_ptr, col, gid, P, group_mask<TPI>(),
                                                      Layout{4, 1}, &ev, &cnt, &wv);
            else
                fp64_row<TPI, false, 1, true, 0, true>(q4, p4, row_ptr, col, gid, P, group_mask<TPI>(),
                                                       Layout{4, 1}, &ev, &cnt, &wv);
        }
    }
    long long c = cnt;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ev += __shfl_xor_sync(0xffffffffu, ev, o);
        wv += __shfl_xor_sync(0xffffffffu, wv, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red_e[threadIdx.x >> 5] = ev;
        red_w[threadIdx.x >> 5] = wv;
        red_c[threadIdx.x >> 5] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double se = 0.0, sw = 0.0;
        long long sc = 0;
        for (int w = 0; w < 8; ++w) {
            se += red_e[w];
            sw += red_w[w];
            sc += red_c[w];
        }
        partial[3 * blockIdx.x] = se;
        partial[3 * blockIdx.x + 1] = static_cast<double>(sc);
        partial[3 * blockIdx.x + 2] = sw;
    }
}

// The force-shifted truncation without the energy (8 lanes per row).
template <bool HALF>
__global__ void __launch_bounds__(256)
force_fs_kernel(const double *__restrict__ q4, const longlong4 *__restrict__ X,
                double *__restrict__ p4, int n, const int *__restrict__ row_ptr,
                const int *__restrict__ col, Fp64Params P, FixParams F)
{
    constexpr int TPI = 8;
    const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / TPI;
    if (gid >= n) return;
    fp64_fixed_row<TPI, HALF, false, true>(q4, X, p4, row_ptr, col, gid, P, F, group_mask<TPI>());
}

// E = scale * (sum of pair energies - vshift * number of in-cutoff entries)
// and, with wout, W = scale * (sum of pair virials); fixed-order sums.
__global__ void energy_partials_kernel(const double *__restrict__ partial, int blocks, double scale,
                                       double vshift, double *__restrict__ out,
                                       double *__restrict__ wout)
{
    __shared__ double se[32], sc[32], sw[32];
    double e = 0.0, c = 0.0, v = 0.0;
    for (int t = threadIdx.x; t < blocks; t += blockDim.x) {
        e += partial[3 * t];
        c += partial[3 * t + 1];
        v += partial[3 * t + 2];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_xor_sync(0xffffffffu, e, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
        v += __shfl_xor_sync(0xffffffffu, v, o);
    }
    if ((threadIdx.x & 31) == 0) {
        se[threadIdx.x >> 5] = e;
        sc[threadIdx.x >> 5] = c;
        sw[threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double te = 0.0, tc = 0.0, tw = 0.0;
        for (int w = 0; w < int(blockDim.x / 32); ++w) {
            te += se[w];
            tc += sc[w];
            tw += sw[w];
        }
        *out = scale * (te - vshift * tc);
        if (wout) *wout = scale * tw;
    }
}

// Rows in order of decreasing length (LJ_SCHED_SORTED): a counting sort on
// min(length, kLenBuckets - 1), so that the groups of one warp walk rows of
// equal length and none idles while another finishes.
constexpr int kLenBuckets = 512;

__global__ void row_len_hist_kernel(const int *__restrict__ row_ptr, int n, int *__restrict__ hist,
                                    int *__restrict__ slot)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int len = min(row_ptr[i + 1] - row_ptr[i], kLenBuckets - 1);
    slot[i] = atomicAdd(&hist[kLenBuckets - 1 - len], 1);
}

__global__ void row_len_scan_kernel(int *__restrict__ hist)
{
    __shared__ int s[kLenBuckets];
    const int t = threadIdx.x;
    s[t] = hist[t];
    __syncthreads();
    for (int o = 1; o < kLenBuckets; o <<= 1) {
        const int v = t >= o ? s[t - o] : 0;
        __syncthreads();
        s[t] += v;
        __syncthreads();
    }
    hist[t] = s[t] - hist[t];  // exclusive
}

__global__ void row_len_scatter_kernel(const int *__restrict__ row_ptr, int n,
                                       const int *__restrict__ start, const int *__restrict__ slot,
                                       int *__restrict__ order)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int len = min(row_ptr[i + 1] - row_ptr[i], kLenBuckets - 1);
    order[start[kLenBuckets - 1 - len] + slot[i]] = i;
}

int sort_rows_by_length(const int *row_ptr, int n, int *hist, int *slot, int *order, cudaStream_t st)
{
    LJ_TRY_CUDA(cudaMemsetAsync(hist, 0, sizeof(int) * kLenBuckets, st));
    const unsigned g = unsigned((n + 255) / 256);
    row_len_hist_kernel<<<g, 256, 0, st>>>(row_ptr, n, hist, slot);
    LJ_TRY_LAUNCH("row_len_hist_kernel");
    row_len_scan_kernel<<<1, kLenBuckets, 0, st>>>(hist);
    LJ_TRY_LAUNCH("row_len_scan_kernel");
    row_len_scatter_kernel<<<g, 256, 0, st>>>(row_ptr, n, hist, slot, order);
    LJ_TRY_LAUNCH("row_len_scatter_kernel");
    return LJ_OK;
}

// Rows in space-filling order (LJ_SCHED_CELLS): the box is cut into at most
// 16 cells per axis of side >= r_c / 2, and the rows are counting-sorted by
// the Morton (bit-interleaved) index of their atom's cell.  The warps of an
// SM then walk rows of nearby atoms, whose neighbour sets overlap, so the
// gathered q_j records are reused from L1 instead of L2 when the atoms are
// numbered in random order.  The order within a cell is the atomic slot
// order; the rows' results do not depend on it.
constexpr int kCellBits = 4;
constexpr int kCellKeys = 1 << (3 * kCellBits);
static_assert(kCellKeys % 1024 == 0, "cell_scan_kernel gives each of 1024 threads whole counts");

struct CellGrid {
    double inv[3];  // cells per unit length
    int nc[3];      // cells per axis (1 .. 16)
};

CellGrid make_cell_grid(const double box[3], double rc)
{
    CellGrid g{};
    for (int a = 0; a < 3; ++a) {
        const int c = static_cast<int>(box[a] / (0.5 * rc));
        g.nc[a] = c < 1 ? 1 : (c > (1 << kCellBits) ? (1 << kCellBits) : c);
        g.inv[a] = g.nc[a] / box[a];
    }
    return g;
}

__device__ __forceinline__ unsigned spread3(unsigned v)  // bit b of v -> bit 3 b
{
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__device__ __forceinline__ int cell_key(const double *__restrict__ q4, int i, const CellGrid &g)
{
    double x, y, z;
    load_xyz(q4, i, x, y, z);
    const int cx = min(max(static_cast<int>(x * g.inv[0]), 0), g.nc[0] - 1);
    const int cy = min(max(static_cast<int>(y * g.inv[1]), 0), g.nc[1] - 1);
    const int cz = min(max(static_cast<int>(z * g.inv[2]), 0), g.nc[2] - 1);
    return static_cast<int>(spread3(cx) | (spread3(cy) << 1) | (spread3(cz) << 2));
}

__global__ void cell_hist_kernel(const double *__restrict__ q4, int n, CellGrid g,
                                 int *__restrict__ hist, int *__restrict__ slot)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    slot[i] = atomicAdd(&hist[cell_key(q4, i, g)], 1);
}

// Exclusive prefix sum of the kCellKeys counts in place: one block of 1024
// threads, kCellKeys / 1024 counts each.
__global__ void cell_scan_kernel(int *__restrict__ hist)
{
    constexpr int kPer = kCellKeys / 1024;
    __shared__ int part[1024];
    const int t = threadIdx.x;
    int v[kPer];
    int sum = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        v[k] = hist[t * kPer + k];
        sum += v[k];
    }
    part[t] = sum;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int u = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += u;
        __syncthreads();
    }
    int run = part[t] - sum;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        hist[t * kPer + k] = run;
        run += v[k];
    }
}

__global__ void cell_scatter_kernel(const double *__restrict__ q4, int n, CellGrid g,
                                    const int *__restrict__ start, const int *__restrict__ slot,
                                    int *__restrict__ order)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    order[start[cell_key(q4, i, g)] + slot[i]] = i;
}

int sort_rows_by_cell(const double *q4, int n, const double box[3], double rc, int *hist,
                      int *slot, int *order, cudaStream_t st)
{
    const CellGrid g = make_cell_grid(box, rc);
    LJ_TRY_CUDA(cudaMemsetAsync(hist, 0, sizeof(int) * kCellKeys, st));
    const unsigned b = unsigned((n + 255) / 256);
    cell_hist_kernel<<<b, 256, 0, st>>>(q4, n, g, hist, slot);
    LJ_TRY_LAUNCH("cell_hist_kernel");
    cell_scan_kernel<<<1, 1024, 0, st>>>(hist);
    LJ_TRY_LAUNCH("cell_scan_kernel");
    cell_scatter_kernel<<<b, 256, 0, st>>>(q4, n, g, hist, slot, order);
    LJ_TRY_LAUNCH("cell_scatter_kernel");
    return LJ_OK;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

template <int TPI, int U, bool IMG = false>
int launch_fp64(const double *q4, double *p4, int n, const int *rp, const int *col, int half,
                const Fp64Params &P, const int *order, cudaStream_t st)
{
    const int64_t threads = int64_t(n) * TPI;
    const unsigned grid = unsigned((threads + 255) / 256);
    if (half)
        force_fp64_kernel<TPI, true, U, IMG><<<grid, 256, 0, st>>>(q4, p4, n, rp, col, P, order);
    else
        force_fp64_kernel<TPI, false, U, IMG><<<grid, 256, 0, st>>>(q4, p4, n, rp, col, P, order);
    LJ_TRY_LAUNCH("force_fp64_kernel");
    return LJ_OK;
}

template <int TPI>
int launch_fixed(const double *q4, const longlong4 *X, double *p4, int n, const int *rp,
                 const int *col, int half, const Fp64Params &P, const FixParams &F, const int *order,
                 cudaStream_t st)
{
    const int64_t threads = int64_t(n) * TPI;
    const unsigned grid = unsigned((threads + 127) / 128);
    if (half)
        force_fixed_kernel<TPI, true><<<grid, 128, 0, st>>>(q4, X, p4, n, rp, col, P, F, order);
    else
        force_fixed_kernel<TPI, false><<<grid, 128, 0, st>>>(q4, X, p4, n, rp, col, P, F, order);
    LJ_TRY_LAUNCH("force_fixed_kernel");
    return LJ_OK;
}

template <int R>
int launch_fixed_stream(const double *q4, const longlong4 *X, double *p4, int n, const int *rp,
                        const int *col, int half, const Fp64Params &P, const FixParams &F,
                        cudaStream_t st)
{
    const int64_t warps = (int64_t(n) + R - 1) / R;
    const unsigned grid = unsigned((warps * 32 + 127) / 128);
    if (half)
        force_fixed_stream_kernel<true, R><<<grid, 128, 0, st>>>(q4, X, p4, n, rp, col, P, F);
    else
        force_fixed_stream_kernel<false, R><<<grid, 128, 0, st>>>(q4, X, p4, n, rp, col, P, F);
    LJ_TRY_LAUNCH("force_fixed_stream_kernel");
    return LJ_OK;
}

template <int TPI, int U = 1>
int launch_mixed(const double *q4, const uint4 *rel, double *p4, int n, const int *rp,
                 const int *col, int half, const MixedParams &P, const int *order, cudaStream_t st)
{
    const int64_t threads = int64_t(n) * TPI;
    const unsigned grid = unsigned((threads + 127) / 128);
    if (half)
        force_mixed_kernel<TPI, true, U><<<grid, 128, 0, st>>>(q4, rel, p4, n, rp, col, P, order);
    else
        force_mixed_kernel<TPI, false, U><<<grid, 128, 0, st>>>(q4, rel, p4, n, rp, col, P, order);
    LJ_TRY_LAUNCH("force_mixed_kernel");
    return LJ_OK;
}

}  // namespace

size_t dfloat_record_bytes(int64_t n);
bool dfloat_params_ok(const double box[3], double dt, double rc, double eps, double sigma);
int force_dfloat(const double *q4, double *p4, int n, const int *row_ptr, const int *col, int half,
                 const double box[3], double dt, double rc, double eps, double sigma, int tpi,
                 const int *order, void *rec_ws, cudaStream_t st);

int check_force_args(const double *q4, const double *p4, int64_t n, const int32_t *row_ptr,
                     const int32_t *col, int64_t nnz, double r_cut, const double box[3], double eps,
                     double sigma, double dt)
{
    if (n < 0 || nnz < 0 || !box) return LJ_ERR_ARG;
    if (n > 0 && (!q4 || !p4 || !row_ptr)) return LJ_ERR_ARG;
    if (nnz > 0 && !col) return LJ_ERR_ARG;
    // AoS4 rows are read with 256-bit loads: 32-byte alignment is required.
    if ((reinterpret_cast<uintptr_t>(q4) | reinterpret_cast<uintptr_t>(p4)) & 31u) return LJ_ERR_ARG;
    if (n >= (int64_t(1) << 31) - 1 || nnz >= (int64_t(1) << 31) - 1) return LJ_ERR_CAPACITY;
    if (!(r_cut > 0.0) || !std::isfinite(r_cut) || !(eps > 0.0) || !(sigma > 0.0) ||
        !std::isfinite(eps) || !std::isfinite(sigma) || !std::isfinite(dt))
        return LJ_ERR_ARG;
    if (r_cut * r_cut > 1e30) return LJ_ERR_ARG;
    return check_box(box, r_cut);
}

// Workspace: [order: n int][slot: n int][histogram] (the row order of
// LJ_SCHED_SORTED or LJ_SCHED_CELLS) and the fixed-point positions
// of the form (LJ_FP64: 64-bit integers; LJ_MIXED: 32-bit; LJ_DFLOAT:
// chunks).
struct ForceWs {
    int *order, *slot, *hist;
    uint4 *rel;
    void *rec;
};

ForceWs carve_force_ws(void *base, int64_t n, int precision)
{
    Carver c(base);
    ForceWs w;
    const size_t nn = size_t(n > 0 ? n : 1);
    w.order = c.take<int>(nn);
    w.slot = c.take<int>(nn);
    w.hist = c.take<int>(kCellKeys);  // the larger of the two counting sorts
    w.rel = precision == LJ_MIXED ? c.take<uint4>(nn) : nullptr;
    w.rec = precision == LJ_DFLOAT ? static_cast<void *>(c.take<char>(dfloat_record_bytes(n)))
            : precision == LJ_FP64 ? static_cast<void *>(c.take<longlong4>(nn))
                                   : nullptr;
    return w;
}

bool valid_schedule(int s, int precision)
{
    // the space-filling row order goes with every row-group schedule (as the
    // length-sorted one does, which it excludes)
    if (s & LJ_SCHED_CELLS) {
        if (s & (LJ_SCHED_SORTED | LJ_SCHED_STREAM)) return false;
        s = (s & ~LJ_SCHED_CELLS) | LJ_SCHED_SORTED;
    }
    const int t = s & 63;
    const bool pow2 = t == 1 || t == 2 || t == 4 || t == 8 || t == 16 || t == 32;
    if (s & LJ_SCHED_STREAM)  // rows per warp; implies the fixed-point rows, not length-sorted
        return precision == LJ_FP64 && (s & ~(LJ_SCHED_FIXED | LJ_SCHED_STREAM | 63)) == 0 &&
               (s & LJ_SCHED_FIXED) && (t == 4 || t == 8 || t == 16 || t == 32);
    if (s & LJ_SCHED_FIXED)
        return precision == LJ_FP64 && (s & ~(LJ_SCHED_FIXED | LJ_SCHED_SORTED | 63)) == 0 &&
               (t == 4 || t == 8 || t == 16);
    if (s & ~(LJ_SCHED_SORTED | LJ_SCHED_SWP2 | LJ_SCHED_IMAGES | 63)) return false;
    if (precision == LJ_DFLOAT) return (s & LJ_SCHED_IMAGES) == 0 && (t == 4 || t == 8 || t == 16);
    if (s & LJ_SCHED_IMAGES) return precision == LJ_FP64 && (t == 4 || t == 8 || t == 16);
    if (s & LJ_SCHED_SWP2) return t == 4 || t == 8 || t == 16;
    return pow2;
}

size_t force_workspace_bytes_impl(int64_t n, int precision)
{
    Carver c(nullptr);
    const size_t nn = size_t(n > 0 ? n : 1);
    c.take<int>(nn);
    c.take<int>(nn);
    c.take<int>(kCellKeys);
    if (precision == LJ_MIXED) c.take<uint4>(nn);
    if (precision == LJ_DFLOAT) c.take<char>(dfloat_record_bytes(n));
    if (precision == LJ_FP64) c.take<longlong4>(nn);
    return c.used + 256;
}

// The FP64 default for a half list of at least this many rows: 32 rows per
// warp walked as one stream (LJ_SCHED_STREAM); below it the 4,864 resident
// warps of a full GPU get fewer than four waves of 32-row windows and the
// grid over rows is as fast (N = 119,164: 0.226 ms against 0.230 for 8-row
// windows), and full lists keep the deterministic grid over rows.
constexpr int64_t kStreamDefaultRows = 524288;

// Every host-side check of lj_force, with no launch: the arguments, the
// form, the schedule (LJ_TPI_AUTO resolved into *tpi) and the workspace.
int force_check(const double *q4, const double *p4, int64_t n, const int32_t *row_ptr,
                const int32_t *col, int64_t nnz, int half, double dt, double rc,
                const double box[3], double eps, double sigma, int precision, int *tpi,
                const void *ws, size_t ws_bytes)
{
    int rcode = check_force_args(q4, p4, n, row_ptr, col, nnz, rc, box, eps, sigma, dt);
    if (rcode != LJ_OK) return rcode;
    if (precision != LJ_FP64 && precision != LJ_MIXED && precision != LJ_DFLOAT) return LJ_ERR_ARG;
    if (n == 0 || nnz == 0) return LJ_OK;
    int t = *tpi;
    if (t == LJ_TPI_AUTO) {
        if (precision == LJ_FP64)
            t = !fixed_point_ok(box, rc) ? (LJ_SCHED_IMAGES | 8)
                : (half && n >= kStreamDefaultRows && nnz <= kStreamMaxEntries)
                    ? (LJ_SCHED_FIXED | LJ_SCHED_STREAM | 32)
                                                     : (LJ_SCHED_FIXED | 8);
        else
            t = precision == LJ_DFLOAT ? (LJ_SCHED_SWP2 | 8) : 8;
    }
    if ((t & LJ_SCHED_FIXED) && !fixed_point_ok(box, rc)) return LJ_ERR_ARG;
    if (!valid_schedule(t, precision)) return LJ_ERR_ARG;
    if ((t & LJ_SCHED_STREAM) && nnz > kStreamMaxEntries) return LJ_ERR_CAPACITY;
    if (!ws || ws_bytes < force_workspace_bytes_impl(n, precision)) return LJ_ERR_CAPACITY;
    if (precision == LJ_DFLOAT && !dfloat_params_ok(box, dt, rc, eps, sigma)) return LJ_ERR_ARG;
    *tpi = t;
    return LJ_OK;
}

int force_impl(const double *q4, double *p4, int64_t n, const int32_t *row_ptr, const int32_t *col,
               int64_t nnz, int half, double dt, double rc, const double box[3], double eps,
               double sigma, int precision, int tpi, void *ws, size_t ws_bytes, cudaStream_t st)
{
    const int rcode = force_check(q4, p4, n, row_ptr, col, nnz, half, dt, rc, box, eps, sigma,
                                  precision, &tpi, ws, ws_bytes);
    if (rcode != LJ_OK) return rcode;
    if (n == 0 || nnz == 0) return LJ_OK;
    const int ni = static_cast<int>(n);
    const ForceWs W = carve_force_ws(ws, n, precision);
    const int *order = nullptr;
    if (tpi & LJ_SCHED_SORTED) {
        const int rc2 = sort_rows_by_length(row_ptr, ni, W.hist, W.slot, W.order, st);
        if (rc2 != LJ_OK) return rc2;
        order = W.order;
        tpi &= ~LJ_SCHED_SORTED;
    } else if (tpi & LJ_SCHED_CELLS) {
        const int rc2 = sort_rows_by_cell(q4, ni, box, rc, W.hist, W.slot, W.order, st);
        if (rc2 != LJ_OK) return rc2;
        order = W.order;
        tpi &= ~LJ_SCHED_CELLS;
    }
    if (precision == LJ_DFLOAT)
        return force_dfloat(q4, p4, ni, row_ptr, col, half, box, dt, rc, eps, sigma, tpi, order,
                            W.rec, st);
    if (precision == LJ_FP64 && (tpi & LJ_SCHED_FIXED)) {
        const Fp64Params P = make_fp64_params(box, dt, rc, eps, sigma);
        const FixParams F = make_fix_params(box);
        longlong4 *X = static_cast<longlong4 *>(W.rec);
        fixed_prepass_kernel<<<unsigned((n + 255) / 256), 256, 0, st>>>(q4, ni, F, X);
        LJ_TRY_LAUNCH("fixed_prepass_kernel");
        if (tpi & LJ_SCHED_STREAM) {
            switch (tpi & 63) {
                case 4: return launch_fixed_stream<4>(q4, X, p4, ni, row_ptr, col, half, P, F, st);
                case 8: return launch_fixed_stream<8>(q4, X, p4, ni, row_ptr, col, half, P, F, st);
                case 16: return launch_fixed_stream<16>(q4, X, p4, ni, row_ptr, col, half, P, F, st);
                case 32: return launch_fixed_stream<32>(q4, X, p4, ni, row_ptr, col, half, P, F, st);
                default: return LJ_ERR_ARG;
            }
        }
        switch (tpi & 63) {
            case 4: return launch_fixed<4>(q4, X, p4, ni, row_ptr, col, half, P, F, order, st);
            case 8: return launch_fixed<8>(q4, X, p4, ni, row_ptr, col, half, P, F, order, st);
            case 16: return launch_fixed<16>(q4, X, p4, ni, row_ptr, col, half, P, F, order, st);
            default: return LJ_ERR_ARG;
        }
    }
    if (precision == LJ_FP64) {
        const Fp64Params P = make_fp64_params(box, dt, rc, eps, sigma);
        switch (tpi) {
            case 1: return launch_fp64<1, 1>(q4, p4, ni, row_ptr, col, half, P, order, st);
            case 2: return launch_fp64<2, 1>(q4, p4, ni, row_ptr, col, half, P, order, st);
            case 4: return launch_fp64<4, 1>(q4, p4, ni, row_ptr, col, half, P, order, st);
            case 8: return launch_fp64<8, 1>(q4, p4, ni, row_ptr, col, half, P, order, st);
            case 16: return launch_fp64<16, 1>(q4, p4, ni, row_ptr, col, half, P, order, st);
            case 32: return launch_fp64<32, 1>(q4, p4, ni, row_ptr, col, half, P, order, st);
            case 4 | LJ_SCHED_SWP2: return launch_fp64<4, 2>(q4, p4, ni, row_ptr, col, half, P, order, st);
            case 8 | LJ_SCHED_SWP2: return launch_fp64<8, 2>(q4, p4, ni, row_ptr, col, half, P, order, st);
            case 16 | LJ_SCHED_SWP2: return launch_fp64<16, 2>(q4, p4, ni, row_ptr, col, half, P, order, st);
            case 4 | LJ_SCHED_IMAGES: return launch_fp64<4, 1, true>(q4, p4, ni, row_ptr, col, half, P, order, st);
            case 8 | LJ_SCHED_IMAGES: return launch_fp64<8, 1, true>(q4, p4, ni, row_ptr, col, half, P, order, st);
            case 16 | LJ_SCHED_IMAGES: return launch_fp64<16, 1, true>(q4, p4, ni, row_ptr, col, half, P, order, st);
            case 4 | LJ_SCHED_SWP2 | LJ_SCHED_IMAGES: return launch_fp64<4, 2, true>(q4, p4, ni, row_ptr, col, half, P, order, st);
            case 8 | LJ_SCHED_SWP2 | LJ_SCHED_IMAGES: return launch_fp64<8, 2, true>(q4, p4, ni, row_ptr, col, half, P, order, st);
            case 16 | LJ_SCHED_SWP2 | LJ_SCHED_IMAGES: return launch_fp64<16, 2, true>(q4, p4, ni, row_ptr, col, half, P, order, st);
            default: return LJ_ERR_ARG;
        }
    }
    const MixedParams P = make_mixed_params(box, dt, rc, eps, sigma);
    uint4 *rel = W.rel;
    mixed_prepass_kernel<<<unsigned((n + 255) / 256), 256, 0, st>>>(q4, ni, P, rel);
    LJ_TRY_LAUNCH("mixed_prepass_kernel");
    switch (tpi) {
        case LJ_SCHED_SWP2 | 4: return launch_mixed<4, 2>(q4, rel, p4, ni, row_ptr, col, half, P, order, st);
        case LJ_SCHED_SWP2 | 8: return launch_mixed<8, 2>(q4, rel, p4, ni, row_ptr, col, half, P, order, st);
        case LJ_SCHED_SWP2 | 16: return launch_mixed<16, 2>(q4, rel, p4, ni, row_ptr, col, half, P, order, st);
        case 1: return launch_mixed<1>(q4, rel, p4, ni, row_ptr, col, half, P, order, st);
        case 2: return launch_mixed<2>(q4, rel, p4, ni, row_ptr, col, half, P, order, st);
        case 4: return launch_mixed<4>(q4, rel, p4, ni, row_ptr, col, half, P, order, st);
        case 8: return launch_mixed<8>(q4, rel, p4, ni, row_ptr, col, half, P, order, st);
        case 16: return launch_mixed<16>(q4, rel, p4, ni, row_ptr, col, half, P, order, st);
        case 32: return launch_mixed<32>(q4, rel, p4, ni, row_ptr, col, half, P, order, st);
        default: return LJ_ERR_ARG;
    }
}

}  // namespace lj

extern "C" size_t lj_force_energy_workspace_bytes(int64_t n)
{
    const int64_t blocks = (std::max<int64_t>(n, 1) * 8 + 255) / 256;
    lj::Carver c(nullptr);
    c.take<double>(3 * size_t(blocks));
    c.take<longlong4>(size_t(std::max<int64_t>(n, 1)));
    return c.used + 256;
}

namespace lj {
namespace {

int force_energy_impl(const double *q4_dev, double *p4_dev, int64_t n, const int32_t *row_ptr_dev,
                      const int32_t *col_dev, int64_t nnz, int half, double dt, double r_cut,
                      const double box[3], double eps, double sigma, int shifted, double *e_out_dev,
                      double *w_out_dev, void *workspace_dev, size_t workspace_bytes,
                      cudaStream_t st)
{
    int rc = check_force_args(q4_dev, p4_dev, n, row_ptr_dev, col_dev, nnz, r_cut, box, eps, sigma,
                              dt);
    if (rc != LJ_OK) return rc;
    if (!e_out_dev || (reinterpret_cast<uintptr_t>(e_out_dev) & 7u)) return LJ_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(w_out_dev) & 7u) return LJ_ERR_ARG;
    if (n == 0 || nnz == 0) {
        LJ_TRY_CUDA(cudaMemsetAsync(e_out_dev, 0, sizeof(double), st));
        if (w_out_dev) LJ_TRY_CUDA(cudaMemsetAsync(w_out_dev, 0, sizeof(double), st));
        return LJ_OK;
    }
    if (!workspace_dev || workspace_bytes < lj_force_energy_workspace_bytes(n)) return LJ_ERR_CAPACITY;
    const Fp64Params P = make_fp64_params(box, dt, r_cut, eps, sigma);
    const FixParams F = make_fix_params(box);
    const int blocks = static_cast<int>((n * 8 + 255) / 256);
    Carver c(workspace_dev);
    double *partial = c.take<double>(3 * size_t(blocks));
    longlong4 *X = c.take<longlong4>(size_t(n));
    if (fixed_point_ok(box, r_cut)) {
        fixed_prepass_kernel<<<unsigned((n + 255) / 256), 256, 0, st>>>(q4_dev, static_cast<int>(n), F, X);
        LJ_TRY_LAUNCH("fixed_prepass_kernel");
    } else {
        X = nullptr;
    }
    force_energy_fp64_kernel<false><<<blocks, 256, 0, st>>>(q4_dev, X, p4_dev, static_cast<int>(n),
                                                            row_ptr_dev, col_dev, P, F, half, partial);
    LJ_TRY_LAUNCH("force_energy_fp64_kernel");
    double vshift = 0.0;
    if (shifted) {
        const double sr2 = sigma * sigma / (r_cut * r_cut), sr6 = sr2 * sr2 * sr2;
        vshift = 4.0 * eps * (sr6 * sr6 - sr6);
    }
    energy_partials_kernel<<<1, 1024, 0, st>>>(partial, blocks, half ? 1.0 : 0.5, vshift, e_out_dev,
                                               w_out_dev);
    LJ_TRY_LAUNCH("energy_partials_kernel");
    return LJ_OK;
}

}  // namespace
}  // namespace lj

extern "C" int lj_force_energy(const double *q4_dev, double *p4_dev, int64_t n,
                               const int32_t *row_ptr_dev, const int32_t *col_dev, int64_t nnz,
                               int half, double dt, double r_cut, const double box[3], double eps,
                               double sigma, int shifted, double *e_out_dev, void *workspace_dev,
                               size_t workspace_bytes, void *stream)
{
    return lj::force_energy_impl(q4_dev, p4_dev, n, row_ptr_dev, col_dev, nnz, half, dt, r_cut, box,
                                 eps, sigma, shifted, e_out_dev, nullptr, workspace_dev,
                                 workspace_bytes, static_cast<cudaStream_t>(stream));
}

extern "C" int lj_force_energy_virial(const double *q4_dev, double *p4_dev, int64_t n,
                                      const int32_t *row_ptr_dev, const int32_t *col_dev,
                                      int64_t nnz, int half, double dt, double r_cut,
                                      const double box[3], double eps, double sigma, int shifted,
                                      double *e_out_dev, double *w_out_dev, void *workspace_dev,
                                      size_t workspace_bytes, void *stream)
{
    if (!w_out_dev) return LJ_ERR_ARG;
    return lj::force_energy_impl(q4_dev, p4_dev, n, row_ptr_dev, col_dev, nnz, half, dt, r_cut, box,
                                 eps, sigma, shifted, e_out_dev, w_out_dev, workspace_dev,
                                 workspace_bytes, static_cast<cudaStream_t>(stream));
}

extern "C" size_t lj_force_shifted_workspace_bytes(int64_t n)
{
    return lj_force_energy_workspace_bytes(n);
}

extern "C" int lj_force_shifted(const double *q4_dev, double *p4_dev, int64_t n,
                                const int32_t *row_ptr_dev, const int32_t *col_dev, int64_t nnz,
                                int half, double dt, double r_cut, const double box[3], double eps,
                                double sigma, double *e_out_dev, void *workspace_dev,
                                size_t workspace_bytes, void *stream)
{
    using namespace lj;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = check_force_args(q4_dev, p4_dev, n, row_ptr_dev, col_dev, nnz, r_cut, box, eps, sigma,
                              dt);
    if (rc != LJ_OK) return rc;
    if (e_out_dev && (reinterpret_cast<uintptr_t>(e_out_dev) & 7u)) return LJ_ERR_ARG;
    if (!fixed_point_ok(box, r_cut)) return LJ_ERR_ARG;
    if (n == 0 || nnz == 0) {
        if (e_out_dev) LJ_TRY_CUDA(cudaMemsetAsync(e_out_dev, 0, sizeof(double), st));
        return LJ_OK;
    }
    if (!workspace_dev || workspace_bytes < lj_force_shifted_workspace_bytes(n)) return LJ_ERR_CAPACITY;
    const Fp64Params P = make_fp64_params(box, dt, r_cut, eps, sigma);
    const FixParams F = make_fix_params(box);
    const int ni = static_cast<int>(n);
    const int blocks = static_cast<int>((n * 8 + 255) / 256);
    Carver c(workspace_dev);
    double *partial = c.take<double>(3 * size_t(blocks));
    longlong4 *X = c.take<longlong4>(size_t(n));
    fixed_prepass_kernel<<<unsigned((n + 255) / 256), 256, 0, st>>>(q4_dev, ni, F, X);
    LJ_TRY_LAUNCH("fixed_prepass_kernel");
    if (e_out_dev) {
        force_energy_fp64_kernel<true><<<blocks, 256, 0, st>>>(q4_dev, X, p4_dev, ni, row_ptr_dev,
                                                               col_dev, P, F, half, partial);
        LJ_TRY_LAUNCH("force_energy_fp64_kernel");
        energy_partials_kernel<<<1, 1024, 0, st>>>(partial, blocks, half ? 1.0 : 0.5, 0.0, e_out_dev,
                                                   nullptr);
        LJ_TRY_LAUNCH("energy_partials_kernel");
    } else {
        if (half)
            force_fs_kernel<true><<<blocks, 256, 0, st>>>(q4_dev, X, p4_dev, ni, row_ptr_dev, col_dev, P, F);
        else
            force_fs_kernel<false><<<blocks, 256, 0, st>>>(q4_dev, X, p4_dev, ni, row_ptr_dev, col_dev, P, F);
        LJ_TRY_LAUNCH("force_fs_kernel");
    }
    return LJ_OK;
}

extern "C" size_t lj_force_workspace_bytes(int64_t n, const double box[3], int precision)
{
    (void)box;
    return lj::force_workspace_bytes_impl(n, precision);
}

extern "C" int lj_force(const double *q4_dev, double *p4_dev, int64_t n, const int32_t *row_ptr_dev,
                        const int32_t *col_dev, int64_t nnz, int half, double dt, double r_cut,
                        const double box[3], double eps, double sigma, int precision, int tpi,
                        void *workspace_dev, size_t workspace_bytes, void *stream)
{
    return lj::force_impl(q4_dev, p4_dev, n, row_ptr_dev, col_dev, nnz, half, dt, r_cut, box, eps,
                          sigma, precision, tpi, workspace_dev, workspace_bytes,
                          static_cast<cudaStream_t>(stream));
}

// lj_pairlist.cu -- GPU construction of the sorted CSR Verlet list.
//
// Paper basis (Watanabe & Nakagawa, arXiv 1806.05713): section "Verlet List
// and Bookkeeping Method" (register every pair closer than the search length
// r_s > r_c; the linked-list cell method makes this O(N)) and section
// "Sorting by Indices" (group the j of each i with a counting sort; Fig.
// "Data layout of a pair list" (b), (c) is this CSR).
//
// GB300 design:
//   1. bin:      one thread per atom -> cell id (cells of side >= r_s / 2,
//                so every partner within r_s lies in the 5 x 5 x 5 cells
//                around an atom's own) and a slot inside the cell (atomic
//                counter); validates q in [0, L).
//   2. scan:     exclusive prefix sum of the cell counts -> cell_start.
//   3. scatter:  atoms in cell order, with an FP32 copy {x, y, z, id} so that
//                the candidate loops below stream 16-byte records.
//   4. walk:     one warp per atom (atoms taken in cell order, so
//                neighbouring warps share their neighbour cells in L1/L2);
//                the five cells of a row of the stencil along x are
//                consecutive in the cell order, so they are walked as one
//                run of candidates (two where the stencil wraps around the
//                box) -- runs of ~27 atoms at density 1 instead of cells of
//                ~5; candidates are screened in FP32 against r_s^2 (1 +-
//                delta) with a proven error bound delta, and only the rare
//                candidates inside the band are decided by the exact FP64
//                definition.  Default (five or more cells on every axis and
//                room for the row slabs): the FORWARD half of the stencil
//                only -- 12.5 runs instead of 25 -- each pair met once and
//                appended, through a per-row atomic slot counter, to the
//                slab of its smaller index (half list) or to both slabs
//                (full list).  Otherwise the full stencil per row i, either
//                into row i's slab or, with no room for slabs, counted
//                first and filled later (the two-walk path).
//   5. scan:     row counts -> row_ptr; total and longest row read back.
//   6. sort:     each slab sorted into its place in col -- a bitonic
//                network in the warp's registers for rows of up to 256
//                entries, a rank sort in shared memory beyond (all j of a
//                row are distinct); the two-walk path instead walks again,
//                compacts the j of the row into shared memory (ballot +
//                popc), sorts them the same way and writes the sorted row.
// The result is bit-exact against the FP64 definition because every
// decision is either certain from the FP32 bound or taken with the exact
// IEEE operations (d = q_j - q_i, minimum image, (dx*dx + dy*dy) + dz*dz,
// no fused multiply-add).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "lj_internal.cuh"
#include "lj_scan.cuh"

namespace lj {
namespace {

constexpr int kWarpsPerBlock = 8;
constexpr int kMaxRowSmem = 56000;  // longest row one warp can sort in shared memory

struct ListStats {
    int64_t nnz;
    int max_row;
    int err;
};

struct Grid {
    int nc[3];
    int noff[3];
    int off[3][5];
    double L[3];
    long long half_bits[3];
    float Lf[3];
    float hLf[3];
    double inv_h[3];
    long long rs2_bits;
    float lo, hi;  // FP32 screening band around r_s^2
    int ncell;
};

// Cells of side >= r_s / 2.
int cells_per_axis(double L, double rs)
{
    const double side = 0.5 * rs;
    int nc = static_cast<int>(std::floor(L / side));
    while (nc > 1 && L / nc < side * (1.0 + 1e-12)) --nc;
    return nc < 1 ? 1 : nc;
}

Grid make_grid(int64_t n, const double box[3], double rs)
{
    Grid g{};
    for (int a = 0; a < 3; ++a) g.nc[a] = cells_per_axis(box[a], rs);
    // Larger cells stay correct (side >= r_s); cap the cell count near 2n.
    const long long limit = 2 * static_cast<long long>(n) + 64;
    while (static_cast<long long>(g.nc[0]) * g.nc[1] * g.nc[2] > limit) {
        int a = 0;
        if (g.nc[1] > g.nc[a]) a = 1;
        if (g.nc[2] > g.nc[a]) a = 2;
        if (g.nc[a] <= 1) break;
        --g.nc[a];
    }
    double Lmax = 0.0;
    for (int a = 0; a < 3; ++a) {
        const int nc = g.nc[a];
        // Offsets -2..2; with fewer than five cells on the axis every cell
        // is a neighbour and each is listed once (offsets 0..nc-1).
        if (nc < 5) {
            g.noff[a] = nc;
            for (int o = 0; o < nc; ++o) g.off[a][o] = o;
        } else {
            g.noff[a] = 5;
            for (int o = 0; o < 5; ++o) g.off[a][o] = o - 2;
        }
        g.L[a] = box[a];
        const double h = 0.5 * box[a];
        std::memcpy(&g.half_bits[a], &h, sizeof(double));
        g.Lf[a] = static_cast<float>(box[a]);
        g.hLf[a] = 0.5f * g.Lf[a];
        g.inv_h[a] = nc / box[a];
        Lmax = std::max(Lmax, box[a]);
    }
    g.ncell = g.nc[0] * g.nc[1] * g.nc[2];
    const double rs2 = rs * rs;
    std::memcpy(&g.rs2_bits, &rs2, sizeof(double));
    // |r2_fp32 - r2| <= ~8.3e-7 (L/r_s) r_s^2 + rounding of the FP32 sum;
    // take four times that.
    const double delta = 4e-6 + 4e-6 * (Lmax / rs);
    g.lo = std::nextafter(static_cast<float>(rs2 * (1.0 - delta)), 0.0f);
    if (!(g.lo > 0.0f)) g.lo = 0.0f;
    g.hi = std::nextafter(static_cast<float>(rs2 * (1.0 + delta)), INFINITY);
    return g;
}

struct Work {
    int *cell_of;
    int *slot;
    int *cell_count;
    int *cell_start;
    int *cell_atoms;
    float4 *pos_f;
    int *row_cnt;
    ListStats *stats;
    int64_t *scan_scratch;
};

Work carve(void *base, int64_t n, int ncell)
{
    Carver c(base);
    Work w;
    const size_t nn = static_cast<size_t>(n > 0 ? n : 1);
    w.cell_of = c.take<int>(nn);
    w.slot = c.take<int>(nn);
    w.cell_count = c.take<int>(size_t(ncell) + 1);
    w.cell_start = c.take<int>(size_t(ncell) + 1);
    w.cell_atoms = c.take<int>(nn);
    w.pos_f = c.take<float4>(nn);
    w.row_cnt = c.take<int>(nn);
    w.stats = c.take<ListStats>(1);
    const size_t words = std::max(scan_scratch_words(n), scan_scratch_words(ncell));
    w.scan_scratch = c.take<int64_t>(words);
    return w;
}

size_t carve_bytes(int64_t n, int ncell)
{
    Carver c(nullptr);
    const size_t nn = static_cast<size_t>(n > 0 ? n : 1);
    c.take<int>(nn);
    c.take<int>(nn);
    c.take<int>(size_t(ncell) + 1);
    c.take<int>(size_t(ncell) + 1);
    c.take<int>(nn);
    c.take<float4>(nn);
    c.take<int>(nn);
    c.take<ListStats>(1);
    c.take<int64_t>(std::max(scan_scratch_words(n), scan_scratch_words(ncell)));
    return c.used + 256;
}

__global__ void bin_kernel(const double *__restrict__ q4, int n, Grid g, int *__restrict__ cell_of,
                           int *__restrict__ slot, int *__restrict__ cell_count,
                           ListStats *__restrict__ stats)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x[3];
    load_xyz(q4, i, x[0], x[1], x[2]);
    int c[3];
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        ok = ok && (x[a] >= 0.0) && (x[a] < g.L[a]);  // false for NaN
        int ca = static_cast<int>(x[a] * g.inv_h[a]);
        ca = ca < 0 ? 0 : (ca >= g.nc[a] ? g.nc[a] - 1 : ca);
        c[a] = ca;
    }
    if (!ok) atomicOr(&stats->err, 1);
    const int id = (c[2] * g.nc[1] + c[1]) * g.nc[0] + c[0];
    cell_of[i] = id;
    slot[i] = atomicAdd(&cell_count[id], 1);
}

__global__ void scatter_kernel(const double *__restrict__ q4, int n, int ncell,
                               const int *__restrict__ cell_of, const int *__restrict__ slot,
                               int *__restrict__ cell_start, int *__restrict__ cell_atoms,
                               float4 *__restrict__ pos_f)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) cell_start[ncell] = n;
    if (i >= n) return;
    const int k = cell_start[cell_of[i]] + slot[i];
    double x, y, z;
    load_xyz(q4, i, x, y, z);
    cell_atoms[k] = i;
    pos_f[k] = make_float4(static_cast<float>(x), static_cast<float>(y), static_cast<float>(z),
                           __int_as_float(i));
}

// Exact FP64 decision, identical operations to the definition.
__device__ __forceinline__ bool exact_within(const double *__restrict__ q4, int j, double xi,
                                             double yi, double zi, const Grid &g)
{
    double xj, yj, zj;
    load_xyz(q4, j, xj, yj, zj);
    const double dx = min_image(__dsub_rn(xj, xi), g.L[0], g.half_bits[0]);
    const double dy = min_image(__dsub_rn(yj, yi), g.L[1], g.half_bits[1]);
    const double dz = min_image(__dsub_rn(zj, zi), g.L[2], g.half_bits[2]);
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return less_nonneg(r2, g.rs2_bits);
}

// Walks every candidate j of row i (the atoms of the distinct neighbour
// cells), calling visit(in_mask) once per 32 candidates with the warp's
// ballot of accepted j (and each lane's j in `jout`).
template <bool HALF, class Visit>
__device__ __forceinline__ void walk_row(const double *__restrict__ q4, const Grid &g,
                                         const int *__restrict__ cell_start,
                                         const float4 *__restrict__ pos_f, int i, float4 pi,
                                         int cell_i, Visit visit)
{
    const int lane = threadIdx.x & 31;
    const int cx = cell_i % g.nc[0];
    const int cy = (cell_i / g.nc[0]) % g.nc[1];
    const int cz = cell_i / (g.nc[0] * g.nc[1]);
    bool have_exact = false;
    double xi = 0.0, yi = 0.0, zi = 0.0;
    // The x-neighbours of a stencil row: cells x0..x1 (consecutive in the
    // cell order), plus x2..x3 where the stencil wraps (empty otherwise).
    int x0, x1, x2 = 0, x3 = -1;
    if (g.noff[0] < 5) {
        x0 = 0;
        x1 = g.nc[0] - 1;
    } else if (cx - 2 < 0) {
        x0 = 0;
        x1 = cx + 2;
        x2 = g.nc[0] + cx - 2;
        x3 = g.nc[0] - 1;
    } else if (cx + 2 >= g.nc[0]) {
        x0 = cx - 2;
        x1 = g.nc[0] - 1;
        x2 = 0;
        x3 = cx + 2 - g.nc[0];
    } else {
        x0 = cx - 2;
        x1 = cx + 2;
    }
    for (int oz = 0; oz < g.noff[2]; ++oz) {
        int nz = cz + g.off[2][oz];
        nz = nz < 0 ? nz + g.nc[2] : (nz >= g.nc[2] ? nz - g.nc[2] : nz);
        for (int oy = 0; oy < g.noff[1]; ++oy) {
            int ny = cy + g.off[1][oy];
            ny = ny < 0 ? ny + g.nc[1] : (ny >= g.nc[1] ? ny - g.nc[1] : ny);
            const int rowc = (nz * g.nc[1] + ny) * g.nc[0];
            for (int run = 0; run < 2; ++run) {
                const int xa = run == 0 ? x0 : x2, xb = run == 0 ? x1 : x3;
                if (xb < xa) continue;  // no second run (warp-uniform)
                const int s = cell_start[rowc + xa], e = cell_start[rowc + xb + 1];
                for (int base = s; base < e; base += 32) {
                    const int k = base + lane;
                    bool in = false;
                    int j = -1;
                    if (k < e) {
                        const float4 pj = pos_f[k];
                        j = __float_as_int(pj.w);
                        if (HALF ? (j > i) : (j != i)) {
                            float dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
                            if (fabsf(dx) > g.hLf[0]) dx -= copysignf(g.Lf[0], dx);
                            if (fabsf(dy) > g.hLf[1]) dy -= copysignf(g.Lf[1], dy);
                            if (fabsf(dz) > g.hLf[2]) dz -= copysignf(g.Lf[2], dz);
                            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                            if (r2 < g.lo) {
                                in = true;
                            } else if (r2 < g.hi) {
                                if (!have_exact) {
                                    load_xyz(q4, i, xi, yi, zi);
                                    have_exact = true;
                                }
                                in = exact_within(q4, j, xi, yi, zi, g);
                            }
                        }
                    }
                    visit(__ballot_sync(0xffffffffu, in), in, j);
                }
            }
        }
    }
}

// A row of len <= 32 E entries (E = 1, 2, 4 or 8) sorted by a bitonic network
// held in registers: entry index u 32 + lane lives in v[u] of that lane,
// pairs 32 or more apart are compared inside a lane, nearer ones across
// lanes with shuffles; padding INT_MAX sorts last.  For long rows it takes
// fewer instructions than ranking every entry against the whole row.
template <int E>
__device__ __forceinline__ void bitonic_row(const int *__restrict__ buf, int len, int lane,
                                            int32_t *__restrict__ out)
{
    constexpr int N = 32 * E;
    int v[E];
#pragma unroll
    for (int u = 0; u < E; ++u) {
        const int e = lane + 32 * u;
        v[u] = e < len ? buf[e] : INT32_MAX;
    }
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
#pragma unroll
                for (int u = 0; u < E; ++u) {
                    const int pu = u ^ (j >> 5);
                    if (pu > u) {
                        const bool asc = ((u * 32) & k) == 0;  // k > 32: set by u alone
                        const int a = v[u], b = v[pu];
                        const bool swap = asc ? (a > b) : (a < b);
                        v[u] = swap ? b : a;
                        v[pu] = swap ? a : b;
                    }
                }
            } else {
#pragma unroll
                for (int u = 0; u < E; ++u) {
                    const int other = __shfl_xor_sync(0xffffffffu, v[u], j);
                    const bool asc = ((u * 32 + lane) & k) == 0;
                    const bool lower = (lane & j) == 0;
                    v[u] = (lower == asc) ? min(v[u], other) : max(v[u], other);
                }
            }
        }
    }
#pragma unroll
    for (int u = 0; u < E; ++u)
        if (lane + 32 * u < len) out[lane + 32 * u] = v[u];
}

// Sorts row `buf` (len distinct j) into out with a bitonic network when it
// has at most 256 entries; returns false for a longer row (left to the
// caller's rank sort).
__device__ __forceinline__ bool bitonic_sort_row(const int *__restrict__ buf, int len, int lane,
                                                 int32_t *__restrict__ out)
{
    switch ((len + 31) >> 5) {
        case 0: return true;
        case 1: bitonic_row<1>(buf, len, lane, out); return true;
        case 2: bitonic_row<2>(buf, len, lane, out); return true;
        case 3:
        case 4: bitonic_row<4>(buf, len, lane, out); return true;
        case 5:
        case 6:
        case 7:
        case 8: bitonic_row<8>(buf, len, lane, out); return true;
        default: return false;
    }
}

template <bool HALF>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
count_kernel(const double *__restrict__ q4, int n, Grid g, const int *__restrict__ cell_of,
             const int *__restrict__ cell_start, const int *__restrict__ cell_atoms,
             const float4 *__restrict__ pos_f, int *__restrict__ row_cnt,
             ListStats *__restrict__ stats)
{
    const int w = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (w >= n) return;
    const int i = cell_atoms[w];
    const float4 pi = pos_f[w];
    int cnt = 0;
    walk_row<HALF>(q4, g, cell_start, pos_f, i, pi, cell_of[i],
                   [&](unsigned mask, bool, int) { cnt += __popc(mask); });
    if ((threadIdx.x & 31) == 0) {
        row_cnt[i] = cnt;
        atomicMax(&stats->max_row, cnt);
    }
}

template <bool HALF>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
fill_kernel(const double *__restrict__ q4, int n, Grid g, const int *__restrict__ cell_of,
            const int *__restrict__ cell_start, const int *__restrict__ cell_atoms,
            const float4 *__restrict__ pos_f, const int *__restrict__ row_ptr,
            int *__restrict__ col, int cap, int warps_per_block, ListStats *__restrict__ stats)
{
    extern __shared__ int smem[];
    const int wib = threadIdx.x >> 5;
    const int w = blockIdx.x * warps_per_block + wib;
    if (w >= n) return;
    const int lane = threadIdx.x & 31;
    int *buf = smem + size_t(wib) * cap;
    const int i = cell_atoms[w];
    const float4 pi = pos_f[w];
    int cnt = 0;
    walk_row<HALF>(q4, g, cell_start, pos_f, i, pi, cell_of[i],
                   [&](unsigned mask, bool in, int j) {
                       const int pos = cnt + __popc(mask & lanemask_lt());
                       if (in && pos < cap) buf[pos] = j;
                       cnt += __popc(mask);
                   });
    __syncwarp();
    const int start = row_ptr[i];
    const int len = row_ptr[i + 1] - start;
    // Unreachable by construction: the count and the fill run the same walk
    // (walk_row, same arithmetic, same inputs), so the fill meets exactly
    // the row's counted entries, and cap is the longest counted row.  Only a
    // caller writing q between the two kernels could break it; the row is
    // then left unwritten and the bit recorded, but the host has already
    // read the statistics, so nothing reports it.
    if (cnt != len || cnt > cap) {
        if (lane == 0) atomicOr(&stats->err, 2);
        return;
    }
    if (bitonic_sort_row(buf, cnt, lane, col + start)) return;
    // Rank sort: the j of a row are distinct, so rank(v) = #{m : buf[m] < v}.
    for (int e = lane; e < cnt; e += 32) {
        const int v = buf[e];
        int r = 0;
        int m = 0;
        for (; m + 4 <= cnt; m += 4)
            r += (buf[m] < v) + (buf[m + 1] < v) + (buf[m + 2] < v) + (buf[m + 3] < v);
        for (; m < cnt; ++m) r += buf[m] < v;
        col[start + r] = v;
    }
}

// One-walk build: the row's accepted j, in walk order, into its slab
// tmp[i * cap .. i * cap + cap) (rows longer than cap are only counted and
// flagged; the caller then finishes with fill_kernel).
template <bool HALF>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
walk_store_kernel(const double *__restrict__ q4, int n, Grid g, const int *__restrict__ cell_of,
                  const int *__restrict__ cell_start, const int *__restrict__ cell_atoms,
                  const float4 *__restrict__ pos_f, int *__restrict__ tmp, int cap,
                  int *__restrict__ row_cnt, ListStats *__restrict__ stats)
{
    const int w = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (w >= n) return;
    const int i = cell_atoms[w];
    const float4 pi = pos_f[w];
    int *dst = tmp + static_cast<size_t>(i) * cap;
    int cnt = 0;
    walk_row<HALF>(q4, g, cell_start, pos_f, i, pi, cell_of[i],
                   [&](unsigned mask, bool in, int j) {
                       const int pos = cnt + __popc(mask & lanemask_lt());
                       if (in && pos < cap) dst[pos] = j;
                       cnt += __popc(mask);
                   });
    if ((threadIdx.x & 31) == 0) {
        row_cnt[i] = cnt;
        atomicMax(&stats->max_row, cnt);
        if (cnt > cap) atomicOr(&stats->err, 4);
    }
}

// One walk over HALF the stencil (every axis with at least five cells, so
// each neighbour cell is one offset in -2..2): the warp of atom a
// (cell-order position w) takes the 62 forward cells -- offset dz > 0, or
// dz = 0 and dy > 0, or dz = dy = 0 and dx > 0 -- and the atoms after it in
// its own cell, so every unordered pair of atoms within reach is met once
// instead of twice.  A pair found closer than r_s goes, for the half list,
// to the row of its smaller index (the larger index into that row's slab),
// for the full list to both rows; each store takes its slot from an atomic
// counter of the row, and the rows are sorted afterwards.  The exact
// decision is the definition's: d = q_b - q_a is the negation of q_a - q_b,
// and the minimum image and the squares are symmetric under it.
__device__ __forceinline__ void append_slab(int row, int val, int *__restrict__ tmp, int cap,
                                            int *__restrict__ row_cnt, ListStats *__restrict__ stats)
{
    const int slot = atomicAdd(&row_cnt[row], 1);
    if (slot < cap)
        tmp[static_cast<size_t>(row) * cap + slot] = val;
    else
        atomicOr(&stats->err, 4);
}

template <bool HALF>
__device__ __forceinline__ void forward_run(const double *__restrict__ q4, const Grid &g,
                                            const float4 *__restrict__ pos_f, int s, int e, int ia,
                                            float4 pa, bool &have_exact, double &xa, double &ya,
                                            double &za, int *__restrict__ tmp, int cap,
                                            int *__restrict__ row_cnt, ListStats *__restrict__ stats)
{
    const int lane = threadIdx.x & 31;
    for (int base = s; base < e; base += 32) {
        const int k = base + lane;
        if (k >= e) break;
        const float4 pj = pos_f[k];
        const int jb = __float_as_int(pj.w);
        float dx = pj.x - pa.x, dy = pj.y - pa.y, dz = pj.z - pa.z;
        if (fabsf(dx) > g.hLf[0]) dx -= copysignf(g.Lf[0], dx);
        if (fabsf(dy) > g.hLf[1]) dy -= copysignf(g.Lf[1], dy);
        if (fabsf(dz) > g.hLf[2]) dz -= copysignf(g.Lf[2], dz);
        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        bool in = r2 < g.lo;
        if (!in && r2 < g.hi) {
            if (!have_exact) {
                load_xyz(q4, ia, xa, ya, za);
                have_exact = true;
            }
            in = exact_within(q4, jb, xa, ya, za, g);
        }
        if (in) {
            if (HALF) {
                append_slab(ia < jb ? ia : jb, ia < jb ? jb : ia, tmp, cap, row_cnt, stats);
            } else {
                append_slab(ia, jb, tmp, cap, row_cnt, stats);
                append_slab(jb, ia, tmp, cap, row_cnt, stats);
            }
        }
    }
}

template <bool HALF>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
walk_forward_store_kernel(const double *__restrict__ q4, int n, Grid g,
                          const int *__restrict__ cell_of, const int *__restrict__ cell_start,
                          const int *__restrict__ cell_atoms, const float4 *__restrict__ pos_f,
                          int *__restrict__ tmp, int cap, int *__restrict__ row_cnt,
                          ListStats *__restrict__ stats)
{
    const int w = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (w >= n) return;
    const int ia = cell_atoms[w];
    const float4 pa = pos_f[w];
    const int cell_a = cell_of[ia];
    const int cx = cell_a % g.nc[0];
    const int cy = (cell_a / g.nc[0]) % g.nc[1];
    const int cz = cell_a / (g.nc[0] * g.nc[1]);
    bool have_exact = false;
    double xa = 0.0, ya = 0.0, za = 0.0;
    auto wrap = [](int c, int nc) { return c < 0 ? c + nc : (c >= nc ? c - nc : c); };
    // x-cells cx-2..cx+2 of a stencil row as up to two consecutive runs
    int x0, x1, x2 = 0, x3 = -1;
    if (cx - 2 < 0) {
        x0 = 0;
        x1 = cx + 2;
        x2 = g.nc[0] + cx - 2;
        x3 = g.nc[0] - 1;
    } else if (cx + 2 >= g.nc[0]) {
        x0 = cx - 2;
        x1 = g.nc[0] - 1;
        x2 = 0;
        x3 = cx + 2 - g.nc[0];
    } else {
        x0 = cx - 2;
        x1 = cx + 2;
    }
    for (int dz = 0; dz <= 2; ++dz) {
        const int nz = wrap(cz + dz, g.nc[2]);
        for (int dy = (dz == 0 ? 0 : -2); dy <= 2; ++dy) {
            const int ny = wrap(cy + dy, g.nc[1]);
            const int rowc = (nz * g.nc[1] + ny) * g.nc[0];
            if (dz == 0 && dy == 0) {
                // own row: the atoms after a in its cell, then cells cx+1, cx+2
                if (cx + 2 < g.nc[0]) {
                    forward_run<HALF>(q4, g, pos_f, w + 1, cell_start[rowc + cx + 3], ia, pa,
                                      have_exact, xa, ya, za, tmp, cap, row_cnt, stats);
                } else {
                    forward_run<HALF>(q4, g, pos_f, w + 1, cell_start[rowc + g.nc[0]], ia, pa,
                                      have_exact, xa, ya, za, tmp, cap, row_cnt, stats);
                    forward_run<HALF>(q4, g, pos_f, cell_start[rowc],
                                      cell_start[rowc + cx + 3 - g.nc[0]], ia, pa, have_exact, xa,
                                      ya, za, tmp, cap, row_cnt, stats);
                }
                continue;
            }
            forward_run<HALF>(q4, g, pos_f, cell_start[rowc + x0], cell_start[rowc + x1 + 1], ia,
                              pa, have_exact, xa, ya, za, tmp, cap, row_cnt, stats);
            if (x3 >= x2)
                forward_run<HALF>(q4, g, pos_f, cell_start[rowc + x2], cell_start[rowc + x3 + 1],
                                  ia, pa, have_exact, xa, ya, za, tmp, cap, row_cnt, stats);
        }
    }
}

// stats->max_row = the longest row (row_cnt filled by atomic slots).
__global__ void max_row_kernel(const int *__restrict__ row_cnt, int n, ListStats *__restrict__ stats)
{
    int m = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        m = max(m, row_cnt[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&stats->max_row, m);
}

// row_ptr[n] = nnz, the total of the row-length scan (clamped to int32; a
// larger total is refused on the host).
__global__ void set_total_kernel(int32_t *__restrict__ row_end, const ListStats *__restrict__ stats)
{
    const int64_t t = stats->nnz;
    *row_end = static_cast<int32_t>(t < INT32_MAX ? t : INT32_MAX);
}

// Row i's slab sorted into col: rows of up to 256 entries by the bitonic
// network above, longer ones staged in shared memory and ranked (the j of
// a row are distinct: rank(v) = #{m : buf[m] < v}).
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
sort_rows_kernel(const int *__restrict__ tmp, int cap, int n, const int32_t *__restrict__ row_ptr,
                 int32_t *__restrict__ col, const ListStats *__restrict__ stats, int64_t col_cap)
{
    // launched before the host has read the list size: nothing to do if the
    // walk overflowed a slab, met a position out of range, or the list does
    // not fit col (the host then reports it or takes the two-walk path)
    {
        const int err = stats->err;
        const int64_t nnz = stats->nnz;
        if ((err & 5) || nnz > col_cap || nnz >= INT32_MAX) return;
    }
    extern __shared__ int4 smem4[];
    int *smem = reinterpret_cast<int *>(smem4);
    const int wib = threadIdx.x >> 5;
    const int i = blockIdx.x * kWarpsPerBlock + wib;
    if (i >= n) return;
    const int lane = threadIdx.x & 31;
    const int start = row_ptr[i];
    const int len = row_ptr[i + 1] - start;
    const int *src = tmp + static_cast<size_t>(i) * cap;
    int32_t *out = col + start;
    // rows of up to 256 entries: a bitonic network straight from the slab
    if (bitonic_sort_row(src, len, lane, out)) return;
    // longer rows: staged in shared memory and ranked
    int *buf = smem + size_t(wib) * cap;
    for (int e = lane; e < len; e += 32) buf[e] = src[e];
    __syncwarp();
    for (int e = lane; e < len; e += 32) {
        const int v = buf[e];
        int r = 0;
        int m = 0;
        for (; m + 4 <= len; m += 4)
            r += (buf[m] < v) + (buf[m + 1] < v) + (buf[m + 2] < v) + (buf[m + 3] < v);
        for (; m < len; ++m) r += buf[m] < v;
        col[start + r] = v;
    }
}

// Slab width of the one-walk build: 1.5 times the mean full-list row of a
// uniform system of this density, plus 32, rounded up to 32 (rows beyond it
// make the build finish with the two-walk path); 0 -- no one-walk build --
// above kMaxSlab, where eight slabs would not fit the sort's shared memory.
constexpr int kMaxSlab = 4096;

int slab_cap(int64_t n, const double box[3], double rs)
{
    const double vol = box[0] * box[1] * box[2];
    const double mean = (vol > 0.0 ? double(n) / vol : 0.0) * (4.0 / 3.0) * 3.14159265358979 * rs * rs * rs;
    const double c = 1.5 * mean + 32.0;
    if (!(c <= double(kMaxSlab))) return 0;
    return (static_cast<int>(c) + 31) & ~31;
}

}  // namespace

// A stream and an event per host thread and device, on which the builder
// reads the list size back while the row sort runs on the caller's stream.
// Created on first use and destroyed when the thread exits (a thread-local
// holder's destructor; errors there are ignored, since the CUDA runtime may
// already be shutting down at process exit).  No limit on the number of
// devices a thread uses.
namespace {
struct SideStreams {
    struct Side {
        int dev;
        cudaStream_t s;
        cudaEvent_t e;
    };
    std::vector<Side> sides;
    ~SideStreams()
    {
        for (const Side &x : sides) {
            int cur = 0;
            if (cudaGetDevice(&cur) != cudaSuccess) break;
            if (cudaSetDevice(x.dev) != cudaSuccess) continue;
            cudaEventDestroy(x.e);
            cudaStreamDestroy(x.s);
            cudaSetDevice(cur);
        }
    }
};
}  // namespace

int side_stream(cudaStream_t &side, cudaEvent_t &ev)
{
    static thread_local SideStreams cache;
    int dev = 0;
    LJ_TRY_CUDA(cudaGetDevice(&dev));
    for (const SideStreams::Side &x : cache.sides)
        if (x.dev == dev) {
            side = x.s;
            ev = x.e;
            return LJ_OK;
        }
    SideStreams::Side x{dev, nullptr, nullptr};
    LJ_TRY_CUDA(cudaStreamCreateWithFlags(&x.s, cudaStreamNonBlocking));
    const cudaError_t err = cudaEventCreateWithFlags(&x.e, cudaEventDisableTiming);
    if (err != cudaSuccess) {
        cudaStreamDestroy(x.s);
        record_cuda_error(err, "cudaEventCreateWithFlags");
        return LJ_ERR_CUDA;
    }
    cache.sides.push_back(x);
    side = x.s;
    ev = x.e;
    return LJ_OK;
}

int build_pairlist_impl(const double *q4, int64_t n, const double box[3], double rs, int half,
                        int32_t *row_ptr, int32_t *col, int64_t cap, void *ws, size_t ws_bytes,
                        int64_t *nnz_out, int64_t *max_row_out, cudaStream_t st)
{
    if (nnz_out) *nnz_out = 0;
    if (max_row_out) *max_row_out = 0;
    if (!box || !row_ptr || !nnz_out || n < 0 || !(rs > 0.0) || !std::isfinite(rs) || cap < 0)
        return LJ_ERR_ARG;
    if (n > 0 && (!q4 || !ws)) return LJ_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(q4) & 31u) || (reinterpret_cast<uintptr_t>(ws) & 255u))
        return LJ_ERR_ARG;
    if (n >= (int64_t(1) << 31) - 1) return LJ_ERR_CAPACITY;
    int rc = check_box(box, rs);
    if (rc != LJ_OK) return rc;
    if (n == 0) {
        LJ_TRY_CUDA(cudaMemsetAsync(row_ptr, 0, sizeof(int32_t), st));
        return LJ_OK;
    }
    const Grid g = make_grid(n, box, rs);
    if (ws_bytes < carve_bytes(n, g.ncell)) return LJ_ERR_CAPACITY;
    const Work w = carve(ws, n, g.ncell);
    const int ni = static_cast<int>(n);

    LJ_TRY_CUDA(cudaMemsetAsync(w.cell_count, 0, sizeof(int) * (size_t(g.ncell) + 1), st));
    LJ_TRY_CUDA(cudaMemsetAsync(w.stats, 0, sizeof(ListStats), st));
    const unsigned gb = unsigned((n + 255) / 256);
    bin_kernel<<<gb, 256, 0, st>>>(q4, ni, g, w.cell_of, w.slot, w.cell_count, w.stats);
    LJ_TRY_LAUNCH("bin_kernel");
    rc = scan_exclusive<int, int>(w.cell_count, w.cell_start, g.ncell, &w.stats->nnz,
                                  w.scan_scratch, st);
    if (rc != LJ_OK) return rc;
    scatter_kernel<<<gb, 256, 0, st>>>(q4, ni, g.ncell, w.cell_of, w.slot, w.cell_start,
                                       w.cell_atoms, w.pos_f);
    LJ_TRY_LAUNCH("scatter_kernel");
    const unsigned gw = unsigned((n + kWarpsPerBlock - 1) / kWarpsPerBlock);
    // One walk (rows stored in slabs, then sorted into place) when the
    // workspace holds the slabs; otherwise count, then fill (two walks).
    const int cap_slab = slab_cap(n, box, rs);
    const size_t base_bytes = carve_bytes(n, g.ncell);
    int *slabs = nullptr;
    if (cap_slab > 0 && ws_bytes >= base_bytes + 256 + size_t(n) * size_t(cap_slab) * sizeof(int))
        slabs = reinterpret_cast<int *>((reinterpret_cast<uintptr_t>(ws) + base_bytes + 255) & ~uintptr_t(255));
    const bool forward_stencil = g.noff[0] == 5 && g.noff[1] == 5 && g.noff[2] == 5;
    if (slabs) {
        if (forward_stencil) {
            LJ_TRY_CUDA(cudaMemsetAsync(w.row_cnt, 0, sizeof(int) * size_t(n), st));
            if (half)
                walk_forward_store_kernel<true><<<gw, kWarpsPerBlock * 32, 0, st>>>(
                    q4, ni, g, w.cell_of, w.cell_start, w.cell_atoms, w.pos_f, slabs, cap_slab, w.row_cnt, w.stats);
            else
                walk_forward_store_kernel<false><<<gw, kWarpsPerBlock * 32, 0, st>>>(
                    q4, ni, g, w.cell_of, w.cell_start, w.cell_atoms, w.pos_f, slabs, cap_slab, w.row_cnt, w.stats);
            LJ_TRY_LAUNCH("walk_forward_store_kernel");
            max_row_kernel<<<unsigned(std::min<int64_t>((n + 255) / 256, 4 * 152)), 256, 0, st>>>(
                w.row_cnt, ni, w.stats);
        } else if (half)
            walk_store_kernel<true><<<gw, kWarpsPerBlock * 32, 0, st>>>(
                q4, ni, g, w.cell_of, w.cell_start, w.cell_atoms, w.pos_f, slabs, cap_slab, w.row_cnt, w.stats);
        else
            walk_store_kernel<false><<<gw, kWarpsPerBlock * 32, 0, st>>>(
                q4, ni, g, w.cell_of, w.cell_start, w.cell_atoms, w.pos_f, slabs, cap_slab, w.row_cnt, w.stats);
        LJ_TRY_LAUNCH("walk_store_kernel");
    } else {
        if (half)
            count_kernel<true><<<gw, kWarpsPerBlock * 32, 0, st>>>(q4, ni, g, w.cell_of, w.cell_start,
                                                                   w.cell_atoms, w.pos_f, w.row_cnt,
                                                                   w.stats);
        else
            count_kernel<false><<<gw, kWarpsPerBlock * 32, 0, st>>>(q4, ni, g, w.cell_of, w.cell_start,
                                                                    w.cell_atoms, w.pos_f, w.row_cnt,
                                                                    w.stats);
        LJ_TRY_LAUNCH("count_kernel");
    }
    rc = scan_exclusive<int, int32_t>(w.row_cnt, row_ptr, n, &w.stats->nnz, w.scan_scratch, st);
    if (rc != LJ_OK) return rc;
    // row_ptr[n] = nnz (the scan writes only the first n entries)
    set_total_kernel<<<1, 1, 0, st>>>(row_ptr + n, w.stats);
    LJ_TRY_LAUNCH("set_total_kernel");
    ListStats hs{};
    if (slabs) {
        // One-walk path: the list size is read on a side stream that waits
        // for the scan only, while the row sort -- which checks the same
        // figures itself and does nothing unless the list fits col -- runs
        // on the caller's stream; the host blocks for the small copy, not
        // for the sort.
        cudaStream_t side;
        cudaEvent_t scanned;
        rc = side_stream(side, scanned);
        if (rc != LJ_OK) return rc;
        LJ_TRY_CUDA(cudaEventRecord(scanned, st));
        if (col && cap > 0) {
            const size_t smem_sort = size_t(kWarpsPerBlock) * cap_slab * sizeof(int);
            if (smem_sort > 48 * 1024)
                LJ_TRY_CUDA(cudaFuncSetAttribute(sort_rows_kernel,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 int(smem_sort)));
            sort_rows_kernel<<<gw, kWarpsPerBlock * 32, smem_sort, st>>>(slabs, cap_slab, ni, row_ptr,
                                                                         col, w.stats, cap);
            LJ_TRY_LAUNCH("sort_rows_kernel");
        }
        LJ_TRY_CUDA(cudaStreamWaitEvent(side, scanned, 0));
        LJ_TRY_CUDA(cudaMemcpyAsync(&hs, w.stats, sizeof(ListStats), cudaMemcpyDeviceToHost, side));
        LJ_TRY_CUDA(cudaStreamSynchronize(side));
    } else {
        // two-walk path (and the allocation-free builder): no side stream
        LJ_TRY_CUDA(cudaMemcpyAsync(&hs, w.stats, sizeof(ListStats), cudaMemcpyDeviceToHost, st));
        LJ_TRY_CUDA(cudaStreamSynchronize(st));
    }
    if (hs.err & 1) return LJ_ERR_RANGE;
    *nnz_out = hs.nnz;
    if (max_row_out) *max_row_out = hs.max_row;
    if (hs.nnz >= (int64_t(1) << 31) - 1) return LJ_ERR_CAPACITY;
    if (hs.nnz > cap || hs.max_row > kMaxRowSmem) return LJ_ERR_CAPACITY;
    if (hs.nnz == 0) return LJ_OK;
    if (slabs && !(hs.err & 4)) return LJ_OK;  // sorted into col by the kernel above
    const int cap_row = std::max(1, hs.max_row);
    int wpb = kWarpsPerBlock;
    while (wpb > 1 && size_t(wpb) * cap_row * sizeof(int) > 200 * 1024) wpb >>= 1;
    const size_t smem = size_t(wpb) * cap_row * sizeof(int);
    const unsigned gf = unsigned((n + wpb - 1) / wpb);
    if (half) {
        if (smem > 48 * 1024)
            LJ_TRY_CUDA(cudaFuncSetAttribute(fill_kernel<true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        fill_kernel<true><<<gf, wpb * 32, smem, st>>>(q4, ni, g, w.cell_of, w.cell_start,
                                                       w.cell_atoms, w.pos_f, row_ptr, col, cap_row,
                                                       wpb, w.stats);
    } else {
        if (smem > 48 * 1024)
            LJ_TRY_CUDA(cudaFuncSetAttribute(fill_kernel<false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        fill_kernel<false><<<gf, wpb * 32, smem, st>>>(q4, ni, g, w.cell_of, w.cell_start,
                                                        w.cell_atoms, w.pos_f, row_ptr, col, cap_row,
                                                        wpb, w.stats);
    }
    LJ_TRY_LAUNCH("fill_kernel");
    return LJ_OK;
}

// The two-walk path's workspace plus the one-walk slabs (n x slab_cap ints);
// a workspace of only carve_bytes() selects the two-walk path.
size_t pairlist_workspace_bytes_impl(int64_t n, const double box[3], double rs)
{
    if (n < 0 || !box || !(rs > 0.0)) return 0;
    if (check_box(box, rs) != LJ_OK) return 256;
    const Grid g = make_grid(n, box, rs);
    return carve_bytes(n, g.ncell) + 256 + size_t(n > 0 ? n : 1) * size_t(slab_cap(n, box, rs)) * sizeof(int);
}

// The two-walk path's workspace alone.
size_t pairlist_workspace_bytes_min_impl(int64_t n, const double box[3], double rs)
{
    if (n < 0 || !box || !(rs > 0.0)) return 0;
    if (check_box(box, rs) != LJ_OK) return 256;
    return carve_bytes(n, make_grid(n, box, rs).ncell);
}

}  // namespace lj

extern "C" size_t lj_pairlist_workspace_bytes(int64_t n, const double box[3], double r_search)
{
    return lj::pairlist_workspace_bytes_impl(n, box, r_search);
}

extern "C" int lj_build_pairlist(const double *q4_dev, int64_t n, const double box[3],
                                 double r_search, int half, int32_t *row_ptr_dev, int32_t *col_dev,
                                 int64_t col_capacity, void *workspace_dev, size_t workspace_bytes,
                                 int64_t *nnz_out, int64_t *max_row_out, void *stream)
{
    return lj::build_pairlist_impl(q4_dev, n, box, r_search, half, row_ptr_dev, col_dev,
                                   col_capacity, workspace_dev, workspace_bytes, nnz_out,
                                   max_row_out, static_cast<cudaStream_t>(stream));
}

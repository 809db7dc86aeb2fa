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
//    small fraction of its FP32 rate, so the kernel spends FP64 operations
//    only where the value needs them: the minimum-image tests and the cutoff
//    test are integer compares of IEEE bit patterns, the division is an FP32
//    seed plus one third-order FP64 correction, and
//    df = u^4 (A - B u^3) with u = 1/r^2 takes five FP64 operations.
//  * MIXED: a pre-pass turns each FP64 position into a cell index and an
//    FP32 offset inside a cell of side ~2-4 sigma (computed in FP64), so the
//    pair displacement m h + (rel_j - rel_i) is accurate to ~1e-7 absolute
//    (absolute FP32 coordinates would lose ~1e-5 at L ~ 100).  The pair
//    arithmetic is FP32, per-lane i-sums are Kahan-compensated FP32,
//    combined across lanes with error-free transformations and added to the
//    FP64 momentum once per row; half-list p_j updates are FP64 atomics.
// In both forms a pair whose r^2 lies within a proven error band of r_c^2
// is re-decided with the exact FP64 definition, so the set of interacting
// pairs is the same as in double precision.
#include <cmath>
#include <cstring>

#include "lj_internal.cuh"

namespace lj {
namespace {

struct Fp64Params {
    double L[3];
    long long half_bits[3];
    long long rc2_bits;
    double A, B;  // df = u^4 (A - B u^3): A = 24 eps sigma^6 dt, B = 48 eps sigma^12 dt
};

struct MixedParams {
    // FP32 cell-relative geometry
    float h[3];      // cell side per axis (FP32 copy of L/nc)
    float hLf[3];    // L/2 in FP32
    int nc[3];       // cells per axis (< 1024)
    int nhalf[3];    // nc / 2
    float rc2f;      // r_c^2 in FP32
    float band;      // |r2f - r_c^2| <= band  => decide in FP64
    float Af, Bf;    // FP32 copies of A, B
    // FP64 geometry for the exact decisions
    double L[3];
    long long half_bits[3];
    double rc2;      // r_c^2 in FP64 (exact definition, no FMA)
    double inv_h[3]; // nc / L
    double hd[3];    // L / nc in FP64
};

// 32-byte read-only gather of one AoS4 record (a single 256-bit load).
__device__ __forceinline__ void load_q4_256(const double *__restrict__ q4, int j, double &x,
                                            double &y, double &z)
{
    double w;
    asm("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];"
        : "=d"(x), "=d"(y), "=d"(z), "=d"(w)
        : "l"(q4 + 4 * static_cast<int64_t>(j)));
}

// Exact definition of "pair within r_c": oracle-identical operations.
__device__ __forceinline__ bool exact_in_cutoff(double dx, double dy, double dz, double rc2)
{
    const double r2 =
        __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return r2 < rc2;
}

// Lanes of this thread's TPI-wide group (groups are aligned inside the warp,
// so a group past the last row exits as a whole and never joins a shuffle).
template <int TPI>
__device__ __forceinline__ unsigned group_mask()
{
    if (TPI == 32) return 0xffffffffu;
    return ((1u << TPI) - 1u) << ((threadIdx.x & 31) & ~(TPI - 1));
}

template <int TPI>
__device__ __forceinline__ double group_sum(double v)
{
    const unsigned m = group_mask<TPI>();
#pragma unroll
    for (int o = TPI / 2; o > 0; o >>= 1) v += __shfl_xor_sync(m, v, o, TPI);
    return v;
}

// ---------------------------------------------------------------------------
// FP64 form
// ---------------------------------------------------------------------------
template <int TPI, bool HALF>
__global__ void __launch_bounds__(256)
force_fp64_kernel(const double *__restrict__ q4, double *__restrict__ p4, int n,
                  const int *__restrict__ row_ptr, const int *__restrict__ col, Fp64Params P)
{
    const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / TPI;
    const int sub = threadIdx.x & (TPI - 1);
    // A group past the last row exits as a whole; the shuffles below name
    // only the group's own lanes.
    if (gid >= n) return;
    const int i = gid;
    double xi, yi, zi;
    load_q4_256(q4, i, xi, yi, zi);
    double ax = 0.0, ay = 0.0, az = 0.0;
    const int kb = row_ptr[i], ke = row_ptr[i + 1];
    for (int k = kb + sub; k < ke; k += TPI) {
        const int j = col[k];
        double xj, yj, zj;
        load_q4_256(q4, j, xj, yj, zj);
        const double dx = min_image(xj - xi, P.L[0], P.half_bits[0]);
        const double dy = min_image(yj - yi, P.L[1], P.half_bits[1]);
        const double dz = min_image(zj - zi, P.L[2], P.half_bits[2]);
        const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
        const long long rb = __double_as_longlong(r2);
        bool in = rb < P.rc2_bits;
        if (static_cast<unsigned long long>(rb - P.rc2_bits + 64) < 128ull) {
            double rc2;
            memcpy(&rc2, &P.rc2_bits, sizeof(double));
            in = exact_in_cutoff(dx, dy, dz, rc2);
        }
        if (in) {
            const double u = rcp_fp64(r2);
            const double u2 = u * u;
            const double u4 = u2 * u2;
            const double u3 = u2 * u;
            const double f = u4 * fma(-P.B, u3, P.A);
            const double fx = f * dx, fy = f * dy, fz = f * dz;
            ax += fx;
            ay += fy;
            az += fz;
            if (HALF) {
                atomicAdd(p4 + 4 * static_cast<int64_t>(j) + 0, -fx);
                atomicAdd(p4 + 4 * static_cast<int64_t>(j) + 1, -fy);
                atomicAdd(p4 + 4 * static_cast<int64_t>(j) + 2, -fz);
            }
        }
    }
    if (TPI > 1) {
        ax = group_sum<TPI>(ax);
        ay = group_sum<TPI>(ay);
        az = group_sum<TPI>(az);
    }
    if (sub == 0) {
        double *pi = p4 + 4 * static_cast<int64_t>(i);
        if (HALF) {
            atomicAdd(pi + 0, ax);
            atomicAdd(pi + 1, ay);
            atomicAdd(pi + 2, az);
        } else {
            pi[0] += ax;
            pi[1] += ay;
            pi[2] += az;
        }
    }
}

// ---------------------------------------------------------------------------
// MIXED form
// ---------------------------------------------------------------------------

// Pre-pass: q (FP64) -> {rel_x, rel_y, rel_z, packed cell} with
// rel = q - c h computed in FP64 and rounded once to FP32.
__global__ void mixed_prepass_kernel(const double *__restrict__ q4, int n, MixedParams P,
                                     float4 *__restrict__ rel)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x[3];
    load_xyz(q4, i, x[0], x[1], x[2]);
    int c[3];
    float r[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int ca = static_cast<int>(x[a] * P.inv_h[a]);
        ca = ca < 0 ? 0 : (ca >= P.nc[a] ? P.nc[a] - 1 : ca);
        c[a] = ca;
        r[a] = __double2float_rn(x[a] - ca * P.hd[a]);
    }
    rel[i] = make_float4(r[0], r[1], r[2], __int_as_float(c[0] | (c[1] << 10) | (c[2] << 20)));
}

// One displacement component from cell-relative coordinates.
__device__ __forceinline__ float mixed_disp(float rj, float ri, int cj, int ci, float h, float hL,
                                            int nc, int nhalf)
{
    int m = cj - ci;
    m = m > nhalf ? m - nc : (m < -nhalf ? m + nc : m);
    const float dr = rj - ri;
    float d = fmaf(static_cast<float>(m), h, dr);
    if (fabsf(d) > hL) d = fmaf(static_cast<float>(d > 0.0f ? m - nc : m + nc), h, dr);
    return d;
}

// Kahan step: (s, c) with true sum ~ s - c.
__device__ __forceinline__ void kahan_add(float &s, float &c, float x)
{
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Combine two compensated sums with an error-free TwoSum of the heads.
__device__ __forceinline__ void kahan_merge(float &s, float &c, float s2, float c2)
{
    const float t = s + s2;
    const float bp = t - s;
    const float e = (s - (t - bp)) + (s2 - bp);  // s + s2 = t + e exactly
    c = (c + c2) - e;
    s = t;
}

template <int TPI>
__device__ __forceinline__ void group_kahan(float &s, float &c)
{
    const unsigned m = group_mask<TPI>();
#pragma unroll
    for (int o = TPI / 2; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(m, s, o, TPI);
        const float c2 = __shfl_xor_sync(m, c, o, TPI);
        kahan_merge(s, c, s2, c2);
    }
}

template <int TPI, bool HALF>
__global__ void __launch_bounds__(256)
force_mixed_kernel(const double *__restrict__ q4, const float4 *__restrict__ rel,
                   double *__restrict__ p4, int n, const int *__restrict__ row_ptr,
                   const int *__restrict__ col, MixedParams P)
{
    const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / TPI;
    const int sub = threadIdx.x & (TPI - 1);
    if (gid >= n) return;
    const int i = gid;
    const float4 pi = rel[i];
    const int ci = __float_as_int(pi.w);
    const int cix = ci & 1023, ciy = (ci >> 10) & 1023, ciz = ci >> 20;
    float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
    const int kb = row_ptr[i], ke = row_ptr[i + 1];
    for (int k = kb + sub; k < ke; k += TPI) {
        const int j = col[k];
        const float4 pj = rel[j];
        const int cj = __float_as_int(pj.w);
        const float dx = mixed_disp(pj.x, pi.x, cj & 1023, cix, P.h[0], P.hLf[0], P.nc[0], P.nhalf[0]);
        const float dy = mixed_disp(pj.y, pi.y, (cj >> 10) & 1023, ciy, P.h[1], P.hLf[1], P.nc[1], P.nhalf[1]);
        const float dz = mixed_disp(pj.z, pi.z, cj >> 20, ciz, P.h[2], P.hLf[2], P.nc[2], P.nhalf[2]);
        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        bool in = r2 < P.rc2f;
        if (fabsf(r2 - P.rc2f) <= P.band) {
            double xi, yi, zi, xj, yj, zj;
            load_xyz(q4, i, xi, yi, zi);
            load_xyz(q4, j, xj, yj, zj);
            const double ex = min_image(__dsub_rn(xj, xi), P.L[0], P.half_bits[0]);
            const double ey = min_image(__dsub_rn(yj, yi), P.L[1], P.half_bits[1]);
            const double ez = min_image(__dsub_rn(zj, zi), P.L[2], P.half_bits[2]);
            in = exact_in_cutoff(ex, ey, ez, P.rc2);
        }
        if (in) {
            const float u = rcp_fp32(r2);
            const float u2 = u * u;
            const float u4 = u2 * u2;
            const float u3 = u2 * u;
            const float f = u4 * fmaf(-P.Bf, u3, P.Af);
            const float fx = f * dx, fy = f * dy, fz = f * dz;
            kahan_add(sx, cx, fx);
            kahan_add(sy, cy, fy);
            kahan_add(sz, cz, fz);
            if (HALF) {
                atomicAdd(p4 + 4 * static_cast<int64_t>(j) + 0, -static_cast<double>(fx));
                atomicAdd(p4 + 4 * static_cast<int64_t>(j) + 1, -static_cast<double>(fy));
                atomicAdd(p4 + 4 * static_cast<int64_t>(j) + 2, -static_cast<double>(fz));
            }
        }
    }
    if (TPI > 1) {
        group_kahan<TPI>(sx, cx);
        group_kahan<TPI>(sy, cy);
        group_kahan<TPI>(sz, cz);
    }
    if (sub == 0) {
        const double ax = static_cast<double>(sx) - static_cast<double>(cx);
        const double ay = static_cast<double>(sy) - static_cast<double>(cy);
        const double az = static_cast<double>(sz) - static_cast<double>(cz);
        double *pp = p4 + 4 * static_cast<int64_t>(i);
        if (HALF) {
            atomicAdd(pp + 0, ax);
            atomicAdd(pp + 1, ay);
            atomicAdd(pp + 2, az);
        } else {
            pp[0] += ax;
            pp[1] += ay;
            pp[2] += az;
        }
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

Fp64Params make_fp64_params(const double box[3], double dt, double rc, double eps, double sigma)
{
    Fp64Params P{};
    for (int a = 0; a < 3; ++a) {
        P.L[a] = box[a];
        const double h = 0.5 * box[a];
        std::memcpy(&P.half_bits[a], &h, sizeof(double));
    }
    const double rc2 = rc * rc;
    std::memcpy(&P.rc2_bits, &rc2, sizeof(double));
    const double s2 = sigma * sigma, s6 = s2 * s2 * s2, s12 = s6 * s6;
    P.A = 24.0 * eps * s6 * dt;
    P.B = 48.0 * eps * s12 * dt;
    return P;
}

MixedParams make_mixed_params(const double box[3], double dt, double rc, double eps, double sigma)
{
    MixedParams P{};
    double hmax = 0.0;
    for (int a = 0; a < 3; ++a) {
        int nc = static_cast<int>(std::floor(box[a] / 2.0));
        nc = nc < 1 ? 1 : (nc > 1023 ? 1023 : nc);
        P.nc[a] = nc;
        P.nhalf[a] = nc / 2;
        P.hd[a] = box[a] / nc;
        P.inv_h[a] = nc / box[a];
        P.h[a] = static_cast<float>(P.hd[a]);
        P.hLf[a] = static_cast<float>(0.5 * box[a]);
        P.L[a] = box[a];
        const double hh = 0.5 * box[a];
        std::memcpy(&P.half_bits[a], &hh, sizeof(double));
        hmax = P.hd[a] > hmax ? P.hd[a] : hmax;
    }
    P.rc2 = rc * rc;
    P.rc2f = static_cast<float>(P.rc2);
    // Per-axis displacement error <= 4 h 2^-23 (offset roundings, FP32 h,
    // the fused add); r^2 error <= 2 sqrt(3) r_c e + 3 e^2 + 4 2^-24 r_c^2
    // plus the rounding of r_c^2 itself; the band is four times that.
    const double e = 4.0 * hmax * std::ldexp(1.0, -23);
    const double err = 2.0 * std::sqrt(3.0) * rc * e + 3.0 * e * e + 4.0 * std::ldexp(1.0, -24) * P.rc2 +
                       std::fabs(static_cast<double>(P.rc2f) - P.rc2);
    P.band = static_cast<float>(4.0 * err);
    const double s2 = sigma * sigma, s6 = s2 * s2 * s2, s12 = s6 * s6;
    P.Af = static_cast<float>(24.0 * eps * s6 * dt);
    P.Bf = static_cast<float>(48.0 * eps * s12 * dt);
    return P;
}

template <int TPI>
int launch_fp64(const double *q4, double *p4, int n, const int *rp, const int *col, int half,
                const Fp64Params &P, cudaStream_t st)
{
    const int64_t threads = int64_t(n) * TPI;
    const unsigned grid = unsigned((threads + 255) / 256);
    if (half)
        force_fp64_kernel<TPI, true><<<grid, 256, 0, st>>>(q4, p4, n, rp, col, P);
    else
        force_fp64_kernel<TPI, false><<<grid, 256, 0, st>>>(q4, p4, n, rp, col, P);
    LJ_TRY_LAUNCH("force_fp64_kernel");
    return LJ_OK;
}

template <int TPI>
int launch_mixed(const double *q4, const float4 *rel, double *p4, int n, const int *rp,
                 const int *col, int half, const MixedParams &P, cudaStream_t st)
{
    const int64_t threads = int64_t(n) * TPI;
    const unsigned grid = unsigned((threads + 255) / 256);
    if (half)
        force_mixed_kernel<TPI, true><<<grid, 256, 0, st>>>(q4, rel, p4, n, rp, col, P);
    else
        force_mixed_kernel<TPI, false><<<grid, 256, 0, st>>>(q4, rel, p4, n, rp, col, P);
    LJ_TRY_LAUNCH("force_mixed_kernel");
    return LJ_OK;
}

}  // namespace

int force_stream_fp64(const double *q4, double *p4, int n, const int *row_ptr, const int *col,
                      int64_t nnz, int half, const double box[3], double dt, double rc, double eps,
                      double sigma, cudaStream_t st);

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

size_t force_workspace_bytes_impl(int64_t n, int precision)
{
    if (precision != LJ_MIXED || n <= 0) return 0;
    return size_t(n) * sizeof(float4) + 256;
}

int force_impl(const double *q4, double *p4, int64_t n, const int32_t *row_ptr, const int32_t *col,
               int64_t nnz, int half, double dt, double rc, const double box[3], double eps,
               double sigma, int precision, int tpi, void *ws, size_t ws_bytes, cudaStream_t st)
{
    int rcode = check_force_args(q4, p4, n, row_ptr, col, nnz, rc, box, eps, sigma, dt);
    if (rcode != LJ_OK) return rcode;
    if (precision != LJ_FP64 && precision != LJ_MIXED) return LJ_ERR_ARG;
    if (n == 0 || nnz == 0) return LJ_OK;
    const int ni = static_cast<int>(n);
    if (tpi == LJ_TPI_AUTO) tpi = (precision == LJ_FP64) ? LJ_SCHED_STREAM : (half ? 8 : 8);
    if (tpi == LJ_SCHED_STREAM) {
        if (precision != LJ_FP64) return LJ_ERR_ARG;
        return force_stream_fp64(q4, p4, ni, row_ptr, col, nnz, half, box, dt, rc, eps, sigma, st);
    }
    if (precision == LJ_FP64) {
        const Fp64Params P = make_fp64_params(box, dt, rc, eps, sigma);
        switch (tpi) {
            case 1: return launch_fp64<1>(q4, p4, ni, row_ptr, col, half, P, st);
            case 2: return launch_fp64<2>(q4, p4, ni, row_ptr, col, half, P, st);
            case 4: return launch_fp64<4>(q4, p4, ni, row_ptr, col, half, P, st);
            case 8: return launch_fp64<8>(q4, p4, ni, row_ptr, col, half, P, st);
            case 16: return launch_fp64<16>(q4, p4, ni, row_ptr, col, half, P, st);
            case 32: return launch_fp64<32>(q4, p4, ni, row_ptr, col, half, P, st);
            default: return LJ_ERR_ARG;
        }
    }
    if (!ws || ws_bytes < force_workspace_bytes_impl(n, precision)) return LJ_ERR_CAPACITY;
    const MixedParams P = make_mixed_params(box, dt, rc, eps, sigma);
    Carver c(ws);
    float4 *rel = c.take<float4>(size_t(n));
    mixed_prepass_kernel<<<unsigned((n + 255) / 256), 256, 0, st>>>(q4, ni, P, rel);
    LJ_TRY_LAUNCH("mixed_prepass_kernel");
    switch (tpi) {
        case 1: return launch_mixed<1>(q4, rel, p4, ni, row_ptr, col, half, P, st);
        case 2: return launch_mixed<2>(q4, rel, p4, ni, row_ptr, col, half, P, st);
        case 4: return launch_mixed<4>(q4, rel, p4, ni, row_ptr, col, half, P, st);
        case 8: return launch_mixed<8>(q4, rel, p4, ni, row_ptr, col, half, P, st);
        case 16: return launch_mixed<16>(q4, rel, p4, ni, row_ptr, col, half, P, st);
        case 32: return launch_mixed<32>(q4, rel, p4, ni, row_ptr, col, half, P, st);
        default: return LJ_ERR_ARG;
    }
}

}  // namespace lj

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

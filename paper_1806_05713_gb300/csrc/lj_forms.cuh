// lj_forms.cuh -- parameters and per-pair helpers of the two arithmetic
// forms (FP64, MIXED), shared by the force, adjoint and batched kernels.
#pragma once

#include <cmath>
#include <cstring>

#include "lj_internal.cuh"

namespace lj {
namespace {

struct Fp64Params {
    double L[3];
    long long half_bits[3];
    long long rc2_bits;
    double rc2;
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
    int wrap_fix;    // nonzero when a pair within r_c can need the second image choice
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
// MIXED form helpers
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

// Small integer (|m| < 2^22) to float without a conversion instruction:
// 1.5 * 2^23 + m has m in its low mantissa bits.
__device__ __forceinline__ float small_int_to_float(int m)
{
    return __int_as_float(0x4B400000 + m) - 12582912.0f;
}

// One displacement component from cell-relative coordinates: the cell
// difference m is wrapped to its nearest representative, d = m h + (rel_j -
// rel_i).  In small boxes (fix != 0, a warp-uniform flag) a pair within r_c
// can still sit across the half-box from that representative; then the other
// image is taken.
__device__ __forceinline__ float mixed_disp(float rj, float ri, int cj, int ci, float h, float hL,
                                            int nc, int nhalf, int fix)
{
    int m = cj - ci;
    m = m > nhalf ? m - nc : (m < -nhalf ? m + nc : m);
    const float dr = rj - ri;
    float d = fmaf(small_int_to_float(m), h, dr);
    if (fix) {
        if (fabsf(d) > hL) d = fmaf(small_int_to_float(d > 0.0f ? m - nc : m + nc), h, dr);
    }
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


// ---------------------------------------------------------------------------
// Host-side parameter blocks
// ---------------------------------------------------------------------------

Fp64Params make_fp64_params(const double box[3], double dt, double rc, double eps, double sigma)
{
    Fp64Params P{};
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
    // With |m| <= nc/2 and |rel_j - rel_i| < h, |d| <= L/2 + h; the other
    // image is then at least L/2 - h away, so it can matter only if
    // L/2 - h < r_c (plus a rounding allowance).
    P.wrap_fix = 0;
    for (int a = 0; a < 3; ++a)
        if (0.5 * box[a] - P.hd[a] < rc * (1.0 + 1e-6) + 1e-6) P.wrap_fix = 1;
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

}  // namespace
}  // namespace lj

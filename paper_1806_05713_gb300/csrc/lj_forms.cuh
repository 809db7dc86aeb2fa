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
    double C12, C6;  // V = u^3 (C12 u^3 - C6): C12 = 4 eps sigma^12, C6 = 4 eps sigma^6
    double W12, W6;  // r F(r) = u^3 (W12 u^3 - W6): W12 = 48 eps sigma^12, W6 = 24 eps sigma^6
    // force-shifted truncation: F_c = -V'(r_c), fs_c = F_c dt, V_c = V(r_c)
    double rc, Fc, fs_c, Vc;
};

struct MixedParams {
    // Fixed-point positions: X = floor(x 2^32 / L) as a 32-bit unsigned
    // integer per axis, so X_j - X_i in wrapping 32-bit arithmetic is the
    // minimum-image displacement in units of L / 2^32, exactly.
    double to_fixed[3];  // 2^32 / L (FP64, pre-pass)
    float scale[3];      // L / 2^32 (FP32, pair loop)
    float rc2f;          // r_c^2 in FP32
    float band;          // |r2f - r_c^2| <= band  => decide in FP64
    float Af, Bf;        // FP32 copies of A, B
    // FP64 geometry for the exact decisions
    double L[3];
    long long half_bits[3];
    double rc2;          // r_c^2 in FP64 (exact definition, no FMA)
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

// Pre-pass: q (FP64) -> {X, Y, Z, 0}, X = floor(x 2^32 / L) computed in
// FP64 (x in [0, L) maps to [0, 2^32); a product that rounds up to 2^32
// saturates to 2^32 - 1).
__global__ void mixed_prepass_kernel(const double *__restrict__ q4, int n, MixedParams P,
                                     uint4 *__restrict__ fx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x[3];
    load_xyz(q4, i, x[0], x[1], x[2]);
    fx[i] = make_uint4(__double2uint_rz(x[0] * P.to_fixed[0]), __double2uint_rz(x[1] * P.to_fixed[1]),
                       __double2uint_rz(x[2] * P.to_fixed[2]), 0u);
}

// One displacement component: the wrapping 32-bit difference is the
// minimum image (exact, in units of L / 2^32); one conversion and one
// multiply round it to FP32.
__device__ __forceinline__ float fixed_disp(unsigned xj, unsigned xi, float scale)
{
    return static_cast<float>(static_cast<int>(xj - xi)) * scale;
}

// Exact float -> double conversion with integer instructions only (GB300
// runs float<->double conversions on its slow FP64 pipe): rebias the
// exponent and shift the mantissa.  Zero and subnormal inputs give +-0
// (their magnitude, below 1.2e-38, is far under any momentum's last digit),
// infinities and NaNs stay non-finite.
__device__ __forceinline__ double f32_to_f64(float x)
{
    const unsigned u = __float_as_uint(x);
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned ed = e == 255u ? 2047u : e + 896u;
    const unsigned hi = (u & 0x80000000u) | (ed << 20) | ((u >> 3) & 0xfffffu);
    const unsigned lo = u << 29;
    return e == 0u ? __hiloint2double(static_cast<int>(u & 0x80000000u), 0)
                   : __hiloint2double(static_cast<int>(hi), static_cast<int>(lo));
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
    P.C12 = 4.0 * eps * s12;
    P.C6 = 4.0 * eps * s6;
    P.W12 = 48.0 * eps * s12;
    P.W6 = 24.0 * eps * s6;
    const double sr = sigma / rc, sr2 = sr * sr, sr6 = sr2 * sr2 * sr2;
    P.rc = rc;
    P.Fc = 24.0 * eps * (2.0 * sr6 * sr6 - sr6) / rc;
    P.fs_c = P.Fc * dt;
    P.Vc = 4.0 * eps * (sr6 * sr6 - sr6);
    return P;
}

MixedParams make_mixed_params(const double box[3], double dt, double rc, double eps, double sigma)
{
    MixedParams P{};
    double Lmax = 0.0;
    for (int a = 0; a < 3; ++a) {
        P.to_fixed[a] = std::ldexp(1.0, 32) / box[a];
        P.scale[a] = static_cast<float>(std::ldexp(box[a], -32));
        P.L[a] = box[a];
        const double hh = 0.5 * box[a];
        std::memcpy(&P.half_bits[a], &hh, sizeof(double));
        Lmax = box[a] > Lmax ? box[a] : Lmax;
    }
    P.rc2 = rc * rc;
    P.rc2f = static_cast<float>(P.rc2);
    // Per-axis displacement error: two position quantisations (< L 2^-32
    // each), the conversion and the scaling (2^-24 |d| each) and the FP32
    // scale (2^-24 |d|); r^2 error <= 2 sqrt(3) r_c e + 3 e^2 + 4 2^-24 r_c^2
    // plus the rounding of r_c^2; the band is four times that.
    const double e = 2.0 * Lmax * std::ldexp(1.0, -32) + 3.0 * std::ldexp(1.0, -24) * rc;
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

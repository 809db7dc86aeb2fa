// lj_dfloat.cuh -- the DFLOAT form of the pair arithmetic: FP64-class
// accuracy from FP32 instructions.
//
// GB300 retires FP32 fused multiply-adds at about 70 times its FP64 rate, so
// the pair impulse of Algorithm 1 is evaluated in double-float arithmetic:
// every quantity is an unevaluated sum hi + lo of two FP32 numbers (|lo| <=
// ulp(hi)/2), carried through the error-free transformations TwoSum
// (Knuth, TAOCP vol. 2, section 4.2.2), FastTwoSum (Dekker 1971) and the
// FMA-based exact product (the rounding error of a*b is fma(a, b, -a*b)).
// Products and sums carry about 46 significand bits.
//
// The displacement is exact.  A pre-pass (FP64, once per atom and call)
// writes each coordinate as a 58-bit fixed-point fraction of its box side,
// X = round(x 2^58 / L) mod 2^58, split into a 24-bit high chunk, a 24-bit
// middle chunk and a 10-bit low chunk:
//   H = X[57:34] 2^(s-24),  M = X[33:10] 2^(s-48),  lo = X[9:0]
// (H and M as FP32, which hold them exactly; the three lo fields packed in
// one 32-bit word), one 32-byte record per atom.  For a pair, H_j - H_i and
// M_j - M_i are exact FP32 subtractions, the periodic wrap of the high part
// is a subtraction of 2^s rint((H_j - H_i) 2^-s), and the low fields give the
// last 10 bits: the minimum-image displacement in units of
// lambda = L 2^-s is recovered to 2^-58 L (1.7e-16 at L = 49), below the
// rounding of an FP64 difference of two coordinates.  s is chosen so that
// r_c <= lambda < 2 r_c, which keeps every pair quantity near 1 in FP32.
//
// In lambda units the impulse of an in-cutoff pair is
//   fn d = (A / lambda^7) u^4 (beta u^3 - 1) delta,  u = 1/|delta|^2,
// with A = 24 eps sigma^6 dt and beta = 2 (sigma/lambda)^6.  The mantissa
// K_m of A / lambda^7 = K_m 2^K_e rides in the constants of g = K_m u^4
// (beta u^3 - 1); the kernels sum g delta in double-float and apply 2^K_e
// exactly when they add into the FP64 momenta (once per row for p_i, per
// pair for the p_j of a half list).
//
// Pairs whose r^2 lies in a band around r_c^2, and pairs closer than the
// range where every intermediate of g stays a normal FP32 number, take the
// FP64 definition and formula, so the DFLOAT form interacts the same pairs
// as the FP64 form and has no input range of its own.
#pragma once

#include <cmath>
#include <cstring>

#include "lj_forms.cuh"

namespace lj {
namespace {

struct DfParams {
    // pre-pass
    double to_fixed[3];  // 2^58 / L_a
    float chunk_hi;      // 2^(s-24): H = X[57:34] * chunk_hi
    float chunk_mid;     // 2^(s-48)
    // pair loop
    float period;        // 2^s: the wrap period of H
    float inv_period;    // 2^-s
    float lo_scale;      // 2^(s-58): value of one unit of the low field
    float lo_offset;     // 2^(s-35) = 2^23 lo_scale (magic-number decode)
    float cx_h[3], cx_l[3];  // L_a / L_0 as double-float (1 for a cubic box)
    float T_h, T_l;      // (r_c / lambda)^2 as double-float
    float band;          // |R_h - T_h| <= band  => decide in FP64
    float r2_min;        // R < r2_min  => FP64 pair formula
    // A / lambda^7 = K_m 2^K_e with K_m in [1, 2): g carries K_m, the FP64
    // side applies 2^K_e (half list: by the exponent of the converted values)
    float ka_h, ka_l;    // K_m
    float kb_h, kb_l;    // K_m beta, beta = 2 (sigma / lambda)^6
    int k_exp;           // K_e
    double k_pow;        // 2^K_e
    // FP64 definitions for the band decisions and the close-pair formula
    double L[3];
    long long half_bits[3];
    double rc2;
    double A, B;         // fn = u^4 (B u^3 - A) in real units (FP64 form)
};

// ---- error-free transformations and double-float operations -------------
// The _rn intrinsics keep the compiler from contracting or re-associating.

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// |a| >= |b| or a == 0.
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

struct df {
    float h, l;
};

__device__ __forceinline__ df df_mul(df a, df b)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    df r;
    fast_two_sum(p, e, r.h, r.l);
    return r;
}

__device__ __forceinline__ df df_sq(df a)
{
    const float p = __fmul_rn(a.h, a.h);
    float e = __fmaf_rn(a.h, a.h, -p);
    e = __fmaf_rn(__fadd_rn(a.h, a.h), a.l, e);
    df r;
    fast_two_sum(p, e, r.h, r.l);
    return r;
}

// a + b with TwoSum on the heads.
__device__ __forceinline__ df df_add(df a, df b)
{
    float s, e;
    two_sum(a.h, b.h, s, e);
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    df r;
    fast_two_sum(s, e, r.h, r.l);
    return r;
}

// 1/a for a normal, positive a: the FP32 approximation y (rcp.approx.ftz,
// 1 ulp), then y (1 + e + e^2) with e = 1 - a y formed by two FMAs
// (relative error ~2^-46).
__device__ __forceinline__ df df_rcp(df a)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a.h));
    float e = __fmaf_rn(-a.h, y, 1.0f);
    e = __fmaf_rn(-a.l, y, e);
    const float q = __fmul_rn(y, e);
    const float l = __fmaf_rn(q, e, q);
    df r;
    fast_two_sum(y, l, r.h, r.l);
    return r;
}

// x 2^k as a double, exactly, with integer instructions only (f32_to_f64
// with the exponent moved by k; |k| < 800 keeps every normal float normal).
__device__ __forceinline__ double f32_to_f64_pow2(float x, int k)
{
    const unsigned u = __float_as_uint(x);
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned ed = e == 255u ? 2047u : e + 896u + static_cast<unsigned>(k);
    const unsigned hi = (u & 0x80000000u) | ((ed & 0x7ffu) << 20) | ((u >> 3) & 0xfffffu);
    const unsigned lo = u << 29;
    return e == 0u ? __hiloint2double(static_cast<int>(u & 0x80000000u), 0)
                   : __hiloint2double(static_cast<int>(hi), static_cast<int>(lo));
}

// (h + l) 2^k rounded once to double: the parts are converted exactly with
// integer instructions, one FP64 addition joins them.
__device__ __forceinline__ double df_to_f64(float h, float l, int k)
{
    return __dadd_rn(f32_to_f64_pow2(h, k), f32_to_f64_pow2(l, k));
}

// ---- fixed-point records ---------------------------------------------------

// One record per atom: H_x, H_y, H_z, M_x, M_y, M_z, packed low fields, 0.
struct __align__(32) DfRec {
    float hx, hy, hz, mx, my, mz;
    unsigned lo, pad;
};

__device__ __forceinline__ DfRec load_rec(const DfRec *__restrict__ rec, int j)
{
    DfRec r;
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(r.hx), "=f"(r.hy), "=f"(r.hz), "=f"(r.mx), "=f"(r.my), "=f"(r.mz),
          "=r"(r.lo), "=r"(r.pad)
        : "l"(rec + j));
    return r;
}

// X = round(x 2^58 / L) mod 2^58: the product and its exact remainder
// (an FMA) are rounded to integers separately, so X is within one unit of
// x 2^58 / L (to the rounding of 2^58 / L itself).
__device__ __forceinline__ long long fixed58(double x, double c)
{
    const double p = x * c;
    const double e = fma(x, c, -p);
    const long long X = __double2ll_rn(p) + __double2ll_rn(e);
    return X & ((1LL << 58) - 1);
}

// The record of one atom at x (FP64 coordinates in [0, L)).
__device__ __forceinline__ DfRec make_rec(const double x[3], const DfParams &P)
{
    float h[3], m[3];
    unsigned lo = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const long long X = fixed58(x[a], P.to_fixed[a]);
        h[a] = __fmul_rn(__int2float_rn(static_cast<int>(X >> 34)), P.chunk_hi);
        m[a] = __fmul_rn(__int2float_rn(static_cast<int>((X >> 10) & 0xffffff)), P.chunk_mid);
        lo |= static_cast<unsigned>(X & 0x3ff) << (10 * a);
    }
    DfRec r;
    r.hx = h[0];
    r.hy = h[1];
    r.hz = h[2];
    r.mx = m[0];
    r.my = m[1];
    r.mz = m[2];
    r.lo = lo;
    r.pad = 0u;
    return r;
}

__global__ void dfloat_prepass_kernel(const double *__restrict__ q4, int n, DfParams P,
                                      DfRec *__restrict__ rec)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x[3];
    load_xyz(q4, i, x[0], x[1], x[2]);
    rec[i] = make_rec(x, P);
}

// Low field a of a record as a float: 2^23 + v by placing v in the mantissa
// of 2^23, then an exact FMA removes 2^23 and scales by 2^(s-58).
__device__ __forceinline__ float lo_field(unsigned w, int a, const DfParams &P)
{
    const unsigned v = ((w >> (10 * a)) & 0x3ffu) | 0x4b000000u;
    return __fmaf_rn(__uint_as_float(v), P.lo_scale, -P.lo_offset);
}

// One displacement component in units of L_a 2^-s from the chunks of j and
// i (li = lo_field of i): exact difference of the chunks, the periodic wrap
// on the high part, then FastTwoSum (|dH| >= 2^(s-24) > |dM| unless dH = 0).
__device__ __forceinline__ df chunk_disp(float hj, float hi, float mj, float mi, float lj, float li,
                                         const DfParams &P)
{
    float dh = __fsub_rn(hj, hi);
    const float k = __fsub_rn(__fmaf_rn(dh, P.inv_period, 12582912.0f), 12582912.0f);
    dh = __fmaf_rn(-k, P.period, dh);
    df d;
    float t;
    fast_two_sum(dh, __fsub_rn(mj, mi), d.h, t);
    d.l = __fadd_rn(t, __fsub_rn(lj, li));
    return d;
}

// |d|^2 of three double-float components: exact squares of the heads,
// TwoSum of the partial sums, all error terms gathered before one
// FastTwoSum.
__device__ __forceinline__ df df_norm2(df x, df y, df z)
{
    const float px = __fmul_rn(x.h, x.h), py = __fmul_rn(y.h, y.h), pz = __fmul_rn(z.h, z.h);
    float e = __fmaf_rn(x.h, x.h, -px);
    e = __fadd_rn(e, __fmaf_rn(y.h, y.h, -py));
    e = __fadd_rn(e, __fmaf_rn(z.h, z.h, -pz));
    float c = __fmul_rn(x.h, x.l);
    c = __fmaf_rn(y.h, y.l, c);
    c = __fmaf_rn(z.h, z.l, c);
    e = __fmaf_rn(2.0f, c, e);
    float s, t1, t2;
    two_sum(px, py, s, t1);
    two_sum(s, pz, s, t2);
    e = __fadd_rn(e, __fadd_rn(t1, t2));
    df r;
    fast_two_sum(s, e, r.h, r.l);
    return r;
}

// g = K_m u^4 (beta u^3 - 1) = u^4 (K_m beta u^3 - K_m), u = 1/R (lambda
// units).
__device__ __forceinline__ df pair_g(df R, const DfParams &P)
{
    const df u = df_rcp(R);
    const df u2 = df_sq(u);
    const df u3 = df_mul(u2, u);
    const df u4 = df_sq(u2);
    const df bu3 = df_mul(df{P.kb_h, P.kb_l}, u3);
    const df v = df_add(bu3, df{-P.ka_h, -P.ka_l});
    return df_mul(u4, v);
}

// Compensated accumulation of a double-float addend: s + c carries the sum.
__device__ __forceinline__ void df_acc(float &s, float &c, df x)
{
    float e;
    two_sum(s, x.h, s, e);
    c = __fadd_rn(c, __fadd_rn(e, x.l));
}

template <int TPI>
__device__ __forceinline__ void group_df_acc(float &s, float &c)
{
    const unsigned m = group_mask<TPI>();
#pragma unroll
    for (int o = TPI / 2; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(m, s, o, TPI);
        const float c2 = __shfl_xor_sync(m, c, o, TPI);
        float e;
        two_sum(s, s2, s, e);
        c = __fadd_rn(c, __fadd_rn(c2, e));
    }
}

// ---- packed form: two entries per lane in f32x2 registers ------------------
// sm_100 and later execute add/sub/mul/fma on a pair of FP32 values held in
// one 64-bit register with one instruction; two list entries of a lane go
// through the double-float sequence side by side, half the instructions.

typedef unsigned long long f2;

__device__ __forceinline__ f2 pk2(float a, float b)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}

__device__ __forceinline__ void up2(f2 v, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}

__device__ __forceinline__ f2 add2(f2 a, f2 b)
{
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ f2 sub2(f2 a, f2 b)
{
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ f2 mul2(f2 a, f2 b)
{
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// Exact negation (sign bits).
__device__ __forceinline__ f2 neg2(f2 a)
{
    return a ^ 0x8000000080000000ull;
}

struct df2 {
    f2 h, l;
};

__device__ __forceinline__ void two_sum2(f2 a, f2 b, f2 &s, f2 &e)
{
    s = add2(a, b);
    const f2 bb = sub2(s, a);
    e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}

__device__ __forceinline__ void fast_two_sum2(f2 a, f2 b, f2 &s, f2 &e)
{
    s = add2(a, b);
    e = sub2(b, sub2(s, a));
}

__device__ __forceinline__ df2 df2_mul(df2 a, df2 b)
{
    const f2 p = mul2(a.h, b.h);
    f2 e = fma2(a.h, b.h, neg2(p));
    e = fma2(a.h, b.l, e);
    e = fma2(a.l, b.h, e);
    df2 r;
    fast_two_sum2(p, e, r.h, r.l);
    return r;
}

__device__ __forceinline__ df2 df2_sq(df2 a)
{
    const f2 p = mul2(a.h, a.h);
    f2 e = fma2(a.h, a.h, neg2(p));
    e = fma2(add2(a.h, a.h), a.l, e);
    df2 r;
    fast_two_sum2(p, e, r.h, r.l);
    return r;
}

__device__ __forceinline__ df2 df2_add(df2 a, df2 b)
{
    f2 s, e;
    two_sum2(a.h, b.h, s, e);
    e = add2(e, add2(a.l, b.l));
    df2 r;
    fast_two_sum2(s, e, r.h, r.l);
    return r;
}

// 1/a as df_rcp, written with t = a y - 1 = -e so that no negation is
// needed: 1/a ~ y + y t (t - 1).
__device__ __forceinline__ df2 df2_rcp(df2 a)
{
    float a0, a1, y0, y1;
    up2(a.h, a0, a1);
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(a0));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y1) : "f"(a1));
    const f2 y = pk2(y0, y1);
    const f2 one = pk2(1.0f, 1.0f), mone = pk2(-1.0f, -1.0f);
    f2 t = fma2(a.h, y, mone);
    t = fma2(a.l, y, t);
    const f2 q = mul2(y, t);
    const f2 l = mul2(q, sub2(t, one));
    df2 r;
    fast_two_sum2(y, l, r.h, r.l);
    return r;
}

__device__ __forceinline__ df2 pair_g2(df2 R, const DfParams &P)
{
    const df2 u = df2_rcp(R);
    const df2 u2 = df2_sq(u);
    const df2 u3 = df2_mul(u2, u);
    const df2 u4 = df2_sq(u2);
    const df2 bu3 = df2_mul(df2{pk2(P.kb_h, P.kb_h), pk2(P.kb_l, P.kb_l)}, u3);
    const df2 v = df2_add(bu3, df2{pk2(-P.ka_h, -P.ka_h), pk2(-P.ka_l, -P.ka_l)});
    return df2_mul(u4, v);
}

// chunk_disp for the two entries of the pair (hj, mj, lj packed; hi, mi,
// li the row's values in both halves).
__device__ __forceinline__ df2 chunk_disp2(f2 hj, f2 hi, f2 mj, f2 mi, f2 lj, f2 li, f2 inv_period,
                                          f2 magic, f2 neg_period)
{
    f2 dh = sub2(hj, hi);
    const f2 k = sub2(fma2(dh, inv_period, magic), magic);
    dh = fma2(k, neg_period, dh);
    df2 d;
    f2 t;
    fast_two_sum2(dh, sub2(mj, mi), d.h, t);
    d.l = add2(t, sub2(lj, li));
    return d;
}

__device__ __forceinline__ df2 df2_norm2(df2 x, df2 y, df2 z)
{
    const f2 px = mul2(x.h, x.h), py = mul2(y.h, y.h), pz = mul2(z.h, z.h);
    f2 e = fma2(x.h, x.h, neg2(px));
    e = add2(e, fma2(y.h, y.h, neg2(py)));
    e = add2(e, fma2(z.h, z.h, neg2(pz)));
    f2 c = mul2(x.h, x.l);
    c = fma2(y.h, y.l, c);
    c = fma2(z.h, z.l, c);
    e = fma2(pk2(2.0f, 2.0f), c, e);
    f2 s, t1, t2;
    two_sum2(px, py, s, t1);
    two_sum2(s, pz, s, t2);
    e = add2(e, add2(t1, t2));
    df2 r;
    fast_two_sum2(s, e, r.h, r.l);
    return r;
}

__device__ __forceinline__ void df2_acc(f2 &s, f2 &c, df2 x)
{
    f2 e;
    two_sum2(s, x.h, s, e);
    c = add2(c, add2(e, x.l));
}

// ---- row walkers (single-system and batched kernels) ----------------------

// The FP64 definition for one entry: the oracle's displacement and cutoff
// decision, the FP64 form's impulse; added to p_i (and p_j for a half list).
template <bool HALF>
__device__ __forceinline__ void dfloat_fp64_pair(const double *__restrict__ q4, double *__restrict__ p4,
                                              int i, int j, const DfParams &P)
{
    double xi, yi, zi, xj, yj, zj;
    load_xyz(q4, i, xi, yi, zi);
    load_xyz(q4, j, xj, yj, zj);
    const double dx = min_image(__dsub_rn(xj, xi), P.L[0], P.half_bits[0]);
    const double dy = min_image(__dsub_rn(yj, yi), P.L[1], P.half_bits[1]);
    const double dz = min_image(__dsub_rn(zj, zi), P.L[2], P.half_bits[2]);
    if (!exact_in_cutoff(dx, dy, dz, P.rc2)) return;
    const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
    const double w = 1.0 / r2;
    const double w2 = w * w, w3 = w2 * w, w4 = w2 * w2;
    const double fn = w4 * fma(P.B, w3, -P.A);  // p_i -= fn d, p_j += fn d
    double *pi = p4 + 4 * static_cast<int64_t>(i);
    atomicAdd(pi + 0, -fn * dx);
    atomicAdd(pi + 1, -fn * dy);
    atomicAdd(pi + 2, -fn * dz);
    if (HALF) {
        double *pj = p4 + 4 * static_cast<int64_t>(j);
        atomicAdd(pj + 0, fn * dx);
        atomicAdd(pj + 1, fn * dy);
        atomicAdd(pj + 2, fn * dz);
    }
}

template <int TPI, bool HALF, bool CUBIC>
__device__ __forceinline__ void dfloat_row(const double *__restrict__ q4,
                                           const DfRec *__restrict__ rec, double *__restrict__ p4,
                                           const int *__restrict__ row_ptr,
                                           const int *__restrict__ col, int i, const DfParams &P,
                                           unsigned gm)
{
    const int sub = threadIdx.x & (TPI - 1);
    const DfRec ri = load_rec(rec, i);
    const float lix = lo_field(ri.lo, 0, P), liy = lo_field(ri.lo, 1, P), liz = lo_field(ri.lo, 2, P);
    float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f, sz = 0.f, cz = 0.f;
    const int kb = row_ptr[i], ke = row_ptr[i + 1];
    // The trip count is the group's (k - sub runs over the row in steps of
    // TPI), so the group's lanes vote together.
    for (int k0 = kb; k0 < ke; k0 += TPI) {
        const int k = k0 + sub;
        const bool valid = k < ke;
        const int j = valid ? col[k] : i;
        const DfRec rj = load_rec(rec, j);
        df dx = chunk_disp(rj.hx, ri.hx, rj.mx, ri.mx, lo_field(rj.lo, 0, P), lix, P);
        df dy = chunk_disp(rj.hy, ri.hy, rj.my, ri.my, lo_field(rj.lo, 1, P), liy, P);
        df dz = chunk_disp(rj.hz, ri.hz, rj.mz, ri.mz, lo_field(rj.lo, 2, P), liz, P);
        if (!CUBIC) {
            dx = df_mul(dx, df{P.cx_h[0], P.cx_l[0]});
            dy = df_mul(dy, df{P.cx_h[1], P.cx_l[1]});
            dz = df_mul(dz, df{P.cx_h[2], P.cx_l[2]});
        }
        df R = df_norm2(dx, dy, dz);
        bool in = valid && (R.h < P.T_h || (R.h == P.T_h && R.l < P.T_l));
        const bool exact = valid && (fabsf(R.h - P.T_h) <= P.band || R.h < P.r2_min);
        if (__any_sync(gm, exact)) {
            if (exact) {
                dfloat_fp64_pair<HALF>(q4, p4, i, j, P);
                in = false;
            }
        }
        if (!in) R = df{1.0f, 0.0f};
        const df g = pair_g(R, P);
        if (in) {
            const df fx = df_mul(g, dx), fy = df_mul(g, dy), fz = df_mul(g, dz);
            df_acc(sx, cx, fx);
            df_acc(sy, cy, fy);
            df_acc(sz, cz, fz);
            if (HALF) {
                double *pj = p4 + 4 * static_cast<int64_t>(j);
                atomicAdd(pj + 0, df_to_f64(fx.h, fx.l, P.k_exp));
                atomicAdd(pj + 1, df_to_f64(fy.h, fy.l, P.k_exp));
                atomicAdd(pj + 2, df_to_f64(fz.h, fz.l, P.k_exp));
            }
        }
    }
    if (TPI > 1) {
        group_df_acc<TPI>(sx, cx);
        group_df_acc<TPI>(sy, cy);
        group_df_acc<TPI>(sz, cz);
    }
    if (sub == 0) {
        double *pi = p4 + 4 * static_cast<int64_t>(i);
        atomicAdd(pi + 0, -df_to_f64(sx, cx, P.k_exp));
        atomicAdd(pi + 1, -df_to_f64(sy, cy, P.k_exp));
        atomicAdd(pi + 2, -df_to_f64(sz, cz, P.k_exp));
    }
}

// Two entries per lane and iteration (k and k + TPI of the row), carried
// through the double-float sequence side by side in f32x2 registers.
template <int TPI, bool HALF, bool CUBIC>
__device__ __forceinline__ void dfloat_row2(const double *__restrict__ q4,
                                            const DfRec *__restrict__ rec, double *__restrict__ p4,
                                            const int *__restrict__ row_ptr,
                                            const int *__restrict__ col, int i, const DfParams &P,
                                            unsigned gm)
{
    const int sub = threadIdx.x & (TPI - 1);
    const DfRec ri = load_rec(rec, i);
    const f2 hix = pk2(ri.hx, ri.hx), hiy = pk2(ri.hy, ri.hy), hiz = pk2(ri.hz, ri.hz);
    const f2 mix = pk2(ri.mx, ri.mx), miy = pk2(ri.my, ri.my), miz = pk2(ri.mz, ri.mz);
    const float l0 = lo_field(ri.lo, 0, P), l1 = lo_field(ri.lo, 1, P), l2 = lo_field(ri.lo, 2, P);
    const f2 lix = pk2(l0, l0), liy = pk2(l1, l1), liz = pk2(l2, l2);
    const f2 inv_period = pk2(P.inv_period, P.inv_period), magic = pk2(12582912.0f, 12582912.0f),
             neg_period = pk2(-P.period, -P.period), lo_scale = pk2(P.lo_scale, P.lo_scale),
             lo_moff = pk2(-P.lo_offset, -P.lo_offset);
    f2 sx = 0ull, cx = 0ull, sy = 0ull, cy = 0ull, sz = 0ull, cz = 0ull;
    const int kb = row_ptr[i], ke = row_ptr[i + 1];
    // Software pipelining of the gathers: the records of the next iteration
    // and the column indices of the one after are requested before the
    // arithmetic of the current iteration, so their L2 latency overlaps it.
    auto col_at = [&](int k) { return k < ke ? __ldg(col + k) : i; };
    int ja = col_at(kb + sub), jb = col_at(kb + sub + TPI);
    DfRec ra = load_rec(rec, ja), rb = load_rec(rec, jb);
    int ja_n = col_at(kb + sub + 2 * TPI), jb_n = col_at(kb + sub + 3 * TPI);
    for (int k0 = kb; k0 < ke; k0 += 2 * TPI) {
        const int ka = k0 + sub, kbb = ka + TPI;
        const bool va = ka < ke, vb = kbb < ke;
        const DfRec ra_n = load_rec(rec, ja_n), rb_n = load_rec(rec, jb_n);
        const int ja_nn = col_at(ka + 4 * TPI), jb_nn = col_at(ka + 5 * TPI);
        const f2 lx = fma2(pk2(__uint_as_float((ra.lo & 0x3ffu) | 0x4b000000u),
                               __uint_as_float((rb.lo & 0x3ffu) | 0x4b000000u)), lo_scale, lo_moff);
        const f2 ly = fma2(pk2(__uint_as_float(((ra.lo >> 10) & 0x3ffu) | 0x4b000000u),
                               __uint_as_float(((rb.lo >> 10) & 0x3ffu) | 0x4b000000u)), lo_scale, lo_moff);
        const f2 lz = fma2(pk2(__uint_as_float(((ra.lo >> 20) & 0x3ffu) | 0x4b000000u),
                               __uint_as_float(((rb.lo >> 20) & 0x3ffu) | 0x4b000000u)), lo_scale, lo_moff);
        df2 dx = chunk_disp2(pk2(ra.hx, rb.hx), hix, pk2(ra.mx, rb.mx), mix, lx, lix, inv_period, magic,
                             neg_period);
        df2 dy = chunk_disp2(pk2(ra.hy, rb.hy), hiy, pk2(ra.my, rb.my), miy, ly, liy, inv_period, magic,
                             neg_period);
        df2 dz = chunk_disp2(pk2(ra.hz, rb.hz), hiz, pk2(ra.mz, rb.mz), miz, lz, liz, inv_period, magic,
                             neg_period);
        if (!CUBIC) {
            dx = df2_mul(dx, df2{pk2(P.cx_h[0], P.cx_h[0]), pk2(P.cx_l[0], P.cx_l[0])});
            dy = df2_mul(dy, df2{pk2(P.cx_h[1], P.cx_h[1]), pk2(P.cx_l[1], P.cx_l[1])});
            dz = df2_mul(dz, df2{pk2(P.cx_h[2], P.cx_h[2]), pk2(P.cx_l[2], P.cx_l[2])});
        }
        const df2 R = df2_norm2(dx, dy, dz);
        float rah, rbh, ral, rbl;
        up2(R.h, rah, rbh);
        up2(R.l, ral, rbl);
        bool ina = va && (rah < P.T_h || (rah == P.T_h && ral < P.T_l));
        bool inb = vb && (rbh < P.T_h || (rbh == P.T_h && rbl < P.T_l));
        const bool exa = va && (fabsf(rah - P.T_h) <= P.band || rah < P.r2_min);
        const bool exb = vb && (fabsf(rbh - P.T_h) <= P.band || rbh < P.r2_min);
        if (__any_sync(gm, exa || exb)) {
            if (exa) {
                dfloat_fp64_pair<HALF>(q4, p4, i, ja, P);
                ina = false;
            }
            if (exb) {
                dfloat_fp64_pair<HALF>(q4, p4, i, jb, P);
                inb = false;
            }
        }
        // entries outside r_c: R = 1 keeps g finite, the mask zeroes it
        const df2 Rs{pk2(ina ? rah : 1.0f, inb ? rbh : 1.0f), pk2(ina ? ral : 0.0f, inb ? rbl : 0.0f)};
        df2 g = pair_g2(Rs, P);
        const f2 m = pk2(ina ? 1.0f : 0.0f, inb ? 1.0f : 0.0f);
        g.h = mul2(g.h, m);
        g.l = mul2(g.l, m);
        const df2 fx = df2_mul(g, dx), fy = df2_mul(g, dy), fz = df2_mul(g, dz);
        df2_acc(sx, cx, fx);
        df2_acc(sy, cy, fy);
        df2_acc(sz, cz, fz);
        if (HALF) {
            float xh0, xh1, xl0, xl1, yh0, yh1, yl0, yl1, zh0, zh1, zl0, zl1;
            up2(fx.h, xh0, xh1);
            up2(fx.l, xl0, xl1);
            up2(fy.h, yh0, yh1);
            up2(fy.l, yl0, yl1);
            up2(fz.h, zh0, zh1);
            up2(fz.l, zl0, zl1);
            if (ina) {
                double *pj = p4 + 4 * static_cast<int64_t>(ja);
                atomicAdd(pj + 0, df_to_f64(xh0, xl0, P.k_exp));
                atomicAdd(pj + 1, df_to_f64(yh0, yl0, P.k_exp));
                atomicAdd(pj + 2, df_to_f64(zh0, zl0, P.k_exp));
            }
            if (inb) {
                double *pj = p4 + 4 * static_cast<int64_t>(jb);
                atomicAdd(pj + 0, df_to_f64(xh1, xl1, P.k_exp));
                atomicAdd(pj + 1, df_to_f64(yh1, yl1, P.k_exp));
                atomicAdd(pj + 2, df_to_f64(zh1, zl1, P.k_exp));
            }
        }
        ra = ra_n;
        rb = rb_n;
        ja = ja_n;
        jb = jb_n;
        ja_n = ja_nn;
        jb_n = jb_nn;
    }
    // the two halves of each packed sum, then the group
    float s0, s1, c0, c1;
    float ax, bx, ay, by, az, bz;
    up2(sx, s0, s1);
    up2(cx, c0, c1);
    two_sum(s0, s1, ax, bx);
    bx = __fadd_rn(bx, __fadd_rn(c0, c1));
    up2(sy, s0, s1);
    up2(cy, c0, c1);
    two_sum(s0, s1, ay, by);
    by = __fadd_rn(by, __fadd_rn(c0, c1));
    up2(sz, s0, s1);
    up2(cz, c0, c1);
    two_sum(s0, s1, az, bz);
    bz = __fadd_rn(bz, __fadd_rn(c0, c1));
    if (TPI > 1) {
        group_df_acc<TPI>(ax, bx);
        group_df_acc<TPI>(ay, by);
        group_df_acc<TPI>(az, bz);
    }
    if (sub == 0) {
        double *pi = p4 + 4 * static_cast<int64_t>(i);
        atomicAdd(pi + 0, -df_to_f64(ax, bx, P.k_exp));
        atomicAdd(pi + 1, -df_to_f64(ay, by, P.k_exp));
        atomicAdd(pi + 2, -df_to_f64(az, bz, P.k_exp));
    }
}

// U = 1: one entry per lane and iteration; U = 2: dfloat_row2.
// ---- host --------------------------------------------------------------

inline void split_df(double v, float &h, float &l)
{
    h = static_cast<float>(v);
    l = static_cast<float>(v - static_cast<double>(h));
}

DfParams make_dfloat_params(const double box[3], double dt, double rc, double eps, double sigma)
{
    DfParams P{};
    const double L0 = box[0];
    // s: r_c <= lambda = L_0 2^-s < 2 r_c (s >= 1 since L >= 2 r_c).
    int s = static_cast<int>(std::floor(std::log2(L0 / rc)));
    if (s < 1) s = 1;
    while (std::ldexp(L0, -s) < rc && s > 1) --s;
    while (std::ldexp(L0, -s) >= 2.0 * rc) ++s;
    const double lambda = std::ldexp(L0, -s);
    double Lmax = 0.0;
    for (int a = 0; a < 3; ++a) {
        P.to_fixed[a] = std::ldexp(1.0, 58) / box[a];
        split_df(box[a] / L0, P.cx_h[a], P.cx_l[a]);
        P.L[a] = box[a];
        const double hh = 0.5 * box[a];
        std::memcpy(&P.half_bits[a], &hh, sizeof(double));
        Lmax = box[a] > Lmax ? box[a] : Lmax;
    }
    P.chunk_hi = static_cast<float>(std::ldexp(1.0, s - 24));
    P.chunk_mid = static_cast<float>(std::ldexp(1.0, s - 48));
    P.period = static_cast<float>(std::ldexp(1.0, s));
    P.inv_period = static_cast<float>(std::ldexp(1.0, -s));
    P.lo_scale = static_cast<float>(std::ldexp(1.0, s - 58));
    P.lo_offset = static_cast<float>(std::ldexp(1.0, s - 35));
    const double T = (rc / lambda) * (rc / lambda);
    split_df(T, P.T_h, P.T_l);
    // Band: the FP64 definition rounds each coordinate difference (and the
    // wrap) to <= 2 ulp(L), the fixed point to 2^-58 L; r^2 moves by at most
    // 2 sqrt(3) r_c times that plus the definition's own three roundings of
    // r^2; double-float keeps ~2^-44 of T.  Sixteen times the sum.
    const double ulpL = std::ldexp(1.0, std::ilogb(Lmax) - 52);
    const double dd = 2.0 * ulpL + 2.0 * std::ldexp(Lmax, -58);
    const double err = 2.0 * std::sqrt(3.0) * rc * dd + 3.0 * dd * dd + 4.0 * std::ldexp(rc * rc, -52);
    P.band = static_cast<float>(16.0 * err / (lambda * lambda) + std::ldexp(T, -36));
    const double sl = sigma / lambda, sl2 = sl * sl, sl6 = sl2 * sl2 * sl2;
    const double beta = 2.0 * sl6;
    // u = 1/R with u^4 <= 2^72 and beta u^7 <= 2^100: every intermediate of
    // pair_g stays a normal FP32 number.
    double umax = std::pow(std::ldexp(1.0, 100) / beta, 1.0 / 7.0);
    if (umax > std::ldexp(1.0, 18)) umax = std::ldexp(1.0, 18);
    P.r2_min = static_cast<float>(1.0 / umax);
    const double A = 24.0 * eps * sigma * sigma * sigma * sigma * sigma * sigma * dt;
    int ke = 0;
    const double km = 2.0 * std::frexp(A / std::pow(lambda, 7), &ke);  // [1, 2)
    P.k_exp = ke - 1;
    P.k_pow = std::ldexp(1.0, P.k_exp);
    split_df(km, P.ka_h, P.ka_l);
    split_df(km * beta, P.kb_h, P.kb_l);
    P.rc2 = rc * rc;
    const double s2 = sigma * sigma, s6 = s2 * s2 * s2, s12 = s6 * s6;
    P.A = 24.0 * eps * s6 * dt;
    P.B = 48.0 * eps * s12 * dt;
    return P;
}

}  // namespace
}  // namespace lj

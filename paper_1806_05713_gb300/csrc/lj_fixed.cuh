// lj_fixed.cuh -- the FP64 form with the displacement and r^2 exact in
// integer fixed point (schedule LJ_SCHED_FIXED).
//
// GB300 issues one FP64 warp instruction per 16 cycles of an SM, its
// integer units four per cycle, so the FP64 kernel is bound by its count of
// FP64 instructions per list entry (20 with image-selected displacement:
// 3 for d, 3 for r^2, 14 for Algorithm 1's impulse and the sums).  Here a
// pre-pass writes each coordinate as the 64-bit integer X = x 2^k (exact for
// x >= L/512, since 2^k L < 2^61 leaves every mantissa bit of x above the
// binary point; a rounding of 2^-(k+1) below that), and per entry
//   D = X_j - X_i, wrapped by one compare against M/2 = L 2^k / 2 (the
//       paper's minimum image, decided exactly),
//   r^2 = (D_x^2 + D_y^2 + D_z^2) 2^-2k exact in 128-bit integers,
// each rounded once to double with integer instructions.  The FP64
// definition rounds d = x_j - x_i (and the wrap) and the three products and
// sums of r^2; these values are at least as accurate.  1/r^2 is formed
// with integer instructions too (rcp_fp64_int: within 0.5 + 2^-12 ulp), and
// the rest -- the powers, df, df d and the momentum sums -- is the FP64
// form's IEEE double arithmetic: 11 FP64 instructions per entry of a half
// list (3 powers, 2 for df, 3 for df d, 3 for the row's sum; 8 for a full
// list, whose products df d fuse into the sum).  Entries whose r^2 lies
// within 64 ulp of r_c^2 take the FP64 definition for the decision and the
// displacement, so the interacting set and every pair near the cutoff are
// the oracle's.
#pragma once

#include <cmath>

#include "lj_rows.cuh"

namespace lj {
namespace {

struct FixParams {
    int k;                   // X = x 2^k
    double scale;            // 2^k
    long long M[3], Mh[3];   // L_a 2^k and floor(M / 2)
};

// The fixed point resolves 2^-k, with 2^k L_max < 2^61; positions below
// 2^(52-k) are rounded to it.  For L_max <= 1024 r_c that is below 2^-50 r_c
// (an FP64 rounding of d), so the fixed-point schedules are offered only
// there; larger boxes take the image-selected FP64 rows.
inline bool fixed_point_ok(const double box[3], double rc)
{
    double Lmax = 0.0;
    for (int a = 0; a < 3; ++a) Lmax = box[a] > Lmax ? box[a] : Lmax;
    return Lmax <= 1024.0 * rc;
}

FixParams make_fix_params(const double box[3])
{
    FixParams F{};
    double Lmax = 0.0;
    for (int a = 0; a < 3; ++a) Lmax = box[a] > Lmax ? box[a] : Lmax;
    int e = 0;
    std::frexp(Lmax, &e);  // Lmax < 2^e
    F.k = 61 - e;          // L 2^k < 2^61: |D| <= 2^60 after the wrap
    F.scale = std::ldexp(1.0, F.k);
    for (int a = 0; a < 3; ++a) {
        F.M[a] = std::llround(std::ldexp(box[a], F.k));
        F.Mh[a] = F.M[a] >> 1;
    }
    return F;
}

__global__ void fixed_prepass_kernel(const double *__restrict__ q4, int n, FixParams F,
                                     longlong4 *__restrict__ X)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x, y, z;
    load_xyz(q4, i, x, y, z);
    X[i] = make_longlong4(__double2ll_rn(x * F.scale), __double2ll_rn(y * F.scale),
                          __double2ll_rn(z * F.scale), 0);
}

__device__ __forceinline__ void load_fixed(const longlong4 *__restrict__ X, int j, long long &x,
                                           long long &y, long long &z)
{
    long long w;
    asm("ld.global.nc.v4.s64 {%0, %1, %2, %3}, [%4];"
        : "=l"(x), "=l"(y), "=l"(z), "=l"(w)
        : "l"(X + j));
}

// The minimum image of D = X_j - X_i (|D| < M): if D > M/2, D - M; if
// D < -M/2, D + M (strict, as the paper's definition; M/2 compared exactly).
__device__ __forceinline__ long long wrap_fixed(long long D, long long M, long long Mh)
{
    return D > Mh ? D - M : (D < -Mh ? D + M : D);
}

// m 2^(n-53-k), m in [2^52, 2^53], as double bits: the exponent field
// absorbs the carry of a mantissa rounded up to 2^53.
__device__ __forceinline__ double assemble_f64(unsigned long long m, int n, int k,
                                               unsigned long long sign)
{
    const unsigned long long ebias = static_cast<unsigned long long>(n - 1 - k + 1023);
    return __longlong_as_double(static_cast<long long>(sign | (((ebias - 1ull) << 52) + m)));
}

// Round-to-nearest-even of the top 53 bits of a (bit length n > 53).
__device__ __forceinline__ unsigned long long round53(unsigned long long top, unsigned long long rem,
                                                      unsigned long long half)
{
    return top + ((rem > half || (rem == half && (top & 1ull))) ? 1ull : 0ull);
}

// (hi 2^64 + lo) 2^-k2 rounded to the nearest double, integer instructions.
__device__ __forceinline__ double fixed128_to_f64(unsigned long long hi, unsigned long long lo, int k2)
{
    if ((hi | lo) == 0ull) return 0.0;
    int n;
    unsigned long long top, rem, half;
    if (hi == 0ull) {
        n = 64 - __clzll(static_cast<long long>(lo));
        if (n <= 53) return assemble_f64(lo << (53 - n), n, k2, 0ull);
        const int sh = n - 53;
        top = lo >> sh;
        rem = lo & ((1ull << sh) - 1ull);
        half = 1ull << (sh - 1);
    } else {
        n = 128 - __clzll(static_cast<long long>(hi));
        const int sh = n - 53;  // 12 .. 75
        if (sh < 64) {
            top = (hi << (64 - sh)) | (lo >> sh);
            rem = lo & ((1ull << sh) - 1ull);
            half = 1ull << (sh - 1);
        } else {
            // sh >= 64: the dropped part spans all of lo and the low bits of hi
            const int s2 = sh - 64;
            top = hi >> s2;
            const unsigned long long rhi = hi & ((1ull << s2) - 1ull);
            // compare (rhi, lo) with the half-way point 2^(sh-1)
            const unsigned long long hh = s2 > 0 ? (1ull << (s2 - 1)) : 0ull;
            const bool gt = s2 > 0 ? (rhi > hh || (rhi == hh && lo > 0ull)) : (lo > (1ull << 63));
            const bool eq = s2 > 0 ? (rhi == hh && lo == 0ull) : (lo == (1ull << 63));
            return assemble_f64(top + ((gt || (eq && (top & 1ull))) ? 1ull : 0ull), n, k2, 0ull);
        }
    }
    return assemble_f64(round53(top, rem, half), n, k2, 0ull);
}

// v 2^-k rounded to the nearest double (|v| < 2^63) with integer
// instructions and no branch: both the exact path (|v| < 2^53, shifted up
// into the significand) and the rounded one (|v| >= 2^53, round to nearest
// even) are computed and one is selected, so the lanes of a warp never
// diverge on the magnitude of their displacement.
__device__ __forceinline__ double fixed_to_f64_sel(long long v, int k)
{
    const unsigned long long sign = v < 0 ? 0x8000000000000000ull : 0ull;
    const unsigned long long a = static_cast<unsigned long long>(v < 0 ? -v : v);
    const int n = 64 - __clzll(static_cast<long long>(a));  // 0 for a = 0
    const int up = max(53 - n, 0), sh = max(n - 53, 0);
    const unsigned long long top = a >> sh;
    const unsigned long long rem = a & ((1ull << sh) - 1ull);
    const unsigned long long half = (1ull << sh) >> 1;       // 0 when sh = 0
    const bool rnd = sh > 0 && (rem > half || (rem == half && (top & 1ull)));
    const unsigned long long m = sh > 0 ? top + (rnd ? 1ull : 0ull) : a << up;
    const double d = assemble_f64(m, n, k, sign);
    return a == 0ull ? 0.0 : d;
}

// fixed128_to_f64 for hi != 0 (a value of 65 to 128 bits), without
// divergence: the 53 kept bits lie across hi and lo when the dropped count
// sh = n - 53 is below 64, in hi alone when it is 64 or more; both forms are
// computed and one is selected, so a warp never diverges on the size of a
// squared distance (the fixed-point scale k ties that size to the box: in
// small boxes list entries fall on both sides).  VOTE: the second form only
// when a lane of the group gm needs it (every lane of gm calls it) -- a gain
// for the whole-warp stream walk, a loss for the 4-16-lane groups, whose
// extra registers cost occupancy.  `fast` is false for
// hi = 0 (a squared distance below 2^(64-2k): coincident atoms, or an idle
// lane), where the caller converts with fixed128_to_f64.  Same values as
// fixed128_to_f64.
template <bool VOTE>
__device__ __forceinline__ double fixed128_to_f64_hi(unsigned long long hi, unsigned long long lo,
                                                     int k2, bool &fast, unsigned gm)
{
    fast = hi != 0ull;
    const int n = 128 - __clzll(static_cast<long long>(hi | 1ull));  // 65 .. 128 when fast
    const int sh = n - 53;
    // dropped bits all in lo (sh = 12 .. 63)
    const int s1 = min(max(sh, 12), 63);
    const unsigned long long top1 = (hi << (64 - s1)) | (lo >> s1);
    const unsigned long long rem1 = lo & ((1ull << s1) - 1ull);
    const unsigned long long half1 = 1ull << (s1 - 1);
    const bool up1 = rem1 > half1 || (rem1 == half1 && (top1 & 1ull));
    // the second form only when a lane of the group needs it (in a box
    // whose squared distances stay below 2^(117 - 2k), none does)
    if constexpr (VOTE) {
        if (__all_sync(gm, sh < 64)) return assemble_f64(top1 + (up1 ? 1ull : 0ull), n, k2, 0ull);
    }
    // dropped bits: all of lo and the low s2 bits of hi (sh = 64 .. 75)
    const int s2 = min(max(sh - 64, 0), 11);
    const unsigned long long top2 = hi >> s2;
    const unsigned long long rhi = hi & ((1ull << s2) - 1ull);
    const unsigned long long hh = (1ull << s2) >> 1;
    const bool gt2 = s2 > 0 ? (rhi > hh || (rhi == hh && lo > 0ull)) : (lo > (1ull << 63));
    const bool eq2 = s2 > 0 ? (rhi == hh && lo == 0ull) : (lo == (1ull << 63));
    const bool up2 = gt2 || (eq2 && (top2 & 1ull));
    const unsigned long long m = sh >= 64 ? top2 + (up2 ? 1ull : 0ull) : top1 + (up1 ? 1ull : 0ull);
    return assemble_f64(m, n, k2, 0ull);
}

// The range of rcp_fp64_int: 2^kRcpIntLo <= a < 2^kRcpIntHi.
constexpr int kRcpIntLo = -119;
constexpr int kRcpIntHi = 120;

// 1/a in double for 2^-119 <= a < 2^120 without an FP64 instruction: one
// Newton step, carried to second order, in integer arithmetic on the
// significands.  The seed y is the FP32 approximate reciprocal of a's
// leading 24 bits, so r = 1 - a y is about 2^-22 in magnitude.  With
// a = A 2^(ea-52) and y = Y 2^(ey-23) (A, Y the integer significands),
// a y = A Y 2^-S with S = 75 - ea - ey (75 or 76), and the residual
// E = 2^S - A Y = 2^S r is below 2^57 in magnitude: it is the low 64 bits
// of -A Y read as a signed number, exactly.  Then
// 1/a = y / (1 - r) = y (1 + r + r^2 + r^3 + ...); the terms
// z1 = Y 2^29 r, z2 = z1 r and z3 = z2 r are formed in integers in units of
// 2^-14 of the ulp of Y 2^29 (z1 from the exact product Y E, z2 and z3 from
// E's leading bits), and u = Y 2^29 + z1 + z2 + z3 is rounded to 53 bits in
// the binade it falls in.  The truncations and the dropped r^4 term leave u
// within about 2^-12 ulp of 1/a, so the result is within 0.5 + 2^-12 ulp
// (and correctly rounded unless 1/a lies that close to a midpoint).  It
// takes a few dozen integer instructions where an FP64 Newton step takes
// two FP64 ones, and leaves the FP64 pipe -- the limit of the FP64 force
// kernels -- to the force arithmetic.  `ok` is false outside the range.
// VOTE as fixed128_to_f64_hi (every lane of gm calls it; gm unused without).
template <bool VOTE>
__device__ __forceinline__ double rcp_fp64_int(double a, bool &ok, unsigned gm)
{
    const long long b = __double_as_longlong(a);
    const int ea = static_cast<int>((b >> 52) & 0x7ff) - 1023;
    ok = ea >= kRcpIntLo && ea < kRcpIntHi;  // the head and y stay normal floats
    const int e = ok ? ea : 0;
    const unsigned long long A =
        (static_cast<unsigned long long>(b) & 0xfffffffffffffull) | 0x10000000000000ull;
    const float head = __uint_as_float(static_cast<unsigned>((e + 127) << 23) |
                                       static_cast<unsigned>((A >> 29) & 0x7fffffull));
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(head));
    const unsigned uy = __float_as_uint(y);
    const int ey = static_cast<int>((uy >> 23) & 0xff) - 127;
    const unsigned Y = (uy & 0x7fffffu) | 0x800000u;
    const int S = 75 - e - ey;
    const long long E = -static_cast<long long>(A * static_cast<unsigned long long>(Y));
    // Q = floor(Y E / 2^32) = 2^(S-61) z1, from two 32 x 32 -> 64-bit products
    const long long Q = static_cast<long long>(Y) * (E >> 32) +
                        static_cast<long long>((static_cast<unsigned long long>(Y) *
                                                (static_cast<unsigned long long>(E) & 0xffffffffull)) >> 32);
    const long long z1 = Q >> (S - 75);  // 2^14 z1 (Q carries S - 61 = 14 or 15 fraction bits)
    const int Qh = static_cast<int>(Q >> 18);
    const int Eh = static_cast<int>(E >> 26);
    const long long z2 = (static_cast<long long>(Qh) * Eh) >> (2 * S - 119);       // 2^14 z2
    const long long z3 = (static_cast<long long>(static_cast<int>(z2)) * Eh) >> (S - 26);  // 2^14 z3
    const long long D = z1 + z2 + z3;
    const long long base = static_cast<long long>(Y) << 29;
    const long long fl = base + (D >> 14);  // floor(u)
    long long m = base + ((D + (1ll << 13)) >> 14);
    int ed = ey;
    const bool up = fl >= (1ll << 53), lo = fl < (1ll << 52);
    // u outside Y's binade (1/a and the seed on either side of a power of
    // two: rare); VOTE: under one vote of the group gm
    if (!VOTE || __any_sync(gm, up || lo)) {
        m = up ? (base >> 1) + ((D + (1ll << 14)) >> 15) : m;  // u in [2^53, 2^54): round u / 2
        m = lo ? 2 * base + ((D + (1ll << 12)) >> 13) : m;     // u below 2^52: round 2 u
        ed += up ? 1 : (lo ? -1 : 0);
    }
    const bool carry = m == (1ll << 53);
    m = carry ? (1ll << 52) : m;
    ed += carry ? 1 : 0;
    return __longlong_as_double((static_cast<long long>(ed + 1023) << 52) | (m & 0xfffffffffffffll));
}

// 1/sqrt(a) in double for 2^-120 < a < 2^120: the FP32 approximation of the
// head of a, then two Newton steps y (3/2 - a y^2 / 2) in FP64 (2^-23 ->
// 2^-46 -> below an ulp).  Outside the range, 1/sqrt by division.
__device__ __forceinline__ double rsqrt_fp64(double a)
{
    const long long b = __double_as_longlong(a);
    const int ea = static_cast<int>((b >> 52) & 0x7ff) - 1023;
    if (!(ea > -120 && ea < 120)) return 1.0 / sqrt(a);
    const float head = __uint_as_float(static_cast<unsigned>((ea + 127) << 23) |
                                       static_cast<unsigned>((b >> 29) & 0x7fffff));
    float y0;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(head));
    double y = f32_to_f64(y0);
    const double h = 0.5 * a;
#pragma unroll
    for (int it = 0; it < 2; ++it) y = fma(y, fma(-h, y * y, 0.5), y);
    return y;
}

// |D|^2 summed over three axes as a 128-bit integer (|D| <= 2^60 each).
__device__ __forceinline__ void norm2_fixed(long long dx, long long dy, long long dz,
                                            unsigned long long &hi, unsigned long long &lo)
{
    const unsigned long long ax = static_cast<unsigned long long>(dx < 0 ? -dx : dx);
    const unsigned long long ay = static_cast<unsigned long long>(dy < 0 ? -dy : dy);
    const unsigned long long az = static_cast<unsigned long long>(dz < 0 ? -dz : dz);
    unsigned long long l0 = ax * ax, h0 = __umul64hi(ax, ax);
    const unsigned long long l1 = ay * ay, h1 = __umul64hi(ay, ay);
    const unsigned long long l2 = az * az, h2 = __umul64hi(az, az);
    unsigned long long s = l0 + l1;
    h0 += h1 + (s < l0 ? 1ull : 0ull);
    l0 = s;
    s = l0 + l2;
    h0 += h2 + (s < l0 ? 1ull : 0ull);
    hi = h0;
    lo = s;
}

// The exact fixed-point displacement of entry j of row i (see the header
// comment): d in double, r^2 in double (1.0 for an invalid lane), and the
// FP64 definition's d, r^2 and decision for entries within 64 ulp of r_c^2.
// The common case (a squared distance of at least 2^(64-2k), away from the
// cutoff band, inside the range of rcp_fp64_int) is computed with selects
// only; the rare lanes -- coincident or nearly coincident atoms, an entry
// within 64 ulp of r_c^2, an r^2 outside the reciprocal's range (a
// division) -- are handled under one vote of the group gm (every lane of
// gm calls it).  Returns whether the pair interacts; *w_div receives 1/r^2
// by division for the lanes that need it (and *use_div says which).  VOTE:
// see fixed128_to_f64_hi.
template <bool VOTE = false>
__device__ __forceinline__ bool fixed_entry_sel(const double *__restrict__ q4, long long xi,
                                                long long yi, long long zi, long long xj,
                                                long long yj, long long zj, bool valid, int i, int j,
                                                const Fp64Params &P, const FixParams &F, unsigned gm,
                                                double &dx, double &dy, double &dz, double &r2,
                                                bool &use_div, double &w_div)
{
    const long long Dx = wrap_fixed(xj - xi, F.M[0], F.Mh[0]);
    const long long Dy = wrap_fixed(yj - yi, F.M[1], F.Mh[1]);
    const long long Dz = wrap_fixed(zj - zi, F.M[2], F.Mh[2]);
    unsigned long long hi, lo;
    norm2_fixed(Dx, Dy, Dz, hi, lo);
    bool fast;
    r2 = fixed128_to_f64_hi<VOTE>(hi, lo, 2 * F.k, fast, gm);
    dx = fixed_to_f64_sel(Dx, F.k);
    dy = fixed_to_f64_sel(Dy, F.k);
    dz = fixed_to_f64_sel(Dz, F.k);
    long long rb = __double_as_longlong(r2);
    bool in = valid && rb < P.rc2_bits;
    bool near = static_cast<unsigned long long>(rb - P.rc2_bits + 64) < 128ull;
    int ea = static_cast<int>((rb >> 52) & 0x7ff) - 1023;
    bool rcp_ok = ea >= kRcpIntLo && ea < kRcpIntHi;
    use_div = false;
    w_div = 0.0;
    const bool special = valid && (!fast || near || !rcp_ok);
    if (__any_sync(gm, special)) {
        if (special) {
            if (!fast) {
                r2 = fixed128_to_f64(hi, lo, 2 * F.k);
                rb = __double_as_longlong(r2);
                in = rb < P.rc2_bits;
                near = static_cast<unsigned long long>(rb - P.rc2_bits + 64) < 128ull;
            }
            if (near) {
                // the FP64 definition: its displacement, its decision
                double qxi, qyi, qzi, qxj, qyj, qzj;
                load_xyz(q4, i, qxi, qyi, qzi);
                load_xyz(q4, j, qxj, qyj, qzj);
                dx = min_image(__dsub_rn(qxj, qxi), P.L[0], P.half_bits[0]);
                dy = min_image(__dsub_rn(qyj, qyi), P.L[1], P.half_bits[1]);
                dz = min_image(__dsub_rn(qzj, qzi), P.L[2], P.half_bits[2]);
                in = exact_in_cutoff(dx, dy, dz, P.rc2);
                r2 = fma(dz, dz, fma(dy, dy, dx * dx));
            }
            ea = static_cast<int>((__double_as_longlong(r2) >> 52) & 0x7ff) - 1023;
            if (in && !(ea >= kRcpIntLo && ea < kRcpIntHi)) {
                use_div = true;
                w_div = 1.0 / r2;
            }
        }
    }
    if (!valid) r2 = 1.0;
    return in;
}

// One row of the FP64 form with the exact fixed-point displacement (see the
// header comment); the arithmetic after r^2 is fp64_row's.  EN: also sum the
// pair energy 4 eps [(sigma/r)^12 - (sigma/r)^6] of every interacting entry
// into *ev, its pair virial r F(r) into *wv, and count them in *ecount.
// FS: the force-shifted truncation -- df - F_c dt / r, and (EN) the pair
// energy V(r) - V(r_c) + (r - r_c) F_c and virial r F(r) - r F_c.
template <int TPI, bool HALF, bool EN = false, bool FS = false>
__device__ __forceinline__ void fp64_fixed_row(const double *__restrict__ q4,
                                               const longlong4 *__restrict__ X,
                                               double *__restrict__ p4,
                                               const int *__restrict__ row_ptr,
                                               const int *__restrict__ col, int i,
                                               const Fp64Params &P, const FixParams &F, unsigned gm,
                                               double *ev = nullptr, int *ecount = nullptr,
                                               double *wv = nullptr)
{
    const int sub = threadIdx.x & (TPI - 1);
    long long xi, yi, zi;
    load_fixed(X, i, xi, yi, zi);
    double ax = 0.0, ay = 0.0, az = 0.0;
    const int kb = row_ptr[i], ke = row_ptr[i + 1];
    for (int k0 = kb; k0 < ke; k0 += TPI) {
        const int k = k0 + sub;
        const bool valid = k < ke;
        const int j = valid ? col[k] : i;
        long long xj, yj, zj;
        load_fixed(X, j, xj, yj, zj);
        double dx, dy, dz, r2, w_div;
        bool use_div;
        const bool in = fixed_entry_sel(q4, xi, yi, zi, xj, yj, zj, valid, i, j, P, F, gm, dx, dy,
                                        dz, r2, use_div, w_div);
        // No vote on `in`: the FP64 chain runs for every lane (a group with
        // no interacting entry at all is rare), lanes outside r_c on r^2 = 1.
        {
            if (!in) r2 = 1.0;
            bool rcp_ok;
            double w = rcp_fp64_int<false>(r2, rcp_ok, gm);
            w = use_div ? w_div : w;
            const double w2 = w * w;
            const double w4 = w2 * w2;
            const double w3 = w2 * w;
            double fn = w4 * fma(P.B, w3, -P.A);  // -df: p_i -= fn d, p_j += fn d
            double inv_r = 0.0;
            if (FS) {
                inv_r = rsqrt_fp64(r2);
                fn = fma(-P.fs_c, inv_r, fn);  // the shifted coefficient: fn - F_c dt / r
            }
            if (in) {
                if (EN) {
                    double v = w3 * fma(P.C12, w3, -P.C6);
                    double vir = w3 * fma(P.W12, w3, -P.W6);
                    if (FS) {
                        v += fma(r2, inv_r, -P.rc) * P.Fc - P.Vc;
                        vir = fma(-P.Fc, r2 * inv_r, vir);
                    }
                    *ev += v;
                    *wv += vir;
                    ++*ecount;
                }
                if (HALF) {
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
    }
    double *pi = p4 + 4 * static_cast<int64_t>(i);
    if (HALF) {
        atomicAdd(pi + 0, ax);
        atomicAdd(pi + 1, ay);
        atomicAdd(pi + 2, az);
    } else {
        if (TPI > 1) {
            ax = group_sum<TPI>(ax);
            ay = group_sum<TPI>(ay);
            az = group_sum<TPI>(az);
        }
        if (sub == 0) {
            atomicAdd(pi + 0, ax);
            atomicAdd(pi + 1, ay);
            atomicAdd(pi + 2, az);
        }
    }
}


// LJ_SCHED_FIXED | LJ_SCHED_STREAM | R: a warp owns R consecutive rows and
// walks their entries as one range -- the rows of a CSR list are
// contiguous, so entries row_ptr[i0] .. row_ptr[i0 + R] are one range --
// cut into 32 contiguous chunks of C entries, one per lane (C a multiple of
// 4 and the chunks aligned to 16 bytes of col, so that a lane reads four
// column indices with one load).  Lanes idle only in the padding of the
// range, not at the end of every row (with 8 lanes per row about 15 % of
// the FP64 instruction slots of a random-order half list went to idle
// lanes).  A lane finds the row of its first entry by a binary search over
// the row pointers and then moves forward through the row boundaries; it
// keeps the partial sum of the row it is in and adds it to p_i with FP64
// atomics when it moves on.  A row is split over the one to three lanes
// whose chunks it spans, so full lists are not deterministic.
// Rows i0 .. i1-1 (i0 < i1) of the calling warp; every lane of the warp calls it.
// The stream walk indexes entries with 32-bit ints up to 128 past the end of
// a warp's range (the padding of the last chunk), so its callers keep a list
// (a system's, in a batch) at or below this many entries.
constexpr long long kStreamMaxEntries = 2147483647LL - 256;

template <bool HALF>
__device__ __forceinline__ void fp64_fixed_stream(const double *__restrict__ q4,
                                                  const longlong4 *__restrict__ X,
                                                  double *__restrict__ p4,
                                                  const int *__restrict__ row_ptr,
                                                  const int *__restrict__ col, int i0, int i1,
                                                  const Fp64Params &P, const FixParams &F)
{
    const int lane = threadIdx.x & 31;
    const int e0 = row_ptr[i0], e1 = row_ptr[i1];
    if (e0 >= e1) return;  // no entries (warp-uniform)
    // chunks start at a0 <= e0, where col + a0 is 16-byte aligned
    const int a0 = e0 - static_cast<int>((reinterpret_cast<uintptr_t>(col + e0) >> 2) & 3u);
    const int C = ((e1 - a0 + 127) >> 7) << 2;  // entries per lane: 32 C >= e1 - a0
    const int s = a0 + lane * C;                // this lane's entries: [s, s + C) within [e0, e1)
    // the row of the lane's first entry: the last row r < i1 with row_ptr[r] <= max(s, e0)
    int row = i0;
    {
        const int first = max(s, e0);
        int hi = i1;
        while (hi - row > 1) {
            const int mid = (row + hi) >> 1;
            if (row_ptr[mid] <= first)
                row = mid;
            else
                hi = mid;
        }
    }
    int row_end = row_ptr[row + 1];
    long long xi = 0, yi = 0, zi = 0;
    bool loaded = false, touched = false;
    double ax = 0.0, ay = 0.0, az = 0.0;
    int c0 = 0, c1 = 0, c2 = 0, c3 = 0;  // the column indices of entries e .. e + 3
    for (int k = 0; k < C; ++k) {
        const int e = s + k;
        if ((k & 3) == 0) {
            if (e >= e0 && e + 4 <= e1) {
                const int4 v = __ldg(reinterpret_cast<const int4 *>(col + e));
                c0 = v.x;
                c1 = v.y;
                c2 = v.z;
                c3 = v.w;
            } else {
                // the range's ends: only the indices inside [e0, e1) are read
                c0 = (e >= e0 && e < e1) ? __ldg(col + e) : 0;
                c1 = (e + 1 >= e0 && e + 1 < e1) ? __ldg(col + e + 1) : 0;
                c2 = (e + 2 >= e0 && e + 2 < e1) ? __ldg(col + e + 2) : 0;
                c3 = (e + 3 >= e0 && e + 3 < e1) ? __ldg(col + e + 3) : 0;
            }
        }
        const bool valid = e >= e0 && e < e1;
        // move to the row that holds entry e (rows may be empty)
        while (valid && e >= row_end) {
            if (touched) {
                double *pr = p4 + 4 * static_cast<int64_t>(row);
                atomicAdd(pr + 0, ax);
                atomicAdd(pr + 1, ay);
                atomicAdd(pr + 2, az);
                ax = ay = az = 0.0;
                touched = false;
            }
            ++row;
            row_end = row_ptr[row + 1];
            loaded = false;
        }
        if (valid && !loaded) {
            load_fixed(X, row, xi, yi, zi);
            loaded = true;
        }
        const int i = row;
        const int j = valid ? c0 : i;
        c0 = c1;
        c1 = c2;
        c2 = c3;
        long long xj, yj, zj;
        load_fixed(X, j, xj, yj, zj);
        double dx, dy, dz, r2, w_div;
        bool use_div;
        const bool in = fixed_entry_sel<true>(q4, xi, yi, zi, xj, yj, zj, valid, i, j, P, F, 0xffffffffu,
                                        dx, dy, dz, r2, use_div, w_div);
        if (!in) r2 = 1.0;
        bool rcp_ok;
        double w = rcp_fp64_int<true>(r2, rcp_ok, 0xffffffffu);
        w = use_div ? w_div : w;
        const double w2 = w * w;
        const double w4 = w2 * w2;
        const double w3 = w2 * w;
        const double fn = w4 * fma(P.B, w3, -P.A);  // -df: p_i -= fn d, p_j += fn d
        if (in) {
            touched = true;
            if (HALF) {
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
    if (touched) {
        double *pr = p4 + 4 * static_cast<int64_t>(row);
        atomicAdd(pr + 0, ax);
        atomicAdd(pr + 1, ay);
        atomicAdd(pr + 2, az);
    }
}

}  // namespace
}  // namespace lj

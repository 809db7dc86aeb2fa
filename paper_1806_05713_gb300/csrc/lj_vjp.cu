// lj_vjp.cu -- hand-written adjoint of the LJ force map.
//
// Forward map (Eq. (1) of Watanabe & Nakagawa differentiated once; the
// impulse of Algorithm 1 divided by dt): with d = q_j - q_i (minimum image),
// s = |d|^2 < r_c^2 and
//     g(s) = 24 eps (2 sigma^12 s^-7 - sigma^6 s^-4),
// each pair adds F_j += g d and F_i -= g d.
//
// Given R = dLoss/dF, the vector-Jacobian product per pair is, with
// w = R_j - R_i,
//     c        = g w + 2 g'(s) (d.w) d,     dLoss/dq_j += c, dLoss/dq_i -= c,
//     dLoss/deps   += (g / eps) (d.w),
//     dLoss/dsigma += (dg/dsigma) (d.w),
//     g'(s)      = 24 eps (-14 sigma^12 s^-8 + 4 sigma^6 s^-5),
//     dg/dsigma  = 24 eps (24 sigma^11 s^-7 - 6 sigma^5 s^-4).
// A full list visits every pair from both ends; c is odd under i <-> j, so
// row i gathers dLoss/dq_i = -sum_j c(d_ij, w_ij) with no atomics, and the
// two scalar gradients take half of the sum over entries.  A half list
// scatters c to q_j with FP64 atomics.
//
// Forms: FP64 (the displacement and s exact in integer fixed point and
// rounded once to double, as lj_force's LJ_SCHED_FIXED; every later step
// double), MIXED (fixed-point displacement rounded once to FP32, R rounded
// to FP32 once per atom, FP32 pair arithmetic as in lj_force,
// Kahan-compensated FP32 row and scalar sums, FP64 outputs).  Pairs within the error band of r_c^2 are
// decided by the exact FP64 definition in both forms.
#include <cmath>
#include <cstring>

#include "lj_fixed.cuh"
#include "lj_forms.cuh"

namespace lj {
namespace {

constexpr int kVjpTpi = 8;
constexpr int kVjpThreads = 256;

struct VjpCoef {
    double G1, G2;  // g      = u^4 (G1 u^3 - G2)
    double H1, H2;  // g'     = u^5 (H2 - H1 u^3)
    double T1, T2;  // 2 g'   = u^5 (T2 - T1 u^3): 2 H1, 2 H2 (exact)
    double S1, S2;  // dg/ds  = u^4 (S1 u^3 - S2)   (s = sigma)
    double inv_eps;
};

VjpCoef make_coef(double eps, double sigma)
{
    const double s2 = sigma * sigma, s5 = s2 * s2 * sigma, s6 = s5 * sigma, s11 = s5 * s6,
                 s12 = s6 * s6;
    VjpCoef C;
    C.G1 = 48.0 * eps * s12;
    C.G2 = 24.0 * eps * s6;
    C.H1 = 336.0 * eps * s12;
    C.H2 = 96.0 * eps * s6;
    C.T1 = 2.0 * C.H1;
    C.T2 = 2.0 * C.H2;
    C.S1 = 576.0 * eps * s11;
    C.S2 = 144.0 * eps * s5;
    C.inv_eps = 1.0 / eps;
    return C;
}

__device__ __forceinline__ void load_r3(const double *__restrict__ R4, int i, double &x, double &y,
                                        double &z)
{
    double w;
    asm("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];"
        : "=d"(x), "=d"(y), "=d"(z), "=d"(w)
        : "l"(R4 + 4 * static_cast<int64_t>(i)));
}

// Block reduction of two doubles into partial[2 * blockIdx.x + {0, 1}].
__device__ __forceinline__ void block_pair_sum(double a, double b, double *__restrict__ partial)
{
    __shared__ double red[2][kVjpThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = a;
        red[1][threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0;
        for (int w = 0; w < kVjpThreads / 32; ++w) {
            sa += red[0][w];
            sb += red[1][w];
        }
        partial[2 * blockIdx.x + 0] = sa;
        partial[2 * blockIdx.x + 1] = sb;
    }
}

// FIX: the exact fixed-point displacement (boxes up to 1024 r_c wide);
// otherwise image selection by integer compares of the FP64 coordinates.
template <bool HALF, bool FIX>
__global__ void __launch_bounds__(kVjpThreads)
vjp_fp64_kernel(const double *__restrict__ q4, const longlong4 *__restrict__ X,
                const double *__restrict__ R4, int n, const int *__restrict__ row_ptr,
                const int *__restrict__ col, Fp64Params P, FixParams F, VjpCoef C,
                double *__restrict__ gq4, double *__restrict__ partial)
{
    constexpr int TPI = kVjpTpi;
    const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / TPI;
    const int sub = threadIdx.x & (TPI - 1);
    const unsigned gm = group_mask<TPI>();
    double ge = 0.0, gs = 0.0;
    if (gid < n) {
        const int i = gid;
        double Rxi, Ryi, Rzi;
        long long fxi = 0, fyi = 0, fzi = 0;
        double ci[3], im[3][2];
        int th[3][2];
        if (FIX) {
            load_fixed(X, i, fxi, fyi, fzi);
        } else {
            load_q4_256(q4, i, ci[0], ci[1], ci[2]);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                im[a][0] = ci[a] - P.L[a];
                im[a][1] = ci[a] + P.L[a];
                double hl;
                memcpy(&hl, &P.half_bits[a], sizeof(double));
                th[a][0] = __double2hiint(ci[a] - hl);
                th[a][1] = __double2hiint(ci[a] + hl);
            }
        }
        load_r3(R4, i, Rxi, Ryi, Rzi);
        double ax = 0.0, ay = 0.0, az = 0.0;
        const int kb = row_ptr[i], ke = row_ptr[i + 1];
        for (int base = kb; base < ke; base += TPI) {
            const int k = base + sub;
            const bool valid = k < ke;
            const int j = valid ? col[k] : i;
            double dx, dy, dz, s, w_div = 0.0;
            bool in, use_div = false;
            if (FIX) {
                // the exact fixed-point displacement and r^2 (the FP64
                // definition within 64 ulp of r_c^2), with selects and one
                // vote for the rare lanes; s = 1 on an invalid lane
                long long fxj, fyj, fzj;
                load_fixed(X, j, fxj, fyj, fzj);
                in = fixed_entry_sel(q4, fxi, fyi, fzi, fxj, fyj, fzj, valid, i, j, P, F, gm, dx, dy,
                                     dz, s, use_div, w_div);
            } else {
                double cj[3];
                load_q4_256(q4, j, cj[0], cj[1], cj[2]);
                double dd[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const int hj = __double2hiint(cj[a]);
                    const double img = hj > th[a][1] ? im[a][1] : (hj < th[a][0] ? im[a][0] : ci[a]);
                    dd[a] = cj[a] - img;
                }
                dx = dd[0];
                dy = dd[1];
                dz = dd[2];
                s = fma(dz, dz, fma(dy, dy, dx * dx));
                const long long sb = __double_as_longlong(s);
                in = valid && sb < P.rc2_bits;
                const bool near = valid && static_cast<unsigned long long>(sb - P.rc2_bits + 64) < 128ull;
                if (__any_sync(gm, near)) {
                    if (near) {
                        const double ex = min_image(cj[0] - ci[0], P.L[0], P.half_bits[0]);
                        const double ey = min_image(cj[1] - ci[1], P.L[1], P.half_bits[1]);
                        const double ez = min_image(cj[2] - ci[2], P.L[2], P.half_bits[2]);
                        in = exact_in_cutoff(ex, ey, ez, P.rc2);
                    }
                }
                if (!valid) s = 1.0;
            }
            // fixed point: no vote on `in` (every lane runs the chain, a lane
            // outside r_c on its own r^2); image selection: skip groups with
            // no interacting entry
            if (FIX || __any_sync(gm, in)) {
                double Rxj, Ryj, Rzj;
                load_r3(R4, j, Rxj, Ryj, Rzj);
                double u;
                if (FIX) {
                    bool rcp_ok;
                    u = rcp_fp64_int<false>(s, rcp_ok, gm);
                    u = use_div ? w_div : u;
                } else {
                    u = rcp_fp64(s, gm);
                }
                const double u2 = u * u, u3 = u2 * u, u4 = u2 * u2, u5 = u4 * u;
                const double g = u4 * fma(C.G1, u3, -C.G2);
                const double gp2 = u5 * fma(-C.T1, u3, C.T2);  // 2 g', bit for bit
                const double dgs = u4 * fma(C.S1, u3, -C.S2);
                const double wx = Rxj - Rxi, wy = Ryj - Ryi, wz = Rzj - Rzi;
                const double rw = fma(dz, wz, fma(dy, wy, dx * wx));
                const double t = gp2 * rw;
                const double cx = fma(g, wx, t * dx), cy = fma(g, wy, t * dy),
                             cz = fma(g, wz, t * dz);
                if (in) {
                    ax -= cx;
                    ay -= cy;
                    az -= cz;
                    ge = fma(g, rw, ge);
                    gs = fma(dgs, rw, gs);
                    if (HALF) {
                        atomicAdd(gq4 + 4 * static_cast<int64_t>(j) + 0, cx);
                        atomicAdd(gq4 + 4 * static_cast<int64_t>(j) + 1, cy);
                        atomicAdd(gq4 + 4 * static_cast<int64_t>(j) + 2, cz);
                    }
                }
            }
        }
        ax = group_sum<TPI>(ax);
        ay = group_sum<TPI>(ay);
        az = group_sum<TPI>(az);
        if (sub == 0) {
            double *g = gq4 + 4 * static_cast<int64_t>(i);
            if (HALF) {
                atomicAdd(g + 0, ax);
                atomicAdd(g + 1, ay);
                atomicAdd(g + 2, az);
            } else {
                g[0] = ax;
                g[1] = ay;
                g[2] = az;
                g[3] = 0.0;
            }
        }
    }
    block_pair_sum(ge, gs, partial);
}

// Half lists of at least kVjpStreamRows rows (fixed point): a warp owns
// kVjpStreamR consecutive rows and cuts their entries into one contiguous
// chunk per lane, as lj_force's LJ_SCHED_STREAM (fp64_fixed_stream): lanes
// idle only in the padding of the last chunk instead of at the end of every
// row, and a lane adds its partial dLoss/dq_i with FP64 atomics when it
// leaves a row.  The pair arithmetic is vjp_fp64_kernel's.
constexpr int kVjpStreamR = 32;
constexpr int64_t kVjpStreamRows = 524288;

__device__ __forceinline__ void vjp_fp64_stream_walk(
    const double *__restrict__ q4, const longlong4 *__restrict__ X, const double *__restrict__ R4,
    const int *__restrict__ row_ptr, const int *__restrict__ col, int i0, int i1, const Fp64Params &P,
    const FixParams &F, const VjpCoef &C, double *__restrict__ gq4, double &ge, double &gs)
{
    const int lane = threadIdx.x & 31;
    const int e0 = row_ptr[i0], e1 = row_ptr[i1];
    if (e0 >= e1) return;  // no entries (warp-uniform)
    // chunks start at a0 <= e0, where col + a0 is 16-byte aligned
    const int a0 = e0 - static_cast<int>((reinterpret_cast<uintptr_t>(col + e0) >> 2) & 3u);
    const int CH = ((e1 - a0 + 127) >> 7) << 2;  // entries per lane: 32 CH >= e1 - a0
    const int s0 = a0 + lane * CH;
    int row = i0;  // the last row r < i1 with row_ptr[r] <= max(s0, e0)
    {
        const int first = max(s0, e0);
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
    long long fxi = 0, fyi = 0, fzi = 0;
    double Rxi = 0.0, Ryi = 0.0, Rzi = 0.0;
    bool loaded = false, touched = false;
    double ax = 0.0, ay = 0.0, az = 0.0;
    int c0 = 0, c1 = 0, c2 = 0, c3 = 0;  // the column indices of entries e .. e + 3
    for (int k = 0; k < CH; ++k) {
        const int e = s0 + k;
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
        while (valid && e >= row_end) {
            if (touched) {
                double *g = gq4 + 4 * static_cast<int64_t>(row);
                atomicAdd(g + 0, ax);
                atomicAdd(g + 1, ay);
                atomicAdd(g + 2, az);
                ax = ay = az = 0.0;
                touched = false;
            }
            ++row;
            row_end = row_ptr[row + 1];
            loaded = false;
        }
        if (valid && !loaded) {
            load_fixed(X, row, fxi, fyi, fzi);
            load_r3(R4, row, Rxi, Ryi, Rzi);
            loaded = true;
        }
        const int i = row;
        const int j = valid ? c0 : i;
        c0 = c1;
        c1 = c2;
        c2 = c3;
        long long fxj, fyj, fzj;
        load_fixed(X, j, fxj, fyj, fzj);
        double dx, dy, dz, sq, w_div;
        bool use_div;
        const bool in = fixed_entry_sel<true>(q4, fxi, fyi, fzi, fxj, fyj, fzj, valid, i, j, P, F,
                                              0xffffffffu, dx, dy, dz, sq, use_div, w_div);
        double Rxj, Ryj, Rzj;
        load_r3(R4, j, Rxj, Ryj, Rzj);
        bool rcp_ok;
        double u = rcp_fp64_int<true>(sq, rcp_ok, 0xffffffffu);
        u = use_div ? w_div : u;
        const double u2 = u * u, u3 = u2 * u, u4 = u2 * u2, u5 = u4 * u;
        const double g = u4 * fma(C.G1, u3, -C.G2);
        const double gp2 = u5 * fma(-C.T1, u3, C.T2);  // 2 g'
        const double dgs = u4 * fma(C.S1, u3, -C.S2);
        const double wx = Rxj - Rxi, wy = Ryj - Ryi, wz = Rzj - Rzi;
        const double rw = fma(dz, wz, fma(dy, wy, dx * wx));
        const double t = gp2 * rw;
        const double cx = fma(g, wx, t * dx), cy = fma(g, wy, t * dy), cz = fma(g, wz, t * dz);
        if (in) {
            touched = true;
            ax -= cx;
            ay -= cy;
            az -= cz;
            ge = fma(g, rw, ge);
            gs = fma(dgs, rw, gs);
            double *gj = gq4 + 4 * static_cast<int64_t>(j);
            atomicAdd(gj + 0, cx);
            atomicAdd(gj + 1, cy);
            atomicAdd(gj + 2, cz);
        }
    }
    if (touched) {
        double *g = gq4 + 4 * static_cast<int64_t>(row);
        atomicAdd(g + 0, ax);
        atomicAdd(g + 1, ay);
        atomicAdd(g + 2, az);
    }
}

__global__ void __launch_bounds__(kVjpThreads, 4)
vjp_fp64_stream_kernel(const double *__restrict__ q4, const longlong4 *__restrict__ X,
                       const double *__restrict__ R4, int n, const int *__restrict__ row_ptr,
                       const int *__restrict__ col, Fp64Params P, FixParams F, VjpCoef C,
                       double *__restrict__ gq4, double *__restrict__ partial)
{
    const long long w = (static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    double ge = 0.0, gs = 0.0;
    if (w * kVjpStreamR < n) {
        const int i0 = static_cast<int>(w * kVjpStreamR);
        vjp_fp64_stream_walk(q4, X, R4, row_ptr, col, i0, min(i0 + kVjpStreamR, n), P, F, C, gq4,
                             ge, gs);
    }
    block_pair_sum(ge, gs, partial);
}

// MIXED form: one 32-byte record per atom, written by a pre-pass -- the
// 32-bit fixed-point position {X, Y, Z} (as lj_force's mixed pre-pass) and
// R = dLoss/dF rounded to FP32 -- so a gathered atom is one 256-bit load
// (one sector) and no float/double conversion runs in the pair loop (those
// run on GB300's FP64 pipe).
__global__ void vjp_mixed_prepass_kernel(const double *__restrict__ q4,
                                         const double *__restrict__ R4, int n, MixedParams P,
                                         ulonglong4 *__restrict__ rec)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x, y, z, rx, ry, rz;
    load_xyz(q4, i, x, y, z);
    load_r3(R4, i, rx, ry, rz);
    const unsigned X = __double2uint_rz(x * P.to_fixed[0]), Y = __double2uint_rz(y * P.to_fixed[1]),
                   Z = __double2uint_rz(z * P.to_fixed[2]);
    const unsigned fx = __float_as_uint(__double2float_rn(rx)),
                   fy = __float_as_uint(__double2float_rn(ry)),
                   fz = __float_as_uint(__double2float_rn(rz));
    rec[i] = make_ulonglong4(static_cast<unsigned long long>(X) | (static_cast<unsigned long long>(Y) << 32),
                             static_cast<unsigned long long>(Z),
                             static_cast<unsigned long long>(fx) | (static_cast<unsigned long long>(fy) << 32),
                             static_cast<unsigned long long>(fz));
}

struct MixedVjpRec {
    unsigned X, Y, Z;
    float rx, ry, rz;
};

__device__ __forceinline__ MixedVjpRec load_mixed_vjp_rec(const ulonglong4 *__restrict__ rec, int j)
{
    unsigned long long a, b, c, d;
    asm("ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];"
        : "=l"(a), "=l"(b), "=l"(c), "=l"(d)
        : "l"(rec + j));
    MixedVjpRec r;
    r.X = static_cast<unsigned>(a);
    r.Y = static_cast<unsigned>(a >> 32);
    r.Z = static_cast<unsigned>(b);
    r.rx = __uint_as_float(static_cast<unsigned>(c));
    r.ry = __uint_as_float(static_cast<unsigned>(c >> 32));
    r.rz = __uint_as_float(static_cast<unsigned>(d));
    return r;
}

// The row walk takes each lane's record one entry ahead and its column
// index two ahead (software pipelining of the gathers, as lj_force's mixed
// row); each lane adds its entries in increasing k as before.
template <bool HALF>
__global__ void __launch_bounds__(kVjpThreads)
vjp_mixed_kernel(const double *__restrict__ q4, const ulonglong4 *__restrict__ rec, int n,
                 const int *__restrict__ row_ptr, const int *__restrict__ col, MixedParams P,
                 float G1, float G2, float H1, float H2, float S1, float S2,
                 double *__restrict__ gq4, double *__restrict__ partial)
{
    constexpr int TPI = kVjpTpi;
    const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / TPI;
    const int sub = threadIdx.x & (TPI - 1);
    const unsigned gm = group_mask<TPI>();
    float es = 0.f, ec = 0.f, ss = 0.f, sc = 0.f;  // Kahan sums of g (d.w), dg/dsigma (d.w)
    if (gid < n) {
        const int i = gid;
        const MixedVjpRec ri = load_mixed_vjp_rec(rec, i);
        float sx = 0.f, sy = 0.f, sz = 0.f, kx = 0.f, ky = 0.f, kz = 0.f;
        const int kb = row_ptr[i], ke = row_ptr[i + 1];
        auto col_at = [&](int k) { return k < ke ? __ldg(col + k) : i; };
        int j = col_at(kb + sub);
        MixedVjpRec rj = load_mixed_vjp_rec(rec, j);
        int jn = col_at(kb + sub + TPI);
        for (int base = kb; base < ke; base += TPI) {
            const MixedVjpRec rn = load_mixed_vjp_rec(rec, jn);
            const int jnn = col_at(base + sub + 2 * TPI);
            const bool valid = base + sub < ke;
            const float dx = fixed_disp(rj.X, ri.X, P.scale[0]);
            const float dy = fixed_disp(rj.Y, ri.Y, P.scale[1]);
            const float dz = fixed_disp(rj.Z, ri.Z, P.scale[2]);
            float s = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            bool in = valid && s < P.rc2f;
            const bool near = valid && fabsf(s - P.rc2f) <= P.band;
            if (__any_sync(gm, near)) {
                if (near) {
                    double xi, yi, zi, xj, yj, zj;
                    load_xyz(q4, i, xi, yi, zi);
                    load_xyz(q4, j, xj, yj, zj);
                    const double ex = min_image(xj - xi, P.L[0], P.half_bits[0]);
                    const double ey = min_image(yj - yi, P.L[1], P.half_bits[1]);
                    const double ez = min_image(zj - zi, P.L[2], P.half_bits[2]);
                    in = exact_in_cutoff(ex, ey, ez, P.rc2);
                }
            }
            if (!valid) s = 1.0f;
            if (in) {
                const float u = rcp_fp32(s);
                const float u2 = u * u, u3 = u2 * u, u4 = u2 * u2, u5 = u4 * u;
                const float g = u4 * fmaf(G1, u3, -G2);
                const float gp = u5 * fmaf(-H1, u3, H2);
                const float dgs = u4 * fmaf(S1, u3, -S2);
                const float wx = rj.rx - ri.rx, wy = rj.ry - ri.ry, wz = rj.rz - ri.rz;
                const float rw = fmaf(dz, wz, fmaf(dy, wy, dx * wx));
                const float t = 2.0f * gp * rw;
                const float cx = fmaf(g, wx, t * dx), cy = fmaf(g, wy, t * dy), cz = fmaf(g, wz, t * dz);
                kahan_add(sx, kx, -cx);
                kahan_add(sy, ky, -cy);
                kahan_add(sz, kz, -cz);
                kahan_add(es, ec, g * rw);
                kahan_add(ss, sc, dgs * rw);
                if (HALF) {
                    atomicAdd(gq4 + 4 * static_cast<int64_t>(j) + 0, f32_to_f64(cx));
                    atomicAdd(gq4 + 4 * static_cast<int64_t>(j) + 1, f32_to_f64(cy));
                    atomicAdd(gq4 + 4 * static_cast<int64_t>(j) + 2, f32_to_f64(cz));
                }
            }
            rj = rn;
            j = jn;
            jn = jnn;
        }
        group_kahan<TPI>(sx, kx);
        group_kahan<TPI>(sy, ky);
        group_kahan<TPI>(sz, kz);
        if (sub == 0) {
            const double ax = f32_to_f64(sx) - f32_to_f64(kx);
            const double ay = f32_to_f64(sy) - f32_to_f64(ky);
            const double az = f32_to_f64(sz) - f32_to_f64(kz);
            double *g = gq4 + 4 * static_cast<int64_t>(i);
            if (HALF) {
                atomicAdd(g + 0, ax);
                atomicAdd(g + 1, ay);
                atomicAdd(g + 2, az);
            } else {
                g[0] = ax;
                g[1] = ay;
                g[2] = az;
                g[3] = 0.0;
            }
        }
    }
    block_pair_sum(static_cast<double>(es) - static_cast<double>(ec),
                   static_cast<double>(ss) - static_cast<double>(sc), partial);
}

// grads[0] = scale * inv_eps * sum(partial[2b]), grads[1] = scale * sum(partial[2b+1]),
// summed in a fixed order.
__global__ void vjp_final_kernel(const double *__restrict__ partial, int blocks, double scale,
                                 double inv_eps, double *__restrict__ grads)
{
    __shared__ double red[2][32];
    double a = 0.0, b = 0.0;
    for (int t = threadIdx.x; t < blocks; t += blockDim.x) {
        a += partial[2 * t];
        b += partial[2 * t + 1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = a;
        red[1][threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0;
        for (int w = 0; w < int(blockDim.x / 32); ++w) {
            sa += red[0][w];
            sb += red[1][w];
        }
        grads[0] = scale * inv_eps * sa;
        grads[1] = scale * sb;
    }
}

int vjp_blocks(int64_t n) { return int((n * kVjpTpi + kVjpThreads - 1) / kVjpThreads); }

}  // namespace

int check_force_args(const double *q4, const double *p4, int64_t n, const int32_t *row_ptr,
                     const int32_t *col, int64_t nnz, double r_cut, const double box[3], double eps,
                     double sigma, double dt);

size_t vjp_dfloat_extra_bytes(int64_t n);
int vjp_dfloat(const double *q4, const double *R4, int n, const int *row_ptr, const int *col,
               int half, double rc, const double box[3], double eps, double sigma, double *gq4,
               double *partial, int blocks, void *extra, cudaStream_t st);

}  // namespace lj

extern "C" size_t lj_force_vjp_workspace_bytes(int64_t n, int precision)
{
    const size_t blocks = size_t(lj::vjp_blocks(n > 0 ? n : 1));
    size_t bytes = 2 * blocks * sizeof(double) + 256;
    if (precision == LJ_MIXED) bytes += size_t(n > 0 ? n : 1) * sizeof(ulonglong4) + 256;
    if (precision == LJ_FP64) bytes += size_t(n > 0 ? n : 1) * sizeof(longlong4) + 256;
    if (precision == LJ_DFLOAT) bytes += lj::vjp_dfloat_extra_bytes(n) + 256;
    return bytes;
}

extern "C" int lj_force_vjp(const double *q4_dev, const double *gradF4_dev, int64_t n,
                            const int32_t *row_ptr_dev, const int32_t *col_dev, int64_t nnz,
                            int half, double r_cut, const double box[3], double eps, double sigma,
                            int precision, double *gradq4_dev, double *grad_eps_sigma_dev,
                            void *workspace_dev, size_t workspace_bytes, void *stream)
{
    using namespace lj;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = check_force_args(q4_dev, gradq4_dev, n, row_ptr_dev, col_dev, nnz, r_cut, box, eps,
                              sigma, 1.0);
    if (rc != LJ_OK) return rc;
    if (!grad_eps_sigma_dev || (n > 0 && !gradF4_dev)) return LJ_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(gradF4_dev) & 31u) return LJ_ERR_ARG;
    if (precision != LJ_FP64 && precision != LJ_MIXED && precision != LJ_DFLOAT) return LJ_ERR_ARG;
    if (n == 0) {
        LJ_TRY_CUDA(cudaMemsetAsync(grad_eps_sigma_dev, 0, 2 * sizeof(double), st));
        return LJ_OK;
    }
    if (!workspace_dev || workspace_bytes < lj_force_vjp_workspace_bytes(n, precision))
        return LJ_ERR_CAPACITY;
    const int ni = static_cast<int>(n);
    const int blocks = vjp_blocks(n);
    int used_blocks = blocks;  // blocks that write a partial sum (the stream walk uses fewer)
    Carver c(workspace_dev);
    double *partial = c.take<double>(2 * size_t(blocks));
    if (half || nnz == 0)
        LJ_TRY_CUDA(cudaMemsetAsync(gradq4_dev, 0, size_t(n) * 4 * sizeof(double), st));
    if (precision == LJ_DFLOAT) {
        void *extra = c.take<char>(vjp_dfloat_extra_bytes(n));
        rc = vjp_dfloat(q4_dev, gradF4_dev, ni, row_ptr_dev, col_dev, half, r_cut, box, eps, sigma,
                        gradq4_dev, partial, blocks, extra, st);
        if (rc != LJ_OK) return rc;
    } else if (precision == LJ_FP64) {
        const Fp64Params P = make_fp64_params(box, 1.0, r_cut, eps, sigma);
        const FixParams F = make_fix_params(box);
        const VjpCoef C = make_coef(eps, sigma);
        longlong4 *X = c.take<longlong4>(size_t(n));
        if (fixed_point_ok(box, r_cut)) {
            fixed_prepass_kernel<<<unsigned((n + 255) / 256), 256, 0, st>>>(q4_dev, ni, F, X);
            LJ_TRY_LAUNCH("fixed_prepass_kernel");
            if (half && n >= kVjpStreamRows && nnz <= kStreamMaxEntries) {
                const int64_t warps = (n + kVjpStreamR - 1) / kVjpStreamR;
                used_blocks = static_cast<int>((warps * 32 + kVjpThreads - 1) / kVjpThreads);
                vjp_fp64_stream_kernel<<<used_blocks, kVjpThreads, 0, st>>>(
                    q4_dev, X, gradF4_dev, ni, row_ptr_dev, col_dev, P, F, C, gradq4_dev, partial);
            } else if (half) {
                vjp_fp64_kernel<true, true><<<blocks, kVjpThreads, 0, st>>>(
                    q4_dev, X, gradF4_dev, ni, row_ptr_dev, col_dev, P, F, C, gradq4_dev, partial);
            } else {
                vjp_fp64_kernel<false, true><<<blocks, kVjpThreads, 0, st>>>(
                    q4_dev, X, gradF4_dev, ni, row_ptr_dev, col_dev, P, F, C, gradq4_dev, partial);
            }
        } else {
            if (half)
                vjp_fp64_kernel<true, false><<<blocks, kVjpThreads, 0, st>>>(
                    q4_dev, X, gradF4_dev, ni, row_ptr_dev, col_dev, P, F, C, gradq4_dev, partial);
            else
                vjp_fp64_kernel<false, false><<<blocks, kVjpThreads, 0, st>>>(
                    q4_dev, X, gradF4_dev, ni, row_ptr_dev, col_dev, P, F, C, gradq4_dev, partial);
        }
        LJ_TRY_LAUNCH("vjp_fp64_kernel");
    } else {
        const MixedParams P = make_mixed_params(box, 1.0, r_cut, eps, sigma);
        const VjpCoef C = make_coef(eps, sigma);
        ulonglong4 *rec = c.take<ulonglong4>(size_t(n));
        vjp_mixed_prepass_kernel<<<unsigned((n + 255) / 256), 256, 0, st>>>(q4_dev, gradF4_dev, ni,
                                                                            P, rec);
        LJ_TRY_LAUNCH("vjp_mixed_prepass_kernel");
        const float G1 = float(C.G1), G2 = float(C.G2), H1 = float(C.H1), H2 = float(C.H2),
                    S1 = float(C.S1), S2 = float(C.S2);
        if (half)
            vjp_mixed_kernel<true><<<blocks, kVjpThreads, 0, st>>>(q4_dev, rec, ni, row_ptr_dev,
                                                                    col_dev, P, G1, G2, H1, H2, S1, S2,
                                                                    gradq4_dev, partial);
        else
            vjp_mixed_kernel<false><<<blocks, kVjpThreads, 0, st>>>(q4_dev, rec, ni, row_ptr_dev,
                                                                     col_dev, P, G1, G2, H1, H2, S1, S2,
                                                                     gradq4_dev, partial);
        LJ_TRY_LAUNCH("vjp_mixed_kernel");
    }
    const double scale = half ? 1.0 : 0.5;
    vjp_final_kernel<<<1, 1024, 0, st>>>(partial, used_blocks, scale, 1.0 / eps, grad_eps_sigma_dev);
    LJ_TRY_LAUNCH("vjp_final_kernel");
    return LJ_OK;
}

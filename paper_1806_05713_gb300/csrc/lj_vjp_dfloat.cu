// lj_vjp_dfloat.cu -- the adjoint of the force map in the DFLOAT form:
// FP64-class gradients from double-float arithmetic on the FP32 pipe.
//
// The map and its vector-Jacobian product are those of lj_vjp.cu (derived
// from Eq. (1)): per pair, with d = q_j - q_i, s = |d|^2, w = R_j - R_i,
//     c = g(s) w + 2 g'(s) (d.w) d,   dL/dq_j += c,  dL/dq_i -= c,
//     dL/deps += g (d.w) / eps,       dL/dsigma += (dg/dsigma) (d.w).
// In units of lambda (lj_dfloat.cuh: d = lambda delta, s = lambda^2 R,
// u = 1/R, beta = 2 (sigma/lambda)^6) the three radial functions are
//     g       = K_g  u^4 (beta u^3 - 1),          K_g = 24 eps sigma^6 / lambda^8,
//     g'      = 4 K_g / lambda^2 u^5 (1 - 7/4 beta u^3),
//     dg/dsig = K_s  u^4 (2 beta u^3 - 1),        K_s = 144 eps sigma^5 / lambda^8,
// so c = K_g [ g^ w + 8 g'^ (delta.w) delta ] with g^ = u^4 (beta u^3 - 1),
// g'^ = u^5 (1 - 7/4 beta u^3), and the scalar sums are K_g lambda sum g^ (delta.w)
// and K_s lambda sum (dg/dsig)^ (delta.w).  The hat quantities and the sums are
// double-float; the K factors are applied in FP64 where the results leave
// the kernel.  Pairs inside the cutoff band, or closer than the range in
// which u^8 stays a normal FP32 number, take the FP64 formulas.
#include <cmath>

#include "lj_dfloat.cuh"

namespace lj {
namespace {

constexpr int kDvTpi = 8;
constexpr int kDvThreads = 256;

struct DfVjp {
    DfParams D;            // geometry, fixed-point chunks, cutoff band
    float b_h, b_l;        // beta
    float c_h, c_l;        // 7/4 beta
    float r2_min;          // R below this: FP64 formulas
    double Kc;             // K_g: gradient of q
    double Ke;             // K_g lambda: d/deps (before 1/eps)
    double Ks;             // K_s lambda: d/dsigma
    double G1, G2, H1, H2, S1, S2;  // FP64 coefficients (as lj_vjp.cu)
};

// The FP64 radial parts of one pair (the fallback): c (into cx, cy, cz),
// g (d.w) and (dg/dsigma) (d.w).
__device__ __forceinline__ bool fp64_vjp_pair(const double *__restrict__ q4,
                                              const double *__restrict__ R4, int i, int j,
                                              const DfVjp &V, double &cx, double &cy, double &cz,
                                              double &ge, double &gs)
{
    const DfParams &D = V.D;
    double xi, yi, zi, xj, yj, zj;
    load_xyz(q4, i, xi, yi, zi);
    load_xyz(q4, j, xj, yj, zj);
    const double dx = min_image(__dsub_rn(xj, xi), D.L[0], D.half_bits[0]);
    const double dy = min_image(__dsub_rn(yj, yi), D.L[1], D.half_bits[1]);
    const double dz = min_image(__dsub_rn(zj, zi), D.L[2], D.half_bits[2]);
    if (!exact_in_cutoff(dx, dy, dz, D.rc2)) return false;
    double rxi, ryi, rzi, rxj, ryj, rzj;
    load_xyz(R4, i, rxi, ryi, rzi);
    load_xyz(R4, j, rxj, ryj, rzj);
    const double s = fma(dz, dz, fma(dy, dy, dx * dx));
    const double u = 1.0 / s;
    const double u2 = u * u, u3 = u2 * u, u4 = u2 * u2, u5 = u4 * u;
    const double g = u4 * fma(V.G1, u3, -V.G2);
    const double gp = u5 * fma(-V.H1, u3, V.H2);
    const double dgs = u4 * fma(V.S1, u3, -V.S2);
    const double wx = rxj - rxi, wy = ryj - ryi, wz = rzj - rzi;
    const double rw = fma(dz, wz, fma(dy, wy, dx * wx));
    const double t = 2.0 * gp * rw;
    cx = fma(g, wx, t * dx);
    cy = fma(g, wy, t * dy);
    cz = fma(g, wz, t * dz);
    ge = g * rw;
    gs = dgs * rw;
    return true;
}

// R (FP64) as double-float, one 32-byte record per atom:
// {Rx_h, Ry_h, Rz_h, Rx_l, Ry_l, Rz_l, 0, 0}.
__global__ void dfloat_r_prepass_kernel(const double *__restrict__ R4, int n, float *__restrict__ rr)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double r[3];
    load_xyz(R4, i, r[0], r[1], r[2]);
    float o[8];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        o[a] = static_cast<float>(r[a]);
        o[3 + a] = static_cast<float>(r[a] - static_cast<double>(o[a]));
    }
    o[6] = 0.f;
    o[7] = 0.f;
    float4 *dst = reinterpret_cast<float4 *>(rr + 8 * static_cast<size_t>(i));
    dst[0] = make_float4(o[0], o[1], o[2], o[3]);
    dst[1] = make_float4(o[4], o[5], o[6], o[7]);
}

__device__ __forceinline__ void load_rr(const float *__restrict__ rr, int j, df &x, df &y, df &z)
{
    float a0, a1, a2, a3, a4, a5, a6, a7;
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(a0), "=f"(a1), "=f"(a2), "=f"(a3), "=f"(a4), "=f"(a5), "=f"(a6), "=f"(a7)
        : "l"(rr + 8 * static_cast<size_t>(j)));
    x = df{a0, a3};
    y = df{a1, a4};
    z = df{a2, a5};
}

__device__ __forceinline__ df df_neg(df a) { return df{-a.h, -a.l}; }

__device__ __forceinline__ df df_scale2(df a, float p2) { return df{a.h * p2, a.l * p2}; }  // exact

template <bool HALF, bool CUBIC>
__global__ void __launch_bounds__(kDvThreads)
vjp_dfloat_kernel(const double *__restrict__ q4, const DfRec *__restrict__ rec,
                  const double *__restrict__ R4, const float *__restrict__ rr, int n,
                  const int *__restrict__ row_ptr, const int *__restrict__ col, DfVjp V,
                  double *__restrict__ gq4, double *__restrict__ partial)
{
    constexpr int TPI = kDvTpi;
    const DfParams &D = V.D;
    const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / TPI;
    const int sub = threadIdx.x & (TPI - 1);
    const unsigned gm = group_mask<TPI>();
    float es = 0.f, ec = 0.f, ss = 0.f, sc = 0.f;  // sums of g^ (delta.w), (dg/dsig)^ (delta.w)
    double e64 = 0.0, s64 = 0.0;                   // FP64 fallback pairs
    if (gid < n) {
        const int i = gid;
        const DfRec ri = load_rec(rec, i);
        const float lix = lo_field(ri.lo, 0, D), liy = lo_field(ri.lo, 1, D), liz = lo_field(ri.lo, 2, D);
        df Rxi, Ryi, Rzi;
        load_rr(rr, i, Rxi, Ryi, Rzi);
        float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f, sz = 0.f, cz = 0.f;
        double fx64 = 0.0, fy64 = 0.0, fz64 = 0.0;
        const int kb = row_ptr[i], ke = row_ptr[i + 1];
        for (int k0 = kb; k0 < ke; k0 += TPI) {
            const int k = k0 + sub;
            const bool valid = k < ke;
            const int j = valid ? col[k] : i;
            const DfRec rj = load_rec(rec, j);
            df dx = chunk_disp(rj.hx, ri.hx, rj.mx, ri.mx, lo_field(rj.lo, 0, D), lix, D);
            df dy = chunk_disp(rj.hy, ri.hy, rj.my, ri.my, lo_field(rj.lo, 1, D), liy, D);
            df dz = chunk_disp(rj.hz, ri.hz, rj.mz, ri.mz, lo_field(rj.lo, 2, D), liz, D);
            if (!CUBIC) {
                dx = df_mul(dx, df{D.cx_h[0], D.cx_l[0]});
                dy = df_mul(dy, df{D.cx_h[1], D.cx_l[1]});
                dz = df_mul(dz, df{D.cx_h[2], D.cx_l[2]});
            }
            df R = df_norm2(dx, dy, dz);
            bool in = valid && (R.h < D.T_h || (R.h == D.T_h && R.l < D.T_l));
            const bool exact = valid && (fabsf(R.h - D.T_h) <= D.band || R.h < V.r2_min);
            if (__any_sync(gm, exact)) {
                if (exact) {
                    double c0, c1, c2, ge, gs;
                    if (fp64_vjp_pair(q4, R4, i, j, V, c0, c1, c2, ge, gs)) {
                        fx64 -= c0;
                        fy64 -= c1;
                        fz64 -= c2;
                        e64 += ge;
                        s64 += gs;
                        if (HALF) {
                            double *g = gq4 + 4 * static_cast<int64_t>(j);
                            atomicAdd(g + 0, c0);
                            atomicAdd(g + 1, c1);
                            atomicAdd(g + 2, c2);
                        }
                    }
                    in = false;
                }
            }
            if (!in) R = df{1.0f, 0.0f};
            const df u = df_rcp(R);
            const df u2 = df_sq(u);
            const df u3 = df_mul(u2, u);
            const df u4 = df_sq(u2);
            const df u5 = df_mul(u4, u);
            const df bu3 = df_mul(df{V.b_h, V.b_l}, u3);
            const df gh = df_mul(u4, df_add(bu3, df{-1.0f, 0.0f}));
            const df gph = df_mul(u5, df_add(df_neg(df_mul(df{V.c_h, V.c_l}, u3)), df{1.0f, 0.0f}));
            const df gsh = df_mul(u4, df_add(df_scale2(bu3, 2.0f), df{-1.0f, 0.0f}));
            if (in) {
                df Rxj, Ryj, Rzj;
                load_rr(rr, j, Rxj, Ryj, Rzj);
                const df wx = df_add(Rxj, df_neg(Rxi)), wy = df_add(Ryj, df_neg(Ryi)),
                         wz = df_add(Rzj, df_neg(Rzi));
                const df dw = df_add(df_add(df_mul(dx, wx), df_mul(dy, wy)), df_mul(dz, wz));
                const df t = df_scale2(df_mul(gph, dw), 8.0f);
                const df c0 = df_add(df_mul(gh, wx), df_mul(t, dx));
                const df c1 = df_add(df_mul(gh, wy), df_mul(t, dy));
                const df c2 = df_add(df_mul(gh, wz), df_mul(t, dz));
                df_acc(sx, cx, c0);
                df_acc(sy, cy, c1);
                df_acc(sz, cz, c2);
                df_acc(es, ec, df_mul(gh, dw));
                df_acc(ss, sc, df_mul(gsh, dw));
                if (HALF) {
                    double *g = gq4 + 4 * static_cast<int64_t>(j);
                    atomicAdd(g + 0, V.Kc * df_to_f64(c0.h, c0.l, 0));
                    atomicAdd(g + 1, V.Kc * df_to_f64(c1.h, c1.l, 0));
                    atomicAdd(g + 2, V.Kc * df_to_f64(c2.h, c2.l, 0));
                }
            }
        }
        group_df_acc<TPI>(sx, cx);
        group_df_acc<TPI>(sy, cy);
        group_df_acc<TPI>(sz, cz);
        fx64 = group_sum<TPI>(fx64);
        fy64 = group_sum<TPI>(fy64);
        fz64 = group_sum<TPI>(fz64);
        if (sub == 0) {
            const double ax = fx64 - V.Kc * df_to_f64(sx, cx, 0);
            const double ay = fy64 - V.Kc * df_to_f64(sy, cy, 0);
            const double az = fz64 - V.Kc * df_to_f64(sz, cz, 0);
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
    // block sums of the two scalar gradients (fixed order)
    __shared__ double red[2][kDvThreads / 32];
    double a = e64 + V.Ke * df_to_f64(es, ec, 0);
    double b = s64 + V.Ks * df_to_f64(ss, sc, 0);
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
        for (int w = 0; w < kDvThreads / 32; ++w) {
            sa += red[0][w];
            sb += red[1][w];
        }
        partial[2 * blockIdx.x + 0] = sa;
        partial[2 * blockIdx.x + 1] = sb;
    }
}

void split_f(double v, float &h, float &l)
{
    h = static_cast<float>(v);
    l = static_cast<float>(v - static_cast<double>(h));
}

}  // namespace

size_t vjp_dfloat_extra_bytes(int64_t n)
{
    const size_t nn = size_t(n > 0 ? n : 1);
    return nn * sizeof(DfRec) + 256 + nn * 8 * sizeof(float) + 256;
}

// Launches the DFLOAT adjoint (two pre-passes and the kernel) writing gq4
// and partial[2 * blocks] in lj_vjp.cu's layout (blocks of 256 threads, 8
// lanes per row).  extra: vjp_dfloat_extra_bytes(n) of workspace.
int vjp_dfloat(const double *q4, const double *R4, int n, const int *row_ptr, const int *col,
               int half, double rc, const double box[3], double eps, double sigma, double *gq4,
               double *partial, int blocks, void *extra, cudaStream_t st)
{
    DfVjp V{};
    V.D = make_dfloat_params(box, 1.0, rc, eps, sigma);
    int s = 0;
    const double L0 = box[0];
    // lambda exactly as make_dfloat_params chose it: L_0 2^-s with the period 2^s
    s = static_cast<int>(std::lround(std::log2(static_cast<double>(V.D.period))));
    const double lambda = std::ldexp(L0, -s);
    const double sl = sigma / lambda, sl2 = sl * sl, sl6 = sl2 * sl2 * sl2;
    const double beta = 2.0 * sl6;
    split_f(beta, V.b_h, V.b_l);
    split_f(1.75 * beta, V.c_h, V.c_l);
    // u^5 <= 2^75 and 7/4 beta u^8 <= 2^100 keep every hat quantity normal
    double umax = std::pow(std::ldexp(1.0, 100) / (1.75 * beta), 1.0 / 8.0);
    if (umax > std::ldexp(1.0, 15)) umax = std::ldexp(1.0, 15);
    V.r2_min = static_cast<float>(1.0 / umax);
    const double s2 = sigma * sigma, s5 = s2 * s2 * sigma, s6 = s5 * sigma, s11 = s5 * s6, s12 = s6 * s6;
    V.Kc = 24.0 * eps * s6 / std::pow(lambda, 8);
    V.Ke = V.Kc * lambda;
    V.Ks = 144.0 * eps * s5 / std::pow(lambda, 8) * lambda;
    V.G1 = 48.0 * eps * s12;
    V.G2 = 24.0 * eps * s6;
    V.H1 = 336.0 * eps * s12;
    V.H2 = 96.0 * eps * s6;
    V.S1 = 576.0 * eps * s11;
    V.S2 = 144.0 * eps * s5;
    Carver c(extra);
    DfRec *rec = c.take<DfRec>(size_t(n));
    float *rr = c.take<float>(8 * size_t(n));
    dfloat_prepass_kernel<<<unsigned((n + 255) / 256), 256, 0, st>>>(q4, n, V.D, rec);
    LJ_TRY_LAUNCH("dfloat_prepass_kernel");
    dfloat_r_prepass_kernel<<<unsigned((n + 255) / 256), 256, 0, st>>>(R4, n, rr);
    LJ_TRY_LAUNCH("dfloat_r_prepass_kernel");
    const bool cubic = box[1] == box[0] && box[2] == box[0];
    if (half) {
        if (cubic)
            vjp_dfloat_kernel<true, true><<<blocks, kDvThreads, 0, st>>>(q4, rec, R4, rr, n, row_ptr, col, V, gq4, partial);
        else
            vjp_dfloat_kernel<true, false><<<blocks, kDvThreads, 0, st>>>(q4, rec, R4, rr, n, row_ptr, col, V, gq4, partial);
    } else {
        if (cubic)
            vjp_dfloat_kernel<false, true><<<blocks, kDvThreads, 0, st>>>(q4, rec, R4, rr, n, row_ptr, col, V, gq4, partial);
        else
            vjp_dfloat_kernel<false, false><<<blocks, kDvThreads, 0, st>>>(q4, rec, R4, rr, n, row_ptr, col, V, gq4, partial);
    }
    LJ_TRY_LAUNCH("vjp_dfloat_kernel");
    return LJ_OK;
}

}  // namespace lj

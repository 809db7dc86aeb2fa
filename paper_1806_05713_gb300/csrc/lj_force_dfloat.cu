// lj_force_dfloat.cu -- the DFLOAT form of the LJ momentum update
// (Algorithm 1 for each entry of the sorted list, Algorithm 3), with the
// pair arithmetic in double-float on the FP32 pipe (lj_dfloat.cuh).
//
// A group of TPI lanes walks row i as in the FP64 and MIXED kernels.  Each
// lane keeps compensated FP32 sums of g delta for p_i; the group combines
// them with error-free shuffles and adds -2^K_e (s + c) to the FP64 p_i
// once.  A half list also sends 2^K_e g delta to p_j through FP64 atomics
// in L2.  Lanes whose pair needs the FP64 definition (r^2 within the band
// around r_c^2, or a pair closer than the double-float range) evaluate it
// in FP64 under a warp-uniform branch and add the result with FP64 atomics.
#include <algorithm>
#include <cmath>

#include "lj_dfloat.cuh"

namespace lj {
namespace {

// The FP64 definition for one entry: the oracle's displacement and cutoff
// decision, the FP64 form's impulse; added to p_i (and p_j for a half list).
template <bool HALF>
__device__ __noinline__ void dfloat_fp64_pair(const double *__restrict__ q4, double *__restrict__ p4,
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
// 128-thread blocks: at ~95 registers a thread (U = 2) five blocks fit an SM.
constexpr int kDfThreads = 128;

template <int TPI, bool HALF, bool CUBIC, int U>
__global__ void __launch_bounds__(kDfThreads)
force_dfloat_kernel(const double *__restrict__ q4, const DfRec *__restrict__ rec,
                    double *__restrict__ p4, int n, const int *__restrict__ row_ptr,
                    const int *__restrict__ col, DfParams P, const int *__restrict__ order)
{
    const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / TPI;
    if (gid >= n) return;
    const int i = order ? order[gid] : gid;
    if (U == 2)
        dfloat_row2<TPI, HALF, CUBIC>(q4, rec, p4, row_ptr, col, i, P, group_mask<TPI>());
    else
        dfloat_row<TPI, HALF, CUBIC>(q4, rec, p4, row_ptr, col, i, P, group_mask<TPI>());
}

template <int TPI, bool CUBIC, int U>
int launch_dfloat_t(const double *q4, const DfRec *rec, double *p4, int n, const int *rp,
                    const int *col, int half, const DfParams &P, const int *order, cudaStream_t st)
{
    const int64_t threads = int64_t(n) * TPI;
    const unsigned grid = unsigned((threads + kDfThreads - 1) / kDfThreads);
    if (half)
        force_dfloat_kernel<TPI, true, CUBIC, U><<<grid, kDfThreads, 0, st>>>(q4, rec, p4, n, rp, col, P, order);
    else
        force_dfloat_kernel<TPI, false, CUBIC, U><<<grid, kDfThreads, 0, st>>>(q4, rec, p4, n, rp, col, P, order);
    LJ_TRY_LAUNCH("force_dfloat_kernel");
    return LJ_OK;
}

}  // namespace

size_t dfloat_record_bytes(int64_t n)
{
    return sizeof(DfRec) * size_t(n > 0 ? n : 1);
}

// precision LJ_DFLOAT; tpi = 4, 8 or 16, optionally | LJ_SCHED_SWP2 (two
// entries per lane, packed); 0 = LJ_SCHED_SWP2 | 8.  rec:
// dfloat_record_bytes(n) of workspace.
int force_dfloat(const double *q4, double *p4, int n, const int *row_ptr, const int *col, int half,
                 const double box[3], double dt, double rc, double eps, double sigma, int tpi,
                 const int *order, void *rec_ws, cudaStream_t st)
{
    const DfParams P = make_dfloat_params(box, dt, rc, eps, sigma);
    if (P.k_exp < -700 || P.k_exp > 700) return LJ_ERR_ARG;
    DfRec *rec = static_cast<DfRec *>(rec_ws);
    dfloat_prepass_kernel<<<unsigned((n + 255) / 256), 256, 0, st>>>(q4, n, P, rec);
    LJ_TRY_LAUNCH("dfloat_prepass_kernel");
    const bool cubic = box[1] == box[0] && box[2] == box[0];
#define LJ_DF(T, U)                                                                        \
    return cubic ? launch_dfloat_t<T, true, U>(q4, rec, p4, n, row_ptr, col, half, P, order, st) \
                 : launch_dfloat_t<T, false, U>(q4, rec, p4, n, row_ptr, col, half, P, order, st)
    switch (tpi) {
        case 4: LJ_DF(4, 1);
        case 8: LJ_DF(8, 1);
        case 16: LJ_DF(16, 1);
        case LJ_SCHED_SWP2 | 4: LJ_DF(4, 2);
        case 0:
        case LJ_SCHED_SWP2 | 8: LJ_DF(8, 2);
        case LJ_SCHED_SWP2 | 16: LJ_DF(16, 2);
        default: return LJ_ERR_ARG;
    }
#undef LJ_DF
}

}  // namespace lj

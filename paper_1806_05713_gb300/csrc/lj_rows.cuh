// lj_rows.cuh -- one CSR row of the LJ momentum update (Algorithm 1 for
// each entry of SortedList[i], Algorithm 3), in the FP64 and MIXED forms,
// walked by a group of TPI lanes of one warp.  Shared by the single-system
// kernels (lj_force.cu) and the batched persistent kernel (lj_batched.cu).
#pragma once

#include "lj_forms.cuh"

namespace lj {
namespace {

// Memory layout of positions and momenta for the FP64 row walk: element
// (i, a) of q or p is at base[i * rs + a * cs].  LAY 0: AoS4 (rs = 4,
// cs = 1, one 256-bit load per atom); LAY 1: any AoS with rs a multiple of 4
// and cs = 1 (e.g. the paper's AoS8, q and p of an atom in one 64-byte
// record); LAY 2: anything else, e.g. SoA (rs = 1, cs = n), three scalar
// loads per atom.
struct Layout {
    long long rs, cs;
};

template <int LAY>
__device__ __forceinline__ void load_pos(const double *__restrict__ q, int i, const Layout &L,
                                         double &x, double &y, double &z)
{
    if (LAY == 0) {
        load_q4_256(q, i, x, y, z);
    } else if (LAY == 1) {
        double w;
        asm("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];"
            : "=d"(x), "=d"(y), "=d"(z), "=d"(w)
            : "l"(q + static_cast<long long>(i) * L.rs));
    } else {
        const double *b = q + static_cast<long long>(i) * L.rs;
        x = __ldg(b);
        y = __ldg(b + L.cs);
        z = __ldg(b + 2 * L.cs);
    }
}

template <int LAY>
__device__ __forceinline__ double *mom_at(double *__restrict__ p, int i, int a, const Layout &L)
{
    if (LAY == 0) return p + 4 * static_cast<long long>(i) + a;
    return p + static_cast<long long>(i) * L.rs + static_cast<long long>(a) * L.cs;
}

// One row i of the FP64 form, walked by the TPI lanes of the calling group
// (gm = their mask).  U independent entries per lane and iteration (U = 2 is
// the paper's software pipelining, section "Software Pipelining": the loads
// and distance work of one entry overlap the force arithmetic of the other,
// so the long dependent FP64 chains of two pairs are in flight together).
// Pointers are the system's own arrays (local indices).
// EN: also accumulate the pair energy 4 eps [(sigma/r)^12 - (sigma/r)^6] of
// every in-cutoff entry into *ev, its pair virial r F(r) into *wv, and
// count the entries into *ecount (the caller applies the shift and, for a
// full list, the factor 1/2).
template <int TPI, bool HALF, int U, bool IMG = false, int LAY = 0, bool EN = false>
__device__ __forceinline__ void fp64_row(const double *__restrict__ q4, double *__restrict__ p4,
                                         const int *__restrict__ row_ptr,
                                         const int *__restrict__ col, int i, const Fp64Params &P,
                                         unsigned gm, const Layout &Lay = Layout{4, 1},
                                         double *ev = nullptr, int *ecount = nullptr,
                                         double *wv = nullptr)
{
    const int sub = threadIdx.x & (TPI - 1);
    double xi, yi, zi;
    load_pos<LAY>(q4, i, Lay, xi, yi, zi);
    // IMG: the two periodic images of q_i per axis and the high words of
    // q_i +- L/2, so that each entry picks the minimum image of q_i with
    // integer compares and needs one FP64 subtraction, never a wrap add.
    // (An entry whose high word ties the threshold lies within 2^-20 of half
    // a box from i, beyond r_c in either image.)
    double im[3][2];
    int th[3][2];
    if (IMG) {
        const double c[3] = {xi, yi, zi};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            im[a][0] = c[a] - P.L[a];
            im[a][1] = c[a] + P.L[a];
            double hl;
            memcpy(&hl, &P.half_bits[a], sizeof(double));
            th[a][0] = __double2hiint(c[a] - hl);
            th[a][1] = __double2hiint(c[a] + hl);
        }
    }
    double ax = 0.0, ay = 0.0, az = 0.0;
    const int kb = row_ptr[i], ke = row_ptr[i + 1];
    for (int base = kb; base < ke; base += TPI * U) {
        int j[U];
        bool valid[U], in[U], near[U];
        double dx[U], dy[U], dz[U], r2[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int k = base + sub + u * TPI;
            valid[u] = k < ke;
            j[u] = valid[u] ? col[k] : i;
        }
        double xj[U], yj[U], zj[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            load_pos<LAY>(q4, j[u], Lay, xj[u], yj[u], zj[u]);
            if (IMG) {
                const double cj[3] = {xj[u], yj[u], zj[u]};
                const double ci[3] = {xi, yi, zi};
                double d[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const int hj = __double2hiint(cj[a]);
                    const double img = hj > th[a][1] ? im[a][1] : (hj < th[a][0] ? im[a][0] : ci[a]);
                    d[a] = cj[a] - img;
                }
                dx[u] = d[0];
                dy[u] = d[1];
                dz[u] = d[2];
            } else {
                dx[u] = xj[u] - xi;
                dy[u] = yj[u] - yi;
                dz[u] = zj[u] - zi;
            }
        }
        bool anynear = false, anyin = false;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (!IMG) min_image3(dx[u], dy[u], dz[u], P.L, P.half_bits, gm);
            r2[u] = fma(dz[u], dz[u], fma(dy[u], dy[u], dx[u] * dx[u]));
            const long long rb = __double_as_longlong(r2[u]);
            in[u] = valid[u] && rb < P.rc2_bits;
            near[u] = valid[u] && static_cast<unsigned long long>(rb - P.rc2_bits + 64) < 128ull;
            anynear |= near[u];
        }
        if (__any_sync(gm, anynear)) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (near[u]) {
                    if (IMG) {
                        // the definition's operations: d = q_j - q_i, then the wrap
                        const double ex = min_image(xj[u] - xi, P.L[0], P.half_bits[0]);
                        const double ey = min_image(yj[u] - yi, P.L[1], P.half_bits[1]);
                        const double ez = min_image(zj[u] - zi, P.L[2], P.half_bits[2]);
                        in[u] = exact_in_cutoff(ex, ey, ez, P.rc2);
                    } else {
                        // dx, dy, dz were formed with exactly those operations
                        in[u] = exact_in_cutoff(dx[u], dy[u], dz[u], P.rc2);
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (!valid[u]) r2[u] = 1.0;
            anyin |= in[u];
        }
        if (__any_sync(gm, anyin)) {
            double fn[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const double w = rcp_fp64(r2[u], gm);
                const double w2 = w * w;
                const double w4 = w2 * w2;
                const double w3 = w2 * w;
                fn[u] = w4 * fma(P.B, w3, -P.A);  // -df: p_i -= fn d, p_j += fn d
                if (EN && in[u]) {
                    *ev += w3 * fma(P.C12, w3, -P.C6);  // 4 eps [(s/r)^12 - (s/r)^6]
                    *wv += w3 * fma(P.W12, w3, -P.W6);  // 24 eps [2 (s/r)^12 - (s/r)^6]
                    ++*ecount;
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (in[u]) {
                    if (HALF) {
                        const double fx = fn[u] * dx[u], fy = fn[u] * dy[u], fz = fn[u] * dz[u];
                        atomicAdd(mom_at<LAY>(p4, j[u], 0, Lay), fx);
                        atomicAdd(mom_at<LAY>(p4, j[u], 1, Lay), fy);
                        atomicAdd(mom_at<LAY>(p4, j[u], 2, Lay), fz);
                        ax -= fx;
                        ay -= fy;
                        az -= fz;
                    } else {
                        ax = fma(-fn[u], dx[u], ax);
                        ay = fma(-fn[u], dy[u], ay);
                        az = fma(-fn[u], dz[u], az);
                    }
                }
            }
        }
    }
    if (HALF) {
        // p_i already receives other rows' atomics: each lane adds its own
        // partial sum in L2 (no FP64 shuffle reduction on the FP64 pipe).
        atomicAdd(mom_at<LAY>(p4, i, 0, Lay), ax);
        atomicAdd(mom_at<LAY>(p4, i, 1, Lay), ay);
        atomicAdd(mom_at<LAY>(p4, i, 2, Lay), az);
    } else {
        // Full list: a fixed-order group reduction keeps p_i deterministic.
        if (TPI > 1) {
            ax = group_sum<TPI>(ax);
            ay = group_sum<TPI>(ay);
            az = group_sum<TPI>(az);
        }
        if (sub == 0) {
            atomicAdd(mom_at<LAY>(p4, i, 0, Lay), ax);
            atomicAdd(mom_at<LAY>(p4, i, 1, Lay), ay);
            atomicAdd(mom_at<LAY>(p4, i, 2, Lay), az);
        }
    }
}

// One row i of the MIXED form with its gathers software-pipelined (the
// paper's section "Software Pipelining", applied to the loads): the lane's
// entries are taken U at a time (k, k + TPI, ..., k + (U-1) TPI); the
// fixed-point records of the next U entries and the column indices of the U
// after those are requested before the arithmetic of the current ones, so
// the two dependent L2 gathers of an entry (col[k], then rel[col[k]]) are in
// flight while the lane computes.  Each lane adds its entries in increasing
// k whatever U is, so the compensated sums do not depend on U.  rel holds
// the fixed-point positions of the system (see lj_force.cu).
template <int TPI, bool HALF, int U>
__device__ __forceinline__ void mixed_row_pf(const double *__restrict__ q4,
                                             const uint4 *__restrict__ rel, double *__restrict__ p4,
                                             const int *__restrict__ row_ptr,
                                             const int *__restrict__ col, int i,
                                             const MixedParams &P)
{
    const int sub = threadIdx.x & (TPI - 1);
    const uint4 pi = __ldg(rel + i);
    float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
    const int kb = row_ptr[i], ke = row_ptr[i + 1];
    // entries past the row end gather atom i itself (r^2 = 0, never used)
    auto col_at = [&](int k) { return k < ke ? __ldg(col + k) : i; };
    int j[U], jn[U];
    uint4 r[U];
#pragma unroll
    for (int u = 0; u < U; ++u) j[u] = col_at(kb + sub + u * TPI);
#pragma unroll
    for (int u = 0; u < U; ++u) r[u] = __ldg(rel + j[u]);
#pragma unroll
    for (int u = 0; u < U; ++u) jn[u] = col_at(kb + sub + (U + u) * TPI);
    for (int k0 = kb; k0 < ke; k0 += U * TPI) {
        uint4 rn[U];
        int jnn[U];
#pragma unroll
        for (int u = 0; u < U; ++u) rn[u] = __ldg(rel + jn[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) jnn[u] = col_at(k0 + sub + (2 * U + u) * TPI);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool valid = k0 + sub + u * TPI < ke;
            const float dx = fixed_disp(r[u].x, pi.x, P.scale[0]);
            const float dy = fixed_disp(r[u].y, pi.y, P.scale[1]);
            const float dz = fixed_disp(r[u].z, pi.z, P.scale[2]);
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            bool in = valid && r2 < P.rc2f;
            if (valid && fabsf(r2 - P.rc2f) <= P.band) {
                double xi, yi, zi, xj, yj, zj;
                load_xyz(q4, i, xi, yi, zi);
                load_xyz(q4, j[u], xj, yj, zj);
                const double ex = min_image(__dsub_rn(xj, xi), P.L[0], P.half_bits[0]);
                const double ey = min_image(__dsub_rn(yj, yi), P.L[1], P.half_bits[1]);
                const double ez = min_image(__dsub_rn(zj, zi), P.L[2], P.half_bits[2]);
                in = exact_in_cutoff(ex, ey, ez, P.rc2);
            }
            if (in) {
                const float w = rcp_fp32(r2);
                const float w2 = w * w;
                const float w4 = w2 * w2;
                const float w3 = w2 * w;
                const float f = w4 * fmaf(-P.Bf, w3, P.Af);
                const float fx = f * dx, fy = f * dy, fz = f * dz;
                kahan_add(sx, cx, fx);
                kahan_add(sy, cy, fy);
                kahan_add(sz, cz, fz);
                if (HALF) {
                    double *pj = p4 + 4 * static_cast<int64_t>(j[u]);
                    atomicAdd(pj + 0, f32_to_f64(-fx));
                    atomicAdd(pj + 1, f32_to_f64(-fy));
                    atomicAdd(pj + 2, f32_to_f64(-fz));
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            r[u] = rn[u];
            j[u] = jn[u];
            jn[u] = jnn[u];
        }
    }
    if (TPI > 1) {
        group_kahan<TPI>(sx, cx);
        group_kahan<TPI>(sy, cy);
        group_kahan<TPI>(sz, cz);
    }
    if (sub == 0) {
        double *pp = p4 + 4 * static_cast<int64_t>(i);
        atomicAdd(pp + 0, f32_to_f64(sx));
        atomicAdd(pp + 1, f32_to_f64(sy));
        atomicAdd(pp + 2, f32_to_f64(sz));
        atomicAdd(pp + 0, f32_to_f64(-cx));
        atomicAdd(pp + 1, f32_to_f64(-cy));
        atomicAdd(pp + 2, f32_to_f64(-cz));
    }
}

}  // namespace
}  // namespace lj

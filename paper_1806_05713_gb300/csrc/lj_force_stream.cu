// lj_force_stream.cu -- FP64 "pair-stream" schedule of the LJ momentum update.
//
// Same arithmetic as the FP64 form in lj_force.cu (Algorithm 1 inside the
// sorted-list loop of Algorithm 3), scheduled for a GPU whose FP64 rate is
// the bottleneck.  In a row-per-group schedule every lane of a warp issues
// the full pair arithmetic in lock step, including lanes whose pair lies in
// the bookkeeping margin (r_c <= r < r_s, about a quarter of the list) and
// lanes past the end of a short row.  Here:
//
//   phase A  the warp walks the entries of R consecutive rows as one flat
//            stream, 32 entries at a time (the lane-counter idea of the
//            paper's remainder-loop elimination, applied across rows);
//            each lane forms d = q_j - q_i (q_i of the R rows is cached in
//            shared memory), r^2 and the cutoff test, and in-cutoff pairs
//            are appended to a per-warp ring queue in shared memory
//            (ballot + popc);
//   phase B  whenever 32 pairs are queued, each lane takes one and computes
//            u = 1/r^2, df and df*d (the expensive FP64 part, now with every
//            lane busy), sends -df*d to p_j (half list, FP64 atomics), and
//            a segmented warp reduction by row adds the p_i parts into
//            per-row accumulators in shared memory;
//   end      each row's accumulated impulse is added to p_i once.
//
// This is the software-pipelining idea of the paper (separate the loads
// and distance work from the force work so that each runs at full width)
// mapped onto a warp and a shared-memory queue.
#include <cmath>
#include <cstring>

#include "lj_internal.cuh"

namespace lj {
namespace {

constexpr int kQ = 64;  // queue slots per warp (power of two, >= 63 needed)

struct StreamParams {
    double L[3];
    long long half_bits[3];
    long long rc2_bits;
    double rc2;
    double A, B;  // df = u^4 (A - B u^3)
};

template <int R>
struct WarpSmem {
    double qx[R], qy[R], qz[R];
    double ax[R], ay[R], az[R];
    int rp[R + 1];
    double dx[kQ], dy[kQ], dz[kQ], r2[kQ];
    int j[kQ];
    int rl[kQ];
};

__device__ __forceinline__ void gather_q(const double *__restrict__ q4, int j, double &x,
                                         double &y, double &z)
{
    double w;
    asm("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];"
        : "=d"(x), "=d"(y), "=d"(z), "=d"(w)
        : "l"(q4 + 4 * static_cast<int64_t>(j)));
}

// Force on the queued pairs head .. head+cnt-1 (one per lane).
template <int R, bool HALF>
__device__ __forceinline__ void process_batch(WarpSmem<R> &S, int head, int cnt,
                                              double *__restrict__ p4, const StreamParams &P)
{
    const int lane = threadIdx.x & 31;
    double fx = 0.0, fy = 0.0, fz = 0.0;
    int rl = -1 - lane;  // distinct sentinel for idle lanes
    if (lane < cnt) {
        const int s = (head + lane) & (kQ - 1);
        rl = S.rl[s];
        const double r2 = S.r2[s];
        const double u = rcp_fp64(r2);
        const double u2 = u * u;
        const double u4 = u2 * u2;
        const double u3 = u2 * u;
        const double f = u4 * fma(-P.B, u3, P.A);
        fx = f * S.dx[s];
        fy = f * S.dy[s];
        fz = f * S.dz[s];
        if (HALF) {
            double *pj = p4 + 4 * static_cast<int64_t>(S.j[s]);
            atomicAdd(pj + 0, -fx);
            atomicAdd(pj + 1, -fy);
            atomicAdd(pj + 2, -fz);
        }
    }
    // Segmented inclusive scan over lanes; rows are non-decreasing along the
    // queue, so "same row" marks the segment.
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int rlo = __shfl_up_sync(0xffffffffu, rl, o);
        const double vx = __shfl_up_sync(0xffffffffu, fx, o);
        const double vy = __shfl_up_sync(0xffffffffu, fy, o);
        const double vz = __shfl_up_sync(0xffffffffu, fz, o);
        if (lane >= o && rlo == rl) {
            fx += vx;
            fy += vy;
            fz += vz;
        }
    }
    const int rln = __shfl_down_sync(0xffffffffu, rl, 1);
    if (lane < cnt && (lane == cnt - 1 || rln != rl)) {
        S.ax[rl] += fx;
        S.ay[rl] += fy;
        S.az[rl] += fz;
    }
    __syncwarp();
}

template <int R, int W, bool HALF>
__global__ void __launch_bounds__(W * 32)
force_stream_kernel(const double *__restrict__ q4, double *__restrict__ p4, int n,
                    const int *__restrict__ row_ptr, const int *__restrict__ col, StreamParams P)
{
    __shared__ WarpSmem<R> smem[W];
    const int wib = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    WarpSmem<R> &S = smem[wib];
    const int64_t r0 = (int64_t(blockIdx.x) * W + wib) * R;
    if (r0 >= n) return;
    const int nr = static_cast<int>(n - r0 < R ? n - r0 : R);
    for (int t = lane; t <= nr; t += 32) S.rp[t] = row_ptr[r0 + t];
    for (int t = lane; t < nr; t += 32) {
        double x, y, z;
        gather_q(q4, static_cast<int>(r0 + t), x, y, z);
        S.qx[t] = x;
        S.qy[t] = y;
        S.qz[t] = z;
        S.ax[t] = 0.0;
        S.ay[t] = 0.0;
        S.az[t] = 0.0;
    }
    __syncwarp();
    const int e0 = S.rp[0], e1 = S.rp[nr];
    int row = 0;
    int head = 0, count = 0;
    for (int base = e0; base < e1; base += 32) {
        const int k = base + lane;
        bool in = false;
        double dx = 0.0, dy = 0.0, dz = 0.0, r2 = 0.0;
        int j = 0;
        if (k < e1) {
            while (S.rp[row + 1] <= k) ++row;
            j = col[k];
            double xj, yj, zj;
            gather_q(q4, j, xj, yj, zj);
            dx = min_image(xj - S.qx[row], P.L[0], P.half_bits[0]);
            dy = min_image(yj - S.qy[row], P.L[1], P.half_bits[1]);
            dz = min_image(zj - S.qz[row], P.L[2], P.half_bits[2]);
            r2 = fma(dz, dz, fma(dy, dy, dx * dx));
            const long long rb = __double_as_longlong(r2);
            in = rb < P.rc2_bits;
            if (static_cast<unsigned long long>(rb - P.rc2_bits + 64) < 128ull) {
                const double e2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                                            __dmul_rn(dz, dz));
                in = e2 < P.rc2;
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, in);
        if (in) {
            const int s = (head + count + __popc(m & lanemask_lt())) & (kQ - 1);
            S.dx[s] = dx;
            S.dy[s] = dy;
            S.dz[s] = dz;
            S.r2[s] = r2;
            S.j[s] = j;
            S.rl[s] = row;
        }
        count += __popc(m);
        __syncwarp();
        if (count >= 32) {
            process_batch<R, HALF>(S, head, 32, p4, P);
            head = (head + 32) & (kQ - 1);
            count -= 32;
        }
    }
    if (count > 0) process_batch<R, HALF>(S, head, count, p4, P);
    for (int t = lane; t < nr; t += 32) {
        double *pi = p4 + 4 * (r0 + t);
        if (HALF) {
            atomicAdd(pi + 0, S.ax[t]);
            atomicAdd(pi + 1, S.ay[t]);
            atomicAdd(pi + 2, S.az[t]);
        } else {
            pi[0] += S.ax[t];
            pi[1] += S.ay[t];
            pi[2] += S.az[t];
        }
    }
}

template <int R, int W>
int launch_stream(const double *q4, double *p4, int n, const int *rp, const int *col, int half,
                  const StreamParams &P, cudaStream_t st)
{
    const int64_t warps = (int64_t(n) + R - 1) / R;
    const unsigned grid = unsigned((warps + W - 1) / W);
    if (half)
        force_stream_kernel<R, W, true><<<grid, W * 32, 0, st>>>(q4, p4, n, rp, col, P);
    else
        force_stream_kernel<R, W, false><<<grid, W * 32, 0, st>>>(q4, p4, n, rp, col, P);
    LJ_TRY_LAUNCH("force_stream_kernel");
    return LJ_OK;
}

}  // namespace

int force_stream_fp64(const double *q4, double *p4, int n, const int *row_ptr, const int *col,
                      int64_t nnz, int half, const double box[3], double dt, double rc, double eps,
                      double sigma, cudaStream_t st)
{
    (void)nnz;
    StreamParams P{};
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
    return launch_stream<16, 2>(q4, p4, n, row_ptr, col, half, P, st);
}

}  // namespace lj

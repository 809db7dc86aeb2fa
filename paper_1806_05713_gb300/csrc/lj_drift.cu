// lj_drift.cu -- the position update around the force call (velocity Verlet
// with unit mass) and the displacement bound of the bookkeeping method.
//
// Section "Verlet List and Bookkeeping Method" of Watanabe & Nakagawa: a list
// built with search length r_s = r_c + margin stays valid while no pair has
// closed the margin, which is guaranteed while twice the largest distance
// any atom has moved since the build is below the margin; monitoring the
// fastest atom (the criterion the paper cites) bounds that distance by the
// sum over steps of the largest per-step displacement.  lj_drift moves the
// atoms, q += dt p, wrapped back into [0, L), and reports that largest
// per-step displacement.  lj_md_steps queues whole leapfrog steps (drift,
// the bound and its test, kick) with the test taken on the device, the
// bound either that sum or the largest displacement since the build
// measured against the positions the list was built from.
#include <cmath>

#include "lj_internal.cuh"

namespace lj {
namespace {

constexpr int kDriftThreads = 256;

// The block's maximum of v >= 0 into *dst (the ordered bit pattern of a
// non-negative double).
__device__ __forceinline__ void block_max_into(double v, unsigned long long *dst)
{
    __shared__ double red[kDriftThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();  // red is reused by a second call
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < kDriftThreads / 32; ++w) m = fmax(m, red[w]);
        atomicMax(dst, static_cast<unsigned long long>(__double_as_longlong(m)));
    }
}

// q += dt p with round-to-nearest double operations (no fused multiply-add),
// then one periodic wrap per axis; *max_d2 = max over atoms of |dt p|^2.
// With qb (the positions of the last list build): *max_dev2 = max over
// atoms of |q - qb|^2, each axis taken as its minimum image.
__device__ __forceinline__ void drift_block(double *__restrict__ q4, const double *__restrict__ p4,
                                            int n, double dt, double Lx, double Ly, double Lz,
                                            unsigned long long *__restrict__ max_d2,
                                            const double *__restrict__ qb = nullptr,
                                            unsigned long long *__restrict__ max_dev2 = nullptr)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double d2 = 0.0, e2 = 0.0;
    if (i < n) {
        double *q = q4 + 4 * static_cast<int64_t>(i);
        const double *p = p4 + 4 * static_cast<int64_t>(i);
        const double L[3] = {Lx, Ly, Lz};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double dq = __dmul_rn(dt, p[a]);
            double x = __dadd_rn(q[a], dq);
            if (x >= L[a]) x = __dsub_rn(x, L[a]);
            else if (x < 0.0) x = __dadd_rn(x, L[a]);
            if (!(x < L[a])) x = 0.0;  // x == L after rounding
            q[a] = x;
            d2 = __dadd_rn(d2, __dmul_rn(dq, dq));
            if (qb) {
                double e = __dsub_rn(x, qb[4 * static_cast<int64_t>(i) + a]);
                const double h = 0.5 * L[a];
                if (e > h) e = __dsub_rn(e, L[a]);
                else if (e < -h) e = __dadd_rn(e, L[a]);
                e2 = __dadd_rn(e2, __dmul_rn(e, e));
            }
        }
    }
    block_max_into(d2, max_d2);
    if (qb) block_max_into(e2, max_dev2);
}

__global__ void __launch_bounds__(kDriftThreads)
drift_kernel(double *__restrict__ q4, const double *__restrict__ p4, int n, double dt, double Lx,
             double Ly, double Lz, unsigned long long *__restrict__ max_d2)
{
    drift_block(q4, p4, n, dt, Lx, Ly, Lz, max_d2);
}

// One step of lj_md_steps, part 1: nothing once the state is stale (every
// block reads the flag before the last block can write it); else the
// drift, and the block that finishes last folds the step into the state:
// moved += sqrt(max |dt p|^2) (the fastest-atom bound), or with qb
// moved = sqrt(max |q - qb|^2) (the largest displacement since the build),
// then the validity test 2 moved < margin.
__global__ void __launch_bounds__(kDriftThreads)
md_drift_kernel(double *__restrict__ q4, const double *__restrict__ p4, int n, double dt, double Lx,
                double Ly, double Lz, double margin, const double *__restrict__ qb,
                lj_md_state *__restrict__ S)
{
    if (*reinterpret_cast<volatile int32_t *>(&S->stale)) return;
    drift_block(q4, p4, n, dt, Lx, Ly, Lz, reinterpret_cast<unsigned long long *>(&S->max_disp2), qb,
                reinterpret_cast<unsigned long long *>(&S->max_dev2));
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();  // this block's maximum before its count
        last = atomicAdd(&S->blocks_done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();  // every block's maximum is visible
        volatile lj_md_state *V = S;
        const double d2 = V->max_disp2;
        const double moved = qb ? sqrt(V->max_dev2) : __dadd_rn(V->moved, sqrt(d2));
        V->moved = moved;
        V->last_disp2 = d2;
        V->max_disp2 = 0.0;
        V->max_dev2 = 0.0;
        V->blocks_done = 0u;
        if (__dmul_rn(2.0, moved) >= margin)
            V->stale = 1;
        else
            V->steps = V->steps + 1;
    }
}

// Part 2: a stale list is emptied (row_ptr[0..n] = 0), so that the force
// calls enqueued after it add nothing until the host rebuilds it.
__global__ void __launch_bounds__(kDriftThreads)
md_empty_kernel(int32_t *__restrict__ row_ptr, int n, const lj_md_state *__restrict__ S)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= n && *reinterpret_cast<const volatile int32_t *>(&S->stale)) row_ptr[i] = 0;
}

}  // namespace
}  // namespace lj

extern "C" int lj_drift(double *q4_dev, const double *p4_dev, int64_t n, double dt,
                        const double box[3], double *max_disp2_dev, void *stream)
{
    using namespace lj;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n < 0 || !box || !max_disp2_dev || !std::isfinite(dt)) return LJ_ERR_ARG;
    if (n > 0 && (!q4_dev || !p4_dev)) return LJ_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(q4_dev) | reinterpret_cast<uintptr_t>(p4_dev)) & 31u)
        return LJ_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(max_disp2_dev) & 7u) return LJ_ERR_ARG;
    if (n >= (int64_t(1) << 31) - 1) return LJ_ERR_CAPACITY;
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(box[a]) || !(box[a] > 0.0)) return LJ_ERR_BOX;
    LJ_TRY_CUDA(cudaMemsetAsync(max_disp2_dev, 0, sizeof(double), st));
    if (n == 0) return LJ_OK;
    drift_kernel<<<unsigned((n + kDriftThreads - 1) / kDriftThreads), kDriftThreads, 0, st>>>(
        q4_dev, p4_dev, static_cast<int>(n), dt, box[0], box[1], box[2],
        reinterpret_cast<unsigned long long *>(max_disp2_dev));
    LJ_TRY_LAUNCH("drift_kernel");
    return LJ_OK;
}

extern "C" int lj_md_steps(double *q4_dev, double *p4_dev, int64_t n, int32_t *row_ptr_dev,
                           const int32_t *col_dev, int64_t nnz, int half, double dt, double r_cut,
                           double r_search, const double box[3], double eps, double sigma,
                           int precision, int tpi, int64_t steps, int flags,
                           const double *q4_build_dev, double *energies_dev,
                           lj_md_state *state_dev, void *workspace_dev, size_t workspace_bytes,
                           void *stream)
{
    using namespace lj;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (steps < 0 || !state_dev || (reinterpret_cast<uintptr_t>(state_dev) & 7u)) return LJ_ERR_ARG;
    if (flags & ~LJ_MD_LAST_HALF_KICK) return LJ_ERR_ARG;
    if (!std::isfinite(r_search) || !(r_search > r_cut)) return LJ_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(q4_build_dev) & 31u) ||
        (reinterpret_cast<uintptr_t>(energies_dev) & 7u))
        return LJ_ERR_ARG;
    if (energies_dev && precision != LJ_FP64) return LJ_ERR_ARG;
    int t = tpi;
    const int rc = force_check(q4_dev, p4_dev, n, row_ptr_dev, col_dev, nnz, half, dt, r_cut, box,
                               eps, sigma, precision, &t, workspace_dev, workspace_bytes);
    if (rc != LJ_OK) return rc;
    if (energies_dev && workspace_bytes < lj_force_energy_workspace_bytes(n)) return LJ_ERR_CAPACITY;
    if (n == 0 || steps == 0) return LJ_OK;
    const int ni = static_cast<int>(n);
    const double margin = r_search - r_cut;
    const unsigned gd = unsigned((n + kDriftThreads - 1) / kDriftThreads);
    const unsigned ge = unsigned((n + 1 + kDriftThreads - 1) / kDriftThreads);
    for (int64_t s = 0; s < steps; ++s) {
        md_drift_kernel<<<gd, kDriftThreads, 0, st>>>(q4_dev, p4_dev, ni, dt, box[0], box[1], box[2],
                                                      margin, q4_build_dev, state_dev);
        LJ_TRY_LAUNCH("md_drift_kernel");
        md_empty_kernel<<<ge, kDriftThreads, 0, st>>>(row_ptr_dev, ni, state_dev);
        LJ_TRY_LAUNCH("md_empty_kernel");
        const double h = (s == steps - 1 && (flags & LJ_MD_LAST_HALF_KICK)) ? 0.5 * dt : dt;
        const int r = energies_dev
                          ? lj_force_energy(q4_dev, p4_dev, n, row_ptr_dev, col_dev, nnz, half, h,
                                            r_cut, box, eps, sigma, 1, energies_dev + s,
                                            workspace_dev, workspace_bytes, stream)
                          : lj_force(q4_dev, p4_dev, n, row_ptr_dev, col_dev, nnz, half, h, r_cut,
                                     box, eps, sigma, precision, t, workspace_dev, workspace_bytes,
                                     stream);
        if (r != LJ_OK) return r;
    }
    return LJ_OK;
}

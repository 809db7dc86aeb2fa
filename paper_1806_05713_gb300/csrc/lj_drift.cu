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
// per-step displacement.
#include <cmath>

#include "lj_internal.cuh"

namespace lj {
namespace {

constexpr int kDriftThreads = 256;

// q += dt p with round-to-nearest double operations (no fused multiply-add),
// then one periodic wrap per axis; *max_d2 = max over atoms of |dt p|^2 (as
// the ordered bit pattern of a non-negative double).
__global__ void __launch_bounds__(kDriftThreads)
drift_kernel(double *__restrict__ q4, const double *__restrict__ p4, int n, double dt, double Lx,
             double Ly, double Lz, unsigned long long *__restrict__ max_d2)
{
    __shared__ double red[kDriftThreads / 32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double d2 = 0.0;
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
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d2 = fmax(d2, __shfl_xor_sync(0xffffffffu, d2, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < kDriftThreads / 32; ++w) m = fmax(m, red[w]);
        atomicMax(max_d2, static_cast<unsigned long long>(__double_as_longlong(m)));
    }
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

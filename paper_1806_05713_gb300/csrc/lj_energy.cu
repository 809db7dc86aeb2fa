// lj_energy.cu -- potential energy of Eq. (1), truncated at r_c and
// optionally shifted so that V(r_c) = 0 (Watanabe & Nakagawa, section
// "Lennard-Jones Potential").  FP64; deterministic: a fixed grid, fixed
// per-thread work and a fixed-order two-level reduction.
#include <cmath>
#include <cstring>

#include "lj_internal.cuh"

namespace lj {
namespace {

constexpr int kEnergyBlocks = 1024;
constexpr int kEnergyThreads = 256;
constexpr int kEnergyTpi = 8;

struct EnergyParams {
    double L[3];
    long long half_bits[3];
    double rc2;
    double s2;      // sigma^2
    double four_eps;
    double vshift;  // shifted * V(r_c)
};

__global__ void __launch_bounds__(kEnergyThreads)
energy_kernel(const double *__restrict__ q4, int n, const int *__restrict__ row_ptr,
              const int *__restrict__ col, int half, EnergyParams P, double *__restrict__ partial)
{
    __shared__ double red[kEnergyThreads / 32];
    const int sub = threadIdx.x & (kEnergyTpi - 1);
    const int groups = gridDim.x * (kEnergyThreads / kEnergyTpi);
    double e = 0.0;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) / kEnergyTpi; i < n; i += groups) {
        double xi, yi, zi;
        load_xyz(q4, i, xi, yi, zi);
        for (int k = row_ptr[i] + sub; k < row_ptr[i + 1]; k += kEnergyTpi) {
            const int j = col[k];
            if (!half && j < i) continue;
            double xj, yj, zj;
            load_xyz(q4, j, xj, yj, zj);
            const double dx = min_image(__dsub_rn(xj, xi), P.L[0], P.half_bits[0]);
            const double dy = min_image(__dsub_rn(yj, yi), P.L[1], P.half_bits[1]);
            const double dz = min_image(__dsub_rn(zj, zi), P.L[2], P.half_bits[2]);
            const double r2 =
                __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
            if (r2 < P.rc2) {
                const double sr2 = P.s2 / r2;
                const double sr6 = sr2 * sr2 * sr2;
                e += P.four_eps * (sr6 * sr6 - sr6) - P.vshift;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kEnergyThreads / 32; ++w) s += red[w];
        partial[blockIdx.x] = s;
    }
}

__global__ void energy_final_kernel(const double *__restrict__ partial, int m, double *__restrict__ out)
{
    __shared__ double red[32];
    double s = 0.0;
    for (int t = threadIdx.x; t < m; t += blockDim.x) s += partial[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < int(blockDim.x / 32); ++w) t += red[w];
        *out = t;
    }
}

}  // namespace

int check_force_args(const double *q4, const double *p4, int64_t n, const int32_t *row_ptr,
                     const int32_t *col, int64_t nnz, double r_cut, const double box[3], double eps,
                     double sigma, double dt);

}  // namespace lj

extern "C" size_t lj_energy_workspace_bytes(int64_t n)
{
    (void)n;
    return size_t(lj::kEnergyBlocks) * sizeof(double) + 256;
}

extern "C" int lj_energy(const double *q4_dev, int64_t n, const int32_t *row_ptr_dev,
                         const int32_t *col_dev, int64_t nnz, int half, double r_cut,
                         const double box[3], double eps, double sigma, int shifted,
                         double *e_out_dev, void *workspace_dev, size_t workspace_bytes,
                         void *stream)
{
    using namespace lj;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!e_out_dev) return LJ_ERR_ARG;
    const int rc = check_force_args(q4_dev, q4_dev, n, row_ptr_dev, col_dev, nnz, r_cut, box, eps,
                                    sigma, 0.0);
    if (rc != LJ_OK) return rc;
    if (n == 0 || nnz == 0) {
        LJ_TRY_CUDA(cudaMemsetAsync(e_out_dev, 0, sizeof(double), st));
        return LJ_OK;
    }
    if (!workspace_dev || workspace_bytes < lj_energy_workspace_bytes(n)) return LJ_ERR_CAPACITY;
    EnergyParams P{};
    for (int a = 0; a < 3; ++a) {
        P.L[a] = box[a];
        const double h = 0.5 * box[a];
        std::memcpy(&P.half_bits[a], &h, sizeof(double));
    }
    P.rc2 = r_cut * r_cut;
    P.s2 = sigma * sigma;
    P.four_eps = 4.0 * eps;
    if (shifted) {
        const double sr2 = P.s2 / P.rc2, sr6 = sr2 * sr2 * sr2;
        P.vshift = P.four_eps * (sr6 * sr6 - sr6);
    }
    Carver c(workspace_dev);
    double *partial = c.take<double>(kEnergyBlocks);
    energy_kernel<<<kEnergyBlocks, kEnergyThreads, 0, st>>>(q4_dev, static_cast<int>(n), row_ptr_dev,
                                                             col_dev, half, P, partial);
    LJ_TRY_LAUNCH("energy_kernel");
    energy_final_kernel<<<1, 1024, 0, st>>>(partial, kEnergyBlocks, e_out_dev);
    LJ_TRY_LAUNCH("energy_final_kernel");
    return LJ_OK;
}

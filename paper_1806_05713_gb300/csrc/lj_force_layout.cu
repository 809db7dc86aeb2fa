// lj_force_layout.cu -- the FP64 force over positions and momenta in any
// strided layout: the paper's central question (section "Optimization before
// vectorization", Fig. "Data layout"; sections "AoS with Padding" and "AoS
// with Eight Elements") asked on GB300.
//
// Element (i, a) of q and of p is at base[i * row_stride + a * comp_stride]:
//   AoS4  row_stride 4, comp_stride 1  -- one 256-bit load per gathered atom
//   AoS8  row_stride 8, comp_stride 1  -- {q, pad, p, pad} in one 64-byte
//         record (q = record, p = record + 4), the paper's best CPU layout
//   SoA   row_stride 1, comp_stride n  -- three separate arrays per vector,
//         three 8-byte gathers per atom
// The arithmetic is that of the default FP64 schedule (t lanes per row,
// image-selected minimum image).
#include <cmath>

#include "lj_rows.cuh"

namespace lj {
namespace {

template <int TPI, bool HALF, int LAY>
__global__ void __launch_bounds__(256)
force_layout_kernel(const double *__restrict__ q, double *__restrict__ p, int n,
                    const int *__restrict__ row_ptr, const int *__restrict__ col, Fp64Params P,
                    Layout Lay)
{
    const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / TPI;
    if (gid >= n) return;
    fp64_row<TPI, HALF, 1, true, LAY>(q, p, row_ptr, col, gid, P, group_mask<TPI>(), Lay);
}

template <int TPI, int LAY>
int launch_layout(const double *q, double *p, int n, const int *rp, const int *col, int half,
                  const Fp64Params &P, const Layout &L, cudaStream_t st)
{
    const unsigned grid = unsigned((int64_t(n) * TPI + 255) / 256);
    if (half)
        force_layout_kernel<TPI, true, LAY><<<grid, 256, 0, st>>>(q, p, n, rp, col, P, L);
    else
        force_layout_kernel<TPI, false, LAY><<<grid, 256, 0, st>>>(q, p, n, rp, col, P, L);
    LJ_TRY_LAUNCH("force_layout_kernel");
    return LJ_OK;
}

}  // namespace

int check_force_args(const double *q4, const double *p4, int64_t n, const int32_t *row_ptr,
                     const int32_t *col, int64_t nnz, double r_cut, const double box[3], double eps,
                     double sigma, double dt);

}  // namespace lj

extern "C" int lj_force_strided(const double *q_dev, double *p_dev, int64_t n, int64_t row_stride,
                                int64_t comp_stride, const int32_t *row_ptr_dev,
                                const int32_t *col_dev, int64_t nnz, int half, double dt,
                                double r_cut, const double box[3], double eps, double sigma,
                                int lanes_per_row, void *stream)
{
    using namespace lj;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const double *fake = reinterpret_cast<const double *>(256);
    int rc = check_force_args(n > 0 ? fake : nullptr, n > 0 ? fake : nullptr, n, row_ptr_dev,
                              col_dev, nnz, r_cut, box, eps, sigma, dt);
    if (rc != LJ_OK) return rc;
    if (n > 0 && (!q_dev || !p_dev)) return LJ_ERR_ARG;
    if (row_stride < 1 || comp_stride < 1) return LJ_ERR_ARG;
    if (((reinterpret_cast<uintptr_t>(q_dev) | reinterpret_cast<uintptr_t>(p_dev)) & 7u) != 0)
        return LJ_ERR_ARG;
    if (lanes_per_row != 4 && lanes_per_row != 8 && lanes_per_row != 16) return LJ_ERR_ARG;
    if (n == 0 || nnz == 0) return LJ_OK;
    const Fp64Params P = make_fp64_params(box, dt, r_cut, eps, sigma);
    const Layout L{row_stride, comp_stride};
    const int ni = static_cast<int>(n);
    const bool vec = comp_stride == 1 && (row_stride % 4) == 0 &&
                     ((reinterpret_cast<uintptr_t>(q_dev) & 31u) == 0);
#define LJ_LAYOUT(T)                                                                            \
    return vec ? launch_layout<T, 1>(q_dev, p_dev, ni, row_ptr_dev, col_dev, half, P, L, st)   \
               : launch_layout<T, 2>(q_dev, p_dev, ni, row_ptr_dev, col_dev, half, P, L, st)
    switch (lanes_per_row) {
        case 4: LJ_LAYOUT(4);
        case 8: LJ_LAYOUT(8);
        default: LJ_LAYOUT(16);
    }
#undef LJ_LAYOUT
}

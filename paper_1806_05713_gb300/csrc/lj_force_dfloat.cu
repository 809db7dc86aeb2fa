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

// K_e (the exponent the double-float impulses are scaled by) within range.
bool dfloat_params_ok(const double box[3], double dt, double rc, double eps, double sigma)
{
    const DfParams P = make_dfloat_params(box, dt, rc, eps, sigma);
    return P.k_exp >= -700 && P.k_exp <= 700;
}

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

// lj_internal.cuh -- helpers shared by the CUDA translation units of the
// library (never by the CPU oracle, which is an independent program).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lj_gb300.h"

namespace lj {

// Records a CUDA error for lj_last_cuda_error() (thread-local text).
void record_cuda_error(cudaError_t err, const char *where);

// Counts kernels this library has enqueued (reported by
// lj_kernel_launch_count); every launch site passes through LJ_TRY_LAUNCH.
void count_launch();

#define LJ_TRY_CUDA(call)                                   \
    do {                                                    \
        cudaError_t lj_err_ = (call);                       \
        if (lj_err_ != cudaSuccess) {                       \
            ::lj::record_cuda_error(lj_err_, #call);        \
            return LJ_ERR_CUDA;                             \
        }                                                   \
    } while (0)

#define LJ_TRY_LAUNCH(where)                                \
    do {                                                    \
        ::lj::count_launch();                               \
        cudaError_t lj_err_ = cudaGetLastError();           \
        if (lj_err_ != cudaSuccess) {                       \
            ::lj::record_cuda_error(lj_err_, where);        \
            return LJ_ERR_CUDA;                             \
        }                                                   \
    } while (0)

// Host-side check of the shared preconditions on the box and the lengths.
int check_box(const double box[3], double r_search);

// Every host-side check lj_force makes before it launches (LJ_TPI_AUTO is
// resolved into *tpi, which may depend on the list kind `half`); LJ_OK or
// the status lj_force would return.
int force_check(const double *q4, const double *p4, int64_t n, const int32_t *row_ptr,
                const int32_t *col, int64_t nnz, int half, double dt, double rc,
                const double box[3], double eps, double sigma, int precision, int *tpi,
                const void *ws, size_t ws_bytes);

// Workspace carving: successive 256-byte-aligned sub-buffers of one block.
struct Carver {
    char *base;
    size_t used = 0;
    explicit Carver(void *b) : base(static_cast<char *>(b)) {}
    template <class T>
    T *take(size_t count) {
        used = (used + 255) & ~size_t(255);
        T *p = base ? reinterpret_cast<T *>(base + used) : nullptr;
        used += count * sizeof(T);
        return p;
    }
};

inline int num_sms()
{
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            sms = 152;
    }
    return sms;
}

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------

// Position x, y, z of atom i from the AoS4 array (one 16-byte and one
// 8-byte read-only load of the same 32-byte record).
__device__ __forceinline__ void load_xyz(const double *__restrict__ q4, int64_t i, double &x,
                                         double &y, double &z)
{
    const double2 a = __ldg(reinterpret_cast<const double2 *>(q4 + 4 * i));
    x = a.x;
    y = a.y;
    z = __ldg(q4 + 4 * i + 2);
}

// Minimum image of one displacement component, exactly as
//   if (d > L/2) d -= L; else if (d < -L/2) d += L;
// but with the two comparisons done on the IEEE bit pattern (|d| > L/2 iff
// the magnitude bits compare greater), so no FP64 compare instruction is
// issued; the subtraction or addition of L is the same rounded operation.
__device__ __forceinline__ double min_image(double d, double L, long long half_bits)
{
    const long long b = __double_as_longlong(d);
    if ((b & 0x7fffffffffffffffLL) > half_bits)
        d = __dadd_rn(d, b < 0 ? L : -L);
    return d;
}

// r2 < c2 for r2 >= 0 and c2 >= 0, on the bit patterns (integer compare).
__device__ __forceinline__ bool less_nonneg(double r2, long long c2_bits)
{
    return __double_as_longlong(r2) < c2_bits;
}

// Reciprocal of a in double precision for 2^-126 <= a < 2^126: an FP32 seed
// (the double truncated to FP32 by bit manipulation, then the hardware
// approximate reciprocal, rcp.approx.ftz.f32, relative error ~2^-22), then
// one third-order correction.  With e = 1 - a x0, 1/a = x0 / (1 - e)
// = x0 (1 + e + e^2 + ...), so x1 = x0 + x0 (e + e^2) has relative error
// ~e^3 < 2^-64 before rounding; the result is within two ulps of 1/a.
// This is the "reciprocal approximation plus correction" the paper's
// summary proposes for AVX-512 (vrcp14pd / vrcp28pd), built on GB300's FP32
// special-function unit: three FP64 instructions instead of a division.
// `ok` is false outside that range (the caller divides there instead).
__device__ __forceinline__ double rcp_fp64_fast(double a, bool &ok)
{
    const int hi = __double2hiint(a);
    ok = (hi >= 0x38100000) && (hi < 0x47d00000);
    const unsigned lo = static_cast<unsigned>(__double2loint(a));
    const unsigned fb = (static_cast<unsigned>(hi - 0x38000000) << 3) | (lo >> 29);
    float xf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(xf) : "f"(__uint_as_float(ok ? fb : 0x3f800000u)));
    const unsigned g = __float_as_uint(xf);
    const double x0 = __hiloint2double(static_cast<int>((g >> 3) + 0x38000000u),
                                       static_cast<int>(g << 29));
    const double e = fma(-a, x0, 1.0);
    return fma(x0, fma(e, e, e), x0);
}

// rcp_fp64_fast with the out-of-range fallback taken only when some lane of
// `mask` needs it (a warp-uniform branch, so the division's instructions are
// not issued in the common case).
__device__ __forceinline__ double rcp_fp64(double a, unsigned mask = 0xffffffffu)
{
    bool ok;
    double x = rcp_fp64_fast(a, ok);
    if (__any_sync(mask, !ok)) {
        if (!ok) x = 1.0 / a;
    }
    return x;
}

// Minimum image of the three components of d, exactly as
//   if (d > L/2) d -= L; else if (d < -L/2) d += L;
// per axis, with the tests on IEEE bit patterns and the adds issued only
// when some lane of `mask` needs a wrap.
__device__ __forceinline__ void min_image3(double &dx, double &dy, double &dz, const double L[3],
                                           const long long hb[3], unsigned mask = 0xffffffffu)
{
    const long long bx = __double_as_longlong(dx), by = __double_as_longlong(dy),
                    bz = __double_as_longlong(dz);
    const bool wx = (bx & 0x7fffffffffffffffLL) > hb[0];
    const bool wy = (by & 0x7fffffffffffffffLL) > hb[1];
    const bool wz = (bz & 0x7fffffffffffffffLL) > hb[2];
    if (__any_sync(mask, wx || wy || wz)) {
        if (wx) dx = __dadd_rn(dx, bx < 0 ? L[0] : -L[0]);
        if (wy) dy = __dadd_rn(dy, by < 0 ? L[1] : -L[1]);
        if (wz) dz = __dadd_rn(dz, bz < 0 ? L[2] : -L[2]);
    }
}

// FP32 reciprocal: hardware approximation plus one Newton step
// x1 = x0 + x0 (1 - a x0), relative error about one ulp.
__device__ __forceinline__ float rcp_fp32(float a)
{
    float x;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(x) : "f"(a));
    const float e = fmaf(-a, x, 1.0f);
    return fmaf(x, e, x);
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

}  // namespace lj

/*
 * lj_measure.h -- measurement and self-check entry points of the GB300 LJ
 * library: the throughput ceilings the force kernels are measured against,
 * and direct evaluation of the reciprocal approximations the kernels use.
 *
 * Conventions are those of lj_gb300.h (device pointers end in _dev, LJ_OK or
 * an LJ_ERR_* code is returned, nothing is allocated by the library).
 */
#ifndef LJ_MEASURE_H
#define LJ_MEASURE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ======================================================================== */
/* Pipe and cache ceilings (the roofline denominators)                      */
/* ======================================================================== */

/* Kinds for lj_measure_peak. */
#define LJ_PEAK_DFMA 0    /* FP64 fused multiply-add: flop/s (2 per FMA) */
#define LJ_PEAK_FFMA 1    /* FP32 fused multiply-add: flop/s */
#define LJ_PEAK_FFMA2 2   /* packed FP32 pair FMA (fma.rn.f32x2): flop/s (4 per lane) */
#define LJ_PEAK_L2_READ 3 /* 16-byte loads of an L2-resident buffer: bytes/s */

/*
 * The paper states the cost of one pair as 27 additions or multiplications,
 * one division, 48 bytes read and 24 written (section "Lennard-Jones
 * Potential"), and rates its kernels by how close they come to the
 * machine's limits.  On GB300 the FP64 force kernel is bound by the FP64
 * pipe, the mixed kernel by the FP32 pipe and by L2 gathers, so the
 * ceilings these kernels are compared with are measured here rather than
 * taken from a data sheet.
 *
 * Runs one timing kernel of the given kind on the current device, on
 * `stream`, and returns its throughput:
 *   LJ_PEAK_DFMA / FFMA / FFMA2: every thread of a full grid (8 blocks of
 *       256 threads per SM) runs 8 independent chains of dependent fused
 *       multiply-adds; `work` = loop trips per thread (each trip is 16 FMAs
 *       per chain); rate_out = flops / s (an FMA counts 2 flops, a packed
 *       pair FMA 4).  buf_dev is not used (may be NULL).
 *   LJ_PEAK_L2_READ: the grid reads buf_dev (buf_bytes, a multiple of 4096,
 *       buf_dev 256-byte aligned; choose it well below the 129 MB L2 so it
 *       stays resident) `work` times over with 16-byte loads; rate_out =
 *       bytes read / s.  The first pass, which brings the buffer into L2,
 *       is run once untimed before the timed ones.  Pass a zero-filled
 *       buffer: it is then only read (the probe keeps its loads alive with a
 *       store that a zero buffer never triggers).
 *  rate_out, ms_out  host out: the rate and the timed kernel's duration
 *                    (CUDA events on `stream`, after one untimed warm-up
 *                    launch).
 * Synchronous (waits for the timed launch).  Errors: LJ_ERR_ARG (unknown
 * kind, work < 1, null outputs, missing or misaligned buffer for
 * LJ_PEAK_L2_READ), LJ_ERR_CUDA.
 */
int lj_measure_peak(int kind, void *buf_dev, size_t buf_bytes, int64_t work, double *rate_out,
                    double *ms_out, void *stream);

/* ======================================================================== */
/* Reciprocal approximations (section "Summary and Discussion")             */
/* ======================================================================== */

/* Kinds for lj_eval_reciprocal.  Each evaluates, element by element, the
 * very device function the force kernels inline.  Kind 0 (a double-float
 * seed with one FP64 Newton step, replaced by LJ_RCP_FP64_INT) is retired
 * and refused. */
#define LJ_RCP_FP64_FAST 1   /* 1/a: FP32 seed + one third-order FP64 correction
                                (the image-selected FP64 kernels); defined for
                                2^-126 <= a < 2^126 */
#define LJ_RSQRT_FP64 2      /* 1/sqrt(a): FP32 seed + two FP64 Newton steps
                                (force-shifted truncation); division outside
                                2^-119 <= a < 2^120 */
#define LJ_RCP_DF 3          /* 1/a in double-float (head + tail of two floats),
                                the DFLOAT kernels' reciprocal, one entry per lane */
#define LJ_RCP_DF2 4         /* the same in packed f32x2 registers, two entries per
                                lane (the DFLOAT kernels' default) */
#define LJ_RCP_FP32 5        /* 1/a in FP32: hardware approximation + one Newton
                                step (the mixed kernels) */
#define LJ_RCP_FP64_INT 6    /* 1/a: FP32 seed + one second-order Newton step in
                                integer arithmetic, no FP64 instruction (the
                                fixed-point FP64 kernels); within 0.5 + 2^-12 ulp
                                for 2^-119 <= a < 2^120 */

/*
 * The paper proposes, as future work for its AVX-512 kernels, replacing the
 * division of Algorithm 1 by a hardware reciprocal approximation followed
 * by a correction (section "Summary and Discussion").  The force kernels do
 * that on GB300; this entry point evaluates each of those reciprocals on
 * caller-chosen inputs so that their error can be measured directly against
 * IEEE division.
 *
 *  a_dev    n doubles (device, 8-byte aligned), the arguments.  For
 *           LJ_RCP_DF and LJ_RCP_DF2 each a is first split into a
 *           double-float head h = fl32(a) and tail l = fl32(a - h); for
 *           LJ_RCP_FP32 it is rounded to FP32 first.
 *  out_dev  2 n doubles (device), overwritten: out[2k] = the result for
 *           a[k] (for the double-float kinds the head), out[2k + 1] = the
 *           double-float tail (0 for the other kinds).  FP32 values are
 *           stored exactly as doubles.
 *  ok_dev   n bytes (device) or NULL: 1 where the input lies in the range
 *           the approximation is defined for (the kernels divide outside
 *           it), else 0; 1 for the kinds without a range.  Outside its range
 *           the value written is unspecified.
 * Asynchronous on `stream`.  Errors: LJ_ERR_ARG (unknown kind, n < 0, null
 * or misaligned pointers), LJ_ERR_CUDA.
 */
int lj_eval_reciprocal(int kind, const double *a_dev, int64_t n, double *out_dev,
                       uint8_t *ok_dev, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* LJ_MEASURE_H */

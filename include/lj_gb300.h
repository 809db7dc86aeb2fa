/*
 * lj_gb300.h -- C ABI of the GB300 (sm_103a) Lennard-Jones force library.
 *
 * The library computes one step of the truncated Lennard-Jones momentum
 * update over a sorted Verlet pair list (Watanabe & Nakagawa, arXiv
 * 1806.05713): for each atom i it walks the j of its list row, forms the
 * minimum-image displacement d = q_j - q_i, skips pairs with r^2 >= r_c^2,
 * and applies
 *
 *     df = (24 eps sigma^6 r^6 - 48 eps sigma^12) dt / r^14,
 *     p_i += df d,   p_j -= df d,
 *
 * which is Algorithm 1 (with the printed sign of the p_j update read as the
 * opposite of p_i's, as Newton's third law requires) inside the sorted-list
 * double loop of Algorithm 3, for the potential of Eq. (1).
 *
 * Conventions for every entry point:
 *  - Pointers named *_dev are device pointers; every other pointer is host.
 *  - Positions and momenta are "AoS4": n rows of 4 doubles {x, y, z, pad}
 *    (the padded layout of the section "AoS with Padding"); their base
 *    pointers must be 32-byte aligned (rows are read with 256-bit loads),
 *    else LJ_ERR_ARG.  Workspaces must be 256-byte aligned.
 *    The pad element of positions is ignored; that of momenta is never
 *    written.
 *  - Positions must lie in [0, L) per axis of the periodic box (L = box[a]),
 *    and every box side must be at least 2 r_search (unique minimum image).
 *  - The pair list is CSR with 32-bit indices: row_ptr[n+1], col[nnz]; row i
 *    holds its j in ascending order; a "half" list holds only j > i, a
 *    "full" list every j != i.
 *  - Caller owns every buffer.  The library never allocates device memory:
 *    scratch space is passed in as `workspace_dev` of at least the size the
 *    matching *_workspace_bytes() function reports (256-byte aligned).
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *    stream).  Entry points that must read a count back say so.
 *  - Return value: LJ_OK (0) or one of the LJ_ERR_* codes; no exception or
 *    abort crosses the ABI.  On error, outputs are unspecified unless stated.
 *    lj_status_string() names each code.
 */
#ifndef LJ_GB300_H
#define LJ_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define LJ_OK 0
#define LJ_ERR_ARG 1      /* null pointer, n < 0, bad flag, r_cut > r_search, ... */
#define LJ_ERR_BOX 2      /* a box side is shorter than 2 r_search (or not finite) */
#define LJ_ERR_RANGE 3    /* a position is outside [0, L) or not finite */
#define LJ_ERR_CAPACITY 4 /* output or workspace too small, or nnz >= 2^31 */
#define LJ_ERR_CUDA 5     /* a CUDA runtime call failed (see lj_last_cuda_error) */
#define LJ_ERR_DEVICE 6   /* no usable sm_103 device for this library build */

/* ---- arithmetic forms of the force kernels ----------------------------- */
#define LJ_FP64 0  /* every step in IEEE double precision */
#define LJ_MIXED 1 /* FP32 pair arithmetic; the displacement formed exactly in
                      32-bit fixed point derived from the FP64 positions and
                      rounded once to FP32; compensated FP32 per-i sums and
                      FP64 momentum updates */
#define LJ_DFLOAT 2 /* FP64-class accuracy from FP32 instructions: the
                       displacement exact from 58-bit fixed-point positions,
                       the pair arithmetic in double-float (unevaluated sums
                       of two FP32 numbers: Dekker 1971, Knuth's TwoSum),
                       compensated per-i sums, FP64 momentum updates; pairs
                       at the cutoff or closer than the FP32 range of r^-14
                       take the FP64 formula.  Not in the paper (which is
                       FP64 throughout): GB300 issues FP32 ~70 times faster
                       than FP64.  lj_force only; tpi = 4, 8, 16. */

/* ---- schedules ---------------------------------------------------------- */
/* `tpi` = threads per i-row: 1, 2, 4, 8, 16 or 32 lanes of one warp walk one
 * row and reduce their partial sums with warp shuffles; 0 = library default
 * (FP64: LJ_SCHED_FIXED | LJ_SCHED_STREAM | 32 for a half list of at least
 * 524,288 rows, else LJ_SCHED_FIXED | 8 -- image selection instead of the
 * fixed point for boxes wider than 1024 r_c; mixed: 8 lanes per row;
 * double-float: LJ_SCHED_SWP2 | 8). */
#define LJ_TPI_AUTO 0
/* LJ_SCHED_SWP2 | tpi (tpi = 4, 8 or 16; FP64 with the IEEE-bit-pattern
 * displacement, LJ_MIXED and LJ_DFLOAT): software pipelining, the paper's
 * section "Software Pipelining" -- each lane carries two independent
 * entries per iteration so that their dependency chains overlap.  (The
 * LJ_MIXED and LJ_DFLOAT rows also request the gathers of the next
 * iteration before the arithmetic of the current one, in every schedule.) */
#define LJ_SCHED_SWP2 128
/* LJ_SCHED_SORTED | (a row-group schedule, FP64 or mixed): rows are walked
 * in order of decreasing length (a counting sort of the row lengths in the
 * workspace, three small kernels per call), so the groups of a warp walk
 * rows of equal length and none waits for a longer one. */
#define LJ_SCHED_SORTED 512
/* LJ_SCHED_IMAGES | 4, 8, 16, optionally | LJ_SCHED_SWP2 (FP64 only): each row
 * precomputes the periodic images q_i +- L and each entry picks the minimum
 * image of q_i with integer compares of IEEE high words, so the
 * displacement costs one FP64 subtraction and no wrap addition. */
#define LJ_SCHED_IMAGES 1024
/* LJ_SCHED_FIXED | 4, 8, 16, optionally | LJ_SCHED_SORTED (FP64 only): the
 * displacement and r^2 computed exactly in 64/128-bit integer fixed point
 * (positions x 2^k, the minimum image by one integer compare) and rounded
 * once to double; the rest of Algorithm 1 in IEEE double as in the other
 * FP64 schedules.  Six fewer FP64 instructions per entry.  Offered for boxes
 * up to 1024 r_c wide (the fixed point then resolves 2^-50 r_c); wider
 * boxes return LJ_ERR_ARG, and the default schedule, lj_force_energy,
 * lj_force_vjp and lj_force_batched use image selection there. */
#define LJ_SCHED_FIXED 2048
/* LJ_SCHED_FIXED | LJ_SCHED_STREAM | r (r = 4, 8, 16 or 32; FP64 only): the
 * fixed-point rows above, but a warp owns r consecutive rows and cuts their
 * entries (contiguous in CSR) into 32 equal chunks, one per lane, each lane
 * moving forward through the row boundaries of its chunk; lanes idle only
 * in the padding of the last chunk instead of at the end of every row.
 * p_i is added with FP64 atomics by every lane whose chunk meets the row,
 * so full lists are not deterministic under this schedule.  Lists of more
 * than 2^31 - 257 entries are refused (LJ_ERR_CAPACITY). */
#define LJ_SCHED_STREAM 8192
/* LJ_SCHED_CELLS | (a row-group schedule, any form; not with LJ_SCHED_SORTED
 * or LJ_SCHED_STREAM): the rows are walked in space-filling order -- counting-
 * sorted per call (three small kernels) by the Morton index of their atom's
 * cell, at most 16 cells per axis of side >= r_cut / 2 -- so that the warps
 * of an SM take nearby atoms, whose neighbour sets overlap, and the gathered
 * q_j records come from L1 when the atoms are numbered in random order.  The
 * results do not depend on the order (each row keeps its own sum). */
#define LJ_SCHED_CELLS 16384

const char *lj_status_string(int status);
/* Text of the last CUDA error seen by this library in this thread. */
const char *lj_last_cuda_error(void);
/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int lj_version(void);
/* Number of CUDA kernels this library has enqueued since it was loaded
 * (all threads; memsets and copies are not counted).  For accounting. */
unsigned long long lj_kernel_launch_count(void);

/* ======================================================================== */
/* Pair list (section "Verlet List and Bookkeeping Method"; Fig. "Data      */
/* layout of a pair list"; the counting sort of section "Sorting by        */
/* Indices").                                                               */
/* ======================================================================== */

/* Bytes of device workspace lj_build_pairlist needs for n atoms. */
size_t lj_pairlist_workspace_bytes(int64_t n, const double box[3], double r_search);

/*
 * Build the sorted CSR Verlet list of every pair closer than r_search:
 * all (i, j), j != i (j > i if half != 0), with minimum-image
 * r^2 < r_search^2, where r^2 = (dx*dx + dy*dy) + dz*dz in round-to-nearest
 * double arithmetic without fused multiply-adds (the list is bit-exact
 * against that definition).  Atoms are binned into cells of side
 * >= r_search / 2 (the linked-list cell method with a 5 x 5 x 5 stencil; with
 * five or more cells on every axis each pair is met once, over the forward
 * half of the stencil), candidates are screened in FP32 with a proven error
 * bound and decided in FP64, and each row is sorted by j.
 *
 *  q4_dev        n x 4 doubles, positions in [0, L).
 *  n             number of atoms (>= 0; n = 0 gives an empty list).
 *  box           host, 3 box sides, each >= 2 r_search.
 *  r_search      search length r_s = r_c + margin (> 0).
 *  half          nonzero: half list (j > i); zero: full list.
 *  row_ptr_dev   out, n + 1 int32.
 *  col_dev       out, col_capacity int32.
 *  col_capacity  entries available in col_dev.
 *  workspace_dev scratch of lj_pairlist_workspace_bytes(n, box, r_search).
 *  nnz_out       host out: number of list entries.  On LJ_ERR_CAPACITY it
 *                holds the number needed (row_ptr_dev is then valid and
 *                col_dev unspecified); retry with a larger col_dev.
 *  max_row_out   host out (may be NULL): longest row.
 *  stream        cudaStream_t.
 * Blocks the calling thread until the list size is known (one small
 * device-to-host copy, read on an internal stream of the library -- one per
 * host thread and device, created on first use -- that waits for the size
 * only, while the rows are sorted on `stream`), and returns: the list is
 * complete in stream order, not yet on return.
 * Errors: LJ_ERR_ARG, LJ_ERR_BOX, LJ_ERR_RANGE (a position outside [0, L) or
 * not finite), LJ_ERR_CAPACITY (col_capacity too small, nnz >= 2^31, or a
 * row longer than the 56,000 entries one warp's shared memory can sort),
 * LJ_ERR_CUDA.
 */
int lj_build_pairlist(const double *q4_dev, int64_t n, const double box[3], double r_search,
                      int half, int32_t *row_ptr_dev, int32_t *col_dev, int64_t col_capacity,
                      void *workspace_dev, size_t workspace_bytes, int64_t *nnz_out,
                      int64_t *max_row_out, void *stream);

/*
 * lj_build_pairlist_static: the same list as lj_build_pairlist, for callers
 * that cannot allocate device memory (no cudaMalloc in their context, no
 * workspace from their host); the paper has no counterpart -- it is a
 * deployment variant of the builder above.
 *
 * The builder's scratch lives in one fixed array of LJ_STATIC_SCRATCH_BYTES
 * inside the library's device memory (every GPU that loads the library holds
 * it until the process exits), so this call allocates nothing: no cudaMalloc,
 * no cudaFree, no allocating library routine.  The caller still passes the
 * positions and the row_ptr / col outputs, exactly as for lj_build_pairlist.
 *  - n must not exceed LJ_STATIC_MAX_ATOMS (LJ_ERR_CAPACITY otherwise; no GPU
 *    work is done).
 *  - The first call on a device looks up the array's device address with that
 *    device current; make that first call before any stream capture.
 *  - All calls share the one array and each call clears what it needs zeroed:
 *    calls whose GPU work overlaps (other streams or host threads) race on it
 *    and must be serialised by the caller.  The array is in use until the
 *    call's work on `stream` has completed -- after the call returns, since
 *    the last kernels still read it -- so serialise through that stream or an
 *    event, not by the order of the host calls alone.
 *  - It always takes the builder's two-walk path (count, scan, fill), and
 *    every operation it enqueues goes on `stream` (no internal stream).
 * Arguments, outputs, blocking behaviour and the other errors are those of
 * lj_build_pairlist.
 */
#define LJ_STATIC_MAX_ATOMS 131072
#define LJ_STATIC_SCRATCH_BYTES (8u << 20)
int lj_build_pairlist_static(const double *q4_dev, int64_t n, const double box[3],
                             double r_search, int half, int32_t *row_ptr_dev, int32_t *col_dev,
                             int64_t col_capacity, int64_t *nnz_out, int64_t *max_row_out,
                             void *stream);

/* ======================================================================== */
/* Force (Algorithm 1 inside Algorithm 3)                                    */
/* ======================================================================== */

/* Bytes of device workspace lj_force needs (about 8 n + 2.5 KB for the
 * length-sorted row order; plus fixed-point positions, 32 n for LJ_FP64
 * and LJ_DFLOAT, 16 n for LJ_MIXED). */
size_t lj_force_workspace_bytes(int64_t n, const double box[3], int precision);

/*
 * One momentum update p += impulses(q) over the list, Algorithms 1 and 3:
 * for each list entry (i, j) with minimum-image r^2 < r_cut^2,
 *   df = (24 eps sigma^6 r^6 - 48 eps sigma^12) dt / r^14,
 *   p_i += df d and, for a half list, p_j -= df d (d = q_j - q_i).
 * A full list applies only the p_i part (the pair appears again in row j).
 * Entries with r_cut <= r < r_search (the bookkeeping margin) contribute
 * nothing.  p4_dev is updated in place and is never zeroed.
 *
 *  q4_dev, p4_dev   n x 4 doubles (positions in [0, L); momenta).
 *  row_ptr_dev, col_dev, nnz, half   the list from lj_build_pairlist.
 *  dt, r_cut        time step and cutoff (0 < r_cut <= L/2).
 *  box              host, 3 box sides.
 *  eps, sigma       Eq. (1) parameters (> 0).
 *  precision        LJ_FP64, LJ_MIXED or LJ_DFLOAT.
 *  tpi              LJ_TPI_AUTO, 1..32 (power of two; LJ_DFLOAT: 4, 8, 16),
 *                   or LJ_SCHED_SWP2 | 4, 8, 16 (every form).
 *                   LJ_SCHED_SORTED may be or-ed into any of these,
 *                   LJ_SCHED_IMAGES into the FP64 4, 8, 16 and SWP2
 *                   schedules; LJ_SCHED_FIXED | 4, 8, 16 (FP64, optionally |
 *                   LJ_SCHED_SORTED); LJ_SCHED_FIXED | LJ_SCHED_STREAM | 4,
 *                   8, 16, 32 (FP64).
 *  workspace_dev    scratch of lj_force_workspace_bytes() (NULL if 0).
 * Half lists add p_j with FP64 atomics, so their rounding order (not their
 * value beyond the last bits) varies between calls; full lists are
 * deterministic (except under LJ_SCHED_STREAM and, for LJ_DFLOAT, rows with
 * two or more pairs that take the FP64 formula).
 * LJ_DFLOAT agrees with LJ_FP64 to ~1e-14 of max |dp|; it returns
 * LJ_ERR_ARG if 24 eps sigma^6 dt / r_c^7 is outside 2^-690 .. 2^690.
 * Asynchronous.  Errors: LJ_ERR_ARG, LJ_ERR_BOX, LJ_ERR_CAPACITY (workspace
 * too small), LJ_ERR_CUDA.
 */
int lj_force(const double *q4_dev, double *p4_dev, int64_t n, const int32_t *row_ptr_dev,
             const int32_t *col_dev, int64_t nnz, int half, double dt, double r_cut,
             const double box[3], double eps, double sigma, int precision, int tpi,
             void *workspace_dev, size_t workspace_bytes, void *stream);

/*
 * lj_force in the FP64 form for positions and momenta in any strided layout
 * -- the data-layout question of the paper (Fig. "Data layout"; sections
 * "AoS with Padding" and "AoS with Eight Elements"): element (i, a) of q and
 * of p is at q_dev[i * row_stride + a * comp_stride] (same strides for p).
 *   AoS4: row_stride 4, comp_stride 1 (lj_force's layout);
 *   AoS8: row_stride 8, comp_stride 1, p_dev = q_dev + 4 (q and p of an atom
 *         in one 64-byte record);
 *   SoA:  row_stride 1, comp_stride n (x[], y[], z[] back to back).
 * Rows are read with one 256-bit load when comp_stride = 1, row_stride is a
 * multiple of 4 and q_dev is 32-byte aligned, else with three 8-byte loads.
 * lanes_per_row: 4, 8 or 16 (the image-selected FP64 schedule).  Pointers
 * 8-byte aligned.  Same semantics and errors as lj_force; no workspace.
 */
int lj_force_strided(const double *q_dev, double *p_dev, int64_t n, int64_t row_stride,
                     int64_t comp_stride, const int32_t *row_ptr_dev, const int32_t *col_dev,
                     int64_t nnz, int half, double dt, double r_cut, const double box[3],
                     double eps, double sigma, int lanes_per_row, void *stream);

/* Bytes of device workspace lj_force_energy needs. */
size_t lj_force_energy_workspace_bytes(int64_t n);

/*
 * lj_force (FP64 form, 8 lanes per row; the exact fixed-point displacement,
 * or image selection for boxes wider than 1024 r_cut) that also returns the
 * potential energy of the same configuration, Eq. (1) truncated at r_cut
 * and, if shifted != 0, shifted so that V(r_cut) = 0 -- the energy a
 * velocity-Verlet loop monitors, as a by-product of the force pass (the pair
 * energy reuses the pass's 1/r^2: three extra FP64 instructions per pair).
 * e_out_dev: one device double, overwritten; a full list counts each pair
 * once (half of its entries' sum).  The energy sum is deterministic
 * (fixed-order reduction).  Asynchronous.  Errors as lj_force and lj_energy.
 */
int lj_force_energy(const double *q4_dev, double *p4_dev, int64_t n, const int32_t *row_ptr_dev,
                    const int32_t *col_dev, int64_t nnz, int half, double dt, double r_cut,
                    const double box[3], double eps, double sigma, int shifted, double *e_out_dev,
                    void *workspace_dev, size_t workspace_bytes, void *stream);

/*
 * lj_force_energy that also returns the pair virial of the same pass,
 *   W = sum over unique pairs with r < r_cut of r F(r),
 *   F(r) = -dV/dr = 24 eps (2 (sigma/r)^12 - (sigma/r)^6) / r
 * (unaffected by the energy shift; positive when the pairs repel), so that
 * with the kinetic energy K the pressure of the box is (2 K + W) / (3 V).
 * w_out_dev: one device double (8-byte aligned), overwritten.  Same
 * workspace (lj_force_energy_workspace_bytes), semantics and errors as
 * lj_force_energy; LJ_ERR_ARG if w_out_dev is NULL.
 */
int lj_force_energy_virial(const double *q4_dev, double *p4_dev, int64_t n,
                           const int32_t *row_ptr_dev, const int32_t *col_dev, int64_t nnz,
                           int half, double dt, double r_cut, const double box[3], double eps,
                           double sigma, int shifted, double *e_out_dev, double *w_out_dev,
                           void *workspace_dev, size_t workspace_bytes, void *stream);

/* Bytes of device workspace lj_force_shifted needs. */
size_t lj_force_shifted_workspace_bytes(int64_t n);

/*
 * The momentum update with the force-shifted truncation the paper recommends
 * for energy conservation but does not use (section "Lennard-Jones
 * Potential"): for r < r_c the pair potential is
 *   V_fs(r) = V(r) - V(r_c) - (r - r_c) V'(r_c),
 * so the pair force -V'(r) + V'(r_c) falls continuously to zero at r_c; the
 * impulse coefficient is lj_force's df minus F_c dt / r with
 * F_c = -V'(r_c).  FP64 (the fixed-point rows of LJ_SCHED_FIXED | 8, plus an
 * FP64 reciprocal square root per pair).  If e_out_dev (device, one double)
 * is not NULL it receives the force-shifted energy sum of V_fs over unique
 * pairs, computed in the same pass (deterministic reduction).  Other
 * arguments as lj_force_energy.  Boxes up to 1024 r_c wide (else
 * LJ_ERR_ARG).  Asynchronous.  Errors: LJ_ERR_ARG, LJ_ERR_BOX,
 * LJ_ERR_CAPACITY, LJ_ERR_CUDA.
 */
int lj_force_shifted(const double *q4_dev, double *p4_dev, int64_t n, const int32_t *row_ptr_dev,
                     const int32_t *col_dev, int64_t nnz, int half, double dt, double r_cut,
                     const double box[3], double eps, double sigma, double *e_out_dev,
                     void *workspace_dev, size_t workspace_bytes, void *stream);

/* ======================================================================== */
/* Energy (Eq. 1, truncated at r_c, optionally shifted)                     */
/* ======================================================================== */

size_t lj_energy_workspace_bytes(int64_t n);

/*
 * E = sum over unique pairs with r < r_cut of V(r) - shifted * V(r_cut),
 * V(r) = 4 eps [(sigma/r)^12 - (sigma/r)^6] (Eq. 1; the shift is the
 * paper's "adding a constant so that V(r_c) = 0").  With a full list only
 * entries with j > i are summed.  FP64, deterministic (fixed-order block
 * reduction).  e_out_dev: one device double, overwritten.  Asynchronous.
 */
int lj_energy(const double *q4_dev, int64_t n, const int32_t *row_ptr_dev,
              const int32_t *col_dev, int64_t nnz, int half, double r_cut, const double box[3],
              double eps, double sigma, int shifted, double *e_out_dev, void *workspace_dev,
              size_t workspace_bytes, void *stream);

/* ======================================================================== */
/* Drift (the position update around the force; bookkeeping criterion)      */
/* ======================================================================== */

/*
 * Velocity-Verlet drift with unit mass: q += dt p per atom and axis (round-
 * to-nearest double operations, no fused multiply-add), then one periodic
 * wrap back into [0, L) (a result equal to L becomes 0).  Writes
 * max_disp2_dev[0] (one device double, overwritten) = max over atoms of
 * |dt p|^2, the squared largest displacement of this step: with the
 * fastest-atom criterion of section "Verlet List and Bookkeeping Method", a
 * list built with margin r_s - r_c stays valid while 2 * (sum over steps of
 * sqrt(max_disp2)) < r_s - r_c.  Requires |dt p| < L per axis.  The pad
 * element of q is untouched.  Asynchronous.  Errors: LJ_ERR_ARG, LJ_ERR_BOX,
 * LJ_ERR_CUDA.
 */
int lj_drift(double *q4_dev, const double *p4_dev, int64_t n, double dt, const double box[3],
             double *max_disp2_dev, void *stream);

/* Bookkeeping state of lj_md_steps, in device memory (caller-owned, 8-byte
 * aligned).  Zero all of it whenever the list is (re)built. */
typedef struct lj_md_state {
    double moved;          /* the displacement bound since the build (see lj_md_steps) */
    double max_disp2;      /* scratch: the current step's largest |dt p|^2 */
    double last_disp2;     /* the largest |dt p|^2 of the last step that moved the atoms */
    double max_dev2;       /* scratch: the current step's largest |q - q_build|^2 */
    int32_t stale;         /* 1 once 2 moved >= r_search - r_cut (see lj_md_steps) */
    int32_t steps;         /* steps completed (drift and kick) since the state was zeroed */
    uint32_t blocks_done;  /* scratch of the drift kernel */
    int32_t reserved;
} lj_md_state;

/* lj_md_steps flag: the last step of the call kicks by dt / 2 (the closing
 * half kick of velocity Verlet). */
#define LJ_MD_LAST_HALF_KICK 1

/*
 * Enqueue `steps` leapfrog steps of velocity Verlet (unit mass) with the
 * bookkeeping method of section "Verlet List and Bookkeeping Method", the
 * validity test taken on the device so that no step waits for the host.
 * Each step, unless state->stale is already set:
 *   1. the drift of lj_drift (q += dt p, wrapped);
 *   2. the displacement bound: with q4_build_dev NULL, moved += the step's
 *      largest |dt p| (the fastest atom's step, summed over the steps since
 *      the build); with q4_build_dev (n x 4, the positions the list was
 *      built from), moved = the largest |q - q_build| over the atoms, each
 *      axis as its minimum image -- the tighter bound, since a pair moves
 *      closer by at most the two atoms' displacements.  If 2 moved >=
 *      r_search - r_cut the list may have lost a pair: stale = 1 and
 *      row_ptr_dev[0..n] is zeroed -- the list is emptied on the device, so
 *      the kick of this step and every later step of the call do nothing;
 *      otherwise steps += 1;
 *   3. the kick p += impulses(q) of lj_force with this dt (dt / 2 on the
 *      call's last step with LJ_MD_LAST_HALF_KICK); with energies_dev
 *      (FP64 only) the kick is lj_force_energy's and writes the shifted
 *      potential energy U(q) of step s to energies_dev[s].
 * After the call the host reads the state: `steps` steps are complete; if
 * stale is 1, the positions are one drift ahead of the momenta -- rebuild
 * the list from q4_dev (lj_build_pairlist), zero the state and apply the
 * kick that step owes with lj_force (same dt, or dt / 2 if it was the last
 * step of a half-kick call), then continue.  The force arguments
 * (precision, tpi, workspace: at least lj_force_workspace_bytes, and with
 * energies also lj_force_energy_workspace_bytes) are all checked before
 * anything is enqueued.  Asynchronous; one small kernel for the drift and
 * bookkeeping, one for the emptying, and the force call's launches, per
 * step.  Errors: LJ_ERR_ARG (also r_search <= r_cut, steps < 0, unknown
 * flags, state NULL or not 8-byte aligned, q4_build_dev not 32-byte
 * aligned, energies with a form other than LJ_FP64), LJ_ERR_BOX,
 * LJ_ERR_CAPACITY, LJ_ERR_CUDA.
 */
int lj_md_steps(double *q4_dev, double *p4_dev, int64_t n, int32_t *row_ptr_dev,
                const int32_t *col_dev, int64_t nnz, int half, double dt, double r_cut,
                double r_search, const double box[3], double eps, double sigma, int precision,
                int tpi, int64_t steps, int flags, const double *q4_build_dev,
                double *energies_dev, lj_md_state *state_dev, void *workspace_dev,
                size_t workspace_bytes, void *stream);

/* ======================================================================== */
/* Batched systems: many independent LJ systems in one persistent launch    */
/* (the Algorithm 3 loop of each system, work-shared across the GPU)        */
/* ======================================================================== */

/* One system of a batch.  Atoms of system s are rows atom_offset ..
 * atom_offset + n - 1 of the packed q4/p4 arrays; its CSR list occupies
 * row_ptr[row_offset .. row_offset + n] (entry indices local to the system,
 * starting at 0) and col[entry_offset .. entry_offset + nnz - 1] (atom
 * indices local to the system) -- exactly what lj_build_pairlist writes when
 * given q4 + 4 atom_offset, row_ptr + row_offset and col + entry_offset. */
typedef struct lj_system {
    int64_t atom_offset;
    int64_t n;
    int64_t row_offset;
    int64_t entry_offset;
    int64_t nnz;
    double box[3];
    double r_cut;
    double eps;
    double sigma;
    int32_t half;
    int32_t reserved;
} lj_system;

/* A batch plan: host-side summary of a device buffer (caller-owned) that
 * holds per-system parameters and the work-item table.  Filled by
 * lj_batch_init; read by lj_force_batched. */
typedef struct lj_batch {
    void *plan_dev;
    size_t plan_bytes;
    int64_t nitems;
    int64_t total_atoms;
    double dt;
    int32_t nsys;
    int32_t precision;
    int32_t tpi;           /* lanes per row: 1, 2, 4, 8, 16, 32; or LJ_SCHED_STREAM
                              (FP64): each work item's rows walked as one stream */
    int32_t rows_per_item; /* rows per work item (>= 1) */
    int32_t blocks;        /* persistent grid size */
    int32_t flags;         /* bit 0: every system has a cubic box */
} lj_batch;

/* Bytes of the device plan for these systems and rows_per_item. */
size_t lj_batch_plan_bytes(const lj_system *systems, int nsys, int rows_per_item);

/*
 * Validate the systems (each as lj_force would), build the work-item table
 * (items of at most rows_per_item rows of one system, ordered by decreasing
 * estimated cost nnz/n * rows, the longest-first rule), and copy it and the
 * per-system constants of Algorithm 1 (dt, eps, sigma, cutoff, box) to
 * plan_dev.  precision: LJ_FP64 (tpi 1 .. 32, or LJ_SCHED_STREAM: the warp
 * that takes an item walks its rows' entries as one stream, as lj_force's
 * LJ_SCHED_STREAM), LJ_MIXED (tpi 1 .. 32) or LJ_DFLOAT (tpi 4, 8 or 16; two
 * entries per lane in packed f32x2 registers).  Blocks until the copy is
 * done.  Errors: LJ_ERR_ARG, LJ_ERR_BOX, LJ_ERR_CAPACITY (plan_bytes too
 * small), LJ_ERR_CUDA.
 */
int lj_batch_init(lj_batch *batch, const lj_system *systems, int nsys, double dt, int precision,
                  int tpi, int rows_per_item, void *plan_dev, size_t plan_bytes, void *stream);

/* Bytes of device workspace lj_force_batched needs (a work counter; for
 * LJ_MIXED also 16 bytes per atom, for LJ_DFLOAT 32). */
size_t lj_force_batched_workspace_bytes(const lj_batch *batch);

/*
 * p += impulses for every system of the batch (lj_force semantics per
 * system) in one persistent launch: warps take work items from a counter in
 * the workspace until none is left.  Enqueues a memset of the counter, (for
 * LJ_MIXED and LJ_DFLOAT) one pre-pass kernel and the force kernel; no host
 * synchronisation and no allocation, so the call can be captured in a CUDA
 * graph and replayed.  Errors: LJ_ERR_ARG, LJ_ERR_CAPACITY, LJ_ERR_CUDA.
 */
int lj_force_batched(const lj_batch *batch, const double *q4_dev, double *p4_dev,
                     const int32_t *row_ptr_dev, const int32_t *col_dev, void *workspace_dev,
                     size_t workspace_bytes, void *stream);

/* ======================================================================== */
/* Autotuning (host-side; times candidate schedules with CUDA events)       */
/* ======================================================================== */

/*
 * Time lj_force over each candidate schedule in `tpis` (values accepted by
 * lj_force's tpi argument) `reps` times on the given system and list, using
 * p4_scratch_dev as the momentum output (its contents are overwritten), and
 * return the fastest in *best_tpi with its median time in *best_ms.
 * ms_out (host, n_tpi floats, may be NULL) receives every candidate's median.
 * Candidates that the precision does not accept are skipped (time +inf).
 * Synchronous.  Errors as lj_force.
 */
int lj_autotune_force(const double *q4_dev, double *p4_scratch_dev, int64_t n,
                      const int32_t *row_ptr_dev, const int32_t *col_dev, int64_t nnz, int half,
                      double dt, double r_cut, const double box[3], double eps, double sigma,
                      int precision, const int *tpis, int n_tpi, int reps, void *workspace_dev,
                      size_t workspace_bytes, int *best_tpi, float *best_ms, float *ms_out,
                      void *stream);

/*
 * Time lj_force_batched for every (tpi, rows_per_item) pair of the
 * candidate lists (re-initialising the plan in plan_dev for each), `reps`
 * times each, on p4_scratch_dev; return the fastest pair and its median
 * time.  plan_bytes must hold the plan for the smallest rows_per_item and
 * the workspace must be sized for the batch.  Candidates the precision does
 * not accept are skipped (LJ_ERR_ARG if none is left).  Synchronous.
 */
int lj_autotune_batched(const lj_system *systems, int nsys, double dt, int precision,
                        const int *tpis, int n_tpi, const int *rows_per_item, int n_rpi,
                        const double *q4_dev, double *p4_scratch_dev, const int32_t *row_ptr_dev,
                        const int32_t *col_dev, void *plan_dev, size_t plan_bytes,
                        void *workspace_dev, size_t workspace_bytes, int reps, int *best_tpi,
                        int *best_rows_per_item, float *best_ms, void *stream);

/* ======================================================================== */
/* Adjoint of the force map (derived from Eq. 1)                            */
/* ======================================================================== */

/* Bytes of device workspace lj_force_vjp needs. */
size_t lj_force_vjp_workspace_bytes(int64_t n, int precision);

/*
 * Vector-Jacobian product of the force map F(q; eps, sigma), the impulse of
 * lj_force with dt = 1 and p = 0: for each unique pair with
 * s = r^2 < r_cut^2 and g(s) = 24 eps (2 sigma^12 s^-7 - sigma^6 s^-4),
 * F_j += g d, F_i -= g d (d = q_j - q_i, minimum image).  Given
 * R = dLoss/dF (gradF4_dev, n x 4, pad ignored) it writes, with w = R_j - R_i
 * and c = g w + 2 g'(s) (d.w) d per pair:
 *   gradq4_dev          n x 4, overwritten: dLoss/dq (pad set to 0);
 *                       dLoss/dq_j += c, dLoss/dq_i -= c;
 *   grad_eps_sigma_dev  2 device doubles, overwritten:
 *                       dLoss/deps = sum (g/eps)(d.w),
 *                       dLoss/dsigma = sum dg/dsigma (d.w).
 * Full lists gather per row without atomics (deterministic); half lists
 * scatter dLoss/dq_j with FP64 atomics (LJ_FP64 half lists of at least
 * 524,288 rows with a box up to 1024 r_cut wide: each warp takes 32 rows and
 * cuts their entries into one chunk per lane, as LJ_SCHED_STREAM, adding
 * dLoss/dq_i with atomics too).  The scalar sums use a fixed-order
 * reduction.  precision: LJ_FP64, LJ_MIXED (FP32 pair arithmetic,
 * compensated FP32 sums, FP64 outputs) or LJ_DFLOAT (double-float pair
 * arithmetic on the FP32 pipe, FP64-class results; needs |dLoss/dF| within
 * the FP32 range).  Asynchronous.  Errors as lj_force.
 */
int lj_force_vjp(const double *q4_dev, const double *gradF4_dev, int64_t n,
                 const int32_t *row_ptr_dev, const int32_t *col_dev, int64_t nnz, int half,
                 double r_cut, const double box[3], double eps, double sigma, int precision,
                 double *gradq4_dev, double *grad_eps_sigma_dev, void *workspace_dev,
                 size_t workspace_bytes, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* LJ_GB300_H */

/*
 * lj_oracle.c -- plain, slow, double-precision CPU oracle for the truncated
 * Lennard-Jones momentum update over a sorted Verlet pair list.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load this file's library.  It shares no code,
 * header, table or constant with the CUDA library and includes none of it.
 * Compile with -ffp-contract=off so that no multiply-add is fused: every
 * product and sum is a separately rounded IEEE-754 double operation.
 *
 * What it follows (Watanabe & Nakagawa, arXiv 1806.05713):
 *   - Eq. (1): V(r) = 4 eps [ (sigma/r)^12 - (sigma/r)^6 ], truncated at r_c
 *     and optionally shifted so that V(r_c) = 0 (section "Lennard-Jones
 *     Potential").
 *   - Algorithm 1 (force of one pair): r = q_j - q_i, r2, r6 = r2*r2*r2,
 *     r14 = r6*r6*r2, df = (48 - 24 r6) dt / r14, with eps = sigma = 1.  The
 *     printed algorithm gives p_i and p_j the same sign, which breaks
 *     Newton's third law; the oracle reads it as p_i -= df r, p_j += df r.
 *   - Algorithm 3 (sorted list): outer loop over i keeps q_i and p_i, inner
 *     loop over SortedList[i] gathers q_j, tests |r| < r_c, updates p_j,
 *     and stores p_i at the end of the row.
 *   - Section "Verlet List and Bookkeeping Method": the list registers every
 *     pair closer than the search length r_s > r_c; the linked-list (cell)
 *     method builds it in O(N); a counting sort groups j by i.
 *
 * Readings where the paper is silent:
 *   - periodic boundaries with the minimum image (branchy form, per axis:
 *     if d > L/2 then d -= L, else if d < -L/2 then d += L);
 *   - strict inequalities r^2 < r_s^2 (list) and r^2 < r_c^2 (force);
 *   - r^2 = (dx*dx + dy*dy) + dz*dz, left to right;
 *   - half list: pairs with i < j; full list: every j != i;
 *   - general eps, sigma: df = (48 eps sigma^12 - 24 eps sigma^6 r6) dt / r14,
 *     which is -dV/dr / r of Eq. (1) and equals Algorithm 1 at eps=sigma=1.
 *
 * Arrays: positions and momenta are rows of `stride` doubles (x, y, z first).
 * CSR: row_ptr[n+1], col[nnz], 32-bit.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Minimum-image component of the displacement d in a periodic box of side L. */
static double min_image(double d, double L)
{
    double h = 0.5 * L;
    if (d > h)
        d -= L;
    else if (d < -h)
        d += L;
    return d;
}

/* r = q_j - q_i with the minimum image; returns r.r (Algorithm 1, lines 1-2). */
static double displacement(const double *qi, const double *qj, const double *L, double r[3])
{
    for (int a = 0; a < 3; ++a)
        r[a] = min_image(qj[a] - qi[a], L[a]);
    double r2 = r[0] * r[0];
    r2 = r2 + r[1] * r[1];
    r2 = r2 + r[2] * r[2];
    return r2;
}

/* ------------------------------------------------------------------------ */
/* Pair list                                                                 */
/* ------------------------------------------------------------------------ */

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/*
 * O(N^2) definition of the list: every (i, j), j != i (j > i for the half
 * list), with minimum-image r^2 < r_s^2, rows in ascending j.
 * Writes row_ptr[0..n] always and col[] while it fits in `cap`; returns the
 * total number of entries (the caller retries with a larger cap if it
 * exceeds cap).
 */
int64_t oracle_pairlist_brute(int64_t n, const double *q, int64_t stride, const double *L,
                              double rs, int half, int32_t *row_ptr, int32_t *col, int64_t cap)
{
    double rs2 = rs * rs;
    int64_t nnz = 0;
    double r[3];
    for (int64_t i = 0; i < n; ++i) {
        row_ptr[i] = (int32_t)nnz;
        for (int64_t j = (half ? i + 1 : 0); j < n; ++j) {
            if (j == i)
                continue;
            double r2 = displacement(q + i * stride, q + j * stride, L, r);
            if (r2 < rs2) {
                if (nnz < cap)
                    col[nnz] = (int32_t)j;
                ++nnz;
            }
        }
    }
    row_ptr[n] = (int32_t)nnz;
    return nnz;
}

/* Number of cells per axis: the largest count whose cell side is at least
 * r_s (with a relative slack of 1e-12 so that rounding of q*nc/L can never
 * separate two atoms closer than r_s by two cells). */
static int cells_per_axis(double L, double rs)
{
    int nc = (int)floor(L / rs);
    while (nc > 1 && L / nc < rs * (1.0 + 1e-12))
        --nc;
    return nc < 1 ? 1 : nc;
}

/* The distinct neighbour-cell offsets along one axis: {0} for one cell,
 * {0, 1} for two cells (where -1 and +1 are the same cell), else {-1, 0, 1}. */
static int axis_offsets(int nc, int off[3])
{
    if (nc == 1) { off[0] = 0; return 1; }
    if (nc == 2) { off[0] = 0; off[1] = 1; return 2; }
    off[0] = -1; off[1] = 0; off[2] = 1;
    return 3;
}

/*
 * Linked-list cell method (section "Verlet List and Bookkeeping Method"):
 * head[c] is the last atom put in cell c and next[i] the atom put before i;
 * each i scans the atoms of its own and neighbouring cells.  The j of each
 * row are then sorted (the paper's counting sort groups by i; within a row
 * the oracle orders by j so that the list is a canonical sorted set).
 * Same output contract as oracle_pairlist_brute, for the rows i0 .. i1-1
 * only: row_ptr has i1 - i0 + 1 entries (starting at 0) and col the j of
 * those rows (global atom indices).  Every atom is binned; only the listed
 * rows are walked (a bounded sample of a large system).
 */
int64_t oracle_pairlist_cells_rows(int64_t n, const double *q, int64_t stride, const double *L,
                                   double rs, int half, int64_t i0, int64_t i1, int32_t *row_ptr,
                                   int32_t *col, int64_t cap)
{
    double rs2 = rs * rs;
    int nc[3], off[3][3], noff[3];
    for (int a = 0; a < 3; ++a) {
        nc[a] = cells_per_axis(L[a], rs);
        noff[a] = axis_offsets(nc[a], off[a]);
    }
    int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    int64_t *head = (int64_t *)malloc(sizeof(int64_t) * ncell);
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    int *cell = (int *)malloc(sizeof(int) * 3 * (n > 0 ? n : 1));
    int32_t *row = (int32_t *)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    for (int64_t c = 0; c < ncell; ++c)
        head[c] = -1;
    for (int64_t i = 0; i < n; ++i) {
        int c3[3];
        for (int a = 0; a < 3; ++a) {
            int c = (int)floor(q[i * stride + a] / L[a] * nc[a]);
            if (c < 0) c = 0;
            if (c >= nc[a]) c = nc[a] - 1;
            c3[a] = c;
            cell[3 * i + a] = c;
        }
        int64_t id = ((int64_t)c3[2] * nc[1] + c3[1]) * nc[0] + c3[0];
        next[i] = head[id];
        head[id] = i;
    }
    int64_t nnz = 0;
    double r[3];
    for (int64_t i = i0; i < i1; ++i) {
        row_ptr[i - i0] = (int32_t)nnz;
        int64_t len = 0;
        for (int oz = 0; oz < noff[2]; ++oz)
            for (int oy = 0; oy < noff[1]; ++oy)
                for (int ox = 0; ox < noff[0]; ++ox) {
                    int cx = (cell[3 * i + 0] + off[0][ox] + nc[0]) % nc[0];
                    int cy = (cell[3 * i + 1] + off[1][oy] + nc[1]) % nc[1];
                    int cz = (cell[3 * i + 2] + off[2][oz] + nc[2]) % nc[2];
                    int64_t id = ((int64_t)cz * nc[1] + cy) * nc[0] + cx;
                    for (int64_t j = head[id]; j >= 0; j = next[j]) {
                        if (j == i || (half && j < i))
                            continue;
                        double r2 = displacement(q + i * stride, q + j * stride, L, r);
                        if (r2 < rs2)
                            row[len++] = (int32_t)j;
                    }
                }
        qsort(row, (size_t)len, sizeof(int32_t), cmp_i32);
        for (int64_t k = 0; k < len; ++k) {
            if (nnz + k < cap)
                col[nnz + k] = row[k];
        }
        nnz += len;
    }
    row_ptr[i1 - i0] = (int32_t)nnz;
    free(head);
    free(next);
    free(cell);
    free(row);
    return nnz;
}

/* The whole list: rows 0 .. n-1 of the cell method above. */
int64_t oracle_pairlist_cells(int64_t n, const double *q, int64_t stride, const double *L,
                              double rs, int half, int32_t *row_ptr, int32_t *col, int64_t cap)
{
    return oracle_pairlist_cells_rows(n, q, stride, L, rs, half, 0, n, row_ptr, col, cap);
}

/* ------------------------------------------------------------------------ */
/* Force (Algorithm 3 with Algorithm 1 inside)                               */
/* ------------------------------------------------------------------------ */

/*
 * p += impulses of one force call.  For a half list (j > i) each entry
 * updates both atoms; for a full list each entry updates only p_i (the pair
 * appears again in row j).  Pairs with r^2 >= r_c^2 (the bookkeeping margin)
 * are skipped.
 */
void oracle_force_rows(int64_t n, const double *q, int64_t qstride, double *p, int64_t pstride,
                       int64_t i0, int64_t i1, const int32_t *row_ptr, const int32_t *col,
                       int half, double dt, double rc, const double *L, double eps, double sigma)
{
    double rc2 = rc * rc;
    double s2 = sigma * sigma;
    double s6 = s2 * s2 * s2;
    double s12 = s6 * s6;
    double c48 = 48.0 * eps * s12;
    double c24 = 24.0 * eps * s6;
    double r[3];
    (void)n;
    for (int64_t i = i0; i < i1; ++i) {
        const double *qi = q + i * qstride;
        double pi[3] = {p[i * pstride + 0], p[i * pstride + 1], p[i * pstride + 2]};
        for (int64_t k = row_ptr[i - i0]; k < row_ptr[i - i0 + 1]; ++k) {
            int64_t j = col[k];
            double r2 = displacement(qi, q + j * qstride, L, r);
            if (r2 < rc2) {
                double r6 = r2 * r2 * r2;
                double r14 = r6 * r6 * r2;
                double df = (c48 - c24 * r6) * dt / r14;
                for (int a = 0; a < 3; ++a)
                    pi[a] -= df * r[a];
                if (half)
                    for (int a = 0; a < 3; ++a)
                        p[j * pstride + a] += df * r[a];
            }
        }
        for (int a = 0; a < 3; ++a)
            p[i * pstride + a] = pi[a];
    }
}

/* One force call over the whole list (rows 0 .. n-1). */
void oracle_force(int64_t n, const double *q, int64_t qstride, double *p, int64_t pstride,
                  const int32_t *row_ptr, const int32_t *col, int half, double dt, double rc,
                  const double *L, double eps, double sigma)
{
    oracle_force_rows(n, q, qstride, p, pstride, 0, n, row_ptr, col, half, dt, rc, L, eps, sigma);
}

/*
 * The momentum change of selected atoms straight from the definition, with
 * no pair list: for each atom i = idx[m], the sum over every other atom j
 * with minimum-image r^2 < r_c^2 of -df r (r = q_j - q_i, Algorithm 1's
 * arithmetic), i.e. what one force call over a complete list adds to p_i,
 * whichever of i and j owns the pair in a half list.  O(n) per atom: it
 * checks sampled atoms of systems too large for the O(N) list to be built
 * on the CPU in seconds.  out: m rows of 3 doubles.
 */
void oracle_force_atoms(int64_t n, const double *q, int64_t qstride, const double *L, double dt,
                        double rc, double eps, double sigma, const int64_t *idx, int64_t m,
                        double *out)
{
    double rc2 = rc * rc;
    double s2 = sigma * sigma;
    double s6 = s2 * s2 * s2;
    double s12 = s6 * s6;
    double c48 = 48.0 * eps * s12;
    double c24 = 24.0 * eps * s6;
    double r[3];
    for (int64_t t = 0; t < m; ++t) {
        int64_t i = idx[t];
        const double *qi = q + i * qstride;
        double pi[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < n; ++j) {
            if (j == i)
                continue;
            double r2 = displacement(qi, q + j * qstride, L, r);
            if (r2 < rc2) {
                double r6 = r2 * r2 * r2;
                double r14 = r6 * r6 * r2;
                double df = (c48 - c24 * r6) * dt / r14;
                for (int a = 0; a < 3; ++a)
                    pi[a] -= df * r[a];
            }
        }
        for (int a = 0; a < 3; ++a)
            out[3 * t + a] = pi[a];
    }
}

/* ------------------------------------------------------------------------ */
/* Energy (Eq. 1, truncated, optionally shifted)                             */
/* ------------------------------------------------------------------------ */

static double lj_v(double r2, double eps, double sigma)
{
    double sr2 = sigma * sigma / r2;
    double sr6 = sr2 * sr2 * sr2;
    return 4.0 * eps * (sr6 * sr6 - sr6);
}

/* Sum over unique pairs with r < r_c of V(r) - shifted*V(r_c).  For a full
 * list only the entries with j > i are counted, so each pair counts once. */
double oracle_energy(int64_t n, const double *q, int64_t qstride, const int32_t *row_ptr,
                     const int32_t *col, int half, double rc, const double *L, double eps,
                     double sigma, int shifted)
{
    double rc2 = rc * rc;
    double vshift = shifted ? lj_v(rc2, eps, sigma) : 0.0;
    double e = 0.0;
    double r[3];
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            int64_t j = col[k];
            if (!half && j < i)
                continue;
            double r2 = displacement(q + i * qstride, q + j * qstride, L, r);
            if (r2 < rc2)
                e += lj_v(r2, eps, sigma) - vshift;
        }
    }
    (void)half;
    return e;
}

/*
 * (Not in the paper; the by-product its bookkeeping MD needs for pressure.)
 * The pair virial of the truncated Eq. (1): W = sum over unique pairs with
 * r < r_c of r F(r), F(r) = -dV/dr = 24 eps (2 (sigma/r)^12 - (sigma/r)^6) / r
 * (positive when repulsive), so W = sum 24 eps (2 (sigma/r)^12 - (sigma/r)^6).
 * With the kinetic energy K, the pressure of the box is (2 K + W) / (3 V).
 */
double oracle_virial(int64_t n, const double *q, int64_t qstride, const int32_t *row_ptr,
                     const int32_t *col, int half, double rc, const double *L, double eps,
                     double sigma)
{
    double rc2 = rc * rc;
    double w = 0.0;
    double r[3];
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            int64_t j = col[k];
            if (!half && j < i)
                continue;
            double r2 = displacement(q + i * qstride, q + j * qstride, L, r);
            if (r2 < rc2) {
                double sr2 = sigma * sigma / r2;
                double sr6 = sr2 * sr2 * sr2;
                w += 24.0 * eps * (2.0 * sr6 * sr6 - sr6);
            }
        }
    }
    return w;
}

/* ------------------------------------------------------------------------ */
/* Force-shifted truncation                                                  */
/* ------------------------------------------------------------------------ */

/*
 * The smooth truncation the paper recommends for energy conservation but
 * does not use (section "Lennard-Jones Potential"): for r < r_c
 *   V_fs(r) = V(r) - V(r_c) - (r - r_c) V'(r_c),
 * whose pair force -V_fs'(r) = -V'(r) + V'(r_c) goes to zero at r_c.  With
 * F_c = -V'(r_c) = 24 eps (2 sigma^12 / r_c^13 - sigma^6 / r_c^7), the
 * impulse coefficient of a pair is the plain one minus F_c dt / r:
 *   df_fs = df - F_c dt / r,   p_i -= df_fs r_vec,  p_j += df_fs r_vec.
 */
static double lj_fc(double rc, double eps, double sigma)
{
    double sr = sigma / rc;
    double sr2 = sr * sr;
    double sr6 = sr2 * sr2 * sr2;
    return 24.0 * eps * (2.0 * sr6 * sr6 - sr6) / rc;
}

void oracle_force_fs(int64_t n, const double *q, int64_t qstride, double *p, int64_t pstride,
                     const int32_t *row_ptr, const int32_t *col, int half, double dt, double rc,
                     const double *L, double eps, double sigma)
{
    double rc2 = rc * rc;
    double s2 = sigma * sigma;
    double s6 = s2 * s2 * s2;
    double s12 = s6 * s6;
    double c48 = 48.0 * eps * s12;
    double c24 = 24.0 * eps * s6;
    double fc = lj_fc(rc, eps, sigma);
    double r[3];
    for (int64_t i = 0; i < n; ++i) {
        const double *qi = q + i * qstride;
        double pi[3] = {p[i * pstride + 0], p[i * pstride + 1], p[i * pstride + 2]};
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            int64_t j = col[k];
            double r2 = displacement(qi, q + j * qstride, L, r);
            if (r2 < rc2) {
                double r6 = r2 * r2 * r2;
                double r14 = r6 * r6 * r2;
                double df = (c48 - c24 * r6) * dt / r14 - fc * dt / sqrt(r2);
                for (int a = 0; a < 3; ++a)
                    pi[a] -= df * r[a];
                if (half)
                    for (int a = 0; a < 3; ++a)
                        p[j * pstride + a] += df * r[a];
            }
        }
        for (int a = 0; a < 3; ++a)
            p[i * pstride + a] = pi[a];
    }
}

/* Sum over unique pairs with r < r_c of V_fs(r). */
double oracle_energy_fs(int64_t n, const double *q, int64_t qstride, const int32_t *row_ptr,
                        const int32_t *col, int half, double rc, const double *L, double eps,
                        double sigma)
{
    double rc2 = rc * rc;
    double vc = lj_v(rc2, eps, sigma);
    double fc = lj_fc(rc, eps, sigma);
    double e = 0.0;
    double r[3];
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            int64_t j = col[k];
            if (!half && j < i)
                continue;
            double r2 = displacement(q + i * qstride, q + j * qstride, L, r);
            if (r2 < rc2)
                e += lj_v(r2, eps, sigma) - vc + (sqrt(r2) - rc) * fc;
        }
    }
    return e;
}

/* ------------------------------------------------------------------------ */
/* Adjoint of the force map                                                  */
/* ------------------------------------------------------------------------ */

/*
 * Forces F (not impulses): for each unique pair with s = r^2 < r_c^2,
 * F_j += g(s) r and F_i -= g(s) r, where r = q_j - q_i (minimum image) and
 * g(s) = 24 eps (2 sigma^12 s^-7 - sigma^6 s^-4) = -(1/r) dV/dr of Eq. (1).
 *
 * Given R = dLoss/dF (rows of `gstride`), this returns
 *   dLoss/dq (rows of 3, overwritten), and dLoss/deps, dLoss/dsigma in
 *   grad_es[0], grad_es[1] (overwritten).
 * Per pair, with w = R_j - R_i:
 *   c = g w + 2 g'(s) (r.w) r,   dLoss/dq_j += c,  dLoss/dq_i -= c,
 *   dLoss/deps += (dg/deps) (r.w),  dLoss/dsigma += (dg/dsigma) (r.w),
 *   g'(s)      = 24 eps (-14 sigma^12 s^-8 + 4 sigma^6 s^-5),
 *   dg/deps    = g / eps,
 *   dg/dsigma  = 24 eps (24 sigma^11 s^-7 - 6 sigma^5 s^-4).
 * For a full list only entries with j > i are used, so each pair counts once.
 */
void oracle_force_vjp(int64_t n, const double *q, int64_t qstride, const double *R,
                      int64_t gstride, const int32_t *row_ptr, const int32_t *col, int half,
                      double rc, const double *L, double eps, double sigma, double *gq,
                      double *grad_es)
{
    double rc2 = rc * rc;
    double s2 = sigma * sigma;
    double s5 = s2 * s2 * sigma;
    double s6 = s5 * sigma;
    double s11 = s5 * s6;
    double s12 = s6 * s6;
    double ge = 0.0, gs = 0.0;
    double r[3];
    memset(gq, 0, sizeof(double) * 3 * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            int64_t j = col[k];
            if (!half && j < i)
                continue;
            double s = displacement(q + i * qstride, q + j * qstride, L, r);
            if (!(s < rc2))
                continue;
            double si = 1.0 / s;
            double si4 = si * si * si * si;
            double si5 = si4 * si;
            double si7 = si4 * si * si * si;
            double si8 = si7 * si;
            double g = 24.0 * eps * (2.0 * s12 * si7 - s6 * si4);
            double gp = 24.0 * eps * (-14.0 * s12 * si8 + 4.0 * s6 * si5);
            double dg_ds = 24.0 * eps * (24.0 * s11 * si7 - 6.0 * s5 * si4);
            double w[3], rw = 0.0;
            for (int a = 0; a < 3; ++a) {
                w[a] = R[j * gstride + a] - R[i * gstride + a];
                rw += r[a] * w[a];
            }
            for (int a = 0; a < 3; ++a) {
                double c = g * w[a] + 2.0 * gp * rw * r[a];
                gq[3 * j + a] += c;
                gq[3 * i + a] -= c;
            }
            ge += (g / eps) * rw;
            gs += dg_ds * rw;
        }
    }
    grad_es[0] = ge;
    grad_es[1] = gs;
}

/*
 * vlref.c -- FP64 CPU oracle of Vlasiator's spatial translation (paper Section 2.1)
 * and of its Ghost Translation form (Section 3).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the CPU
 * baseline of the benchmark, never by the CUDA path, with which it shares nothing.
 *
 * Written for reading, not speed: every velocity cell is advanced as an independent
 * scalar field on the spatial grid (the translation speed v_d of a velocity cell is
 * constant, Section 2.1), one dimension at a time, with plain loops.
 */
#include "vlref.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------------
 * PPM on one line (Section 2.1: "piece-wise parabolic fitting ... stencil of 2 cells";
 * formulas from Colella & Woodward 1984, eqs. 1.6-1.12)
 * ---------------------------------------------------------------------------- */

/* Value at the face between cells 0 and 1 from the averages of cells -1, 0, 1, 2:
 * the fourth-order interpolant of the cell averages (CW84 eq. 1.6 with the plain
 * centred slope).  With the limiter on, it is clamped into the interval spanned by
 * the two cells that share the face, so that no new extremum is created there. */
double vlref_face(double am1, double a0, double a1, double a2, int limiter)
{
    double f = (7.0 / 12.0) * (a0 + a1) - (1.0 / 12.0) * (am1 + a2);
    if (limiter) {
        double lo = a0 < a1 ? a0 : a1;
        double hi = a0 < a1 ? a1 : a0;
        if (f < lo) f = lo;
        if (f > hi) f = hi;
    }
    return f;
}

/* CW84 monotonicity limiter (eq. 1.10): a cell whose average is a local extremum
 * relative to its edge values becomes flat; otherwise the edge value on the side of
 * the parabola's interior extremum is moved so that the extremum reaches the edge. */
void vlref_limit(double a, double* aL, double* aR)
{
    if ((*aR - a) * (a - *aL) <= 0.0) {
        *aL = a;
        *aR = a;
        return;
    }
    double d = *aR - *aL;
    double m = a - 0.5 * (*aL + *aR);
    if (d * m > d * d / 6.0)
        *aL = 3.0 * a - 2.0 * (*aR);
    else if (d * m < -(d * d) / 6.0)
        *aR = 3.0 * a - 2.0 * (*aL);
}

/* Mass that leaves a cell through its downwind face in one sweep: the integral of the
 * cell's parabola a(xi) = aL + xi (da + a6 (1 - xi)), xi in [0,1], over the fraction
 * |c| of the cell next to the downwind face (CW84 eq. 1.12).  c > 0 moves content to
 * the right neighbour, c < 0 to the left one; |c| <= 1 so one face neighbour receives
 * everything that leaves (Section 2.1). */
double vlref_outflow(double aL, double a, double aR, double c)
{
    double da = aR - aL;
    double a6 = 6.0 * (a - 0.5 * (aL + aR));
    if (c >= 0.0)
        return c * (aR - 0.5 * c * (da - (1.0 - 2.0 * c / 3.0) * a6));
    double g = -c;
    return g * (aL + 0.5 * g * (da + (1.0 - 2.0 * g / 3.0) * a6));
}

/* Outflow of cell j of a line whose averages are a[j-3 .. j+3] (a points at cell 0). */
static double outflow_at(const double* a, long j, double c, int limiter)
{
    double aL = vlref_face(a[j - 2], a[j - 1], a[j], a[j + 1], limiter);
    double aR = vlref_face(a[j - 1], a[j], a[j + 1], a[j + 2], limiter);
    if (limiter)
        vlref_limit(a[j], &aL, &aR);
    return vlref_outflow(aL, a[j], aR, c);
}

/* New averages of cells lo..hi-1 of a line: each cell keeps what does not leave it and
 * receives what leaves its upwind neighbour (mass-conserving remap, Section 2.1).
 * a must be readable on [lo-3, hi+3); out is written on [lo, hi). flux is scratch of
 * hi-lo+2 values. */
static void remap_range(const double* a, double* out, long lo, long hi, double c,
                        int limiter, double* flux)
{
    for (long j = lo - 1; j <= hi; j++)
        flux[j - (lo - 1)] = outflow_at(a, j, c, limiter);
    for (long i = lo; i < hi; i++) {
        double own = flux[i - (lo - 1)];
        double upwind = c >= 0.0 ? flux[i - 1 - (lo - 1)] : flux[i + 1 - (lo - 1)];
        out[i] = a[i] - own + upwind;
    }
}

int vlref_sweep_line(int n, int periodic, const double* in, double* out, double c, int limiter)
{
    if (n <= 0 || !in || !out) return 1;
    if (fabs(c) > 1.0) return 2;
    double* ext = (double*)malloc(sizeof(double) * (size_t)(n + 6));
    double* flux = (double*)malloc(sizeof(double) * (size_t)(n + 2));
    for (long j = -3; j < n + 3; j++) {
        double v;
        if (periodic) v = in[((j % n) + n) % n];
        else v = (j >= 0 && j < n) ? in[j] : 0.0;
        ext[j + 3] = v;
    }
    double* res = (double*)malloc(sizeof(double) * (size_t)(n + 6));
    remap_range(ext + 3, res + 3, 0, n, c, limiter, flux);
    memcpy(out, res + 3, sizeof(double) * (size_t)n);
    free(res);
    free(flux);
    free(ext);
    return 0;
}

/* ------------------------------------------------------------------------------
 * One scalar field on a box (one velocity cell of the phase space)
 * ---------------------------------------------------------------------------- */

static long cell_index(const int n[3], long x, long y, long z)
{
    return x + (long)n[0] * (y + (long)n[1] * z);
}

/* One Cartesian shear of the whole field along dim (Section 2.1). */
static void sweep_field(const int n[3], int periodic, const double* in, double* out, int dim,
                        double c, int limiter, double* line, double* res, double* flux)
{
    int o1 = (dim + 1) % 3, o2 = (dim + 2) % 3;
    long nd = n[dim];
    for (long p = 0; p < n[o2]; p++)
        for (long q = 0; q < n[o1]; q++) {
            long pos[3];
            pos[o1] = q;
            pos[o2] = p;
            for (long j = -3; j < nd + 3; j++) {
                long jj = j;
                double v = 0.0;
                if (periodic) jj = ((j % nd) + nd) % nd;
                if (jj >= 0 && jj < nd) {
                    pos[dim] = jj;
                    v = in[cell_index(n, pos[0], pos[1], pos[2])];
                }
                line[j + 3] = v;
            }
            remap_range(line + 3, res + 3, 0, nd, c, limiter, flux);
            for (long j = 0; j < nd; j++) {
                pos[dim] = j;
                out[cell_index(n, pos[0], pos[1], pos[2])] = res[j + 3];
            }
        }
}

static long max3l(const int n[3])
{
    long m = n[0];
    if (n[1] > m) m = n[1];
    if (n[2] > m) m = n[2];
    return m;
}

int vlref_sweep_field(const int n[3], int periodic, const double* in, double* out, int dim,
                      double c, int limiter)
{
    if (!n || n[0] <= 0 || n[1] <= 0 || n[2] <= 0 || dim < 0 || dim > 2) return 1;
    if (fabs(c) > 1.0) return 2;
    long m = max3l(n) + 6;
    double* line = (double*)malloc(sizeof(double) * (size_t)m);
    double* res = (double*)malloc(sizeof(double) * (size_t)m);
    double* flux = (double*)malloc(sizeof(double) * (size_t)m);
    sweep_field(n, periodic, in, out, dim, c, limiter, line, res, flux);
    free(flux);
    free(res);
    free(line);
    return 0;
}

static int valid_order(const int order[3])
{
    if (!order) return 0;
    int seen[3] = {0, 0, 0};
    for (int j = 0; j < 3; j++) {
        if (order[j] < 0 || order[j] > 2 || seen[order[j]]) return 0;
        seen[order[j]] = 1;
    }
    return 1;
}

/* One translation step of one field: the three shears in the given order, each on the
 * result of the previous one (Section 2.1, the classical form). */
static void step_field(const int n[3], int periodic, double* f, const double c[3],
                       const int order[3], int limiter, double* tmp, double* line,
                       double* res, double* flux)
{
    long total = (long)n[0] * n[1] * n[2];
    for (int j = 0; j < 3; j++) {
        int d = order[j];
        sweep_field(n, periodic, f, tmp, d, c[d], limiter, line, res, flux);
        memcpy(f, tmp, sizeof(double) * (size_t)total);
    }
}

int vlref_step_field(const int n[3], int periodic, double* f, const double c[3],
                     const int order[3], int limiter)
{
    if (!n || n[0] <= 0 || n[1] <= 0 || n[2] <= 0 || !valid_order(order)) return 1;
    for (int d = 0; d < 3; d++)
        if (fabs(c[d]) > 1.0) return 2;
    long total = (long)n[0] * n[1] * n[2];
    long m = max3l(n) + 6;
    double* tmp = (double*)malloc(sizeof(double) * (size_t)total);
    double* line = (double*)malloc(sizeof(double) * (size_t)m);
    double* res = (double*)malloc(sizeof(double) * (size_t)m);
    double* flux = (double*)malloc(sizeof(double) * (size_t)m);
    step_field(n, periodic, f, c, order, limiter, tmp, line, res, flux);
    free(flux);
    free(res);
    free(line);
    free(tmp);
    return 0;
}

/* ------------------------------------------------------------------------------
 * Ghost Translation (Section 3)
 * ---------------------------------------------------------------------------- */

/* Cell sets of Section 3.1 for a box of extents local[] (real numbers allowed, so
 * that the ideal cubic domains of Section 3.3 can be evaluated at any edge length).
 * Walking the sweeps in reverse order d2, d1, d0:
 *   active_2 = local cells and their face neighbours along d2;
 *   source_j = active_j widened by the 2-cell stencil along d_j;
 *   active_j (j < 2) = active_{j+1} widened by k-1 cells along d_{j+1} (GT3: all of
 *   source_{j+1}; GT1: active_{j+1} itself, Section 3.2), plus face neighbours along d_j.
 * Outputs are the volumes of active_j and source_j. */
void vlref_gt_regions(const double local[3], int k, const int order[3], double active[3],
                      double source[3])
{
    double ext[3] = {local[0], local[1], local[2]};
    for (int j = 2; j >= 0; j--) {
        int d = order[j];
        if (j < 2) ext[order[j + 1]] += 2.0 * (k - 1);
        ext[d] += 2.0; /* face neighbours along d_j */
        active[j] = ext[0] * ext[1] * ext[2];
        double s[3] = {ext[0], ext[1], ext[2]};
        s[d] += 4.0; /* +-2 stencil along d_j */
        source[j] = s[0] * s[1] * s[2];
    }
}

/* Gather-form update regions of the GT-k tiled step, as half-widths around the box
 * along each dimension.  A cell's new value is computed from its own outflow and its
 * upwind neighbour's, so the cells that must hold correct values after sweep j are:
 * after d2, the local box; after d1, the local box widened by k along d2; after d0,
 * that region widened by k along d1.  Widening each by one face neighbour along the
 * sweep's own dimension gives exactly active_j above; for k = 3 these are the
 * source_{j+1} sets, so every stencil value of every later sweep is up to date. */
static void gt_update_halfwidths(int k, const int order[3], int hw[3][3])
{
    for (int j = 0; j < 3; j++)
        for (int d = 0; d < 3; d++) hw[j][d] = 0;
    hw[1][order[2]] = k;
    hw[0][order[2]] = k;
    hw[0][order[1]] = k;
}

/* GT-k step of one periodic field, box by box.  Each box loads itself plus a ghost
 * layer of 3 cells per side from the pre-step field in one go (the single coalesced
 * ghost update of Section 3), runs the three sweeps on its update regions only (cells
 * outside keep the values they were loaded with, Section 3.2), and writes its local
 * cells back.  Boxes that do not divide the grid are ragged at the high end.
 * box[d] = 0 makes every box span the whole periodic axis d with no neighbour along
 * it: all cells along d are local, so its ghost layer only mirrors the box's own
 * cells and is refreshed from them after every sweep (a domain that wraps onto itself
 * has nothing to exchange along that axis). */
static void refresh_wrapped_ghosts(double* buf, const long e[3], const long ext[3], int d, int H)
{
    long pos[3];
    for (pos[2] = 0; pos[2] < e[2]; pos[2]++)
        for (pos[1] = 0; pos[1] < e[1]; pos[1]++)
            for (pos[0] = 0; pos[0] < e[0]; pos[0]++) {
                long t = pos[d] - H;
                if (t >= 0 && t < ext[d]) continue;
                long src[3] = {pos[0], pos[1], pos[2]};
                src[d] = ((t % ext[d]) + ext[d]) % ext[d] + H;
                buf[pos[0] + e[0] * (pos[1] + e[1] * pos[2])] = buf[src[0] + e[0] * (src[1] + e[1] * src[2])];
            }
}

int vlref_step_field_gt(const int n[3], double* f, const double c[3], const int order[3],
                        int limiter, int k, const int box_in[3])
{
    if (!n || n[0] <= 0 || n[1] <= 0 || n[2] <= 0 || !valid_order(order)) return 1;
    if (k < 1 || k > 3 || !box_in || box_in[0] < 0 || box_in[1] < 0 || box_in[2] < 0) return 1;
    int box[3], whole[3];
    for (int d = 0; d < 3; d++) {
        whole[d] = box_in[d] == 0;
        box[d] = whole[d] ? n[d] : box_in[d];
    }
    for (int d = 0; d < 3; d++)
        if (fabs(c[d]) > 1.0) return 2;
    const int H = 3;
    long total = (long)n[0] * n[1] * n[2];
    double* pre = (double*)malloc(sizeof(double) * (size_t)total);
    memcpy(pre, f, sizeof(double) * (size_t)total);
    int hw[3][3];
    gt_update_halfwidths(k, order, hw);
    long e[3] = {box[0] + 2 * H, box[1] + 2 * H, box[2] + 2 * H};
    long esz = e[0] * e[1] * e[2];
    double* buf = (double*)calloc((size_t)esz, sizeof(double));
    double* nxt = (double*)calloc((size_t)esz, sizeof(double));
    long m = e[0] > e[1] ? e[0] : e[1];
    if (e[2] > m) m = e[2];
    double* line = (double*)malloc(sizeof(double) * (size_t)m);
    double* res = (double*)malloc(sizeof(double) * (size_t)m);
    double* flux = (double*)malloc(sizeof(double) * (size_t)m);

    for (long bz = 0; bz < n[2]; bz += box[2])
        for (long by = 0; by < n[1]; by += box[1])
            for (long bx = 0; bx < n[0]; bx += box[0]) {
                long org[3] = {bx, by, bz};
                long ext[3];
                for (int d = 0; d < 3; d++) {
                    ext[d] = n[d] - org[d];
                    if (ext[d] > box[d]) ext[d] = box[d];
                }
                /* load local + ghost layer (periodic wrap) */
                for (long z = -H; z < ext[2] + H; z++)
                    for (long y = -H; y < ext[1] + H; y++)
                        for (long x = -H; x < ext[0] + H; x++) {
                            long gx = ((org[0] + x) % n[0] + n[0]) % n[0];
                            long gy = ((org[1] + y) % n[1] + n[1]) % n[1];
                            long gz = ((org[2] + z) % n[2] + n[2]) % n[2];
                            buf[(x + H) + e[0] * ((y + H) + e[1] * (z + H))] =
                                pre[cell_index(n, gx, gy, gz)];
                        }
                for (int j = 0; j < 3; j++) {
                    int d = order[j];
                    int o1 = (d + 1) % 3, o2 = (d + 2) % 3;
                    memcpy(nxt, buf, sizeof(double) * (size_t)esz);
                    long lo[3], hi[3];
                    for (int q = 0; q < 3; q++) {
                        lo[q] = -hw[j][q];
                        hi[q] = ext[q] + hw[j][q];
                    }
                    for (long p = lo[o2]; p < hi[o2]; p++)
                        for (long q = lo[o1]; q < hi[o1]; q++) {
                            long pos[3];
                            pos[o1] = q + H;
                            pos[o2] = p + H;
                            for (long t = 0; t < e[d]; t++) {
                                pos[d] = t;
                                line[t] = buf[pos[0] + e[0] * (pos[1] + e[1] * pos[2])];
                            }
                            /* line[t] holds box coordinate t - H along d */
                            remap_range(line + H, res + H, lo[d], hi[d], c[d], limiter, flux);
                            for (long t = lo[d]; t < hi[d]; t++) {
                                pos[d] = t + H;
                                nxt[pos[0] + e[0] * (pos[1] + e[1] * pos[2])] = res[t + H];
                            }
                        }
                    double* sw = buf;
                    buf = nxt;
                    nxt = sw;
                    for (int q = 0; q < 3; q++)
                        if (whole[q]) refresh_wrapped_ghosts(buf, e, ext, q, H);
                }
                for (long z = 0; z < ext[2]; z++)
                    for (long y = 0; y < ext[1]; y++)
                        for (long x = 0; x < ext[0]; x++)
                            f[cell_index(n, org[0] + x, org[1] + y, org[2] + z)] =
                                buf[(x + H) + e[0] * ((y + H) + e[1] * (z + H))];
            }
    free(flux);
    free(res);
    free(line);
    free(nxt);
    free(buf);
    free(pre);
    return 0;
}

/* ------------------------------------------------------------------------------
 * Sparse velocity space (Section 2: 64-element blocks added where necessary and
 * removed where the density falls below the sparsity threshold)
 * ---------------------------------------------------------------------------- */

/* Block set each cell needs before a step: every block present in any cell of its
 * 3x3x3 neighbourhood.  Content moves at most one face neighbour per sweep
 * (|c| <= 1, Section 2.1), so after the three sweeps a block can only have arrived
 * from within one cell in each dimension; new blocks start at zero.  Open boxes
 * (periodic = 0) have no neighbours outside.  With ids_u == NULL only the offsets
 * (off_u, ncells+1 entries) are written; ids come out sorted per cell. */
int vlref_union(const int n[3], int periodic, int64_t nb, const int64_t* off_in,
                const uint16_t* ids_in, int64_t* off_u, uint16_t* ids_u)
{
    if (!n || n[0] <= 0 || n[1] <= 0 || n[2] <= 0 || nb <= 0 || nb > 65536) return 1;
    if (!off_in || !off_u) return 1;
    unsigned char* mark = (unsigned char*)calloc((size_t)nb, 1);
    int64_t pos = 0;
    off_u[0] = 0;
    for (long z = 0; z < n[2]; z++)
        for (long y = 0; y < n[1]; y++)
            for (long x = 0; x < n[0]; x++) {
                memset(mark, 0, (size_t)nb);
                for (int dz = -1; dz <= 1; dz++)
                    for (int dy = -1; dy <= 1; dy++)
                        for (int dx = -1; dx <= 1; dx++) {
                            long q[3] = {x + dx, y + dy, z + dz};
                            int inside = 1;
                            for (int d = 0; d < 3; d++) {
                                if (periodic) q[d] = ((q[d] % n[d]) + n[d]) % n[d];
                                else if (q[d] < 0 || q[d] >= n[d]) inside = 0;
                            }
                            if (!inside) continue;
                            long cq = cell_index(n, q[0], q[1], q[2]);
                            for (int64_t t = off_in[cq]; t < off_in[cq + 1]; t++) mark[ids_in[t]] = 1;
                        }
                for (int64_t b = 0; b < nb; b++)
                    if (mark[b]) {
                        if (ids_u) ids_u[pos] = (uint16_t)b;
                        pos++;
                    }
                off_u[cell_index(n, x, y, z) + 1] = pos;
            }
    free(mark);
    return 0;
}

/* Per block id, the list of (cell, row) pairs of a per-cell block layout. */
typedef struct {
    int64_t* start; /* nb + 1 */
    int64_t* cell;
    int64_t* row;
} by_id_t;

static void index_by_id(long ncell, int64_t nb, const int64_t* off, const uint16_t* ids,
                        by_id_t* ix)
{
    int64_t total = off[ncell];
    ix->start = (int64_t*)calloc((size_t)nb + 1, sizeof(int64_t));
    ix->cell = (int64_t*)malloc(sizeof(int64_t) * (size_t)(total > 0 ? total : 1));
    ix->row = (int64_t*)malloc(sizeof(int64_t) * (size_t)(total > 0 ? total : 1));
    for (int64_t t = 0; t < total; t++) ix->start[ids[t] + 1]++;
    for (int64_t b = 0; b < nb; b++) ix->start[b + 1] += ix->start[b];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)nb);
    memcpy(fill, ix->start, sizeof(int64_t) * (size_t)nb);
    for (long c = 0; c < ncell; c++)
        for (int64_t t = off[c]; t < off[c + 1]; t++) {
            int64_t k = fill[ids[t]]++;
            ix->cell[k] = c;
            ix->row[k] = t;
        }
    free(fill);
}

static void free_index(by_id_t* ix)
{
    free(ix->start);
    free(ix->cell);
    free(ix->row);
}

/* One translation step of the sparse phase space.  The input blocks (off_in/ids_in/
 * val_in, 64 values per block) are advanced into the caller-allocated union layout
 * (off_u/ids_u/val_u, from vlref_union).  Each of the 64 velocity cells of each block
 * id is one scalar field on the box, zero where the block is absent, advanced by the
 * three shears; its values are then stored into the cells whose union set holds that
 * id.  Anything left in cells outside the union (nothing, with the limiter on and
 * f >= 0, since a flat zero cell sends nothing) is added to *leaked.
 * gt_k = 0 uses the sweep-by-sweep form; 1..3 the tiled GT-k form with boxes gt_box
 * (periodic boxes only). */
int vlref_translate(const int n[3], int periodic, const double dx[3], const int nv[3],
                    const double vmin[3], const double dv[3], double dt, const int order[3],
                    int limiter, int gt_k, const int gt_box[3], const int64_t* off_in,
                    const uint16_t* ids_in, const double* val_in, const int64_t* off_u,
                    const uint16_t* ids_u, double* val_u, double* leaked, int nthreads)
{
    if (!n || n[0] <= 0 || n[1] <= 0 || n[2] <= 0 || !valid_order(order)) return 1;
    for (int d = 0; d < 3; d++)
        if (nv[d] <= 0 || nv[d] % 4 != 0 || dx[d] <= 0.0 || dv[d] <= 0.0) return 1;
    if (gt_k < 0 || gt_k > 3 || (gt_k > 0 && !periodic)) return 1;
    /* Section 2.1: the step must keep every velocity cell within one face neighbour */
    for (int d = 0; d < 3; d++) {
        double vlo = fabs(vmin[d] + 0.5 * dv[d]);
        double vhi = fabs(vmin[d] + (nv[d] - 0.5) * dv[d]);
        double vmax = vlo > vhi ? vlo : vhi;
        if (vmax * dt / dx[d] > 1.0) return 2;
    }
    long ncell = (long)n[0] * n[1] * n[2];
    int nbx = nv[0] / 4, nby = nv[1] / 4, nbz = nv[2] / 4;
    int64_t nb = (int64_t)nbx * nby * nbz;
    by_id_t in_ix, u_ix;
    index_by_id(ncell, nb, off_in, ids_in, &in_ix);
    index_by_id(ncell, nb, off_u, ids_u, &u_ix);
    double leak = 0.0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) reduction(+ : leak)
#endif
    for (int64_t b = 0; b < nb; b++) {
        if (u_ix.start[b] == u_ix.start[b + 1] && in_ix.start[b] == in_ix.start[b + 1]) continue;
        int bx = (int)(b % nbx), by = (int)((b / nbx) % nby), bz = (int)(b / ((int64_t)nbx * nby));
        double* field = (double*)malloc(sizeof(double) * (size_t)ncell);
        unsigned char* inu = (unsigned char*)calloc((size_t)ncell, 1);
        for (int64_t k = u_ix.start[b]; k < u_ix.start[b + 1]; k++) inu[u_ix.cell[k]] = 1;
        long m = max3l(n) + 6;
        double* tmp = (double*)malloc(sizeof(double) * (size_t)ncell);
        double* line = (double*)malloc(sizeof(double) * (size_t)m);
        double* res = (double*)malloc(sizeof(double) * (size_t)m);
        double* flux = (double*)malloc(sizeof(double) * (size_t)m);
        for (int v = 0; v < 64; v++) {
            int iv[3] = {bx * 4 + (v & 3), by * 4 + ((v >> 2) & 3), bz * 4 + (v >> 4)};
            double c[3];
            for (int d = 0; d < 3; d++) {
                double vel = vmin[d] + (iv[d] + 0.5) * dv[d];
                c[d] = vel * dt / dx[d];
            }
            memset(field, 0, sizeof(double) * (size_t)ncell);
            for (int64_t k = in_ix.start[b]; k < in_ix.start[b + 1]; k++)
                field[in_ix.cell[k]] = val_in[in_ix.row[k] * 64 + v];
            if (gt_k == 0)
                step_field(n, periodic, field, c, order, limiter, tmp, line, res, flux);
            else
                vlref_step_field_gt(n, field, c, order, limiter, gt_k, gt_box);
            for (int64_t k = u_ix.start[b]; k < u_ix.start[b + 1]; k++)
                val_u[u_ix.row[k] * 64 + v] = field[u_ix.cell[k]];
            for (long cc = 0; cc < ncell; cc++)
                if (!inu[cc]) leak += fabs(field[cc]);
        }
        free(flux);
        free(res);
        free(line);
        free(tmp);
        free(inu);
        free(field);
    }
    free_index(&in_ix);
    free_index(&u_ix);
    if (leaked) *leaked = leak;
    return 0;
}

/* Sparsity rule (Section 2): a block stays iff the largest of its 64 values reaches
 * the threshold (ties stay).  The mass of removed blocks, sum f times the phase-space
 * cell volume, is reported so that conservation can be checked up to it. */
int vlref_prune(int64_t nblocks, const double* val, double threshold, double cell_volume,
                uint8_t* keep, double* dropped_mass)
{
    if (nblocks < 0 || (nblocks > 0 && (!val || !keep))) return 1;
    double dropped = 0.0;
    for (int64_t t = 0; t < nblocks; t++) {
        double mx = val[t * 64];
        for (int v = 1; v < 64; v++)
            if (val[t * 64 + v] > mx) mx = val[t * 64 + v];
        keep[t] = mx >= threshold ? 1 : 0;
        if (!keep[t])
            for (int v = 0; v < 64; v++) dropped += val[t * 64 + v] * cell_volume;
    }
    if (dropped_mass) *dropped_mass = dropped;
    return 0;
}

/* Total mass: the sum of all cell averages times the phase-space cell volume
 * (dx dy dz dvx dvy dvz). */
double vlref_mass(int64_t nblocks, const double* val, double phase_cell_volume)
{
    double s = 0.0;
    for (int64_t t = 0; t < nblocks * 64; t++) s += val[t];
    return s * phase_cell_volume;
}

/* Velocity moments per spatial cell (particle mass 1): n = sum f dv^3,
 * n V_d = sum v_d f dv^3, P_dd = sum (v_d - V_d)^2 f dv^3.  out holds 7 values per
 * cell: n, nVx, nVy, nVz, Pxx, Pyy, Pzz. */
int vlref_moments(int64_t ncells, const int nv[3], const double vmin[3], const double dv[3],
                  const int64_t* off, const uint16_t* ids, const double* val, double* out)
{
    if (ncells < 0 || !off || !out) return 1;
    int nbx = nv[0] / 4, nby = nv[1] / 4;
    double dv3 = dv[0] * dv[1] * dv[2];
    for (int64_t c = 0; c < ncells; c++) {
        double s[4] = {0, 0, 0, 0};
        for (int64_t t = off[c]; t < off[c + 1]; t++) {
            int b = ids[t];
            int bx = b % nbx, by = (b / nbx) % nby, bz = b / (nbx * nby);
            for (int v = 0; v < 64; v++) {
                double f = val[t * 64 + v];
                double vel[3] = {vmin[0] + (bx * 4 + (v & 3) + 0.5) * dv[0],
                                 vmin[1] + (by * 4 + ((v >> 2) & 3) + 0.5) * dv[1],
                                 vmin[2] + (bz * 4 + (v >> 4) + 0.5) * dv[2]};
                s[0] += f;
                for (int d = 0; d < 3; d++) s[1 + d] += vel[d] * f;
            }
        }
        double nn = s[0] * dv3;
        double V[3];
        for (int d = 0; d < 3; d++) V[d] = nn != 0.0 ? s[1 + d] * dv3 / nn : 0.0;
        double p[3] = {0, 0, 0};
        for (int64_t t = off[c]; t < off[c + 1]; t++) {
            int b = ids[t];
            int bx = b % nbx, by = (b / nbx) % nby, bz = b / (nbx * nby);
            for (int v = 0; v < 64; v++) {
                double f = val[t * 64 + v];
                double vel[3] = {vmin[0] + (bx * 4 + (v & 3) + 0.5) * dv[0],
                                 vmin[1] + (by * 4 + ((v >> 2) & 3) + 0.5) * dv[1],
                                 vmin[2] + (bz * 4 + (v >> 4) + 0.5) * dv[2]};
                for (int d = 0; d < 3; d++) p[d] += (vel[d] - V[d]) * (vel[d] - V[d]) * f;
            }
        }
        out[c * 7 + 0] = nn;
        for (int d = 0; d < 3; d++) out[c * 7 + 1 + d] = s[1 + d] * dv3;
        for (int d = 0; d < 3; d++) out[c * 7 + 4 + d] = p[d] * dv3;
    }
    return 0;
}

int vlref_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * vlref.h -- FP64 CPU oracle of Vlasiator's spatial translation step and of its
 * coalesced-ghost ("Ghost Translation") form.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline of the benchmark may load this library.  It shares no code, header,
 * table or helper with the CUDA path, and the CUDA path never calls it.
 *
 * What it computes (paper sections cited per function in vlref.c):
 *   - Section 2 / Eq. 1: the v . grad_x f part of the Vlasov equation, split into three
 *     Cartesian shears per time step; each shear is a mass-conserving semi-Lagrangian
 *     remap with a piecewise-parabolic (PPM) fit on a stencil of 2 cells, writing to the
 *     cell itself and its downwind face neighbour; |v_d| dt / dx_d <= 1 (Section 2.1).
 *   - The PPM face value, limiter and flux integral are not printed in the paper; they
 *     follow Colella & Woodward (1984), J. Comput. Phys. 54:174, eqs. 1.5-1.12, with a
 *     fourth-order face value clamped between its two neighbours.
 *   - Section 2 (sparse velocity space): 4x4x4 velocity blocks that appear where a
 *     neighbour may send content and vanish below the sparsity threshold.
 *   - Section 3.1-3.3: active/source cell selection in reverse sweep order, the GT-k
 *     region sizes, and the tiled Ghost Translation form.
 *
 * Conventions: spatial cell index c = x + nx*(y + ny*z); block id
 * b = bx + nbx*(by + nby*bz); the 64 values of a block are ordered vx fastest,
 * then vy, then vz.  A velocity cell's speed is taken at its centre,
 * v_d = vmin_d + (i_d + 1/2) dv_d.  All arithmetic is IEEE double; the library is
 * compiled without floating-point contraction so that results are reproducible.
 * Return codes: 0 = ok, 1 = bad argument, 2 = Courant number above 1.
 */
#ifndef VLREF_H
#define VLREF_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- PPM pieces (one dimension) -------------------------------------------- */
double vlref_face(double am1, double a0, double a1, double a2, int limiter);
void   vlref_limit(double a, double* aL, double* aR);
double vlref_outflow(double aL, double a, double aR, double c);

/* One periodic (periodic=1) or open (periodic=0, outside = 0) line of n cells. */
int vlref_sweep_line(int n, int periodic, const double* in, double* out, double c, int limiter);

/* ---- one scalar field (one velocity cell) on an nx*ny*nz box ----------------- */
int vlref_sweep_field(const int n[3], int periodic, const double* in, double* out,
                      int dim, double c, int limiter);
int vlref_step_field(const int n[3], int periodic, double* f, const double c[3],
                     const int order[3], int limiter);
/* GT-k (k = 1..3) tiled step with boxes of extents box[]; box[d] = 0: every box spans
 * the whole periodic axis d and has no ghosts along it. */
int vlref_step_field_gt(const int n[3], double* f, const double c[3], const int order[3],
                        int limiter, int k, const int box[3]);

/* ---- Section 3.1/3.3 region sizes -------------------------------------------- */
void vlref_gt_regions(const double local[3], int k, const int order[3],
                      double active[3], double source[3]);

/* ---- sparse block-structured phase space --------------------------------------- */
int vlref_union(const int n[3], int periodic, int64_t nb,
                const int64_t* off_in, const uint16_t* ids_in,
                int64_t* off_u, uint16_t* ids_u);
int vlref_translate(const int n[3], int periodic, const double dx[3],
                    const int nv[3], const double vmin[3], const double dv[3],
                    double dt, const int order[3], int limiter, int gt_k, const int gt_box[3],
                    const int64_t* off_in, const uint16_t* ids_in, const double* val_in,
                    const int64_t* off_u, const uint16_t* ids_u, double* val_u,
                    double* leaked, int nthreads);
int vlref_prune(int64_t nblocks, const double* val, double threshold, double cell_volume,
                uint8_t* keep, double* dropped_mass);
double vlref_mass(int64_t nblocks, const double* val, double phase_cell_volume);
int vlref_moments(int64_t ncells, const int nv[3], const double vmin[3], const double dv[3],
                  const int64_t* off, const uint16_t* ids, const double* val, double* out);
int vlref_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif

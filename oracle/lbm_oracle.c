/*
 * FP64 CPU oracle for one LBMTau1 time step on the D2Q9 lattice.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke check
 * and the benchmark's CPU-baseline leg may load this library.  It shares no
 * code, header or constant table with the CUDA path.
 *
 * What it computes (Matyka & Dzikowski, arXiv:1912.09327):
 *   - Eq. (LBMTau1): with tau = 1 the post-collision populations are the
 *     equilibria, f_k(x + e_k, t + 1) = f^eq_k(x, t), so only the density R and
 *     the momentum (U, V) of every node are stored (Section 2).
 *   - Eqs. (rhotau1), (utau1): the new moments of a fluid node are the sums of
 *     the equilibria f^eq_ik pulled from its nine neighbours x + e_k, with
 *     i_k the direction opposite to k.
 *   - Eq. (maxwellboltzmann): f^eq_k = w_k rho (1 + 3 e_k.u + 9/2 (e_k.u)^2
 *     - 3/2 u^2).
 *   - Eq. (feqnoslip): when x + e_k is a no-slip (solid) node, the pulled term
 *     is the zero-velocity equilibrium of the node itself, w_k rho(x).
 *   - Algorithm 1: the body force is added to the neighbour's momentum before
 *     the division by its density, u = (U + f_x) / r, v = (V + f_y) / r.
 *
 * Readings where the paper is silent or inconsistent:
 *   - the rest direction k = 0 is part of the sum (the k < 9 loop of the
 *     Appendix A code); the north-wall worked example of Section 2 omits it;
 *   - the moments are accumulated inside the direction loop (Appendix A);
 *     Algorithm 1 prints the three accumulations after its inner loop;
 *   - "(i_p, i_p)" in Algorithm 1 is read as (i_p, j_p);
 *   - U and V hold momentum (rho u), as Eq. (utau1) sums e_k f_k;
 *   - node types: 0 = fluid (updated), 1 = solid (no-slip, never updated),
 *     2 = fixed-equilibrium node such as the moving lid of Section 3 (acts as
 *     a fluid neighbour, never updated, as the lid row of Appendix A);
 *   - an axis marked periodic wraps (the channel of Section 3); on an axis
 *     that is not periodic, a neighbour outside the domain is solid.
 *
 * Layout: every field is row-major, idx = y * nx + x.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { NODE_FLUID = 0, NODE_SOLID = 1, NODE_FIXED = 2 };

/* D2Q9 velocity set in the order of Section 2, the direction inverse to each,
 * and the direction weights (4/9 rest, 1/9 axis, 1/36 diagonal). */
static const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int inv_dir[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double omega[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                                1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                                1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

typedef struct {
  int64_t nx, ny;
  int periodic_x, periodic_y;
  double fx, fy;
  const uint8_t *mask;
} domain;

/* Copies the lattice tables out, so tests can pin them against the paper. */
void oracle_lattice(int32_t *out_ex, int32_t *out_ey, int32_t *out_inv,
                    double *out_w) {
  for (int k = 0; k < 9; ++k) {
    out_ex[k] = ex[k];
    out_ey[k] = ey[k];
    out_inv[k] = inv_dir[k];
    out_w[k] = omega[k];
  }
}

/* Neighbour lookup.  Returns the flat index of (x, y) after periodic wrap, or
 * -1 when the point lies outside a non-periodic edge (treated as solid). */
static int64_t neighbour_index(const domain *d, int64_t x, int64_t y) {
  if (x < 0 || x >= d->nx) {
    if (!d->periodic_x) return -1;
    x = ((x % d->nx) + d->nx) % d->nx;
  }
  if (y < 0 || y >= d->ny) {
    if (!d->periodic_y) return -1;
    y = ((y % d->ny) + d->ny) % d->ny;
  }
  return y * d->nx + x;
}

/* One node of Algorithm 1: the new (R, U, V) of node (x, y) from the old
 * fields.  Nodes that are not fluid keep their old values. */
static void update_node(const domain *d, const double *R, const double *U,
                        const double *V, int64_t x, int64_t y, double *r_out,
                        double *u_out, double *v_out) {
  const int64_t i = y * d->nx + x;
  if (d->mask[i] != NODE_FLUID) {
    *r_out = R[i];
    *u_out = U[i];
    *v_out = V[i];
    return;
  }
  double r_new = 0.0, u_new = 0.0, v_new = 0.0;
  for (int k = 0; k < 9; ++k) {
    const int ik = inv_dir[k];
    const int64_t p = neighbour_index(d, x + ex[k], y + ey[k]);
    double feq;
    if (p >= 0 && d->mask[p] != NODE_SOLID) {
      /* Eq. (maxwellboltzmann) at the neighbour, force added first. */
      const double r = R[p];
      const double u = (U[p] + d->fx) / r;
      const double v = (V[p] + d->fy) / r;
      const double eu = ex[ik] * u + ey[ik] * v;
      feq = omega[ik] * r *
            (1.0 - 1.5 * (u * u + v * v) + 3.0 * eu + 4.5 * eu * eu);
    } else {
      /* Eq. (feqnoslip): zero-velocity equilibrium of this node. */
      feq = omega[k] * R[i];
    }
    r_new += feq;
    u_new += ex[ik] * feq;
    v_new += ey[ik] * feq;
  }
  *r_out = r_new;
  *u_out = u_new;
  *v_out = v_new;
}

static domain make_domain(int64_t nx, int64_t ny, int32_t periodic_x,
                          int32_t periodic_y, double fx, double fy,
                          const uint8_t *mask) {
  domain d;
  d.nx = nx;
  d.ny = ny;
  d.periodic_x = periodic_x != 0;
  d.periodic_y = periodic_y != 0;
  d.fx = fx;
  d.fy = fy;
  d.mask = mask;
  return d;
}

/* One full time step: reads (R0, U0, V0), writes (R1, U1, V1). */
void oracle_step(int64_t nx, int64_t ny, int32_t periodic_x, int32_t periodic_y,
                 double fx, double fy, const uint8_t *mask, const double *R0,
                 const double *U0, const double *V0, double *R1, double *U1,
                 double *V1) {
  const domain d = make_domain(nx, ny, periodic_x, periodic_y, fx, fy, mask);
#pragma omp parallel for schedule(static)
  for (int64_t y = 0; y < ny; ++y)
    for (int64_t x = 0; x < nx; ++x) {
      const int64_t i = y * nx + x;
      update_node(&d, R0, U0, V0, x, y, &R1[i], &U1[i], &V1[i]);
    }
}

/* nsteps time steps in place on (R, U, V), ping-ponging through a scratch
 * copy (the two grids c = 0, 1 of Section 2.1).  Returns 0, or -1 when the
 * scratch copy cannot be allocated. */
int oracle_run(int64_t nx, int64_t ny, int32_t periodic_x, int32_t periodic_y,
               double fx, double fy, const uint8_t *mask, double *R, double *U,
               double *V, int64_t nsteps) {
  const size_t n = (size_t)nx * (size_t)ny;
  double *tmp = (double *)malloc(3 * n * sizeof(double));
  if (!tmp) return -1;
  double *src[3] = {R, U, V};
  double *dst[3] = {tmp, tmp + n, tmp + 2 * n};
  for (int64_t s = 0; s < nsteps; ++s) {
    oracle_step(nx, ny, periodic_x, periodic_y, fx, fy, mask, src[0], src[1],
                src[2], dst[0], dst[1], dst[2]);
    for (int f = 0; f < 3; ++f) {
      double *t = src[f];
      src[f] = dst[f];
      dst[f] = t;
    }
  }
  if (src[0] != R)
    for (int f = 0; f < 3; ++f) memcpy(dst[f], src[f], n * sizeof(double));
  free(tmp);
  return 0;
}

/* The new moments of the listed nodes only (flat indices), from the old
 * fields: lets a test check sampled outputs of a domain too large to step
 * whole on the CPU.  out holds 3 * count values (R, U, V per node). */
void oracle_step_nodes(int64_t nx, int64_t ny, int32_t periodic_x,
                       int32_t periodic_y, double fx, double fy,
                       const uint8_t *mask, const double *R0, const double *U0,
                       const double *V0, const int64_t *nodes, int64_t count,
                       double *out) {
  const domain d = make_domain(nx, ny, periodic_x, periodic_y, fx, fy, mask);
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < count; ++j) {
    const int64_t i = nodes[j];
    update_node(&d, R0, U0, V0, i % nx, i / nx, &out[3 * j], &out[3 * j + 1],
                &out[3 * j + 2]);
  }
}

/* ---- Shan-Chen multiphase step (Section 4, Eq. f_sc) ----
 *
 * Section 4 adds the pseudo-potential interaction force
 *   F_SC(x) = psi(x) sum_i alpha_i psi(x + e_i) G(e_i)        (Eq. f_sc)
 * to the step: with tau = 1 the populations leaving a node are the
 * equilibria of its density and of its velocity shifted by the force, so
 * F_SC enters exactly where Algorithm 1 adds the body force, before the
 * division by the density.  (Kupershtokh's exact-difference forcing, which
 * the paper's performance test uses, adds f^eq(rho, u + F / rho) -
 * f^eq(rho, u) to the collision; at tau = 1 that is the same shift.)
 * The paper leaves psi, alpha_i and G(e_i) to the model of Shan and Chen;
 * the readings taken here are that model's own:
 *   psi(rho) = 1 - exp(-rho),  alpha_i = w_i,  G(e_i) = -g e_i,
 * so F_SC(x) = -g psi(x) sum_i w_i psi(x + e_i) e_i, with a scalar coupling
 * g (g < -4 separates phases).  A solid node, or a point outside a
 * non-periodic edge, has psi = 0.  The rest of the step is Algorithm 1 as in
 * update_node above; the force on every pulled neighbour needs the
 * potentials of that neighbour's own neighbours, the two-fold loop that
 * Section 3 names. */

/* psi of flat index p (-1: outside a non-periodic edge). */
static double sc_psi(const domain *d, const double *R, int64_t p) {
  if (p < 0 || d->mask[p] == NODE_SOLID) return 0.0;
  return 1.0 - exp(-R[p]);
}

/* Eq. (f_sc) at node (x, y): the inner loop over its neighbours. */
static void sc_force(const domain *d, double g, const double *R, int64_t x,
                     int64_t y, double *fsx, double *fsy) {
  double sx = 0.0, sy = 0.0;
  for (int i = 0; i < 9; ++i) {
    const double ps = sc_psi(d, R, neighbour_index(d, x + ex[i], y + ey[i]));
    sx += omega[i] * ps * ex[i];
    sy += omega[i] * ps * ey[i];
  }
  const double own = sc_psi(d, R, y * d->nx + x);
  *fsx = -g * own * sx;
  *fsy = -g * own * sy;
}

/* One node of the multiphase step: as update_node, with F_SC of each pulled
 * neighbour added to its momentum beside the body force. */
static void update_node_sc(const domain *d, double g, const double *R,
                           const double *U, const double *V, int64_t x,
                           int64_t y, double *r_out, double *u_out,
                           double *v_out) {
  const int64_t i = y * d->nx + x;
  if (d->mask[i] != NODE_FLUID) {
    *r_out = R[i];
    *u_out = U[i];
    *v_out = V[i];
    return;
  }
  double r_new = 0.0, u_new = 0.0, v_new = 0.0;
  for (int k = 0; k < 9; ++k) {
    const int ik = inv_dir[k];
    const int64_t px = x + ex[k], py = y + ey[k];
    const int64_t p = neighbour_index(d, px, py);
    double feq;
    if (p >= 0 && d->mask[p] != NODE_SOLID) {
      double fsx, fsy;
      sc_force(d, g, R, p % d->nx, p / d->nx, &fsx, &fsy);
      const double r = R[p];
      const double u = (U[p] + d->fx + fsx) / r;
      const double v = (V[p] + d->fy + fsy) / r;
      const double eu = ex[ik] * u + ey[ik] * v;
      feq = omega[ik] * r *
            (1.0 - 1.5 * (u * u + v * v) + 3.0 * eu + 4.5 * eu * eu);
    } else {
      feq = omega[k] * R[i];
    }
    r_new += feq;
    u_new += ex[ik] * feq;
    v_new += ey[ik] * feq;
  }
  *r_out = r_new;
  *u_out = u_new;
  *v_out = v_new;
}

/* One multiphase time step with coupling g: reads (R0, U0, V0), writes
 * (R1, U1, V1). */
void oracle_step_sc(int64_t nx, int64_t ny, int32_t periodic_x,
                    int32_t periodic_y, double fx, double fy, double g,
                    const uint8_t *mask, const double *R0, const double *U0,
                    const double *V0, double *R1, double *U1, double *V1) {
  const domain d = make_domain(nx, ny, periodic_x, periodic_y, fx, fy, mask);
#pragma omp parallel for schedule(static)
  for (int64_t y = 0; y < ny; ++y)
    for (int64_t x = 0; x < nx; ++x) {
      const int64_t i = y * nx + x;
      update_node_sc(&d, g, R0, U0, V0, x, y, &R1[i], &U1[i], &V1[i]);
    }
}

/* nsteps multiphase steps in place on (R, U, V); 0, or -1 without memory. */
int oracle_run_sc(int64_t nx, int64_t ny, int32_t periodic_x,
                  int32_t periodic_y, double fx, double fy, double g,
                  const uint8_t *mask, double *R, double *U, double *V,
                  int64_t nsteps) {
  const size_t n = (size_t)nx * (size_t)ny;
  double *tmp = (double *)malloc(3 * n * sizeof(double));
  if (!tmp) return -1;
  double *src[3] = {R, U, V};
  double *dst[3] = {tmp, tmp + n, tmp + 2 * n};
  for (int64_t s = 0; s < nsteps; ++s) {
    oracle_step_sc(nx, ny, periodic_x, periodic_y, fx, fy, g, mask, src[0],
                   src[1], src[2], dst[0], dst[1], dst[2]);
    for (int f = 0; f < 3; ++f) {
      double *t = src[f];
      src[f] = dst[f];
      dst[f] = t;
    }
  }
  if (src[0] != R)
    for (int f = 0; f < 3; ++f) memcpy(dst[f], src[f], n * sizeof(double));
  free(tmp);
  return 0;
}

/* The multiphase force F_SC of every node (0 at nodes that are not fluid or
 * fixed), for tests of its sum and symmetry. */
void oracle_sc_force(int64_t nx, int64_t ny, int32_t periodic_x,
                     int32_t periodic_y, double g, const uint8_t *mask,
                     const double *R, double *FX, double *FY) {
  const domain d = make_domain(nx, ny, periodic_x, periodic_y, 0.0, 0.0, mask);
  for (int64_t y = 0; y < ny; ++y)
    for (int64_t x = 0; x < nx; ++x) {
      const int64_t i = y * nx + x;
      FX[i] = FY[i] = 0.0;
      if (mask[i] != NODE_SOLID) sc_force(&d, g, R, x, y, &FX[i], &FY[i]);
    }
}

/* Steady-state measures over fluid nodes (type 0), velocity u = (U, V) / R:
 *   residual = sqrt(sum |u_new - u_old|^2 / sum |u_new|^2)  (Section 3 uses
 *   the relative velocity change between consecutive steps; here it is taken
 *   over the whole field), or sqrt(sum |u_new - u_old|^2) when the flow is at
 *   rest;  mass = sum R_new. */
void oracle_residual(int64_t n, const uint8_t *mask, const double *R0,
                     const double *U0, const double *V0, const double *R1,
                     const double *U1, const double *V1, double *residual,
                     double *mass) {
  double num = 0.0, den = 0.0, m = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    if (mask[i] != NODE_FLUID) continue;
    const double ux0 = U0[i] / R0[i], uy0 = V0[i] / R0[i];
    const double ux1 = U1[i] / R1[i], uy1 = V1[i] / R1[i];
    num += (ux1 - ux0) * (ux1 - ux0) + (uy1 - uy0) * (uy1 - uy0);
    den += ux1 * ux1 + uy1 * uy1;
    m += R1[i];
  }
  *residual = den > 0.0 ? sqrt(num / den) : sqrt(num);
  *mass = m;
}

void oracle_set_threads(int32_t n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int32_t oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

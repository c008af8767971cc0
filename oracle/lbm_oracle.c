/*
 * FP64 reference ("oracle") of the D2Q9 single-relaxation-time lattice
 * Boltzmann method of Sec. 2.1 of "Hybrid Fourier Neural Operator-Lattice
 * Boltzmann Method" (arXiv 2604.27158), plus the re-initialisation of the
 * populations from macroscopic fields used by the hybrid framework (Sec. 2.3).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, obviously-correct
 * restatement of the method in double precision.  It shares no code, header or
 * table with the CUDA path; only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark call it.
 *
 * Notation follows the paper: f_i populations, f_i^eq equilibrium (Eq. for
 * f_i^eq in Sec. 2.1), f_i^* post-collision populations (SRT collision
 * equation), streaming f_i(x + c_i dt, t + dt) = f_i^*(x, t), moments
 * rho = sum_i f_i and rho u = sum_i c_i f_i.  Lattice units dx = dt = 1.
 *
 * Readings of points the paper leaves open (each restated in the design notes):
 *  - D2Q9 ordering 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1)
 *    7:(-1,-1) 8:(1,-1); weights 4/9, 1/9, 1/36; c_s^2 = 1/3.
 *  - The SRT collision is printed with a "(1 + dt/tau)" factor; it is read as
 *    the standard BGK relaxation f* = f (1 - dt/tau) + f^eq dt/tau (the printed
 *    sign neither conserves mass nor is stable).
 *  - No-slip obstacle walls: halfway bounce-back, f_i(x, t+1) = f*_opp(i)(x, t)
 *    whenever x - c_i is solid.  Solid cells carry no dynamics.
 *  - Inlet / outlet columns (x = 0, x = nx-1) when not periodic: Zou-He
 *    completion of the populations streaming in from outside the domain, with
 *    a prescribed density (pressure) or a prescribed normal velocity (u_y = 0).
 *    Completion is applied to every post-stream state and to the initial
 *    state, i.e. to every state moments are taken from.
 *  - The y direction is always periodic; channel walls are solid mask rows.
 *  - Body force (not in the paper): Guo forcing with a constant force density
 *    F; u = (sum_i c_i f_i + F/2) / rho and source
 *    S_i = (1 - 1/(2 tau)) w_i [3 (c_i - u) + 9 (c_i . u) c_i] . F.
 *  - Re-initialisation: f_i = f_i^eq(rho, u) + f_i^neq with the first-order
 *    Chapman-Enskog estimate f_i^neq = -(tau w_i rho / c_s^2) Q_iab d_a u_b,
 *    Q_iab = c_ia c_ib - c_s^2 delta_ab, derivatives by second-order central
 *    differences, one-sided where a neighbour is solid or outside the domain,
 *    zero where neither neighbour is fluid.  neq_mode = 0 gives f = f^eq.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OL_Q 9

static const int OL_CX[OL_Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int OL_CY[OL_Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OL_OPP[OL_Q] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double OL_W[OL_Q] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                                  1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double OL_CS2 = 1.0 / 3.0;

/* boundary kinds for the x-ends; y is always periodic */
enum { OL_BC_PERIODIC = 0, OL_BC_PRESSURE = 1, OL_BC_VELOCITY = 2 };

typedef struct {
  int nx, ny;
  double tau;
  double fx, fy;        /* body-force density */
  int bc_west, bc_east; /* OL_BC_*; periodic must be set on both ends */
  double west_value;    /* rho (pressure) or u_x (velocity) at x = 0 */
  double east_value;    /* rho (pressure) or u_x (velocity) at x = nx-1 */
} ol_grid;

/* populations are stored f[i][y][x], i.e. f[(i * ny + y) * nx + x] */
static inline size_t ol_idx(const ol_grid* g, int i, int x, int y) {
  return ((size_t)i * g->ny + (size_t)y) * g->nx + (size_t)x;
}
static inline int ol_solid(const ol_grid* g, const uint8_t* solid, int x, int y) {
  return solid[(size_t)y * g->nx + x] != 0;
}
static inline int ol_wrap(int v, int n) { return ((v % n) + n) % n; }

void ol_lattice(int* cx, int* cy, int* opp, double* w) {
  for (int i = 0; i < OL_Q; ++i) {
    cx[i] = OL_CX[i];
    cy[i] = OL_CY[i];
    opp[i] = OL_OPP[i];
    w[i] = OL_W[i];
  }
}

/* f_i^eq (Sec. 2.1): w_i rho (1 + u.c/cs2 + (u.c)^2/(2 cs4) - u.u/(2 cs2)) */
void ol_equilibrium(double rho, double ux, double uy, double* feq) {
  const double uu = ux * ux + uy * uy;
  for (int i = 0; i < OL_Q; ++i) {
    const double cu = ux * OL_CX[i] + uy * OL_CY[i];
    feq[i] = OL_W[i] * rho *
             (1.0 + cu / OL_CS2 + (cu * cu) / (2.0 * OL_CS2 * OL_CS2) - uu / (2.0 * OL_CS2));
  }
}

/* moments (Sec. 2.1) of one cell with the half-force correction of Guo forcing */
static void ol_cell_moments(const ol_grid* g, const double* fc, double* rho, double* ux,
                            double* uy) {
  double r = 0.0, jx = 0.0, jy = 0.0;
  for (int i = 0; i < OL_Q; ++i) {
    r += fc[i];
    jx += OL_CX[i] * fc[i];
    jy += OL_CY[i] * fc[i];
  }
  *rho = r;
  *ux = (jx + 0.5 * g->fx) / r;
  *uy = (jy + 0.5 * g->fy) / r;
}

static void ol_gather(const ol_grid* g, const double* f, int x, int y, double* fc) {
  for (int i = 0; i < OL_Q; ++i) fc[i] = f[ol_idx(g, i, x, y)];
}
static void ol_scatter(const ol_grid* g, double* f, int x, int y, const double* fc) {
  for (int i = 0; i < OL_Q; ++i) f[ol_idx(g, i, x, y)] = fc[i];
}

/*
 * Zou-He completion of one boundary cell.  West (x = 0): unknown i = 1, 5, 8.
 * East (x = nx-1): unknown i = 3, 6, 7.  With u_y = 0 the density / velocity
 * follows from the known populations and the unknown ones from bounce-back of
 * the non-equilibrium part.
 */
static void ol_zou_he(int west, int kind, double value, double* f) {
  if (west) {
    const double known = f[0] + f[2] + f[4] + 2.0 * (f[3] + f[6] + f[7]);
    double rho, ux;
    if (kind == OL_BC_PRESSURE) {
      rho = value;
      ux = 1.0 - known / rho;
    } else {
      ux = value;
      rho = known / (1.0 - ux);
    }
    f[1] = f[3] + (2.0 / 3.0) * rho * ux;
    f[5] = f[7] - 0.5 * (f[2] - f[4]) + (1.0 / 6.0) * rho * ux;
    f[8] = f[6] + 0.5 * (f[2] - f[4]) + (1.0 / 6.0) * rho * ux;
  } else {
    const double known = f[0] + f[2] + f[4] + 2.0 * (f[1] + f[5] + f[8]);
    double rho, ux;
    if (kind == OL_BC_PRESSURE) {
      rho = value;
      ux = -1.0 + known / rho;
    } else {
      ux = value;
      rho = known / (1.0 + ux);
    }
    f[3] = f[1] - (2.0 / 3.0) * rho * ux;
    f[7] = f[5] + 0.5 * (f[2] - f[4]) - (1.0 / 6.0) * rho * ux;
    f[6] = f[8] - 0.5 * (f[2] - f[4]) - (1.0 / 6.0) * rho * ux;
  }
}

/* apply the Zou-He completion to the fluid cells of the non-periodic end columns */
void ol_boundary(const ol_grid* g, const uint8_t* solid, double* f) {
  double fc[OL_Q];
  if (g->bc_west != OL_BC_PERIODIC) {
    for (int y = 0; y < g->ny; ++y) {
      if (ol_solid(g, solid, 0, y)) continue;
      ol_gather(g, f, 0, y, fc);
      ol_zou_he(1, g->bc_west, g->west_value, fc);
      ol_scatter(g, f, 0, y, fc);
    }
  }
  if (g->bc_east != OL_BC_PERIODIC) {
    for (int y = 0; y < g->ny; ++y) {
      if (ol_solid(g, solid, g->nx - 1, y)) continue;
      ol_gather(g, f, g->nx - 1, y, fc);
      ol_zou_he(0, g->bc_east, g->east_value, fc);
      ol_scatter(g, f, g->nx - 1, y, fc);
    }
  }
}

/*
 * SRT collision (Sec. 2.1) on every fluid cell: f* = f - (f - f^eq)/tau + S.
 * Solid cells are copied unchanged.
 */
void ol_collide(const ol_grid* g, const uint8_t* solid, const double* f, double* fstar) {
  const double inv_tau = 1.0 / g->tau;
  const double guo = 1.0 - 0.5 * inv_tau;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < g->ny; ++y) {
    double fc[OL_Q], feq[OL_Q];
    for (int x = 0; x < g->nx; ++x) {
      ol_gather(g, f, x, y, fc);
      if (!ol_solid(g, solid, x, y)) {
        double rho, ux, uy;
        ol_cell_moments(g, fc, &rho, &ux, &uy);
        ol_equilibrium(rho, ux, uy, feq);
        for (int i = 0; i < OL_Q; ++i) {
          const double cu = OL_CX[i] * ux + OL_CY[i] * uy;
          const double sx = 3.0 * (OL_CX[i] - ux) + 9.0 * cu * OL_CX[i];
          const double sy = 3.0 * (OL_CY[i] - uy) + 9.0 * cu * OL_CY[i];
          const double src = guo * OL_W[i] * (sx * g->fx + sy * g->fy);
          fc[i] = fc[i] - (fc[i] - feq[i]) * inv_tau + src;
        }
      }
      ol_scatter(g, fstar, x, y, fc);
    }
  }
}

/*
 * Streaming (Sec. 2.1) with halfway bounce-back: for every fluid cell x,
 * f_i(x) = f*_i(x - c_i) if x - c_i is a fluid cell of the domain (periodic
 * wrap where the axis is periodic), f*_opp(i)(x) if it is solid.  Populations
 * that would enter from outside the domain are completed by ol_boundary.
 * Solid cells are copied unchanged.
 */
void ol_stream(const ol_grid* g, const uint8_t* solid, const double* fstar, double* f) {
  const int periodic_x = (g->bc_west == OL_BC_PERIODIC);
#pragma omp parallel for schedule(static)
  for (int y = 0; y < g->ny; ++y) {
    for (int x = 0; x < g->nx; ++x) {
      if (ol_solid(g, solid, x, y)) {
        for (int i = 0; i < OL_Q; ++i) f[ol_idx(g, i, x, y)] = fstar[ol_idx(g, i, x, y)];
        continue;
      }
      for (int i = 0; i < OL_Q; ++i) {
        int xs = x - OL_CX[i];
        const int ys = ol_wrap(y - OL_CY[i], g->ny);
        if (xs < 0 || xs >= g->nx) {
          if (!periodic_x) {
            f[ol_idx(g, i, x, y)] = NAN; /* filled by the Zou-He completion */
            continue;
          }
          xs = ol_wrap(xs, g->nx);
        }
        if (ol_solid(g, solid, xs, ys))
          f[ol_idx(g, i, x, y)] = fstar[ol_idx(g, OL_OPP[i], x, y)];
        else
          f[ol_idx(g, i, x, y)] = fstar[ol_idx(g, i, xs, ys)];
      }
    }
  }
  ol_boundary(g, solid, f);
}

/* nsteps of the loop of Fig. 1: equilibrium -> collision -> streaming -> moments */
void ol_run(const ol_grid* g, const uint8_t* solid, double* f, int nsteps) {
  const size_t n = (size_t)OL_Q * g->nx * g->ny;
  double* fstar = (double*)malloc(n * sizeof(double));
  for (int s = 0; s < nsteps; ++s) {
    ol_collide(g, solid, f, fstar);
    ol_stream(g, solid, fstar, f);
  }
  free(fstar);
}

/* macroscopic fields; solid cells report rho = 1, u = 0 */
void ol_macro(const ol_grid* g, const uint8_t* solid, const double* f, double* rho, double* ux,
              double* uy) {
  double fc[OL_Q];
  for (int y = 0; y < g->ny; ++y) {
    for (int x = 0; x < g->nx; ++x) {
      const size_t c = (size_t)y * g->nx + x;
      if (ol_solid(g, solid, x, y)) {
        rho[c] = 1.0;
        ux[c] = 0.0;
        uy[c] = 0.0;
        continue;
      }
      ol_gather(g, f, x, y, fc);
      ol_cell_moments(g, fc, &rho[c], &ux[c], &uy[c]);
    }
  }
}

/*
 * derivative of field v along one axis at (x, y): central where both
 * neighbours are fluid cells of the domain, one-sided where only one is,
 * zero otherwise.  axis 0 = x, 1 = y.
 */
static double ol_deriv(const ol_grid* g, const uint8_t* solid, const double* v, int x, int y,
                       int axis) {
  const int periodic_x = (g->bc_west == OL_BC_PERIODIC);
  int xp = x, yp = y, xm = x, ym = y;
  int okp = 1, okm = 1;
  if (axis == 0) {
    xp = x + 1;
    xm = x - 1;
    if (periodic_x) {
      xp = ol_wrap(xp, g->nx);
      xm = ol_wrap(xm, g->nx);
    } else {
      if (xp >= g->nx) okp = 0;
      if (xm < 0) okm = 0;
    }
  } else {
    yp = ol_wrap(y + 1, g->ny);
    ym = ol_wrap(y - 1, g->ny);
  }
  if (okp && ol_solid(g, solid, xp, yp)) okp = 0;
  if (okm && ol_solid(g, solid, xm, ym)) okm = 0;
  const double vc = v[(size_t)y * g->nx + x];
  if (okp && okm) return 0.5 * (v[(size_t)yp * g->nx + xp] - v[(size_t)ym * g->nx + xm]);
  if (okp) return v[(size_t)yp * g->nx + xp] - vc;
  if (okm) return vc - v[(size_t)ym * g->nx + xm];
  return 0.0;
}

/*
 * Re-initialise f from macroscopic fields (hybrid framework, Sec. 2.3):
 * fluid cells get f^eq(rho, u) (+ f^neq if neq_mode != 0); solid cells get
 * the rest state w_i.  The Zou-He completion is then applied.
 */
void ol_reinit(const ol_grid* g, const uint8_t* solid, const double* rho, const double* ux,
               const double* uy, int neq_mode, double* f) {
  double feq[OL_Q];
  for (int y = 0; y < g->ny; ++y) {
    for (int x = 0; x < g->nx; ++x) {
      const size_t c = (size_t)y * g->nx + x;
      if (ol_solid(g, solid, x, y)) {
        for (int i = 0; i < OL_Q; ++i) f[ol_idx(g, i, x, y)] = OL_W[i];
        continue;
      }
      ol_equilibrium(rho[c], ux[c], uy[c], feq);
      double grad[2][2] = {{0.0, 0.0}, {0.0, 0.0}}; /* grad[a][b] = d_a u_b */
      if (neq_mode) {
        grad[0][0] = ol_deriv(g, solid, ux, x, y, 0);
        grad[0][1] = ol_deriv(g, solid, uy, x, y, 0);
        grad[1][0] = ol_deriv(g, solid, ux, x, y, 1);
        grad[1][1] = ol_deriv(g, solid, uy, x, y, 1);
      }
      for (int i = 0; i < OL_Q; ++i) {
        const int c_[2] = {OL_CX[i], OL_CY[i]};
        double qd = 0.0; /* Q_iab d_a u_b */
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b)
            qd += (c_[a] * c_[b] - (a == b ? OL_CS2 : 0.0)) * grad[a][b];
        const double fneq = -(g->tau * OL_W[i] * rho[c] / OL_CS2) * qd;
        f[ol_idx(g, i, x, y)] = feq[i] + fneq;
      }
    }
  }
  ol_boundary(g, solid, f);
}

/*
 * shasta_oracle.c -- plain FP64 reference of the relativistic SHASTA step.
 *
 * TEST INFRASTRUCTURE.  This oracle exists only to check the CUDA path.  Only
 * the test suite, the smoke check of the package entry point and the CPU
 * baseline leg of the benchmark may build, load or call it.  It shares no code
 * with the CUDA library and is never reached from the product path.
 *
 * It follows the paper step by step, line by line, with no blocking and no
 * fusion:  for every sweep it fills the ghost cells of the old state, recovers
 * the primitives, takes the half step, fills the ghost cells of the half-step
 * state, recovers again and takes the full step from the old state.
 *
 * Build: gcc -O2 -ffp-contract=off (no FMA contraction, IEEE division and
 * square root), optionally -fopenmp to spread independent lines of one sweep
 * over threads (the arithmetic of every line is unchanged by that).
 *
 * Readings of points the paper leaves open (each also listed in the design
 * notes of the repository):
 *  - a "step" is three sweeps taken from consecutive triples of the axis
 *    permutation table of Sec. 3.1.4;
 *  - the half step is a complete SHASTA pass (transport, source,
 *    antidiffusion, limiter) with lambda/2, velocities and pressure at level n;
 *    the full step transports the OLD state with velocities and pressure
 *    recovered from the half-step state (Sec. 3, staggered time level);
 *  - the inner 1/8 term of the phoenical antidiffusion acts on the
 *    differences of the old state;
 *  - |M| is clamped to (1-delta)*E before recovery (never written back);
 *    E <= 0 recovers to vacuum;
 *  - the bag EoS gap (no root on either branch) resolves to the mixed-phase
 *    point e = e_c;
 *  - the ghost cells of the half-step state are filled by the boundary rule
 *    after the half step (reflecting, periodic) or keep their frozen values;
 *  - a tabulated EoS is linear between its nodes and continued from its last
 *    interval; its fixed-point iteration starts from v = M/(E + p(E)) and
 *    stops at a change of at most 1e-14.
 *
 * Parity unpinned: the clamp margin delta, the bag-EoS gap rule and the
 * choice of a half step with antidiffusion are readings the paper does not
 * fix; no pin can confirm them, and the tests compare the GPU with this
 * oracle under the same readings.
 */
#include "shasta_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NG 3 /* ghost depth = stencil radius of one SHASTA pass (Sec. 3.1.2) */
#define NFLD 5

static int g_threads = 1;

void or_set_threads(int n) { g_threads = n < 1 ? 1 : n; }
int or_get_threads(void) { return g_threads; }

/* Sec. 3.1.4 (and the enqueue routine of App. A): fixed permutation of axes. */
static const int k_axis_table[18] = {0, 1, 2, 0, 2, 1, 2, 0, 1, 2, 1, 0, 1, 2, 0, 1, 0, 2};

int or_axis(long step, int sub) { return k_axis_table[3 * (int)(step % 6) + sub]; }

/* ---------------------------------------------------------------- EoS ---- */

/* Tabulated p(e) (Sec. 2: parametrised or tabulated EoS, interpolated):
 * piecewise linear through (k de, table[k]); the last interval continues
 * above the table, the first below it. */
static double table_p(const or_params* P, double e) {
  double x = e / P->table_de;
  int k = (int)floor(x);
  if (k < 0) k = 0;
  if (k > P->table_n - 2) k = P->table_n - 2;
  double f = x - (double)k;
  return P->table[k] + f * (P->table[k + 1] - P->table[k]);
}

/* Sec. 2 closes the system with the ideal gas p = e/3.  The bag model
 * p = (e - 4B)/3 above e_c is an added workload, not from the paper. */
double or_eos_p(const or_params* P, double e) {
  if (P->eos == OR_EOS_TABLE) return table_p(P, e);
  if (P->eos == OR_EOS_BAG && e > P->bag_ec) return (e - 4.0 * P->bag_B) / 3.0;
  return e / 3.0;
}

/* Sec. 3: the paper finds the velocity by a fixed-point iteration so that a
 * tabulated EoS can replace p = e/3: from M = (E + p) v and e = E - M v,
 * |v| = M / (E + p(E - M |v|)).  Returns the number of iterations. */
int or_fixed_point(const or_params* P, double E, double M, double* e_out, double* p_out) {
  double v = M / (E + table_p(P, E));
  int it = 0;
  while (it < OR_FP_MAXIT) {
    double vn = M / (E + table_p(P, E - M * v));
    ++it;
    double d = vn - v;
    v = vn;
    if (fabs(d) <= OR_FP_TOL) break;
  }
  double e = E - M * v;
  *e_out = e;
  *p_out = table_p(P, e);
  return it;
}

/* Rest-frame energy density and pressure from E and |M| (already clamped).
 * Uses M = (E + p) v and e = E - M v (Sec. 2, Eqs. cf-momentum, cf-energy),
 * which for p = e/3 gives the closed root written here without the
 * E - |M| cancellation.  (The paper finds the same root by fixed-point
 * iteration, Sec. 3; the closed form is its exact limit.) */
static void eos_solve(const or_params* P, double E, double M, double* e_out, double* p_out) {
  if (P->eos == OR_EOS_TABLE) {
    or_fixed_point(P, E, M, e_out, p_out);
    return;
  }
  double s = sqrt(4.0 * E * E - 3.0 * M * M);
  double pa = ((E - M) * (E + M)) / (s + E);
  double ea = 3.0 * pa;
  if (P->eos != OR_EOS_BAG || ea <= P->bag_ec) {
    *e_out = ea;
    *p_out = pa;
    return;
  }
  /* bag branch: p = (e - 4B)/3, root e = 2B - E + sqrt(4(E-B)^2 - 3M^2),
   * written as a quotient to avoid cancellation; only reachable for E > e_c */
  double B = P->bag_B;
  if (E > P->bag_ec) {
    double r = 4.0 * (E - B) * (E - B) - 3.0 * M * M;
    if (r >= 0.0) {
      double sb = sqrt(r);
      double eb = (3.0 * ((E - M) * (E + M)) - 4.0 * B * E) / (sb + (E - 2.0 * B));
      if (eb > P->bag_ec) {
        *e_out = eb;
        *p_out = (eb - 4.0 * B) / 3.0;
        return;
      }
    }
  }
  /* mixed-phase point: e = e_c, v = (E - e_c)/M, p = M/v - E */
  *e_out = P->bag_ec;
  *p_out = M * M / (E - P->bag_ec) - E;
}

/* Clamp of |M| and the momentum scale it implies (reading: applied to the
 * recovery inputs only).  Returns the clamped |M|; *scale multiplies M_i. */
static double clamp_momentum(const or_params* P, double E, double Mx, double My, double Mz,
                             double* scale) {
  double M = sqrt((Mx * Mx + My * My) + Mz * Mz);
  double lim = (1.0 - P->delta) * E;
  *scale = 1.0;
  if (M > lim) {
    *scale = lim / M;
    M = lim;
  }
  return M;
}

/* Sec. 3 phases 3-4 for one cell: boost to the rest frame, EoS. */
static void recover_cell(const or_params* P, const double u[NFLD], double* e, double v[3],
                         double* nb, double* p) {
  double E = u[0];
  if (!(E > 0.0)) {
    *e = 0.0;
    v[0] = v[1] = v[2] = 0.0;
    *nb = 0.0;
    *p = 0.0;
    return;
  }
  double scale;
  double M = clamp_momentum(P, E, u[1], u[2], u[3], &scale);
  double ee, pp;
  eos_solve(P, E, M, &ee, &pp);
  double h = E + pp; /* = (e + p) gamma^2 */
  for (int a = 0; a < 3; ++a) {
    double m = (scale == 1.0) ? u[1 + a] : u[1 + a] * scale;
    v[a] = m / h;
  }
  *e = ee;
  *p = pp;
  *nb = u[4] * sqrt((ee + pp) / h); /* R / gamma, 1 - v^2 = (e+p)/(E+p) */
}

void or_recover(const or_params* P, size_t n, const double* E, const double* Mx,
                const double* My, const double* Mz, const double* R, double* e, double* vx,
                double* vy, double* vz, double* nb, double* p) {
  for (size_t i = 0; i < n; ++i) {
    double u[NFLD] = {E[i], Mx[i], My[i], Mz[i], R[i]};
    double ee, v[3], nn, pp;
    recover_cell(P, u, &ee, v, &nn, &pp);
    if (e) e[i] = ee;
    if (vx) vx[i] = v[0];
    if (vy) vy[i] = v[1];
    if (vz) vz[i] = v[2];
    if (nb) nb[i] = nn;
    if (p) p[i] = pp;
  }
}

/* Sec. 2, Eqs. (cf-density), (cf-momentum), (cf-energy). */
void or_prim2cons(const or_params* P, size_t n, const double* e, const double* vx,
                  const double* vy, const double* vz, const double* nb, double* E, double* Mx,
                  double* My, double* Mz, double* R) {
  for (size_t i = 0; i < n; ++i) {
    double v2 = (vx[i] * vx[i] + vy[i] * vy[i]) + vz[i] * vz[i];
    double g2 = 1.0 / (1.0 - v2);
    double p = or_eos_p(P, e[i]);
    double w = (e[i] + p) * g2;
    E[i] = w - p;
    Mx[i] = w * vx[i];
    My[i] = w * vy[i];
    Mz[i] = w * vz[i];
    R[i] = nb[i] * sqrt(g2);
  }
}

/* ------------------------------------------------------- one SHASTA pass -- */

/* Sec. 3: geometric transport with the factors Q+- of Eq. (shasta-diff), the
 * transported value of Eq. (shasta-geo) including the source lambda*Delta(f)
 * with Delta(f) = -(f_{j+1} - f_{j-1})/2, the phoenical antidiffusion, the
 * flux limiter and the update of Eq. (shasta-n).  Index j of the padded
 * arrays sits at position j + NG; valid j = -3 .. n+2. */
void or_line(int n, const double* u, const double* w, const double* f, double tau, double eta,
             double* out) {
  const double* U = u + NG;
  const double* W = w + NG;
  const double* F = f ? f + NG : NULL;
  int len = n + 2 * NG;
  double* uh_buf = (double*)malloc(sizeof(double) * (size_t)len);
  double* a_buf = (double*)malloc(sizeof(double) * (size_t)len);
  double* UH = uh_buf + NG;
  double* A = a_buf + NG;

  /* transported value on j = -2 .. n+1 */
  for (int j = -2; j <= n + 1; ++j) {
    double em = tau * W[j - 1];
    double e0 = tau * W[j];
    double ep = tau * W[j + 1];
    double qp = (0.5 - e0) / (1.0 + (ep - e0));
    double qm = (0.5 + e0) / (1.0 - (em - e0));
    double d = U[j + 1] - U[j];
    double dm = U[j] - U[j - 1];
    double t1 = (0.5 * qp * qp) * d;
    double t2 = (0.5 * qm * qm) * dm;
    double v = (t1 - t2) + (qp + qm) * U[j];
    if (F) v = v + (0.5 * tau) * (F[j - 1] - F[j + 1]);
    UH[j] = v;
  }
  /* limited antidiffusive flux through face j+1/2, j = -1 .. n-1 */
  for (int j = -1; j <= n - 1; ++j) {
    double dh = UH[j + 1] - UH[j];
    double dhp = UH[j + 2] - UH[j + 1];
    double dhm = UH[j] - UH[j - 1];
    double d = U[j + 1] - U[j];
    double dp = U[j + 2] - U[j + 1];
    double dm = U[j] - U[j - 1];
    double aph = eta * (dh - 0.125 * ((dp + dm) - 2.0 * d));
    double sg = (aph > 0.0) ? 1.0 : ((aph < 0.0) ? -1.0 : 0.0);
    double m = fmin(fmin(sg * dhp, fabs(aph)), sg * dhm);
    A[j] = sg * fmax(0.0, m);
  }
  for (int j = 0; j < n; ++j) out[j] = UH[j] - (A[j] - A[j - 1]);
  free(uh_buf);
  free(a_buf);
}

/* ------------------------------------------------------------- sweeps ---- */

static void line_geometry(const or_params* P, int axis, long* nlines, int* n, long* stride) {
  long nx = P->nx, ny = P->ny, nz = P->nz;
  if (axis == 0) {
    *n = (int)nx;
    *stride = 1;
    *nlines = ny * nz;
  } else if (axis == 1) {
    *n = (int)ny;
    *stride = nx;
    *nlines = nx * nz;
  } else {
    *n = (int)nz;
    *stride = nx * ny;
    *nlines = nx * ny;
  }
}

/* First element of line t (transverse index, lower axis fastest). */
static long line_base(const or_params* P, int axis, long t) {
  long nx = P->nx, ny = P->ny;
  if (axis == 0) return t * nx;             /* t = j + ny*k */
  if (axis == 1) return (t % nx) + nx * ny * (t / nx); /* t = i + nx*k */
  return t;                                  /* t = i + nx*j */
}

static long plane_size(const or_params* P, int axis) {
  long nx = P->nx, ny = P->ny, nz = P->nz;
  return axis == 0 ? ny * nz : (axis == 1 ? nx * nz : nx * ny);
}

size_t or_frozen_size(const or_params* P) {
  size_t s = 0;
  for (int a = 0; a < 3; ++a) s += (size_t)2 * NG * NFLD * (size_t)plane_size(P, a);
  return s;
}

static size_t frozen_offset(const or_params* P, int axis, int side, int layer, int field, long t) {
  size_t off = 0;
  for (int a = 0; a < axis; ++a) off += (size_t)2 * NG * NFLD * (size_t)plane_size(P, a);
  long pl = plane_size(P, axis);
  return off + ((((size_t)side * NG + (size_t)layer) * NFLD + (size_t)field) * (size_t)pl) +
         (size_t)t;
}

void or_frozen_capture(const or_params* P, const double* E, const double* Mx, const double* My,
                       const double* Mz, const double* R, double* frozen) {
  const double* f[NFLD] = {E, Mx, My, Mz, R};
  for (int a = 0; a < 3; ++a) {
    long nl, st;
    int n;
    line_geometry(P, a, &nl, &n, &st);
    for (long t = 0; t < nl; ++t) {
      long b = line_base(P, a, t);
      for (int side = 0; side < 2; ++side) {
        long edge = b + (side == 0 ? 0 : (long)(n - 1) * st);
        for (int layer = 0; layer < NG; ++layer)
          for (int k = 0; k < NFLD; ++k)
            frozen[frozen_offset(P, a, side, layer, k, t)] = f[k][edge];
      }
    }
  }
}

/* Ghost cells of a padded line (Sec. 3.1.3: halo cells).  Reflecting: the
 * mirror image through the wall with the momentum along the line negated
 * (repeated mirrors when n < 3).  Periodic: wrap.  Frozen: stored values. */
static void fill_ghosts(const or_params* P, int axis, long t, int n, double* ln[NFLD],
                        const double* frozen) {
  for (int side = 0; side < 2; ++side) {
    for (int layer = 0; layer < NG; ++layer) {
      int g = side == 0 ? -1 - layer : n + layer;
      for (int k = 0; k < NFLD; ++k) {
        double val;
        if (P->bc == OR_BC_PERIODIC) {
          int src = ((g % n) + n) % n;
          val = ln[k][NG + src];
        } else if (P->bc == OR_BC_FROZEN) {
          val = frozen[frozen_offset(P, axis, side, layer, k, t)];
        } else {
          int m = ((g % (2 * n)) + 2 * n) % (2 * n);
          int src = m < n ? m : 2 * n - 1 - m;
          double par = (m < n || k != 1 + axis) ? 1.0 : -1.0;
          val = par * ln[k][NG + src];
        }
        ln[k][NG + g] = val;
      }
    }
  }
}

/* Velocity along the sweep and pressure at every padded position. */
static void recover_line(const or_params* P, int axis, int len, double* ln[NFLD], double* w,
                         double* p) {
  for (int i = 0; i < len; ++i) {
    double u[NFLD] = {ln[0][i], ln[1][i], ln[2][i], ln[3][i], ln[4][i]};
    double e, v[3], nb, pp;
    recover_cell(P, u, &e, v, &nb, &pp);
    w[i] = v[axis];
    p[i] = pp;
  }
}

/* Both time levels of one sweep on one line (Sec. 3, staggered half step;
 * Sec. 3.1.3, half steps through a changed lambda).  Sources: +p for the
 * momentum along the line, +p v for the energy, none for the others. */
static void sweep_line(const or_params* P, int axis, long t, int n, double* old[NFLD],
                       double* half[NFLD], double* w, double* p, double* fe, const double* frozen) {
  int len = n + 2 * NG;
  fill_ghosts(P, axis, t, n, old, frozen);
  recover_line(P, axis, len, old, w, p);
  for (int i = 0; i < len; ++i) fe[i] = p[i] * w[i];
  for (int k = 0; k < NFLD; ++k) {
    const double* f = k == 0 ? fe : (k == 1 + axis ? p : NULL);
    or_line(n, old[k], w, f, 0.5 * P->lambda, P->eta, half[k] + NG);
  }
  fill_ghosts(P, axis, t, n, half, frozen);
  recover_line(P, axis, len, half, w, p);
  for (int i = 0; i < len; ++i) fe[i] = p[i] * w[i];
  for (int k = 0; k < NFLD; ++k) {
    const double* f = k == 0 ? fe : (k == 1 + axis ? p : NULL);
    /* the full step writes its result over the half-step buffer */
    or_line(n, old[k], w, f, P->lambda, P->eta, half[k] + NG);
  }
}

void or_sweep(const or_params* P, int axis, double* E, double* Mx, double* My, double* Mz,
              double* R, const double* frozen) {
  double* fld[NFLD] = {E, Mx, My, Mz, R};
  long nlines, stride;
  int n;
  line_geometry(P, axis, &nlines, &n, &stride);
  int len = n + 2 * NG;
#ifdef _OPENMP
#pragma omp parallel num_threads(g_threads)
#endif
  {
    double* buf = (double*)malloc(sizeof(double) * (size_t)len * (2 * NFLD + 3));
    double* old[NFLD];
    double* half[NFLD];
    for (int k = 0; k < NFLD; ++k) {
      old[k] = buf + (size_t)k * len;
      half[k] = buf + (size_t)(NFLD + k) * len;
    }
    double* w = buf + (size_t)(2 * NFLD) * len;
    double* p = w + len;
    double* fe = p + len;
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
    for (long t = 0; t < nlines; ++t) {
      long b = line_base(P, axis, t);
      for (int k = 0; k < NFLD; ++k)
        for (int i = 0; i < n; ++i) old[k][NG + i] = fld[k][b + (long)i * stride];
      sweep_line(P, axis, t, n, old, half, w, p, fe, frozen);
      for (int k = 0; k < NFLD; ++k)
        for (int i = 0; i < n; ++i) fld[k][b + (long)i * stride] = half[k][NG + i];
    }
    free(buf);
  }
}

int or_step(const or_params* P, double* E, double* Mx, double* My, double* Mz, double* R,
            const double* frozen, long step0, long nsteps) {
  if (P->nx < 1 || P->ny < 1 || P->nz < 1) return 1;
  if (P->bc == OR_BC_FROZEN && !frozen) return 2;
  if (P->eos == OR_EOS_TABLE && (!P->table || P->table_n < 2 || !(P->table_de > 0.0))) return 3;
  for (long s = step0; s < step0 + nsteps; ++s)
    for (int sub = 0; sub < 3; ++sub) or_sweep(P, or_axis(s, sub), E, Mx, My, Mz, R, frozen);
  return 0;
}

/* ------------------------------------------------------------- totals ---- */

static double neumaier(size_t n, const double* x) {
  double s = 0.0, c = 0.0;
  for (size_t i = 0; i < n; ++i) {
    double t = s + x[i];
    if (fabs(s) >= fabs(x[i]))
      c += (s - t) + x[i];
    else
      c += (x[i] - t) + s;
    s = t;
  }
  return s + c;
}

void or_totals(size_t n, const double* E, const double* Mx, const double* My, const double* Mz,
               const double* R, double out[5]) {
  out[0] = neumaier(n, E);
  out[1] = neumaier(n, Mx);
  out[2] = neumaier(n, My);
  out[3] = neumaier(n, Mz);
  out[4] = neumaier(n, R);
}

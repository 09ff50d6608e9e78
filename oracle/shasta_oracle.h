/*
 * shasta_oracle.h -- plain FP64 reference of the relativistic SHASTA step.
 *
 * TEST INFRASTRUCTURE.  This oracle exists only to check the CUDA path.  Only
 * the test suite, the smoke check of the package entry point and the CPU
 * baseline leg of the benchmark may build, load or call it.  It shares no code
 * with the CUDA library and must never be reached from the product path.
 *
 * Paper: J. Gerhard, V. Lindenstruth, M. Bleicher, "Relativistic
 * Hydrodynamics on Graphic Cards" (arXiv:1206.0919), Sec. 2 (conserved
 * variables) and Sec. 3 (the four-phase relativistic SHASTA).
 *
 * Storage: five conserved fields E, Mx, My, Mz, R, each a dense
 * nx*ny*nz array with x fastest (index i + nx*(j + ny*k)).
 */
#ifndef SHASTA_ORACLE_H
#define SHASTA_ORACLE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_BC_REFLECT = 0, OR_BC_PERIODIC = 1, OR_BC_FROZEN = 2 };
enum { OR_EOS_IDEAL = 0, OR_EOS_BAG = 1, OR_EOS_TABLE = 2 };

typedef struct {
  int nx, ny, nz;
  int bc;        /* OR_BC_* */
  int eos;       /* OR_EOS_* */
  double lambda; /* dt/dx, the CFL number of Sec. 3 */
  double eta;    /* outer antidiffusion coefficient (1/8 in Sec. 3) */
  double bag_B;  /* bag constant B (bag EoS only) */
  double bag_ec; /* energy density where the bag EoS switches branch */
  double delta;  /* |M| is clamped to (1-delta)*E before recovery */
  /* OR_EOS_TABLE: p at e_k = k * table_de, k = 0 .. table_n-1, linear in
   * between and linearly extrapolated from the last interval above; the
   * recovery then finds |v| by the fixed-point iteration of Sec. 3. */
  const double* table;
  int table_n;
  double table_de;
} or_params;

/* Fixed-point iteration of the tabulated recovery: start v = M/(E + p(E)),
 * iterate v <- M/(E + p(E - M v)) until |change| <= OR_FP_TOL or
 * OR_FP_MAXIT iterations. */
#define OR_FP_TOL 1e-14
#define OR_FP_MAXIT 200

/* Equation of state p(e). */
double or_eos_p(const or_params* P, double e);

/* Tabulated EoS: rest-frame e and p of a cell with energy E > 0 and |M| < E
 * by the fixed-point iteration; returns the iterations taken. */
int or_fixed_point(const or_params* P, double E, double M, double* e_out, double* p_out);

/* Sec. 2, Eqs. (cf-density), (cf-momentum), (cf-energy): primitives -> conserved. */
void or_prim2cons(const or_params* P, size_t n, const double* e, const double* vx,
                  const double* vy, const double* vz, const double* nb, double* E,
                  double* Mx, double* My, double* Mz, double* R);

/* Sec. 3 phases 3-4: conserved -> primitives (e, v, n, p).  Any output may be NULL. */
void or_recover(const or_params* P, size_t n, const double* E, const double* Mx,
                const double* My, const double* Mz, const double* R, double* e,
                double* vx, double* vy, double* vz, double* nb, double* p);

/* One SHASTA pass of a single field along one line (Sec. 3, Eqs. shasta-diff,
 * shasta-geo, the phoenical antidiffusion and the flux limiter, shasta-n).
 * u, w, f point at padded arrays of length n+6 (3 ghosts per side, ghost and
 * interior values already in place); f may be NULL for a source-free field.
 * out receives the n interior values. */
void or_line(int n, const double* u, const double* w, const double* f, double tau,
             double eta, double* out);

/* One sweep along axis (0=x, 1=y, 2=z): half step + full step. */
void or_sweep(const or_params* P, int axis, double* E, double* Mx, double* My,
              double* Mz, double* R, const double* frozen);

/* nsteps full split steps starting at step counter step0 (axis order from
 * the permutation table of Sec. 3.1.4).  frozen: ghost store for
 * OR_BC_FROZEN (see or_frozen_size), else NULL.  Returns 0 on success. */
int or_step(const or_params* P, double* E, double* Mx, double* My, double* Mz,
            double* R, const double* frozen, long step0, long nsteps);

/* Number of doubles in the frozen ghost store and its capture from a state:
 * per axis a, per side (low, high), per ghost layer (3), per field (5), one
 * transverse plane (the other two axes, lower axis fastest).  Every ghost
 * layer holds the edge cell of the state it was captured from. */
size_t or_frozen_size(const or_params* P);
void or_frozen_capture(const or_params* P, const double* E, const double* Mx,
                       const double* My, const double* Mz, const double* R,
                       double* frozen);

/* Compensated (Neumaier) sums of the five fields. */
void or_totals(size_t n, const double* E, const double* Mx, const double* My,
               const double* Mz, const double* R, double out[5]);

/* Axis permutation table of Sec. 3.1.4 (18 entries). */
int or_axis(long step, int sub);

/* Worker threads used by or_sweep (OpenMP over independent lines); 1 = serial. */
void or_set_threads(int n);
int or_get_threads(void);

#ifdef __cplusplus
}
#endif
#endif

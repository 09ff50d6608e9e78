// sweep.cuh -- fused relativistic SHASTA sweep along one axis (sm_103a).
//
// One sweep (arXiv:1206.0919, Sec. 3) on every line of the grid along the
// sweep axis: recovery of velocity and pressure at level n, a half step of
// SHASTA with lambda/2 (transport factors Q+- of Eq. shasta-diff, transported
// value of Eq. shasta-geo with the pressure source, phoenical antidiffusion,
// flux limiter, update of Eq. shasta-n), recovery at level n+1/2, and the
// full step that transports the OLD state with the half-step velocity and
// pressure (staggered time level, Sec. 3; double buffering, Sec. 3.1.3).
//
// Design (differs from the paper's one-work-item-per-cell-per-quantity
// kernels, Sec. 3.1.2): one thread owns one grid line and streams along it
// once.  Each quantity (recovered v and p, transported value, limited flux)
// is computed once per cell and kept in a short register window, instead of
// being recomputed five times (transport) and twice (antiflux) per cell.
// All five conserved fields share the transport factors.  The state at level
// n+1/2 never touches memory.  Ghost cells are not stored: the loader maps
// an index outside the line to its mirror (reflecting), its wrap (periodic)
// or the frozen ghost store.  For mirror and wrap the half-step state at a
// ghost position is computed from the extended line, which equals the mirror
// / wrap of the interior half-step state because the arithmetic below is
// ordered symmetrically (second difference as (d+ + d-) - 2d, flux
// differences as A_j - A_{j-1}).
//
// Pipeline (q = position of the newest loaded cell, q = -6 .. n+5):
//   U^n_q loaded, (w, p)^n_q recovered
//   Uhat^h_{q-1}     transported half-step value
//   A^h_{q-3}        limited half-step flux; U^h_{q-3} = Uhat - (A_{q-3} - A_{q-4})
//   (w, p)^h_{q-3}   recovered at n+1/2
//   Uhat^f_{q-4}     transported full-step value (from U^n)
//   A^f_{q-6}        limited full-step flux; U^{n+1}_{q-6} stored if inside
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace shasta {

constexpr int NF = 5;  // E, M_x, M_y, M_z, R
constexpr int NG = 3;  // ghost depth of one SHASTA pass

enum { BC_REFLECT = 0, BC_PERIODIC = 1, BC_FROZEN = 2 };
enum { EOS_IDEAL = 0, EOS_BAG = 1, EOS_TABLE = 2 };

// Tabulated EoS (EOS_TABLE): p at e = k de, k = 0 .. n-1, linear in
// between, the last interval continued above the table (device copies in
// double and float).
struct EosTable {
  const double* p64;
  const float* p32;
  int n;
  double de;
  float inv_de32;  // 1 / de in float (FP32 lookups)
};

// Geometry and constants of one sweep launch (filled on the host).
struct SweepParams {
  const void* in[NF];  // fields of U^n, storage type T, global order E,Mx,My,Mz,R
  void* out[NF];       // fields of U^{n+1}
  const void* frozen;  // frozen ghosts of this axis: [side][layer][field][plane], or null
  long long plane;     // number of lines (= size of the transverse plane)
  long long stride;    // element stride along the line
  long long sb, sc;    // first element of line t = b + nb*c is b*sb + c*sc
  int n;               // cells along the line
  int nb;              // extent of the faster transverse axis
  int bc;              // BC_*
  double tau_h, tau_f;    // lambda/2 and lambda
  double htau_h, htau_f;  // half of each (source coefficient)
  double eta;             // outer antidiffusion coefficient
  double omd;             // 1 - delta (clamp of |M|)
  double bag_B, bag_ec;
  unsigned long long* clamp_count;  // cells recovered with |M| clamped or E <= 0
  long long range_len;              // fast kernels: positions per work range (>= 1; batches: 0
                                    // = whole line groups, BatchList.prefix then counts groups)
  const int* ranges;                // one event, when set: range r is positions
  long long nranges;                // [ranges[r], ranges[r+1]), r < nranges (balanced cuts)
  int variant;                      // fast kernels: launch variant (0: capped registers, 1: not)
  long long blocks;                 // fast kernels: grid size (one wave of resident warps)
  // fast kernels: state as (E, Mx, My, Mz) quads per cell plus an R array
  const float* qin;
  const float* rin;
  float* qout;
  float* rout;
  EosTable tab;  // EOS_TABLE only
  // fast kernels: the scalars above rounded to float (set_float_scalars), so
  // that the kernels take them as constant-bank operands instead of holding
  // converted copies in registers
  float f_tau_h, f_tau_f, f_htau_h, f_htau_f, f_eta, f_omd, f_bag_B, f_bag_ec;
  // checked builds (SHASTA_CHECKED): cells in each of qin / rin / qout / rout,
  // and the record [count, first code, first index] of refused accesses
  long long ncap;
  unsigned long long* chk;
};

// Fills the float copies of the launch scalars (host side, after the
// doubles are set).
inline void set_float_scalars(SweepParams& P) {
  P.f_tau_h = (float)P.tau_h;
  P.f_tau_f = (float)P.tau_f;
  P.f_htau_h = (float)P.htau_h;
  P.f_htau_f = (float)P.htau_f;
  P.f_eta = (float)P.eta;
  P.f_omd = (float)P.omd;
  P.f_bag_B = (float)P.bag_B;
  P.f_bag_ec = (float)P.bag_ec;
}

// Checked builds (-DSHASTA_CHECKED): each global access of the streaming
// sweeps (FP64 and FP32 / MIXED), and each shared-memory access of the fast
// sweeps at a computed offset, is first tested against the bounds of its
// buffer; a miss is counted in P.chk (count, first code, first index) and
// the access is skipped.  The tests run them to
// show that the index arithmetic stays in bounds; other builds compile the
// tests away.  Codes: 1 state load, 2 frozen-ghost load, 3 state store,
// 4 shared-memory ring, 5 range table.
#ifdef SHASTA_CHECKED
__device__ __forceinline__ bool chk_ok(unsigned long long* rec, bool ok, int code, long long idx) {
  if (!ok && rec && atomicAdd(rec, 1ull) == 0ull) {
    rec[1] = (unsigned long long)code;
    rec[2] = (unsigned long long)idx;
  }
  return ok;
}
#define SH_OK(P, cond, code, idx) ::shasta::chk_ok((P).chk, (cond), (code), (long long)(idx))
#else
#define SH_OK(P, cond, code, idx) true
#endif

// Batched sweeps: one event of a batch.  All events of a batch share the
// batch's state arrays (qin/rin/qout/rout of SweepParams); the event's cells
// are [off, off + nx*ny*nz) of each, x fastest.
struct EvDesc {
  long long off;
  int nx, ny, nz, bc;
  float tau_h, tau_f;               // lambda/2 and lambda
  float htau_h, htau_f;             // half of each
  float bag_B, bag_ec;
  const float* frozen[3];           // frozen ghosts per axis (as SweepParams::frozen), or null
  unsigned long long* clamp_count;  // the event's clamp counter
};

// Work list of one batched launch: list entry k is event idx[k], whose
// (line group, position) pairs along the axis are numbered prefix[k] ..
// prefix[k+1]-1 (group-major: ceil(lines / 32) groups of n positions), or,
// when the launch takes whole line groups, whose line groups are.
struct BatchList {
  const EvDesc* ev;
  const int* idx;
  const int* prefix;  // nlist + 1 entries
  int nlist;
};

// ------------------------------------------------------------- recovery ----

// Rest-frame e and p from E and the clamped |M| (Sec. 2: M = (E + p) v,
// e = E - M v; closed root of that fixed point for p = e/3; bag branch
// p = (e - 4B)/3 above e_c; mixed-phase point in the gap).
template <class R, int EOS>
__device__ __forceinline__ void eos_solve(R E, R M, R B, R ec, R& e, R& p) {
  R s = sqrt(R(4) * E * E - R(3) * M * M);
  R pa = ((E - M) * (E + M)) / (s + E);
  R ea = R(3) * pa;
  if (EOS == EOS_IDEAL) {
    e = ea;
    p = pa;
    return;
  } else {
    if (ea <= ec) {
      e = ea;
      p = pa;
      return;
    }
    if (E > ec) {
      R r = R(4) * (E - B) * (E - B) - R(3) * M * M;
      if (r >= R(0)) {
        R sb = sqrt(r);
        R eb = (R(3) * ((E - M) * (E + M)) - R(4) * B * E) / (sb + (E - R(2) * B));
        if (eb > ec) {
          e = eb;
          p = (eb - R(4) * B) / R(3);
          return;
        }
      }
    }
    e = ec;
    p = M * M / (E - ec) - E;
  }
}

// p(e) of the table, the lookup written as in the oracle.
__device__ __forceinline__ double table_p64(const EosTable& T, double e) {
  double x = e / T.de;
  int k = (int)floor(x);
  if (k < 0) k = 0;
  if (k > T.n - 2) k = T.n - 2;
  double f = x - (double)k;
  const double a = T.p64[k], b = T.p64[k + 1];
  return a + f * (b - a);
}

// Tabulated EoS: |v| by the fixed-point iteration of Sec. 3 (kept by the
// paper so that a table can replace p = e/3): from v = M/(E + p(E)),
// v <- M/(E + p(E - M v)) until the change is at most 1e-14 (200 at most),
// then e = E - M v and p = p(e).
__device__ __forceinline__ void eos_table_solve(double E, double M, const EosTable& T, double& e,
                                                double& p) {
  double v = M / (E + table_p64(T, E));
  for (int it = 0; it < 200; ++it) {
    const double vn = M / (E + table_p64(T, E - M * v));
    const double d = vn - v;
    v = vn;
    if (fabs(d) <= 1e-14) break;
  }
  e = E - M * v;
  p = table_p64(T, e);
}

// Velocity along the sweep axis and pressure of one cell.  m1 is the
// momentum along the sweep, m2/m3 the other two in increasing axis order;
// |M|^2 is summed in x, y, z order.
// Returns 1 if |M| was clamped or E <= 0, else 0.
template <class R, int EOS, int AXIS>
__device__ __forceinline__ unsigned recover_wp(R E, R m1, R m2, R m3, R omd, R B, R ec,
                                               const EosTable& T, R& w, R& p) {
  if (!(E > R(0))) {
    w = R(0);
    p = R(0);
    return 1;
  }
  R X = AXIS == 0 ? m1 : m2;
  R Y = AXIS == 0 ? m2 : (AXIS == 1 ? m1 : m3);
  R Z = AXIS == 2 ? m1 : m3;
  R M = sqrt((X * X + Y * Y) + Z * Z);
  R lim = omd * E;
  R m = m1;
  unsigned clamped = 0;
  if (M > lim) {
    m = m1 * (lim / M);
    M = lim;
    clamped = 1;
  }
  R e, pp;
  if constexpr (EOS == EOS_TABLE)
    eos_table_solve(E, M, T, e, pp);
  else
    eos_solve<R, EOS>(E, M, B, ec, e, pp);
  R h = E + pp;
  w = m / h;
  p = pp;
  return clamped;
}

// ------------------------------------------------------------ transport ----

// Transport factors Q+ and Q- at a cell from eps = tau*w at j-1, j, j+1
// (Eq. shasta-diff).
template <class C>
__device__ __forceinline__ void qfactors(C wm, C w0, C wp, C tau, C& qp, C& qm) {
  C em = tau * wm;
  C e0 = tau * w0;
  C ep = tau * wp;
  qp = (C(0.5) - e0) / (C(1) + (ep - e0));
  qm = (C(0.5) + e0) / (C(1) - (em - e0));
}

// Transported value without source (Eq. shasta-geo).
template <class C>
__device__ __forceinline__ C transport(C a, C b, C c, C um, C u0, C up) {
  C t1 = a * (up - u0);
  C t2 = b * (u0 - um);
  return (t1 - t2) + c * u0;
}

// Limited phoenical antidiffusive flux through face j+1/2 from transported
// values at j-1..j+2 and old values at j-1..j+2 (Sec. 3).
template <class C, bool FAST>
__device__ __forceinline__ C antiflux(C h0, C h1, C h2, C h3, C u0, C u1, C u2, C u3, C eta) {
  C dhm = h1 - h0;
  C dh = h2 - h1;
  C dhp = h3 - h2;
  C dm = u1 - u0;
  C d = u2 - u1;
  C dp = u3 - u2;
  C aph = eta * (dh - C(0.125) * ((dp + dm) - C(2) * d));
  if (!FAST) {
    C sg = (aph > C(0)) ? C(1) : ((aph < C(0)) ? C(-1) : C(0));
    C m = fmin(fmin(sg * dhp, fabs(aph)), sg * dhm);
    return sg * fmax(C(0), m);
  } else {
    // sign of aph applied by flipping sign bits; for aph == 0 this returns 0
    uint32_t s = __float_as_uint(float(aph)) & 0x80000000u;
    float a = fabsf(float(aph));
    float p1 = __uint_as_float(__float_as_uint(float(dhp)) ^ s);
    float p2 = __uint_as_float(__float_as_uint(float(dhm)) ^ s);
    float m = fmaxf(0.0f, fminf(fminf(p1, a), p2));
    return C(__uint_as_float(__float_as_uint(m) ^ s));
  }
}

// ---------------------------------------------------------------- loads ----

template <class T>
__device__ __forceinline__ T ldv(const void* p, long long i) {
  return __ldg(static_cast<const T*>(p) + i);
}

// Loads the five fields of extended position q of the line starting at
// `base`, in sweep order (E, M_par, M_t1, M_t2, R), applying the boundary
// rule for positions outside [0, n).
template <class T, int AXIS>
__device__ __forceinline__ void load_ext(const SweepParams& P, long long base, long long t, int q,
                                         T v[NF]) {
  constexpr int FPAR = 1 + AXIS;                  // momentum along the sweep
  constexpr int FT1 = AXIS == 0 ? 2 : 1;          // transverse, lower axis
  constexpr int FT2 = AXIS == 2 ? 2 : 3;          // transverse, higher axis
  const int n = P.n;
  if (q >= 0 && q < n) {
    long long i = base + (long long)q * P.stride;
#ifdef SHASTA_CHECKED
    if (!SH_OK(P, i >= 0 && i < P.ncap, 1, i)) {
      for (int k = 0; k < NF; ++k) v[k] = T(0);
      return;
    }
#endif
    v[0] = ldv<T>(P.in[0], i);
    v[1] = ldv<T>(P.in[FPAR], i);
    v[2] = ldv<T>(P.in[FT1], i);
    v[3] = ldv<T>(P.in[FT2], i);
    v[4] = ldv<T>(P.in[4], i);
    return;
  }
  if (P.bc == BC_FROZEN) {
    int side = q < 0 ? 0 : 1;
    int layer = q < 0 ? -1 - q : q - n;
    layer = layer > NG - 1 ? NG - 1 : layer;
    long long o = ((long long)(side * NG + layer) * NF) * P.plane + t;
#ifdef SHASTA_CHECKED
    if (!SH_OK(P, o >= 0 && t < P.plane && o + 4 * P.plane < 2LL * NG * NF * P.plane, 2, o)) {
      for (int k = 0; k < NF; ++k) v[k] = T(0);
      return;
    }
#endif
    v[0] = ldv<T>(P.frozen, o + 0 * P.plane);
    v[1] = ldv<T>(P.frozen, o + (long long)FPAR * P.plane);
    v[2] = ldv<T>(P.frozen, o + (long long)FT1 * P.plane);
    v[3] = ldv<T>(P.frozen, o + (long long)FT2 * P.plane);
    v[4] = ldv<T>(P.frozen, o + 4 * P.plane);
    return;
  }
  int src;
  bool neg = false;
  if (P.bc == BC_PERIODIC) {
    src = ((q % n) + n) % n;
  } else {
    int n2 = 2 * n;
    int m = ((q % n2) + n2) % n2;
    src = m < n ? m : n2 - 1 - m;
    neg = m >= n;
  }
  long long i = base + (long long)src * P.stride;
#ifdef SHASTA_CHECKED
  if (!SH_OK(P, i >= 0 && i < P.ncap, 1, i)) {
    for (int k = 0; k < NF; ++k) v[k] = T(0);
    return;
  }
#endif
  v[0] = ldv<T>(P.in[0], i);
  T par = ldv<T>(P.in[FPAR], i);
  v[1] = neg ? -par : par;
  v[2] = ldv<T>(P.in[FT1], i);
  v[3] = ldv<T>(P.in[FT2], i);
  v[4] = ldv<T>(P.in[4], i);
}

// --------------------------------------------------------------- kernel ----

// T: storage and transport type.  R: recovery type.  FAST: float limiter
// with sign-bit arithmetic (same values as the branchy form).
// One thread streams positions [s0, s1) of one line (the segment seg of
// line t; P.range_len cells per segment, whole lines when it is 0 or >= n),
// starting 2 NG positions early: the pipeline windows then hold exactly what
// a whole-line pass holds at s0, so segments give the same bits.
template <class T, class R, int EOS, int AXIS, bool FAST>
__global__ void __launch_bounds__(128) sweep_kernel(SweepParams P) {
  constexpr int FPAR = 1 + AXIS;
  constexpr int FT1 = AXIS == 0 ? 2 : 1;
  constexpr int FT2 = AXIS == 2 ? 2 : 3;
  const int n = P.n;
  const int L = P.range_len > 0 && P.range_len < n ? (int)P.range_len : n;
  const int nseg = (n + L - 1) / L;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= P.plane * nseg) return;
  const long long t = tid % P.plane;
  const int s0 = (int)(tid / P.plane) * L;
  const int s1 = s0 + L < n ? s0 + L : n;
  const long long b = t % P.nb;
  const long long c = t / P.nb;
  const long long base = b * P.sb + c * P.sc;
  const bool frozen = P.bc == BC_FROZEN;

  const T tau_h = T(P.tau_h), tau_f = T(P.tau_f);
  const T htau_h = T(P.htau_h), htau_f = T(P.htau_f);
  const T eta = T(P.eta);
  const R omd = R(P.omd), B = R(P.bag_B), ec = R(P.bag_ec);
  unsigned nclamp = 0;

  // register windows (index 0 = oldest)
  T u[8][NF];           // U^n at q-7 .. q
  T wn[3], pn[3];       // (w, p)^n at q-2 .. q
  T uh[4][NF];          // Uhat^h at q-4 .. q-1
  T ah[NF];             // A^h at q-4
  T wh[3], ph[3];       // (w, p)^h at q-5 .. q-3
  T uf[4][NF];          // Uhat^f at q-7 .. q-4
  T af[NF];             // A^f at q-7
#pragma unroll
  for (int k = 0; k < NF; ++k) {
#pragma unroll
    for (int s = 0; s < 8; ++s) u[s][k] = T(k == 0 ? 1 : 0);
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      uh[s][k] = T(0);
      uf[s][k] = T(0);
    }
    ah[k] = T(0);
    af[k] = T(0);
  }
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    wn[s] = pn[s] = wh[s] = ph[s] = T(0);
  }

  T nxt[NF];
  load_ext<T, AXIS>(P, base, t, s0 - 2 * NG, nxt);

  for (int q = s0 - 2 * NG; q <= s1 + 2 * NG - 1; ++q) {
    // ---- stage 0: ingest U^n_q, prefetch q+1, recover (w, p)^n_q
#pragma unroll
    for (int s = 0; s < 7; ++s)
#pragma unroll
      for (int k = 0; k < NF; ++k) u[s][k] = u[s + 1][k];
#pragma unroll
    for (int k = 0; k < NF; ++k) u[7][k] = nxt[k];
    if (q + 1 <= s1 + 2 * NG - 1) load_ext<T, AXIS>(P, base, t, q + 1, nxt);
    wn[0] = wn[1];
    wn[1] = wn[2];
    pn[0] = pn[1];
    pn[1] = pn[2];
    {
      R w, p;
      const unsigned c0 = recover_wp<R, EOS, AXIS>(R(u[7][0]), R(u[7][1]), R(u[7][2]),
                                                   R(u[7][3]), omd, B, ec, P.tab, w, p);
      nclamp += (q >= s0 && q < s1) ? c0 : 0u;
      wn[2] = T(w);
      pn[2] = T(p);
    }
    // ---- stage 1: half-step transported value at q-1
#pragma unroll
    for (int s = 0; s < 3; ++s)
#pragma unroll
      for (int k = 0; k < NF; ++k) uh[s][k] = uh[s + 1][k];
    {
      T qp, qm;
      qfactors<T>(wn[0], wn[1], wn[2], tau_h, qp, qm);
      T a = T(0.5) * qp * qp, bq = T(0.5) * qm * qm, cq = qp + qm;
#pragma unroll
      for (int k = 0; k < NF; ++k) uh[3][k] = transport<T>(a, bq, cq, u[5][k], u[6][k], u[7][k]);
      uh[3][0] = uh[3][0] + htau_h * (pn[0] * wn[0] - pn[2] * wn[2]);
      uh[3][1] = uh[3][1] + htau_h * (pn[0] - pn[2]);
    }
    // ---- stage 2: half-step flux at q-3, half-step state at q-3
    T hs[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      T an = antiflux<T, FAST>(uh[0][k], uh[1][k], uh[2][k], uh[3][k], u[3][k], u[4][k], u[5][k],
                               u[6][k], eta);
      hs[k] = uh[1][k] - (an - ah[k]);
      ah[k] = an;
    }
    const int jh = q - NG;
    if (frozen && (jh < 0 || jh >= n)) {
#pragma unroll
      for (int k = 0; k < NF; ++k) hs[k] = u[4][k];
    }
    // ---- stage 3: recovery at n+1/2, position q-3
    wh[0] = wh[1];
    wh[1] = wh[2];
    ph[0] = ph[1];
    ph[1] = ph[2];
    {
      R w, p;
      // (the counter counts level-n recoveries only, as the FP32 kernels)
      recover_wp<R, EOS, AXIS>(R(hs[0]), R(hs[1]), R(hs[2]), R(hs[3]), omd, B, ec, P.tab, w, p);
      wh[2] = T(w);
      ph[2] = T(p);
    }
    // ---- stage 4: full-step transported value at q-4 (old state, half-step velocity)
#pragma unroll
    for (int s = 0; s < 3; ++s)
#pragma unroll
      for (int k = 0; k < NF; ++k) uf[s][k] = uf[s + 1][k];
    {
      T qp, qm;
      qfactors<T>(wh[0], wh[1], wh[2], tau_f, qp, qm);
      T a = T(0.5) * qp * qp, bq = T(0.5) * qm * qm, cq = qp + qm;
#pragma unroll
      for (int k = 0; k < NF; ++k) uf[3][k] = transport<T>(a, bq, cq, u[2][k], u[3][k], u[4][k]);
      uf[3][0] = uf[3][0] + htau_f * (ph[0] * wh[0] - ph[2] * wh[2]);
      uf[3][1] = uf[3][1] + htau_f * (ph[0] - ph[2]);
    }
    // ---- stage 5: full-step flux at q-6, new state at q-6
    T outv[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      T an = antiflux<T, FAST>(uf[0][k], uf[1][k], uf[2][k], uf[3][k], u[0][k], u[1][k], u[2][k],
                               u[3][k], eta);
      outv[k] = uf[1][k] - (an - af[k]);
      af[k] = an;
    }
    const int jo = q - 2 * NG;
    if (jo >= s0 && SH_OK(P, base + (long long)jo * P.stride < P.ncap, 3, base + (long long)jo * P.stride)) {
      long long i = base + (long long)jo * P.stride;
      static_cast<T*>(P.out[0])[i] = outv[0];
      static_cast<T*>(P.out[FPAR])[i] = outv[1];
      static_cast<T*>(P.out[FT1])[i] = outv[2];
      static_cast<T*>(P.out[FT2])[i] = outv[3];
      static_cast<T*>(P.out[4])[i] = outv[4];
    }
  }
  if (nclamp && P.clamp_count) atomicAdd(P.clamp_count, (unsigned long long)nclamp);
}

}  // namespace shasta

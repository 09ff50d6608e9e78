// sweep_fast.cuh -- FP32 fused SHASTA sweep tuned for sm_103a.
//
// Same sweep as sweep.cuh (arXiv:1206.0919, Sec. 3: half step with lambda/2,
// recovery at n+1/2, full step from the old state), reorganised for
// throughput on Blackwell:
//
//  * State layout: (E, Mx, My, Mz) as one 16-byte quad per cell and R as a
//    separate array.  A cell moves with one 16-byte and one 4-byte access,
//    and the quad splits into the register pairs (E, Mx), (My, Mz).
//  * One warp streams 32 lines (one per lane) along the sweep axis.  The
//    positions of all line groups are cut into equal ranges, one or more
//    per warp, so that every warp has the same amount of work; a range
//    touches one or two line groups (each piece with its own 6-cell halo
//    per side).
//  * Input cells are staged through a per-warp shared-memory ring filled
//    with cp.async ahead of use.  For y/z sweeps each lane copies its own
//    line (the lanes of one position are adjacent in memory).  For x sweeps
//    the warp copies chunks of 8 positions x 32 rows cooperatively (8 lanes
//    per 128-byte row segment of quads) and writes results back the same way
//    from ring entries it no longer needs, so global accesses stay
//    sector-complete.
//  * Transport, differences and the antidiffusive flux run on the field
//    pairs (E, Mx), (My, Mz) as plain FP32 scalar operations; the flux
//    limiter uses the three-input min.  (The packed f32x2 arithmetic of
//    sm_100+ measured no faster here: the kernel is latency-bound at 12
//    warps per SM, and forming register pairs cost one move for every two
//    packed operations.)
//  * The pass is written with differences (Delta, their first and second
//    differences, Delta-hat) so that every carried quantity spans at most two
//    positions: the loop is unrolled by 2 and all windows are renamed
//    registers.  Old values are consumed before a same-parity slot is
//    overwritten, so no copies are needed.
//  * The old state for the full step is re-read from the ring (it is still
//    resident) instead of being carried in registers.
//  * Transport factors use Q-_j = 1 - Q+_{j-1}, exact for Eq. shasta-diff
//    (the two share the denominator 1 + eps_j - eps_{j-1}), so each cell
//    needs one division per pass.
//  * The baryon density R is not transported at the half step: only E and M
//    enter the recovery at n+1/2.
//  * Recoveries at n (newest cell) and n+1/2 (four cells back) are two
//    independent scalar chains.  For p = e/3 with D = E^2 - |M|^2:
//    s = sqrt(E^2 + 3D), p = D/(E + s), v = M/(E + p).  The clamp counter
//    is only touched on the rare clamped path.  MIXED evaluates D in double-float
//    (error-free products and sums on the FP32 pipe), which removes the
//    cancellation as v -> 1 at about FP64 accuracy of D.
//  * The including units are built with -fmad=false: every fused
//    multiply-add is explicit, so all instantiations of the streaming step
//    (position parity, boundary variant, register variant) round alike and
//    the result does not depend on how lines are cut into pieces.
#pragma once

#include <type_traits>

#include "sweep.cuh"

namespace shasta {
namespace fast {


constexpr int LANES = 32;
constexpr int CH = 8;      // x sweep: positions per cooperative chunk
constexpr int XSLOTS = 3;  // x sweep: chunk slots (previous, current, next)
// x ring slot: quad plane [row][pos][4] with row stride 36 (16-byte units
// 9 apart: conflict-free 128-bit accesses down a column), R plane [row][pos]
// with row stride 9.
constexpr int XQSTR = 4 * CH + 4;
constexpr int XRSTR = CH + 1;
constexpr int XQ = LANES * XQSTR;         // 1152 floats
constexpr int XSLOT = XQ + LANES * XRSTR; // 1440 floats
// y/z ring slot: quad row [lane][4] (128 floats), R row [lane]
constexpr int YQ = 4 * LANES;
constexpr int YSLOT = YQ + LANES;         // 160 floats

// ----------------------------------------------------------- field pairs ----

// Two fields of a cell, (E, Mx) or (My, Mz), or one field of two cells.
struct f2 {
  float x, y;
};

__device__ __forceinline__ f2 pk(float lo, float hi) { return f2{lo, hi}; }
__device__ __forceinline__ void up(f2 v, float& lo, float& hi) {
  lo = v.x;
  hi = v.y;
}
__device__ __forceinline__ float lo_of(f2 v) {
  float a, b;
  up(v, a, b);
  return a;
}
__device__ __forceinline__ float hi_of(f2 v) {
  float a, b;
  up(v, a, b);
  return b;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return f2{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ f2 sub2(f2 a, f2 b) { return f2{a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return f2{a.x * b.x, a.y * b.y}; }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  return f2{fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y)};
}
__device__ __forceinline__ float max3f(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ float min3f(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// ---------------------------------------------------------- cp.async ----

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ------------------------------------------------------ position maps ----

// Source index of extended position q on a reflecting / periodic line.
__device__ __forceinline__ int map_pos(int q, int n, int bc) {
  if (q >= 0 && q < n) return q;
  if (bc == BC_PERIODIC) return ((q % n) + n) % n;
  const int n2 = 2 * n;
  const int m = ((q % n2) + n2) % n2;
  return m >= n ? n2 - 1 - m : m;
}

// Whether the mirror image at extended position q negates the momentum along
// the line (reflecting lines only).
__device__ __forceinline__ bool flips(int q, int n, int bc) {
  if (bc != BC_REFLECT || (q >= 0 && q < n)) return false;
  const int n2 = 2 * n;
  const int m = ((q % n2) + n2) % n2;
  return m >= n;
}

// Negates the momentum along the sweep in the pair that holds it:
// x -> hi of (E, Mx); y -> lo of (My, Mz); z -> hi of (My, Mz).
template <int AXIS>
__device__ __forceinline__ void negate_par(f2& A, f2& B) {
  if (AXIS == 0) A.y = -A.y;
  if (AXIS == 1) B.x = -B.x;
  if (AXIS == 2) B.y = -B.y;
}

// Geometry and coefficients of the event a piece of work belongs to, held
// in registers (one event of a batch).
struct ItemGeo {
  long long off;     // first cell of the event in the state arrays
  long long stride;  // cell stride along the line
  long long plane;   // lines along this axis
  long long sb, sc;  // first cell of line t = b + nb*c: off + b*sb + c*sc
  int n, nb, bc;
  const float* frozen;
  float tau_h, tau_f, htau_h, htau_f, B, ec;
  unsigned long long* clamp;
};

// Geometry accessors.  GeoP reads the launch parameters at each use
// (the single event of a launch: the values stay constant-bank operands);
// GeoR returns the registers of an ItemGeo.
struct GeoP {
  const SweepParams& P;
  __device__ __forceinline__ long long off() const { return 0; }
  __device__ __forceinline__ long long stride() const { return P.stride; }
  __device__ __forceinline__ long long plane() const { return P.plane; }
  __device__ __forceinline__ long long sb() const { return P.sb; }
  __device__ __forceinline__ long long sc() const { return P.sc; }
  __device__ __forceinline__ int n() const { return P.n; }
  __device__ __forceinline__ int nb() const { return P.nb; }
  __device__ __forceinline__ int bc() const { return P.bc; }
  __device__ __forceinline__ const float* frozen() const { return static_cast<const float*>(P.frozen); }
  __device__ __forceinline__ float tau_h() const { return P.f_tau_h; }
  __device__ __forceinline__ float tau_f() const { return P.f_tau_f; }
  __device__ __forceinline__ float htau_h() const { return P.f_htau_h; }
  __device__ __forceinline__ float htau_f() const { return P.f_htau_f; }
  __device__ __forceinline__ float B() const { return P.f_bag_B; }
  __device__ __forceinline__ float ec() const { return P.f_bag_ec; }
};
struct GeoR {
  ItemGeo g;
  __device__ __forceinline__ long long off() const { return g.off; }
  __device__ __forceinline__ long long stride() const { return g.stride; }
  __device__ __forceinline__ long long plane() const { return g.plane; }
  __device__ __forceinline__ long long sb() const { return g.sb; }
  __device__ __forceinline__ long long sc() const { return g.sc; }
  __device__ __forceinline__ int n() const { return g.n; }
  __device__ __forceinline__ int nb() const { return g.nb; }
  __device__ __forceinline__ int bc() const { return g.bc; }
  __device__ __forceinline__ const float* frozen() const { return g.frozen; }
  __device__ __forceinline__ float tau_h() const { return g.tau_h; }
  __device__ __forceinline__ float tau_f() const { return g.tau_f; }
  __device__ __forceinline__ float htau_h() const { return g.htau_h; }
  __device__ __forceinline__ float htau_f() const { return g.htau_f; }
  __device__ __forceinline__ float B() const { return g.B; }
  __device__ __forceinline__ float ec() const { return g.ec; }
};

template <int AXIS>
__device__ __forceinline__ ItemGeo geo_of(const EvDesc& D) {
  ItemGeo G;
  const long long nx = D.nx, ny = D.ny, nz = D.nz;
  G.off = D.off;
  if (AXIS == 0) {
    G.n = D.nx;
    G.stride = 1;
    G.plane = ny * nz;
    G.nb = D.ny;
    G.sb = nx;
    G.sc = nx * ny;
  } else if (AXIS == 1) {
    G.n = D.ny;
    G.stride = nx;
    G.plane = nx * nz;
    G.nb = D.nx;
    G.sb = 1;
    G.sc = nx * ny;
  } else {
    G.n = D.nz;
    G.stride = nx * ny;
    G.plane = nx * ny;
    G.nb = D.nx;
    G.sb = 1;
    G.sc = nx;
  }
  G.bc = D.bc;
  G.frozen = D.frozen[AXIS];
  G.tau_h = D.tau_h;
  G.tau_f = D.tau_f;
  G.htau_h = D.htau_h;
  G.htau_f = D.htau_f;
  G.B = D.bag_B;
  G.ec = D.bag_ec;
  G.clamp = D.clamp_count;
  return G;
}

// Copies extended position q of a line (first cell `cell0`, cell stride
// `stride`) into a ring entry (quad at dq, R at dr).  Ghost positions follow
// the boundary rule; frozen ghosts come from the frozen store (line t).
template <class Geo>
__device__ __forceinline__ void copy_cell(const SweepParams& P, const Geo& G, float* dq,
                                          float* dr, long long cell0, long long stride,
                                          long long t, int q, int n) {
  if (G.bc() == BC_FROZEN && (q < 0 || q >= n)) {
    const int side = q < 0 ? 0 : 1;
    int layer = q < 0 ? -1 - q : q - n;
    layer = layer > NG - 1 ? NG - 1 : layer;
#ifdef SHASTA_CHECKED
    const long long fi = (long long)(side * NG + layer) * NF * G.plane() + t;
    if (!SH_OK(P, fi >= 0 && t < G.plane() && fi + 4 * G.plane() < 2LL * NG * NF * G.plane(), 2, fi))
      return;
#endif
    const float* fz = G.frozen() + (long long)(side * NG + layer) * NF * G.plane() + t;
#pragma unroll
    for (int f = 0; f < 4; ++f) cp_async4(dq + f, fz + f * G.plane());
    cp_async4(dr, fz + 4 * G.plane());
    return;
  }
  const long long c = cell0 + (long long)map_pos(q, n, G.bc()) * stride;
  if (!SH_OK(P, c >= 0 && c < P.ncap, 1, c)) return;
  cp_async16(dq, P.qin + 4 * c);
  cp_async4(dr, P.rin + c);
}

// ----------------------------------------------------------- recovery ----

// p(e) of a tabulated EoS in float: linear between the nodes k de, the
// last interval continued above (the index stays inside the table for any
// e, NaN included); *slope receives dp/de of the interval.
__device__ __forceinline__ float tab32(const EosTable& T, float e, float* slope = nullptr) {
  const float x = e * T.inv_de32;
  int k = (int)x;
  k = k < 0 ? 0 : (k > T.n - 2 ? T.n - 2 : k);
  const float f = x - (float)k;
  const float a = __ldg(T.p32 + k), b = __ldg(T.p32 + k + 1);
  if (slope) *slope = (b - a) * T.inv_de32;
  return fmaf(f, b - a, a);
}

// Tabulated EoS: p from E and |M|^2.  The root is the fixed point of Sec. 3,
// |v| = |M| / (E + p(E - |M| |v|)), started as there from |M| / (E + p(E)).
// In float the root is found by Newton steps on g(v) = v - |M| / (E + p),
// g'(v) = 1 - |M|^2 p'(e) / (E + p)^2 >= 1 - v^2 p' > 0 (exact within one
// interval of the piecewise-linear table), until the change is at most
// 1e-7 (12 steps at most), then p = p(E - |M| |v|).
__device__ __forceinline__ float table_p32(const EosTable& T, float E, float M2) {
  const float M = sqrtf(M2);
  float v = M * __fdividef(1.0f, E + tab32(T, E));
#pragma unroll 1
  for (int it = 0; it < 12; ++it) {
    float dp;
    const float pe = tab32(T, fmaf(-M, v, E), &dp);
    const float r = __fdividef(1.0f, E + pe);
    const float g = fmaf(-M, r, v);               // v - M / (E + p)
    const float mr = M * r;
    const float gp = fmaf(-mr * mr, dp, 1.0f);    // 1 - M^2 p' / (E + p)^2
    const float d = __fdividef(g, gp);
    v -= d;
    if (fabsf(d) <= 1e-7f) break;
  }
  return tab32(T, fmaf(-M, v, E));
}

// Recovery arithmetic of the kernels on a float state: REC_F32 all in
// float (precision FP32); REC_DF |M|^2 and D = E^2 - |M|^2 in double-float,
// the rest in float (MIXED); REC_F64 D, the root s, p and w in double from
// the float state, rounded to float for the transport (MIXED_FP64).
constexpr int REC_F32 = 0, REC_DF = 1, REC_F64 = 2;

// REC_F64: velocity along the sweep and pressure of one cell, every
// operation in double (IEEE division and square root) on the float state;
// the same closed forms as rec32 below.  omd = 1 - delta in double.
template <int EOS>
__device__ __forceinline__ unsigned rec64(float Ef, float mxf, float myf, float mzf, float m1f,
                                          double omd, double B, double ec, float& w, float& p) {
  const double E = Ef, mx = mxf, my = myf, mz = mzf;
  unsigned clamped = 0;
  double M2 = fma(mx, mx, fma(my, my, mz * mz));
  const double lim = omd * E;
  const double L2 = lim * lim;
  double m = m1f;
  if (M2 > L2) {
    m = m * (lim / sqrt(M2));
    M2 = L2;
    clamped = 1;
  }
  double D = fmax(fma(E, E, -M2), 0.0);
  double pp;
  if constexpr (EOS == EOS_BAG) {
    const bool bag = 3.0 * D > ec * fma(2.0, E, ec);
    const double b = bag ? B : 0.0;
    const double q = fma(-4.0, b, E);
    const double r = fma(3.0, D, fma(q, q, -12.0 * (b * b)));
    const double s = sqrt(fmax(r, 0.0));
    pp = fma(-(4.0 / 3.0) * b, E, D) / fma(-2.0, b, E + s) - (4.0 / 3.0) * b;
    if (bag && !(E > ec && r >= 0.0 && fma(3.0, pp, 4.0 * B) > ec)) pp = M2 / (E - ec) - E;
  } else {
    const double s = sqrt(fma(3.0, D, E * E));
    pp = D / (E + s);
  }
  w = (float)(m / (E + pp));
  p = (float)pp;
  if (!(E > 0.0)) {
    w = 0.0f;
    p = 0.0f;
    clamped = 1;
  }
  return clamped;
}

// Velocity along the sweep and pressure of one cell, FP32 (REC_DF: D in
// double-float; REC_F64: rec64).  mx, my, mz are the momenta, m1 the one
// along the sweep.  Returns 1 if |M| was clamped or E <= 0.
template <int EOS, int REC>
__device__ __forceinline__ unsigned rec32(float E, float mx, float my, float mz, float m1,
                                          float omd, double omd64, float B, float ec,
                                          const EosTable& T, float& w, float& p) {
  if constexpr (REC == REC_F64 && EOS != EOS_TABLE)
    return rec64<EOS>(E, mx, my, mz, m1, omd64, B, ec, w, p);
  unsigned clamped = 0;
  float M2, M2lo = 0.0f;  // |M|^2; REC_DF: an unevaluated sum M2 + M2lo
  if constexpr (REC == REC_DF) {
    // |M|^2 = hi + lo from error-free products and compensated sums
    const float a = mx * mx, a_l = fmaf(mx, mx, -a);
    const float b = my * my, b_l = fmaf(my, my, -b);
    const float c = mz * mz, c_l = fmaf(mz, mz, -c);
    const float s1 = a + b;
    float bb = s1 - a;
    const float r1 = (a - (s1 - bb)) + (b - bb);
    M2 = s1 + c;
    bb = M2 - s1;
    const float r2 = (s1 - (M2 - bb)) + (c - bb);
    M2lo = ((a_l + b_l) + c_l) + (r1 + r2);
  } else {
    M2 = fmaf(mx, mx, fmaf(my, my, mz * mz));
  }
  const float E2 = E * E;
  const float lim = omd * E;
  const float L2 = lim * lim;
  float m = m1;
  float D;
  if (M2 > L2) {
    // |M| clamped to (1 - delta) E (rare): scale the momentum
    m = m1 * (lim * rsqrtf(M2));
    M2 = L2;
    D = E2 - M2;
    clamped = 1;
  } else if (REC == REC_DF) {
    // D = E^2 - |M|^2: E^2 - hi in one fused multiply-add (one rounding of
    // the exact difference), then lo
    D = fmaf(E, E, -M2) - M2lo;
  } else {
    D = E2 - M2;
  }
  float pp;
  if constexpr (EOS == EOS_TABLE) {
    pp = table_p32(T, E, M2);
  } else if constexpr (EOS == EOS_BAG) {
    // One root for both branches.  With R0 = E^2 + 3D the ideal-gas root
    // e = sqrt(R0) - E lies above e_c exactly when R0 > (E + e_c)^2; then
    // the bag root with p = (e - 4b)/3, else b = 0, which is the ideal-gas
    // root itself (p = D / (E + sqrt(R0))):
    //   p = (D - 4bE/3) / (E - 2b + sqrt(r)) - 4b/3,  r = R0 - 4b (2E - b)
    // (r = 3D + (E - 4b)^2 - 12b^2).
    D = fmaxf(D, 0.0f);
    const float R0 = fmaf(3.0f, D, E2);
    const float te = E + ec;
    const bool bag = R0 > te * te;
    const float b = bag ? B : 0.0f;
    const float r = fmaf(-4.0f * b, fmaf(2.0f, E, -b), R0);
    const float s = sqrtf(fmaxf(r, 0.0f));
    const float b43 = (4.0f / 3.0f) * b;
    pp = fmaf(fmaf(-b43, E, D), __fdividef(1.0f, fmaf(-2.0f, b, E + s)), -b43);
    // the bag root must exist and lie above e_c; else the mixed-phase point
    if (bag && !(E > ec && r >= 0.0f && fmaf(3.0f, pp, 4.0f * B) > ec))
      pp = __fdividef(M2, E - ec) - E;
  } else {
    D = fmaxf(D, 0.0f);
    const float s = sqrtf(fmaf(3.0f, D, E2));
    pp = D * __fdividef(1.0f, E + s);
  }
  w = m * __fdividef(1.0f, E + pp);
  p = pp;
  if (!(E > 0.0f)) {
    w = 0.0f;
    p = 0.0f;
    clamped = 1;
  }
  return clamped;
}

// The two recoveries of a streaming step (halves lo: U^n of the newest
// cell, hi: U^(n+1/2) four cells back): E, the three momenta and the
// momentum along the sweep.  cnt counts the lo cell when in_seg (a cell of
// the piece's own positions) and it was clamped or vacuum.
template <int EOS, int REC>
__device__ __forceinline__ void rec2(f2 E, f2 mx, f2 my, f2 mz, f2 mpar, float omd, double omd64,
                                     float B, float ec, const EosTable& T, f2& w, f2& p,
                                     unsigned& cnt, bool in_seg) {
  float wl, wh, pl, ph;
  const unsigned c =
      rec32<EOS, REC>(E.x, mx.x, my.x, mz.x, mpar.x, omd, omd64, B, ec, T, wl, pl);
  if (c) cnt += in_seg ? 1u : 0u;
  rec32<EOS, REC>(E.y, mx.y, my.y, mz.y, mpar.y, omd, omd64, B, ec, T, wh, ph);
  w = f2{wl, wh};
  p = f2{pl, ph};
}

// ------------------------------------------------------- antidiffusion ----

// Flux limiter of Sec. 3 on one field: A = s max(0, min(s dhp, |aph|, s dhm))
// with s = sgn(aph) (aph = 0 gives 0), written without the sign as
// max(lo, min(hi, 0)) with lo = min3(dhp, aph, dhm), hi = max3(...): for
// aph > 0, hi >= aph > 0 and the result is max(lo, 0); for aph < 0,
// lo <= aph <= min(hi, 0) and the result is min(hi, 0); for aph = 0 it is 0.
__device__ __forceinline__ float limit(float aph, float dhp, float dhm) {
  return fmaxf(min3f(dhp, aph, dhm), fminf(max3f(dhp, aph, dhm), 0.0f));
}

// ------------------------------------------------------ line pipeline ----
//
// One SHASTA pass of a field pair along the line, written with differences
// so that every carried quantity is needed for at most two positions.  With
// the newest cell k (U_k just read), one step computes
//   Delta_{k-1} = U_k - U_{k-1}
//   Uhat_{k-1}  = a Delta_{k-1} + nb Delta_{k-2} + c U_{k-1} (+ source)      [Eq. shasta-geo]
//   DD_{k-1}    = Delta_{k-1} - Delta_{k-2},  D2_{k-2} = DD_{k-1} - DD_{k-2}
//   Dh_{k-2}    = Uhat_{k-1} - Uhat_{k-2}                                   [Delta-hat]
//   A_{k-3}     = limit(eta (Dh_{k-3} - D2_{k-3}/8), Dh_{k-2}, Dh_{k-4})    [phoenical + limiter]
//   out_{k-3}   = (Uhat_{k-3} + A_{k-4}) - A_{k-3}                          [Eq. shasta-n]
// Two-slot arrays are indexed by position parity; K is the parity of k.
// With AF false the antidiffusion stage is left out (A = 0, the result of
// eta = 0): out_{k-3} = Uhat_{k-3}, the transport alone.
struct Line2 {
  f2 Up[2];  // U by parity
  f2 D[2];   // Delta
  f2 DD[2];  // first difference of Delta
  f2 D2[2];  // second difference of Delta
  f2 Uh[2];  // transported values
  f2 Dh[2];  // their differences
  f2 A[2];   // limited fluxes
};
struct Line1 {
  float Up[2], D[2], DD[2], D2[2], Uh[2], Dh[2], A[2];
};

template <int K, bool SRC, bool AF>
__device__ __forceinline__ f2 step2(Line2& s, f2 u, f2 a2, f2 nb2, f2 c2, f2 src, f2 eta2, f2 m8) {
  constexpr int P0 = K & 1, P1 = (K + 1) & 1;  // parity of k (= k-2, k-4) and of k-1 (= k-3)
  if constexpr (!AF) {
    const f2 out = s.Uh[P1];                                     // Uhat_{k-3}
    const f2 d = sub2(u, s.Up[P1]);
    s.Uh[P1] = fma2(c2, s.Up[P1], fma2(a2, d, SRC ? fma2(nb2, s.D[P0], src) : mul2(nb2, s.D[P0])));
    s.Up[P0] = u;
    s.D[P1] = d;
    return out;
  }
  // values whose slots are overwritten below are consumed first
  const f2 aph = mul2(eta2, fma2(m8, s.D2[P1], s.Dh[P1]));        // A^ph_{k-3}
  const f2 t = add2(s.Uh[P1], s.A[P0]);                          // Uhat_{k-3} + A_{k-4}
  const f2 d = sub2(u, s.Up[P1]);                                // Delta_{k-1}
  // Uhat_{k-1}, the source folded into the innermost term
  const f2 uh = fma2(c2, s.Up[P1], fma2(a2, d, SRC ? fma2(nb2, s.D[P0], src) : mul2(nb2, s.D[P0])));
  const f2 dd = sub2(d, s.D[P0]);                                // DD_{k-1}
  const f2 d2 = sub2(dd, s.DD[P0]);                              // D2_{k-2}
  const f2 dh = sub2(uh, s.Uh[P0]);                              // Dh_{k-2}
  const f2 A = f2{limit(aph.x, dh.x, s.Dh[P0].x), limit(aph.y, dh.y, s.Dh[P0].y)};
  s.A[P1] = A;
  s.Up[P0] = u;
  s.D[P1] = d;
  s.DD[P1] = dd;
  s.D2[P0] = d2;
  s.Uh[P1] = uh;
  s.Dh[P0] = dh;
  return sub2(t, A);
}

template <int K, bool AF>
__device__ __forceinline__ float step1(Line1& s, float u, float a, float nb, float c, float eta) {
  constexpr int P0 = K & 1, P1 = (K + 1) & 1;
  if constexpr (!AF) {
    const float out = s.Uh[P1];
    const float d = u - s.Up[P1];
    s.Uh[P1] = fmaf(c, s.Up[P1], fmaf(a, d, nb * s.D[P0]));
    s.Up[P0] = u;
    s.D[P1] = d;
    return out;
  }
  const float aph = eta * fmaf(-0.125f, s.D2[P1], s.Dh[P1]);
  const float qm = s.Dh[P0];
  const float t = s.Uh[P1] + s.A[P0];
  const float d = u - s.Up[P1];
  const float uh = fmaf(c, s.Up[P1], fmaf(a, d, nb * s.D[P0]));
  const float dd = d - s.D[P0];
  const float d2 = dd - s.DD[P0];
  const float dh = uh - s.Uh[P0];
  const float A = limit(aph, dh, qm);
  s.A[P1] = A;
  s.Up[P0] = u;
  s.D[P1] = d;
  s.DD[P1] = dd;
  s.D2[P0] = d2;
  s.Uh[P1] = uh;
  s.Dh[P0] = dh;
  return t - A;
}

__device__ __forceinline__ void init2(Line2& s, f2 u0) {
  const f2 z = pk(0.0f, 0.0f);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    s.Up[k] = u0;
    s.A[k] = s.D[k] = s.DD[k] = s.D2[k] = s.Uh[k] = s.Dh[k] = z;
  }
}
__device__ __forceinline__ void init1(Line1& s) {
#pragma unroll
  for (int k = 0; k < 2; ++k) s.Up[k] = s.A[k] = s.D[k] = s.DD[k] = s.D2[k] = s.Uh[k] = s.Dh[k] = 0.0f;
}

// Transport coefficients of cell k-1 from w_{k-1}, w_k and Q+_{k-2}:
// Q+ of Eq. shasta-diff and Q-_{k-1} = 1 - Q+_{k-2}.  Every fused
// multiply-add is written out (the unit is built without contraction), so
// each instantiation of the streaming step rounds identically.
__device__ __forceinline__ void coeffs(float tau, float w1, float w0, float& qprev, float& a,
                                       float& nb, float& c) {
  const float num = fmaf(-tau, w1, 0.5f);          // 1/2 - eps_{k-1}
  const float den = fmaf(tau, w0 - w1, 1.0f);      // 1 + (eps_k - eps_{k-1})
  const float qp = num * __fdividef(1.0f, den);
  const float qm = 1.0f - qprev;
  qprev = qp;
  a = 0.5f * (qp * qp);
  nb = -0.5f * (qm * qm);
  c = qp + qm;
}

// Pressure sources of the pairs (E, Mx) and (My, Mz) from the difference of
// (p w, p) two cells apart: E gets the p w term, the momentum along the
// sweep the p term.
template <int AXIS>
__device__ __forceinline__ void sources(f2 ht2, float ht, f2 fdiff, f2& sA, f2& sB) {
  if (AXIS == 0) {
    sA = mul2(ht2, fdiff);
    sB = pk(0.0f, 0.0f);
  } else {
    float pwd, pd;
    up(fdiff, pwd, pd);
    sA = pk(ht * pwd, 0.0f);
    sB = AXIS == 1 ? pk(ht * pd, 0.0f) : pk(0.0f, ht * pd);
  }
}

// Shared memory per warp, in floats.
template <int AXIS, int RING>
struct Smem {
  static constexpr int per_warp = AXIS == 0 ? XSLOTS * XSLOT : RING * YSLOT;
};

template <int V>
using ic = std::integral_constant<int, V>;
template <bool V>
using bc_ = std::integral_constant<bool, V>;

// ------------------------------------------------------------- kernel ----
//
// Pipeline (q = newest loaded position; lag 7):
//   U^n_q read; (w, p)^n_q and (w, p)^h_{q-4} recovered (two scalar chains)
//   half-step pass of (E, M) with newest cell q      -> U^h_{q-3}
//   full-step pass of (E, M, R) with newest cell q-4 -> U^{n+1}_{q-7}

// One piece of work: positions [s0, s1) of the 32 lines of line group g of
// the event described by G (x path: s0 and, unless s1 = n, s1 on 8-cell
// chunk boundaries).
template <int EOS, int AXIS, int REC, int RING, int DIST, bool AF, class Geo>
__device__ __forceinline__ void sweep_item(const SweepParams& P, const Geo& G, int g, int s0, int s1,
                                           float* wsm, int lane, unsigned& nclamp) {
  constexpr bool XP = AXIS == 0;
  constexpr int LAG = 7;
  static_assert(RING == 8 && DIST == 3, "ring layout assumes 8 slots, 3 ahead");
  const int n = G.n();
  const long long t = (long long)g * LANES + lane;
  const bool valid = t < G.plane();
  const long long tl = valid ? t : G.plane() - 1;
  // cells of the piece this lane owns: q - s0 in [0, span) (none past the last line)
  const unsigned span = valid ? (unsigned)(s1 - s0) : 0u;
  const long long base = G.off() + (tl % G.nb()) * G.sb() + (tl / G.nb()) * G.sc();  // first cell of the line
  // positions streamed: qs .. qe (the x path starts on a chunk boundary)
  const int qs = XP ? ((s0 - 2 * NG) & ~(CH - 1)) : s0 - 2 * NG;
  const int qe = s1 + LAG - 1;
  const int trip = ((qe - qs + 1) + 7) & ~7;
  // steady blocks [i1, i2): every position they touch is inside [0, n)
  // (reads q, q-3 and q-4, prefetch ahead, store q-7)
  const int ahead = XP ? 2 * CH : DIST;
  int i1 = (4 - qs) > 0 ? ((4 - qs) + 7) & ~7 : 0;
  int i2 = (n - 1 - ahead) - qs + 1;
  i2 = i2 > 0 ? (i2 & ~7) : 0;
  i2 = i2 < trip ? i2 : trip;
  if (i2 < i1) i2 = i1;

  const float tau_h = G.tau_h(), tau_f = G.tau_f();
  const float eta = P.f_eta;
  const float omd = P.f_omd, B = G.B(), ec = G.ec();
  const float htau_h = G.htau_h(), htau_f = G.htau_f();
  const f2 eta2 = pk(eta, eta), m8c = pk(-0.125f, -0.125f);
  const f2 ht_h2 = pk(htau_h, htau_h), ht_f2 = pk(htau_f, htau_f);
  const bool frozen = G.bc() == BC_FROZEN;

#ifdef SHASTA_CHECKED
  // whether nf floats at p lie in this warp's ring
  auto sm_in = [&](const float* p, int nf) {
    const long long o = p - wsm;
    constexpr long long kRing = Smem<AXIS, RING>::per_warp;
    return SH_OK(P, o >= 0 && o + nf <= kRing, 4, o);
  };
#endif

  auto x_slot = [&](int C) -> float* { return wsm + ((C + 3 * 4) % XSLOTS) * XSLOT; };
  // x path: cooperative copy of chunk C = positions [8C, 8C+8) of 32 rows
  // (the ghost variant, rare, stays a rolled loop: the x kernel is
  // sensitive to code size)
  auto x_issue = [&](int C, bool ghost) {
    float* ring = x_slot(C);
    const int r0 = lane >> 3, pc = lane & 7;
    const int pos = C * CH + pc;
    if (ghost) {
#pragma unroll 1
      for (int k = 0; k < 8; ++k) {
        const int row = r0 + 4 * k;
        long long tr = g * LANES + row;
        tr = tr < G.plane() ? tr : G.plane() - 1;
        copy_cell(P, G, ring + row * XQSTR + pc * 4, ring + XQ + row * XRSTR + pc,
                  G.off() + tr * G.sb(), 1, tr, pos, n);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int row = r0 + 4 * k;
        long long tr = g * LANES + row;
        tr = tr < G.plane() ? tr : G.plane() - 1;
        const unsigned c = (unsigned)G.off() + (unsigned)tr * (unsigned)G.sb() + (unsigned)pos;
        if (!SH_OK(P, (long long)c < P.ncap, 1, c)) continue;
        cp_async16(ring + row * XQSTR + pc * 4, P.qin + 4 * (size_t)c);
        cp_async4(ring + XQ + row * XRSTR + pc, P.rin + c);
      }
    }
  };
  const unsigned base32 = (unsigned)base, stride32 = (unsigned)G.stride();
  // y/z path: own-lane copy of position q into ring slot `slot`
  auto yz_issue = [&](float* slot, int q, bool ghost) {
    float* dq = slot + lane * 4;
    float* dr = slot + YQ + lane;
#ifdef SHASTA_CHECKED
    if (!sm_in(dq, 4) || !sm_in(dr, 1)) return;
#endif
    if (ghost) {
      copy_cell(P, G, dq, dr, base, G.stride(), tl, q, n);
    } else {
      const unsigned c = base32 + (unsigned)q * stride32;
      if (!SH_OK(P, (long long)c < P.ncap, 1, c)) return;
      cp_async16(dq, P.qin + 4 * (size_t)c);
      cp_async4(dr, P.rin + c);
    }
  };
  // quad (as the pairs (E, Mx), (My, Mz)) and R of a ring entry
  auto rdq = [&](const float* slot, int pos, f2& A, f2& Bp) {
#ifdef SHASTA_CHECKED
    if (!sm_in(XP ? slot + lane * XQSTR + pos * 4 : slot + lane * 4, 4)) {
      A = Bp = pk(0.0f, 0.0f);
      return;
    }
#endif
    const float4 v = *reinterpret_cast<const float4*>(XP ? slot + lane * XQSTR + pos * 4 : slot + lane * 4);
    A = pk(v.x, v.y);
    Bp = pk(v.z, v.w);
  };
  auto rdr = [&](const float* slot, int pos) -> float {
#ifdef SHASTA_CHECKED
    if (!sm_in(XP ? slot + XQ + lane * XRSTR + pos : slot + YQ + lane, 1)) return 0.0f;
#endif
    return XP ? slot[XQ + lane * XRSTR + pos] : slot[YQ + lane];
  };

  // prologue
  if (XP) {
    x_issue(qs >> 3, true);
    cp_commit();
  } else {
#pragma unroll 1
    for (int d = 0; d < DIST; ++d) {
      if (qs + d <= qe) yz_issue(wsm + d * YSLOT, qs + d, true);
      cp_commit();
    }
  }

  // per-line state: pairs A = (E, Mx), B = (My, Mz)
  Line2 hA, hB, fA, fB;  // half-step and full-step passes
  Line1 fR;              // full-step pass of R
  init2(hA, pk(1.0f, 0.0f));
  init2(hB, pk(0.0f, 0.0f));
  init2(fA, pk(1.0f, 0.0f));
  init2(fB, pk(0.0f, 0.0f));
  init1(fR);
  f2 HA = pk(1.0f, 0.0f), HB = pk(0.0f, 0.0f);  // U^h_{q-4}, recovered next step
  float wn1 = 0.0f, wh1 = 0.0f;                 // w^n_{q-1}, w^h_{q-5}
  f2 fn[2], fh[2];                               // (p w, p) by parity
  fn[0] = fn[1] = fh[0] = fh[1] = pk(0.0f, 0.0f);
  float qph = 0.5f, qpf = 0.5f;                 // Q+ of the previous cell

  // One streaming step at position q = qs + i + K (K = parity of q - qs).
  //   sq, sq4: ring slots of positions q and q-4; sjo: slot of output
  //   position q-7 (x path); siss: slot receiving position q + DIST (y/z).
  auto body = [&](int i, auto Kc, auto Gc, const float* sq, const float* sq4, float* sjo,
                  float* siss) {
    constexpr int K = decltype(Kc)::value;
    constexpr bool GH = decltype(Gc)::value;
    constexpr int P0 = K & 1;
    const int q = qs + i + K;
    const int pq = XP ? (q & 7) : 0;
    const int pq4 = XP ? ((q - 4) & 7) : 0;
    if (!XP) cp_wait<DIST - 1>();
    // ---- U^n_q (E, M)
    f2 uA, uB;
    rdq(sq, pq, uA, uB);
    if (GH && flips(q, n, G.bc())) negate_par<AXIS>(uA, uB);
    if (!XP) {
      if (GH) {
        if (q + DIST <= qe) yz_issue(siss, q + DIST, true);
      } else {
        yz_issue(siss, q + DIST, false);
      }
      cp_commit();
    }
    // ---- recovery of U^n_q (lo) and U^h_{q-4} (hi) together
    float wn0, wh0;
    f2 fn0, fh0;
    {
      const f2 E = pk(lo_of(uA), lo_of(HA));
      const f2 mx = pk(hi_of(uA), hi_of(HA));
      const f2 my = pk(lo_of(uB), lo_of(HB));
      const f2 mz = pk(hi_of(uB), hi_of(HB));
      const f2 mpar = AXIS == 0 ? mx : (AXIS == 1 ? my : mz);
      f2 w2, p2;
      // count each cell of the piece once (lanes past the last line only
      // repeat it)
      rec2<EOS, REC>(E, mx, my, mz, mpar, omd, P.omd, B, ec, P.tab, w2, p2, nclamp,
                       (unsigned)(q - s0) < span);
      float pl, phi, pwl, pwh;
      up(w2, wn0, wh0);
      up(p2, pl, phi);
      up(mul2(p2, w2), pwl, pwh);
      fn0 = pk(pwl, pl);
      fh0 = pk(pwh, phi);
    }
    // ---- half-step pass, newest cell q: U^h_{q-3}
    {
      float a, nb, c;
      coeffs(tau_h, wn1, wn0, qph, a, nb, c);
      f2 sA, sB;
      sources<AXIS>(ht_h2, htau_h, sub2(fn[P0], fn0), sA, sB);  // f_{q-2} - f_q
      fn[P0] = fn0;
      wn1 = wn0;
      const f2 a2 = pk(a, a), nb2 = pk(nb, nb), c2 = pk(c, c);
      HA = step2<K, true, AF>(hA, uA, a2, nb2, c2, sA, eta2, m8c);
      HB = step2<K, AXIS != 0, AF>(hB, uB, a2, nb2, c2, sB, eta2, m8c);
      if (GH && frozen && (q - NG < 0 || q - NG >= n)) {
        // frozen ghost: the half-step state is the stored ghost value
        const float* s3 = XP ? x_slot((q - NG) >> 3) : wsm + ((q - NG - qs) & (RING - 1)) * YSLOT;
        rdq(s3, XP ? ((q - NG) & 7) : 0, HA, HB);
      }
    }
    // ---- full-step pass, newest cell q-4 (old state re-read): U^{n+1}_{q-7}
    f2 oA, oB;
    float oR;
    {
      f2 vA, vB;
      rdq(sq4, pq4, vA, vB);
      const float vR = rdr(sq4, pq4);
      if (GH && flips(q - 4, n, G.bc())) negate_par<AXIS>(vA, vB);
      float a, nb, c;
      coeffs(tau_f, wh1, wh0, qpf, a, nb, c);
      f2 sA, sB;
      sources<AXIS>(ht_f2, htau_f, sub2(fh[P0], fh0), sA, sB);  // f_{q-6} - f_{q-4}
      fh[P0] = fh0;
      wh1 = wh0;
      const f2 a2 = pk(a, a), nb2 = pk(nb, nb), c2 = pk(c, c);
      oA = step2<K, true, AF>(fA, vA, a2, nb2, c2, sA, eta2, m8c);
      oB = step2<K, AXIS != 0, AF>(fB, vB, a2, nb2, c2, sB, eta2, m8c);
      oR = step1<K, AF>(fR, vR, a, nb, c, eta);
    }
    const int jo = q - LAG;
    if (XP) {
      // the ring entry of position jo is dead: stage the result there
      if ((unsigned)(jo - s0) < (unsigned)(s1 - s0)) {
        const int pj = jo & 7;
        float o0, o1, o2, o3;
        up(oA, o0, o1);
        up(oB, o2, o3);
#ifdef SHASTA_CHECKED
        if (!sm_in(sjo + lane * XQSTR + pj * 4, 4) || !sm_in(sjo + XQ + lane * XRSTR + pj, 1)) return;
#endif
        *reinterpret_cast<float4*>(sjo + lane * XQSTR + pj * 4) = make_float4(o0, o1, o2, o3);
        sjo[XQ + lane * XRSTR + pj] = oR;
      }
    } else if ((unsigned)(jo - s0) < span) {
      const unsigned c = base32 + (unsigned)jo * stride32;
      if (!SH_OK(P, (long long)c < P.ncap, 3, c)) return;
      float o0, o1, o2, o3;
      up(oA, o0, o1);
      up(oB, o2, o3);
      *reinterpret_cast<float4*>(P.qout + 4 * (size_t)c) = make_float4(o0, o1, o2, o3);
      P.rout[c] = oR;
    }
  };

  // two steps: positions qs+i and qs+i+1 (i even)
  auto duo = [&](int i, auto Gc) {
    if (XP) {
      const int C = (qs + i) >> 3;  // chunk of both positions
      float* pC = x_slot(C);
      float* pCm = x_slot(C - 1);
      const float* s4 = ((qs + i) & 4) ? pC : pCm;  // chunk of positions q-4
      body(i, ic<0>{}, Gc, pC, s4, pCm, nullptr);
      body(i, ic<1>{}, Gc, pC, s4, ((qs + i + 1) & 7) == 7 ? pC : pCm, nullptr);
    } else {
      const int r = i & 7;  // ring slot of position qs+i
      float* yb = wsm + r * YSLOT;
      float* yb4 = wsm + (r ^ 4) * YSLOT;
      body(i, ic<0>{}, Gc, yb, yb4, nullptr, wsm + ((r + 3) & 7) * YSLOT);
      body(i, ic<1>{}, Gc, yb + YSLOT, yb4 + YSLOT, nullptr, wsm + ((r + 4) & 7) * YSLOT);
    }
  };
  // steps actually needed: positions qs .. qe, in whole duos; the x path
  // starts its first chunk at s0 - 6 (the sweep's reach), not at the chunk
  // boundary below it
  const int steps = ((qe - qs + 1) + 1) & ~1;
  const int hbeg0 = ((s0 - 2 * NG) - qs) & ~1;

  int fl = s0;  // x path: next output position to write back
#pragma unroll 1
  for (int i0 = 0; i0 < trip; i0 += 8) {
    const bool steady = i0 >= i1 && i0 + 8 <= i2;
    if (XP) {
      // chunk (qs + i0) / 8 becomes resident; prefetch the next one
      const int C = (qs + i0) >> 3;
      cp_wait<0>();
      __syncwarp();
      if (steady)
        x_issue(C + 1, false);
      else if (C + 1 <= (qe >> 3))
        x_issue(C + 1, true);
      cp_commit();
    }
    // the last block stops after the last needed duo
    const int hend = min(8, steps - i0);
#pragma unroll 1
    for (int h = i0 == 0 ? hbeg0 : 0; h < hend; h += 2) {
      if (steady)
        duo(i0 + h, bc_<false>{});
      else
        duo(i0 + h, bc_<true>{});
    }
    if (XP) {
      // write back completed output chunks (positions [fl, avail))
      const int avail = min(qs + i0 + 8 - LAG, s1);
#pragma unroll 1
      while (fl < s1 && (avail - fl >= CH || avail == s1)) {
        __syncwarp();
        const float* ring = x_slot(fl >> 3);
        const int r0 = lane >> 3, pc = lane & 7;
        const int pos = fl + pc;
        if (pos < avail && (long long)(g + 1) * LANES <= G.plane()) {
          // a full line group: every row exists
          const unsigned sb4 = 4u * (unsigned)G.sb();
          unsigned c = (unsigned)G.off() + (unsigned)(g * LANES + r0) * (unsigned)G.sb() + (unsigned)pos;
#pragma unroll 4
          for (int k = 0; k < 8; ++k, c += sb4) {
            const int row = r0 + 4 * k;
            if (!SH_OK(P, (long long)c < P.ncap, 3, c)) continue;
            *reinterpret_cast<float4*>(P.qout + 4 * (size_t)c) =
                *reinterpret_cast<const float4*>(ring + row * XQSTR + pc * 4);
            P.rout[c] = ring[XQ + row * XRSTR + pc];
          }
        } else if (pos < avail) {
#pragma unroll 2
          for (int k = 0; k < 8; ++k) {
            const int row = r0 + 4 * k;
            const long long tr = g * LANES + row;
            if (tr < G.plane()) {
              const unsigned c = (unsigned)G.off() + (unsigned)tr * (unsigned)G.sb() + (unsigned)pos;
              if (!SH_OK(P, (long long)c < P.ncap, 3, c)) continue;
              *reinterpret_cast<float4*>(P.qout + 4 * (size_t)c) =
                  *reinterpret_cast<const float4*>(ring + row * XQSTR + pc * 4);
              P.rout[c] = ring[XQ + row * XRSTR + pc];
            }
          }
        }
        __syncwarp();
        fl = min(fl + CH, s1);
      }
    }
  }
  cp_wait<0>();
  __syncwarp();
}

// Work of one launch: the positions of all line groups of the single event
// of P, or of the events of the work list L (BATCH), numbered group by group
// (event after event) and cut into ranges of P.range_len positions; warp w
// takes ranges w, w + warps, ...  A range is streamed piece by piece (one
// piece per line group it touches, each with its own halo); on the x path
// range boundaries are moved down to 8-cell chunk boundaries of their line.
// One event may instead take the host's table of range bounds (P.ranges:
// ranges of equal streaming cost, chunk-aligned on the x path); a batch may
// take whole line groups as work units (range_len 0).
template <int EOS, int AXIS, int REC, int WARPS, int RING, int DIST, bool BATCH, bool AF = true>
__device__ __forceinline__ void sweep_items(const SweepParams& P, const BatchList& L) {
  constexpr bool XP = AXIS == 0;
  extern __shared__ __align__(16) float smem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  float* wsm = smem + (size_t)warp * Smem<AXIS, RING>::per_warp;
  // position counts of one launch stay below 2^31 (checked on the host)
  const int nwarps = (int)gridDim.x * WARPS;
  const int first = (int)blockIdx.x * WARPS + warp;
  const int len = (int)P.range_len;
  unsigned nclamp = 0;
  if constexpr (BATCH) {
    const int total = L.nlist > 0 ? L.prefix[L.nlist] : 0;
    // list entry holding position x: the largest k with prefix[k] <= x
    auto entry = [&](int x) {
      int lo = 0, hi = L.nlist - 1;
#pragma unroll 1
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (L.prefix[mid] <= x)
          lo = mid;
        else
          hi = mid - 1;
      }
      return lo;
    };
    auto bound = [&](int x) -> int {
      if (!XP || x >= total) return x;
      const int k = entry(x);
      return x - ((x - L.prefix[k]) % L.ev[L.idx[k]].nx) % CH;
    };
    if (len <= 0) {
      // line-group mode: prefix counts line groups; a work unit is one
      // whole line group
#pragma unroll 1
      for (int r = first; r < total; r += nwarps) {
        const int k = entry(r);
        const GeoR G{geo_of<AXIS>(L.ev[L.idx[k]])};
        sweep_item<EOS, AXIS, REC, RING, DIST, AF>(P, G, r - L.prefix[k], 0, G.n(), wsm, lane, nclamp);
        if (nclamp && G.g.clamp) atomicAdd(G.g.clamp, (unsigned long long)nclamp);
        nclamp = 0;
      }
      return;
    }
    const int nranges = (total + len - 1) / len;
#pragma unroll 1
    for (int r = first; r < nranges; r += nwarps) {
      int x = bound(r * len);
      const int end = bound(min(r * len + len, total));
#pragma unroll 1
      while (x < end) {
        const int k = entry(x);
        const GeoR G{geo_of<AXIS>(L.ev[L.idx[k]])};
        const int n = G.n();
        const int loc = x - L.prefix[k];
        const int g = loc / n;
        const int s0 = loc - g * n;
        const int pe = min(end, x - s0 + n);  // the piece ends with the range or the line group
        sweep_item<EOS, AXIS, REC, RING, DIST, AF>(P, G, g, s0, s0 + (pe - x), wsm, lane, nclamp);
        if (nclamp && G.g.clamp) atomicAdd(G.g.clamp, (unsigned long long)nclamp);
        nclamp = 0;
        x = pe;
      }
    }
  } else {
    const GeoP G{P};
    const int n = P.n;
    const int total = (int)((P.plane + LANES - 1) / LANES) * n;
    auto bound = [&](int x) -> int { return XP && x < total ? x - (x % n) % CH : x; };
    // uniform ranges of len positions, or the host's table of balanced bounds
    const int nranges = P.ranges ? (int)P.nranges : (total + len - 1) / len;
#pragma unroll 1
    for (int r = first; r < nranges; r += nwarps) {
      int x, end;
      if (P.ranges) {
        if (!SH_OK(P, r + 1 <= P.nranges, 5, r)) break;
        x = P.ranges[r];
        end = P.ranges[r + 1];
      } else {
        x = bound(r * len);
        end = bound(min(r * len + len, total));
      }
#pragma unroll 1
      while (x < end) {
        const int g = x / n;
        const int s0 = x - g * n;
        const int pe = min(end, x - s0 + n);
        sweep_item<EOS, AXIS, REC, RING, DIST, AF>(P, G, g, s0, s0 + (pe - x), wsm, lane, nclamp);
        x = pe;
      }
    }
    if (nclamp && P.clamp_count) atomicAdd(P.clamp_count, (unsigned long long)nclamp);
  }
}

// One event: the launch's work is that of P.
template <int EOS, int AXIS, int REC, int WARPS, int RING, int DIST, int MINB>
__global__ void __launch_bounds__(WARPS * 32, MINB) sweep_fast_kernel(SweepParams P) {
  sweep_items<EOS, AXIS, REC, WARPS, RING, DIST, false>(P, BatchList{});
}

// One event without the antidiffusion stage (the transport alone): an
// ablation measuring what antidiffusion and limiter cost.
template <int EOS, int AXIS, int WARPS, int RING, int DIST, int MINB>
__global__ void __launch_bounds__(WARPS * 32, MINB) sweep_noaf_kernel(SweepParams P) {
  sweep_items<EOS, AXIS, REC_F32, WARPS, RING, DIST, false, false>(P, BatchList{});
}

// A batch: the work of every event of the work list L, all swept along
// AXIS; P supplies the batch's state arrays, eta and 1 - delta.
template <int EOS, int AXIS, int REC, int WARPS, int RING, int DIST, int MINB>
__global__ void __launch_bounds__(WARPS * 32, MINB) sweep_batch_kernel(SweepParams P, BatchList L) {
  sweep_items<EOS, AXIS, REC, WARPS, RING, DIST, true>(P, L);
}

}  // namespace fast
}  // namespace shasta

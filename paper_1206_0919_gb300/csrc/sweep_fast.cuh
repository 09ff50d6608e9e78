// sweep_fast.cuh -- FP32 fused SHASTA sweep tuned for sm_103a.
//
// Same sweep as sweep.cuh (arXiv:1206.0919, Sec. 3: half step with lambda/2,
// recovery at n+1/2, full step from the old state), reorganised for
// throughput:
//
//  * One warp streams 32 lines (one per lane) along the sweep axis.  Lines
//    may be cut into segments (each with its own 6-cell halo per side) so
//    that small grids still fill the machine.
//  * Input cells are staged through a per-warp shared-memory ring filled
//    with cp.async ahead of use.  For y/z sweeps each lane copies its own
//    line (the lanes of one position are adjacent in memory).  For x sweeps
//    the warp copies chunks of 8 positions x 32 rows cooperatively (8 lanes
//    per 32-byte row segment) and writes results back the same way from the
//    ring entries it no longer needs, so global accesses stay
//    sector-complete.
//  * The loop is unrolled by 4 and every register window is a circular
//    buffer indexed at compile time: no window shifting.
//  * The old state for the full step is re-read from the ring (it is still
//    resident) instead of being carried in registers.
//  * Transport factors use Q-_j = 1 - Q+_{j-1}, exact for Eq. shasta-diff
//    (the two share the denominator 1 + eps_j - eps_{j-1}), so each cell
//    needs one division per pass.
//  * The baryon density R is not transported at the half step: only E and M
//    enter the recovery at n+1/2.
//  * Recovery for p = e/3 uses D = E^2 - |M|^2:  s = sqrt(E^2 + 3D),
//    p = D/(E + s), v = M/(E + p).  MIXED evaluates D in double-float
//    (error-free products and sums on the FP32 pipe), which removes the
//    cancellation as v -> 1 at about FP64 accuracy of D.
#pragma once

#include <type_traits>

#include "sweep.cuh"

namespace shasta {
namespace fast {

constexpr int LANES = 32;
constexpr int CH = 8;         // x sweep: positions per cooperative chunk
constexpr int XSTR = CH + 1;  // padded row of a chunk tile (conflict-free reads)
constexpr int XSLOTS = 3;     // x sweep: chunk slots (previous, current, next)

// ---------------------------------------------------------- cp.async ----

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(dst)), "l"(src)
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

// Global field index of sweep-order field f.
template <int AXIS>
__device__ __forceinline__ int gfield(int f) {
  constexpr int FPAR = 1 + AXIS;
  constexpr int FT1 = AXIS == 0 ? 2 : 1;
  constexpr int FT2 = AXIS == 2 ? 2 : 3;
  return f == 0 ? 0 : (f == 1 ? FPAR : (f == 2 ? FT1 : (f == 3 ? FT2 : 4)));
}

// Global address of sweep-order field f at extended position q of line t.
template <int AXIS>
__device__ __forceinline__ const float* src_addr(const SweepParams& P, int f, long long base,
                                                 long long t, int q, int n) {
  const int gf = gfield<AXIS>(f);
  if (P.bc == BC_FROZEN && (q < 0 || q >= n)) {
    const int side = q < 0 ? 0 : 1;
    int layer = q < 0 ? -1 - q : q - n;
    layer = layer > NG - 1 ? NG - 1 : layer;
    return static_cast<const float*>(P.frozen) + ((long long)(side * NG + layer) * NF + gf) * P.plane + t;
  }
  return static_cast<const float*>(P.in[gf]) + base + (long long)map_pos(q, n, P.bc) * P.stride;
}

// ----------------------------------------------------------- recovery ----

// Velocity along the sweep and pressure, FP32 (MIXED: D in double-float).
// Returns 1 if |M| was clamped or E <= 0, else 0.
template <int EOS, bool MIXED>
__device__ __forceinline__ unsigned rec32(float E, float m1, float m2, float m3, float omd,
                                          float B, float ec, float& w, float& p) {
  unsigned clamped = 0;
  float M2 = fmaf(m1, m1, fmaf(m2, m2, m3 * m3));
  const float E2 = E * E;
  const float lim = omd * E;
  float m = m1;
  float D;
  if (M2 > lim * lim) {
    // |M| clamped to (1 - delta) E (rare): scale the momentum
    m = m1 * (lim * rsqrtf(M2));
    M2 = lim * lim;
    D = fmaf(E, E, -M2);
    clamped = 1;
  } else if (MIXED) {
    // D = E^2 - m1^2 - m2^2 - m3^2 from exact products and compensated sums
    const float e_l = fmaf(E, E, -E2);
    const float a = m1 * m1, a_l = fmaf(m1, m1, -a);
    const float b = m2 * m2, b_l = fmaf(m2, m2, -b);
    const float c = m3 * m3, c_l = fmaf(m3, m3, -c);
    const float s1 = E2 - a;
    float bb = s1 - E2;
    const float r1 = (E2 - (s1 - bb)) + (-a - bb);
    const float s2 = s1 - b;
    bb = s2 - s1;
    const float r2 = (s1 - (s2 - bb)) + (-b - bb);
    const float s3 = s2 - c;
    bb = s3 - s2;
    const float r3 = (s2 - (s3 - bb)) + (-c - bb);
    D = s3 + (((r1 + r2) + r3) + (((e_l - a_l) - b_l) - c_l));
  } else {
    D = fmaf(E, E, -M2);
  }
  D = fmaxf(D, 0.0f);
  const float s = sqrtf(fmaf(3.0f, D, E2));
  float pp = __fdividef(D, E + s);
  if (EOS == EOS_BAG) {
    if (3.0f * pp > ec) {
      const float r = 4.0f * (E - B) * (E - B) - 3.0f * M2;
      bool ok = false;
      if (E > ec && r >= 0.0f) {
        const float eb = __fdividef(3.0f * D - 4.0f * B * E, sqrtf(r) + (E - 2.0f * B));
        if (eb > ec) {
          pp = (eb - 4.0f * B) * (1.0f / 3.0f);
          ok = true;
        }
      }
      if (!ok) pp = __fdividef(M2, E - ec) - E;
    }
  }
  w = __fdividef(m, E + pp);
  p = pp;
  if (!(E > 0.0f)) {
    w = 0.0f;
    p = 0.0f;
    clamped = 1;
  }
  return clamped;
}

// Limited phoenical antidiffusive flux through face j+1/2 (Sec. 3) from the
// transported values at j-1..j+2 and the old differences Delta_{j-1},
// Delta_j, Delta_{j+1}; the sign of A^ph is applied with sign-bit flips.
__device__ __forceinline__ float afx(float h0, float h1, float h2, float h3, float dm, float d,
                                     float dp, float eta) {
  const float dhm = h1 - h0;
  const float dh = h2 - h1;
  const float dhp = h3 - h2;
  const float aph = eta * fmaf(-0.125f, (dp + dm) - 2.0f * d, dh);
  const uint32_t sg = __float_as_uint(aph) & 0x80000000u;
  const float p1 = __uint_as_float(__float_as_uint(dhp) ^ sg);
  const float p2 = __uint_as_float(__float_as_uint(dhm) ^ sg);
  const float mm = fmaxf(0.0f, fminf(fminf(p1, fabsf(aph)), p2));
  return __uint_as_float(__float_as_uint(mm) ^ sg);
}

// Shared memory per warp, in floats.
template <int AXIS, int RING>
struct Smem {
  static constexpr int per_warp =
      AXIS == 0 ? XSLOTS * NF * LANES * XSTR : RING * NF * LANES;
};

// ------------------------------------------------------------- kernel ----

template <int V>
using ic = std::integral_constant<int, V>;
template <bool V>
using bc_ = std::integral_constant<bool, V>;

template <int EOS, int AXIS, bool MIXED, int WARPS, int RING, int DIST, int MINB>
__global__ void __launch_bounds__(WARPS * 32, MINB) sweep_fast_kernel(SweepParams P) {
  constexpr bool XP = AXIS == 0;
  static_assert(RING >= DIST + 4 && (RING & (RING - 1)) == 0, "ring too small");
  extern __shared__ __align__(16) float smem[];

  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const long long gw = (long long)blockIdx.x * WARPS + warp;
  const long long ngroups = (P.plane + LANES - 1) / LANES;
  const long long g = gw % ngroups;
  const int seg = (int)(gw / ngroups);
  if (seg >= P.nseg) return;  // whole warp
  float* wsm = smem + (size_t)warp * Smem<AXIS, RING>::per_warp;

  const int n = P.n;
  const long long t = g * LANES + lane;
  const bool valid = t < P.plane;
  const long long tl = valid ? t : P.plane - 1;
  const long long base = (tl % P.nb) * P.sb + (tl / P.nb) * P.sc;
  const int s0 = seg * P.seg_len;
  const int s1 = min(s0 + P.seg_len, n);
  // positions streamed: qs .. qe (the x path starts on a chunk boundary)
  const int qs = XP ? ((s0 - 2 * NG) & ~(CH - 1)) : s0 - 2 * NG;
  const int qe = s1 + 2 * NG - 1;
  const int trip = ((qe - qs + 1) + 3) & ~3;
  // steady iterations [i1, i2): every position they touch is inside [0, n)
  // (reads q and q-3, frozen override at q-3, prefetch ahead, store q-6)
  const int ahead = XP ? 2 * CH : DIST;
  int i1 = (3 - qs) > 0 ? ((3 - qs) + 3) & ~3 : 0;
  int i2 = ((n - 1 - ahead) - qs + 1);
  i2 = i2 > 0 ? (i2 & ~3) : 0;
  i2 = i2 < trip ? i2 : trip;
  if (i2 < i1) i2 = i1;

  const float* in0 = static_cast<const float*>(P.in[0]);
  float* out0 = static_cast<float*>(P.out[0]);
  const long long fs = P.fstride;
  const float tau_h = float(P.tau_h), tau_f = float(P.tau_f);
  const float htau_h = float(P.htau_h), htau_f = float(P.htau_f);
  const float eta = float(P.eta);
  const float omd = float(P.omd), B = float(P.bag_B), ec = float(P.bag_ec);
  const bool frozen = P.bc == BC_FROZEN;
  unsigned nclamp = 0;

  // x path: cooperative copy of chunk C = positions [8C, 8C+8) of 32 rows
  auto x_slot = [&](int C) -> float* { return wsm + ((C + 3 * 4) % XSLOTS) * (NF * LANES * XSTR); };
  auto x_issue = [&](int C, bool ghost) {
    float* ring = x_slot(C);
    const int r0 = lane >> 3, pc = lane & 7;
    const int pos = C * CH + pc;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int row = r0 + 4 * k;
      long long tr = g * LANES + row;
      tr = tr < P.plane ? tr : P.plane - 1;
      if (ghost) {
#pragma unroll
        for (int f = 0; f < NF; ++f)
          cp_async4(ring + (f * LANES + row) * XSTR + pc, src_addr<AXIS>(P, f, tr * P.sb, tr, pos, n));
      } else {
        const float* rp = in0 + tr * P.sb + pos;
#pragma unroll
        for (int f = 0; f < NF; ++f)
          cp_async4(ring + (f * LANES + row) * XSTR + pc, rp + gfield<AXIS>(f) * fs);
      }
    }
  };
  // y/z path: own-lane copy of position q
  auto yz_issue = [&](int q, bool ghost) {
    float* ring = wsm + ((q - qs) & (RING - 1)) * (NF * LANES) + lane;
    if (ghost) {
#pragma unroll
      for (int f = 0; f < NF; ++f) cp_async4(ring + f * LANES, src_addr<AXIS>(P, f, base, tl, q, n));
    } else {
      const float* rp = in0 + base + (long long)q * P.stride;
#pragma unroll
      for (int f = 0; f < NF; ++f) cp_async4(ring + f * LANES, rp + gfield<AXIS>(f) * fs);
    }
  };
  auto at = [&](int q, int f) -> float& {
    if (XP) return x_slot(q >> 3)[(f * LANES + lane) * XSTR + (q & 7)];
    return wsm[((q - qs) & (RING - 1)) * (NF * LANES) + f * LANES + lane];
  };

  // prologue
  if (XP) {
    x_issue(qs >> 3, true);
    cp_commit();
  } else {
#pragma unroll 1
    for (int d = 0; d < DIST; ++d) {
      if (qs + d <= qe) yz_issue(qs + d, true);
      cp_commit();
    }
  }

  // register windows, slot = (position - qs) & 3
  float Uh_prev[4];     // U^n_{q-1}: E, M_par, M_t1, M_t2
  float dn[4][4];       // Delta^n_j, j = q-4 .. q-1 (E, M)
  float wn[4], pn[4];   // (w, p)^n at q-3 .. q
  float uh[4][4];       // Uhat^h_j, j = q-4 .. q-1 (E, M)
  float ah[4];          // A^h_{q-4}
  float Uf_prev[NF];    // U^n_{q-4}
  float df[4][NF];      // Delta^n_j, j = q-7 .. q-4
  float wh[4], ph[4];   // (w, p)^h at q-6 .. q-3
  float uf[4][NF];      // Uhat^f_j, j = q-7 .. q-4
  float af[NF];         // A^f_{q-7}
  float qph = 0.5f, qpf = 0.5f;  // Q+ of the previous cell, half and full step
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    Uh_prev[k] = k == 0 ? 1.0f : 0.0f;
    ah[k] = 0.0f;
    wn[k] = pn[k] = wh[k] = ph[k] = 0.0f;
#pragma unroll
    for (int s = 0; s < 4; ++s) dn[s][k] = uh[s][k] = 0.0f;
  }
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    Uf_prev[f] = f == 0 ? 1.0f : 0.0f;
    af[f] = 0.0f;
#pragma unroll
    for (int s = 0; s < 4; ++s) df[s][f] = uf[s][f] = 0.0f;
  }

  // One streaming step at position q = qs + i0 + K.  GH: positions outside
  // [0, n) may be touched (boundary rule, frozen ghosts, segment edges).
  auto body = [&](int i0, auto Kc, auto Gc) {
    constexpr int K = decltype(Kc)::value;
    constexpr bool GH = decltype(Gc)::value;
    const int q = qs + i0 + K;
#define SL(o) ((K - (o) + 16) & 3)
    // ---- staging: make position q resident, prefetch ahead
    if (XP) {
      if ((q & 7) == 0) {
        cp_wait<0>();
        __syncwarp();
        if (GH) {
          if ((q >> 3) + 1 <= (qe >> 3)) x_issue((q >> 3) + 1, true);
        } else {
          x_issue((q >> 3) + 1, false);
        }
        cp_commit();
      }
    } else {
      cp_wait<DIST - 1>();
    }
    // ---- stage 0: U^n_q (E, M), recovery at level n
    float uq[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) uq[f] = at(q, f);
    if (GH && flips(q, n, P.bc)) uq[1] = -uq[1];
    if (!XP) {
      if (GH) {
        if (q + DIST <= qe) yz_issue(q + DIST, true);
      } else {
        yz_issue(q + DIST, false);
      }
      cp_commit();
    }
    {
      float w, p;
      const unsigned c0 = rec32<EOS, MIXED>(uq[0], uq[1], uq[2], uq[3], omd, B, ec, w, p);
      nclamp += (q >= s0 && q < s1) ? c0 : 0u;
      wn[SL(0)] = w;
      pn[SL(0)] = p;
    }
    // ---- stage 1: half-step transported value at q-1 (E, M only)
    {
      const float e1 = tau_h * wn[SL(1)], e0 = tau_h * wn[SL(0)];
      const float qp = __fdividef(0.5f - e1, 1.0f + (e0 - e1));  // Q+_{q-1}
      const float qm = 1.0f - qph;                                // Q-_{q-1}
      qph = qp;
      const float a = 0.5f * qp * qp, b = 0.5f * qm * qm, c = qp + qm;
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const float d = uq[f] - Uh_prev[f];  // Delta_{q-1}
        uh[SL(1)][f] = fmaf(c, Uh_prev[f], fmaf(a, d, -b * dn[SL(2)][f]));
        dn[SL(1)][f] = d;
        Uh_prev[f] = uq[f];
      }
      uh[SL(1)][0] += htau_h * (pn[SL(2)] * wn[SL(2)] - pn[SL(0)] * wn[SL(0)]);
      uh[SL(1)][1] += htau_h * (pn[SL(2)] - pn[SL(0)]);
    }
    // ---- stage 2: half-step flux at q-3, state U^h_{q-3}
    float hs[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const float an = afx(uh[SL(4)][f], uh[SL(3)][f], uh[SL(2)][f], uh[SL(1)][f], dn[SL(4)][f],
                           dn[SL(3)][f], dn[SL(2)][f], eta);
      hs[f] = uh[SL(3)][f] - (an - ah[f]);
      ah[f] = an;
    }
    if (GH && frozen && (q - NG < 0 || q - NG >= n)) {
#pragma unroll
      for (int f = 0; f < 4; ++f) hs[f] = at(q - NG, f);
    }
    // ---- stage 3: recovery at n+1/2, position q-3
    {
      float w, p;
      const unsigned c3 = rec32<EOS, MIXED>(hs[0], hs[1], hs[2], hs[3], omd, B, ec, w, p);
      nclamp += (q - NG >= s0 && q - NG < s1) ? c3 : 0u;
      wh[SL(3)] = w;
      ph[SL(3)] = p;
    }
    // ---- stage 4: full-step transported value at q-4 from U^n
    {
      float u3[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) u3[f] = at(q - 3, f);
      if (GH && flips(q - 3, n, P.bc)) u3[1] = -u3[1];
      const float e4 = tau_f * wh[SL(4)], e3 = tau_f * wh[SL(3)];
      const float qp = __fdividef(0.5f - e4, 1.0f + (e3 - e4));  // Q+_{q-4}
      const float qm = 1.0f - qpf;
      qpf = qp;
      const float a = 0.5f * qp * qp, b = 0.5f * qm * qm, c = qp + qm;
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const float d = u3[f] - Uf_prev[f];  // Delta_{q-4}
        uf[SL(4)][f] = fmaf(c, Uf_prev[f], fmaf(a, d, -b * df[SL(5)][f]));
        df[SL(4)][f] = d;
        Uf_prev[f] = u3[f];
      }
      uf[SL(4)][0] += htau_f * (ph[SL(5)] * wh[SL(5)] - ph[SL(3)] * wh[SL(3)]);
      uf[SL(4)][1] += htau_f * (ph[SL(5)] - ph[SL(3)]);
    }
    // ---- stage 5: full-step flux at q-6, new state U^{n+1}_{q-6}
    float ov[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const float an = afx(uf[SL(7)][f], uf[SL(6)][f], uf[SL(5)][f], uf[SL(4)][f], df[SL(7)][f],
                           df[SL(6)][f], df[SL(5)][f], eta);
      ov[f] = uf[SL(6)][f] - (an - af[f]);
      af[f] = an;
    }
    const int jo = q - 2 * NG;
    if (XP) {
      // the ring entry of position jo is dead: stage the result there
      if (jo >= s0 && jo < s1) {
#pragma unroll
        for (int f = 0; f < NF; ++f) at(jo, f) = ov[f];
      }
      if (jo >= s0 && ((jo & 7) == 7 || jo == s1 - 1)) {
        __syncwarp();
        const float* ring = x_slot(jo >> 3);
        const int r0 = lane >> 3, pc = lane & 7;
        const int pos = (jo & ~7) + pc;
        if (pos >= s0 && pos <= jo) {
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int row = r0 + 4 * k;
            const long long tr = g * LANES + row;
            if (tr < P.plane) {
              float* op = out0 + tr * P.sb + pos;
#pragma unroll
              for (int f = 0; f < NF; ++f) op[gfield<AXIS>(f) * fs] = ring[(f * LANES + row) * XSTR + pc];
            }
          }
        }
        __syncwarp();
      }
    } else if (valid && jo >= s0 && jo < s1) {
      float* op = out0 + base + (long long)jo * P.stride;
#pragma unroll
      for (int f = 0; f < NF; ++f) op[gfield<AXIS>(f) * fs] = ov[f];
    }
#undef SL
  };

#pragma unroll 1
  for (int i0 = 0; i0 < trip; i0 += 4) {
    if (i0 >= i1 && i0 < i2) {
      body(i0, ic<0>{}, bc_<false>{});
      body(i0, ic<1>{}, bc_<false>{});
      body(i0, ic<2>{}, bc_<false>{});
      body(i0, ic<3>{}, bc_<false>{});
    } else {
      body(i0, ic<0>{}, bc_<true>{});
      body(i0, ic<1>{}, bc_<true>{});
      body(i0, ic<2>{}, bc_<true>{});
      body(i0, ic<3>{}, bc_<true>{});
    }
  }
  cp_wait<0>();
  if (nclamp && P.clamp_count) atomicAdd(P.clamp_count, (unsigned long long)nclamp);
}

}  // namespace fast
}  // namespace shasta

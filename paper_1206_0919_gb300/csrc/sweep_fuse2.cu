// sweep_fuse2.cu -- the first two sweeps of a step in one launch (temporal
// blocking of two sweeps on 2.5D tiles; FP32).
//
// Sec. 3.1.4 trades memory traffic for recomputation.  Fusing the sweeps of
// a step along axes A then B cuts the traffic of the pair from two reads
// and two writes of the state to one of each: a warp takes a tile of
// TA x TB output cells of one plane of the third axis C, loads it with a
// halo of H = 6 cells on each side in A and B (the reach of one sweep: two
// SHASTA passes of radius 3) into shared memory, sweeps the TB + 2H rows
// along A in place (one lane per row), then the TA columns along B (one
// lane per column), and writes the TA x TB results.  Planes of C are taken
// one after another.  The halo rows are swept along A by every tile that
// needs them: the price of the fusion is that recomputation.
//
// Every cell is computed by the functions of the one-lane kernel
// (sweep_fast.cuh) in the same order and from the same inputs, so the state
// after the two sweeps is bitwise that of two separate sweeps.  Ghost cells
// follow the boundary rule when the tile is loaded: along A by the mirror
// or wrap of the line (momentum along A negated in a mirror), along B by
// loading the mirrored or wrapped rows themselves (their momentum along B
// negated in a mirror), which the A sweep maps exactly as it maps the rows
// they mirror (negating a transported field commutes with the transport,
// and |M|^2 does not see the sign).  Reflecting and periodic walls only.
#include "kernels.h"
#include "sweep_fast.cuh"

namespace shasta {
namespace fuse2 {

using namespace fast;

constexpr int H = 2 * NG;       // halo of one sweep
constexpr int TA = 32;          // output cells along A (= lanes of the B sweep)
constexpr int TBL = 32;         // rows of the tile (= lanes of the A sweep)
constexpr int TB = TBL - 2 * H; // output cells along B: 20
constexpr int LA = TA + 2 * H;  // cells of a tile row: 44
// shared tile: [row b][cell a] quads with a row stride of LA + 1 quads (odd:
// the 32 rows read at one a by the A sweep fall in different bank groups),
// then R as [row b][cell a]
constexpr int QROW = 4 * (LA + 1);
constexpr int RROW = LA + 1;
constexpr int TILE_FLOATS = TBL * QROW + TBL * RROW;
constexpr size_t SMEM = (size_t)TILE_FLOATS * sizeof(float);

// Geometry of one fused pair.
struct Geo2 {
  int nA, nB, nC;                 // cells along A, B, C
  long long sA, sB, sC;           // element strides of A, B, C
  int bc;
};

// Source index of extended position q of a line of n cells (reflect or wrap)
// and whether the mirror negates the momentum along that line.
__device__ __forceinline__ int src_of(int q, int n, int bc, bool& flip) {
  flip = flips(q, n, bc);
  return map_pos(q, n, bc);
}

// Streams one line of L tile cells (extended positions 0 .. L-1 of the
// tile, the line's outputs at [H, L - H)), newest cell q = 0 .. L, with the
// one-lane kernel's step.  load(k, A, B, R) reads tile cell k (k clamped to
// the line), store(k, A, B, R) receives output k; count(k) says whether the
// level-n recovery of cell k is counted.
template <int EOS, int AXIS, class Load, class Store, class Count>
__device__ __forceinline__ void stream_line(const SweepParams& P, int L, float tau_h, float tau_f,
                                            float htau_h, float htau_f, Load load, Store store,
                                            Count count, unsigned& nclamp) {
  constexpr int LAG = 7;
  const float eta = float(P.eta);
  const float omd = float(P.omd), B = float(P.bag_B), ec = float(P.bag_ec);
  const f2 eta2 = pk(eta, eta), m8c = pk(-0.125f, -0.125f);
  const f2 ht_h2 = pk(htau_h, htau_h), ht_f2 = pk(htau_f, htau_f);
  Line2 hA, hB, fA, fB;
  Line1 fR;
  init2(hA, pk(1.0f, 0.0f));
  init2(hB, pk(0.0f, 0.0f));
  init2(fA, pk(1.0f, 0.0f));
  init2(fB, pk(0.0f, 0.0f));
  init1(fR);
  f2 HA = pk(1.0f, 0.0f), HB = pk(0.0f, 0.0f);
  float wn1 = 0.0f, wh1 = 0.0f;
  f2 fn[2], fh[2];
  fn[0] = fn[1] = fh[0] = fh[1] = pk(0.0f, 0.0f);
  float qph = 0.5f, qpf = 0.5f;

  auto body = [&](int q, auto Kc) {
    constexpr int K = decltype(Kc)::value;
    constexpr int P0 = K & 1;
    f2 uA, uB;
    float uR;
    load(q < L ? q : L - 1, uA, uB, uR);
    float wn0, wh0;
    f2 fn0, fh0;
    {
      const f2 E = pk(uA.x, HA.x);
      const f2 mx = pk(uA.y, HA.y);
      const f2 my = pk(uB.x, HB.x);
      const f2 mz = pk(uB.y, HB.y);
      const f2 mpar = AXIS == 0 ? mx : (AXIS == 1 ? my : mz);
      f2 w2, p2;
      rec2<EOS, REC_F32>(E, mx, my, mz, mpar, omd, P.omd, B, ec, P.tab, w2, p2, nclamp,
                         q < L && count(q));
      float pl, phi, pwl, pwh;
      up(w2, wn0, wh0);
      up(p2, pl, phi);
      up(mul2(p2, w2), pwl, pwh);
      fn0 = pk(pwl, pl);
      fh0 = pk(pwh, phi);
    }
    {
      float a, nb, c;
      coeffs(tau_h, wn1, wn0, qph, a, nb, c);
      f2 sA, sB;
      sources<AXIS>(ht_h2, htau_h, sub2(fn[P0], fn0), sA, sB);
      fn[P0] = fn0;
      wn1 = wn0;
      const f2 a2 = pk(a, a), nb2 = pk(nb, nb), c2 = pk(c, c);
      HA = step2<K, true, true>(hA, uA, a2, nb2, c2, sA, eta2, m8c);
      HB = step2<K, AXIS != 0, true>(hB, uB, a2, nb2, c2, sB, eta2, m8c);
    }
    f2 oA, oB;
    float oR;
    {
      f2 vA, vB;
      float vR;
      load(q - 4 < 0 ? 0 : q - 4, vA, vB, vR);
      float a, nb, c;
      coeffs(tau_f, wh1, wh0, qpf, a, nb, c);
      f2 sA, sB;
      sources<AXIS>(ht_f2, htau_f, sub2(fh[P0], fh0), sA, sB);
      fh[P0] = fh0;
      wh1 = wh0;
      const f2 a2 = pk(a, a), nb2 = pk(nb, nb), c2 = pk(c, c);
      oA = step2<K, true, true>(fA, vA, a2, nb2, c2, sA, eta2, m8c);
      oB = step2<K, AXIS != 0, true>(fB, vB, a2, nb2, c2, sB, eta2, m8c);
      oR = step1<K, true>(fR, vR, a, nb, c, eta);
    }
    const int jo = q - LAG;
    if (jo >= H && jo < L - H) store(jo, oA, oB, oR);
  };
#pragma unroll 1
  for (int q = 0; q <= L; q += 2) {
    body(q, ic<0>{});
    body(q + 1, ic<1>{});
  }
}

// One warp per tile; warps loop over (tile, plane of C) work items.
template <int EOS, int AA, int AB>
__global__ void __launch_bounds__(32, 8) fuse2_kernel(SweepParams P, Geo2 G) {
  extern __shared__ __align__(16) float tile[];
  float* tq = tile;
  float* tr = tile + TBL * QROW;
  const int lane = threadIdx.x;
  const int tilesA = (G.nA + TA - 1) / TA, tilesB = (G.nB + TB - 1) / TB;
  const long long items = (long long)tilesA * tilesB * G.nC;
  unsigned nclamp = 0;
  const float tau_h = float(P.tau_h), tau_f = float(P.tau_f);
  const float htau_h = float(P.htau_h), htau_f = float(P.htau_f);
#pragma unroll 1
  for (long long it = blockIdx.x; it < items; it += gridDim.x) {
    const int c = (int)(it / ((long long)tilesA * tilesB));
    const int rest = (int)(it - (long long)c * tilesA * tilesB);
    const int a0 = (rest % tilesA) * TA, b0 = (rest / tilesA) * TB;
    const long long plane0 = (long long)c * G.sC;
    // ---- load the tile: rows b0 - H .. b0 + TB + H - 1, cells a0 - H ..
    // a0 + TA + H - 1, ghosts by the boundary rule (each lane one row)
    {
      const int rb = b0 - H + lane;
      bool flipB;
      const int sb = src_of(rb, G.nB, G.bc, flipB);
#pragma unroll 1
      for (int k = 0; k < LA; ++k) {
        bool flipA;
        const int sa = src_of(a0 - H + k, G.nA, G.bc, flipA);
        const long long cell = plane0 + (long long)sb * G.sB + (long long)sa * G.sA;
        cp_async16(tq + lane * QROW + 4 * k, P.qin + 4 * cell);
        cp_async4(tr + lane * RROW + k, P.rin + cell);
      }
      cp_commit();
      cp_wait<0>();
      __syncwarp();
      // mirrored ghosts (tiles at a reflecting wall): negate the momentum
      // along the mirrored line
      if (G.bc == BC_REFLECT && (a0 - H < 0 || a0 + TA + H > G.nA || b0 - H < 0 ||
                                 b0 + TB + H > G.nB)) {
#pragma unroll 1
        for (int k = 0; k < LA; ++k) {
          bool flipA;
          src_of(a0 - H + k, G.nA, G.bc, flipA);
          float* qd = tq + lane * QROW + 4 * k;
          if (flipA) qd[1 + AA] = -qd[1 + AA];
          if (flipB) qd[1 + AB] = -qd[1 + AB];
        }
      }
      __syncwarp();
    }
    // ---- sweep along A: lane = row b of the tile, in place
    {
      const int b = lane;
      const bool row_in = b >= H && b < TBL - H && b0 - H + b < G.nB;
      float* rq = tq + b * QROW;
      float* rr = tr + b * RROW;
      auto load = [&](int k, f2& A, f2& Bp, float& R) {
        const float4 v = *reinterpret_cast<const float4*>(rq + 4 * k);
        A = pk(v.x, v.y);
        Bp = pk(v.z, v.w);
        R = rr[k];
      };
      auto store = [&](int k, f2 A, f2 Bp, float R) {
        *reinterpret_cast<float4*>(rq + 4 * k) = make_float4(A.x, A.y, Bp.x, Bp.y);
        rr[k] = R;
      };
      auto count = [&](int k) { return row_in && k >= H && k < LA - H && a0 - H + k < G.nA; };
      stream_line<EOS, AA>(P, LA, tau_h, tau_f, htau_h, htau_f, load, store, count, nclamp);
    }
    __syncwarp();
    // ---- sweep along B: lane = column a0 + lane, results to the output
    {
      const int k = H + lane;  // tile cell of this column
      const bool col_in = a0 + lane < G.nA;
      auto load = [&](int b, f2& A, f2& Bp, float& R) {
        const float4 v = *reinterpret_cast<const float4*>(tq + b * QROW + 4 * k);
        A = pk(v.x, v.y);
        Bp = pk(v.z, v.w);
        R = tr[b * RROW + k];
      };
      const long long col0 = plane0 + (long long)(col_in ? a0 + lane : 0) * G.sA;
      auto store = [&](int b, f2 A, f2 Bp, float R) {
        const int gb = b0 - H + b;
        if (col_in && gb < G.nB) {
          const long long cell = col0 + (long long)gb * G.sB;
          *reinterpret_cast<float4*>(P.qout + 4 * cell) = make_float4(A.x, A.y, Bp.x, Bp.y);
          P.rout[cell] = R;
        }
      };
      auto count = [&](int b) { return col_in && b >= H && b < TBL - H && b0 - H + b < G.nB; };
      stream_line<EOS, AB>(P, TBL, tau_h, tau_f, htau_h, htau_f, load, store, count, nclamp);
    }
    __syncwarp();
  }
  if (nclamp && P.clamp_count) atomicAdd(P.clamp_count, (unsigned long long)nclamp);
}

template <int EOS, int AA, int AB>
cudaError_t launch_one(const SweepParams& P, const Geo2& G, int blocks, cudaStream_t s) {
  fuse2_kernel<EOS, AA, AB><<<blocks, 32, SMEM, s>>>(P, G);
  return cudaGetLastError();
}

template <int EOS>
cudaError_t prepare_eos() {
  const void* ks[6] = {(const void*)fuse2_kernel<EOS, 0, 1>, (const void*)fuse2_kernel<EOS, 0, 2>,
                       (const void*)fuse2_kernel<EOS, 1, 0>, (const void*)fuse2_kernel<EOS, 1, 2>,
                       (const void*)fuse2_kernel<EOS, 2, 0>, (const void*)fuse2_kernel<EOS, 2, 1>};
  for (const void* k : ks) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int EOS>
cudaError_t launch_pair(const SweepParams& P, const Geo2& G, int aa, int ab, int blocks,
                        cudaStream_t s) {
  switch (aa * 3 + ab) {
    case 1: return launch_one<EOS, 0, 1>(P, G, blocks, s);
    case 2: return launch_one<EOS, 0, 2>(P, G, blocks, s);
    case 3: return launch_one<EOS, 1, 0>(P, G, blocks, s);
    case 5: return launch_one<EOS, 1, 2>(P, G, blocks, s);
    case 6: return launch_one<EOS, 2, 0>(P, G, blocks, s);
    case 7: return launch_one<EOS, 2, 1>(P, G, blocks, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fuse2

cudaError_t prepare_fuse2() {
  cudaError_t e = fuse2::prepare_eos<EOS_IDEAL>();
  return e == cudaSuccess ? fuse2::prepare_eos<EOS_BAG>() : e;
}

cudaError_t launch_fuse2(const SweepParams& P, int nx, int ny, int nz, int axis_a, int axis_b,
                         int eos, int sm_count, cudaStream_t s) {
  const int n[3] = {nx, ny, nz};
  const long long st[3] = {1, (long long)nx, (long long)nx * ny};
  if (axis_a == axis_b || axis_a < 0 || axis_a > 2 || axis_b < 0 || axis_b > 2)
    return cudaErrorInvalidValue;
  const int axis_c = 3 - axis_a - axis_b;
  fuse2::Geo2 G;
  G.nA = n[axis_a];
  G.nB = n[axis_b];
  G.nC = n[axis_c];
  G.sA = st[axis_a];
  G.sB = st[axis_b];
  G.sC = st[axis_c];
  G.bc = P.bc;
  const long long items = (long long)((G.nA + fuse2::TA - 1) / fuse2::TA) *
                          ((G.nB + fuse2::TB - 1) / fuse2::TB) * G.nC;
  long long blocks = (long long)sm_count * 8;
  if (blocks > items) blocks = items;
  if (blocks < 1) return cudaSuccess;
  if (eos == EOS_IDEAL) return fuse2::launch_pair<EOS_IDEAL>(P, G, axis_a, axis_b, (int)blocks, s);
  if (eos == EOS_BAG) return fuse2::launch_pair<EOS_BAG>(P, G, axis_a, axis_b, (int)blocks, s);
  return cudaErrorInvalidValue;
}

}  // namespace shasta

// sweep_split.cu -- the alternative decomposition of Sec. 3.1: one sweep as
// separate kernels (recovery, geometric transport, antidiffusion) that pass
// their intermediate results through device memory, FP32.  An ablation of
// the fused sweep (sweep_fast.cuh): the same method, six launches and
// about 260 bytes of traffic per cell instead of one launch and 40 bytes.
//
// Per pass (half step with lambda/2 from U^n, then full step with lambda
// from U^n with the n+1/2 velocity and pressure):
//   recover:   w = v along the sweep and p at extended positions [-3, n+3)
//   transport: Uhat_j (Eq. shasta-geo, with the pressure source) at [-2, n+2)
//   antidiff:  A_j, A_{j-1} (phoenical flux and limiter) and
//              U'_j = Uhat_j - A_j + A_{j-1} (Eq. shasta-n) on [0, n)
// Ghost positions follow the boundary rule (mirror with the momentum along
// the line negated, periodic wrap, or the frozen store).
#include "kernels.h"
#include "sweep_fast.cuh"

namespace shasta {
namespace {

using fast::flips;
using fast::map_pos;

constexpr int kThreads = 256;

// One state: (E, Mx, My, Mz) quads and R.
struct St {
  const float* q;
  const float* r;
};

// Where extended position j of line t lives in a buffer of m positions
// starting at j0: x sweeps keep a line contiguous (threads run along it),
// y / z sweeps keep a position's lines contiguous (threads run across lines).
struct Ext {
  long long plane;
  int j0, m;
  bool along;
  __device__ __forceinline__ long long at(int j, long long t) const {
    return along ? t * m + (j - j0) : (long long)(j - j0) * plane + t;
  }
  __device__ __forceinline__ long long size() const { return plane * m; }
  // thread g -> (j, t)
  __device__ __forceinline__ void of(long long g, int& j, long long& t) const {
    if (along) {
      t = g / m;
      j = j0 + (int)(g - t * m);
    } else {
      j = j0 + (int)(g / plane);
      t = g - (long long)(j - j0) * plane;
    }
  }
};

__device__ __forceinline__ long long cell0(const SweepParams& P, long long t) {
  return (t % P.nb) * P.sb + (t / P.nb) * P.sc;
}

// The five fields of extended position j of line t (ghosts by the boundary
// rule; `frozen` ghosts come from the store).
__device__ __forceinline__ void load(const SweepParams& P, St s, long long t, int j, int axis,
                                     float u[5]) {
  const int n = P.n;
  if (P.bc == BC_FROZEN && (j < 0 || j >= n)) {
    const int side = j < 0 ? 0 : 1;
    int layer = j < 0 ? -1 - j : j - n;
    layer = layer > NG - 1 ? NG - 1 : layer;
    const float* fz = static_cast<const float*>(P.frozen) + (long long)(side * NG + layer) * NF * P.plane + t;
#pragma unroll
    for (int f = 0; f < 5; ++f) u[f] = fz[f * P.plane];
    return;
  }
  const long long c = cell0(P, t) + (long long)map_pos(j, n, P.bc) * P.stride;
  const float4 v = *reinterpret_cast<const float4*>(s.q + 4 * c);
  u[0] = v.x;
  u[1] = v.y;
  u[2] = v.z;
  u[3] = v.w;
  u[4] = s.r[c];
  if (flips(j, n, P.bc)) u[1 + axis] = -u[1 + axis];
}

// Velocity along the sweep and pressure at [-3, n+3); counts clamped
// recoveries of interior cells when `count`.
template <int EOS>
__global__ void k_recover(SweepParams P, St s, int axis, Ext X, float* w, float* p, int count) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  unsigned c = 0;
  if (g < X.size()) {
    int j;
    long long t;
    X.of(g, j, t);
    float u[5];
    load(P, s, t, j, axis, u);
    float wv, pv;
    c = fast::rec32<EOS, fast::REC_F32>(u[0], u[1], u[2], u[3], u[1 + axis], float(P.omd), P.omd,
                                        float(P.bag_B), float(P.bag_ec), P.tab, wv, pv);
    w[X.at(j, t)] = wv;
    p[X.at(j, t)] = pv;
    c = count && j >= 0 && j < P.n ? c : 0u;
  }
  const unsigned k = __popc(__ballot_sync(0xffffffffu, c != 0));
  if (k && (threadIdx.x & 31) == 0 && P.clamp_count) atomicAdd(P.clamp_count, (unsigned long long)k);
}

// Uhat at [-2, n+2) from U^n and the pass's w, p (buffer W of [-3, n+3)).
__global__ void k_transport(SweepParams P, St s, int axis, Ext X, Ext W, const float* w,
                            const float* p, float tau, float htau, float* uh) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= X.size()) return;
  int j;
  long long t;
  X.of(g, j, t);
  float um[5], u0[5], up[5];
  load(P, s, t, j - 1, axis, um);
  load(P, s, t, j, axis, u0);
  load(P, s, t, j + 1, axis, up);
  const float wm = w[W.at(j - 1, t)], w0 = w[W.at(j, t)], wp = w[W.at(j + 1, t)];
  const float pm = p[W.at(j - 1, t)], pp = p[W.at(j + 1, t)];
  // Q+_j and Q-_j = 1 - Q+_{j-1} (Eq. shasta-diff; both share 1 + eps_j - eps_{j-1})
  const float qp = fmaf(-tau, w0, 0.5f) / fmaf(tau, wp - w0, 1.0f);
  const float qm = 1.0f - fmaf(-tau, wm, 0.5f) / fmaf(tau, w0 - wm, 1.0f);
  const float a = 0.5f * (qp * qp), nb = -0.5f * (qm * qm), c = qp + qm;
  const long long o = X.at(j, t);
#pragma unroll
  for (int f = 0; f < 5; ++f) {
    const float dj = up[f] - u0[f], dm = u0[f] - um[f];
    float v = fmaf(c, u0[f], fmaf(a, dj, nb * dm));
    // pressure source -(tau/2)(f_{j+1} - f_{j-1}): E carries p w, the
    // momentum along the sweep p
    if (f == 0) v = fmaf(-htau, pp * wp - pm * wm, v);
    if (f == 1 + axis) v = fmaf(-htau, pp - pm, v);
    uh[(long long)f * X.size() + o] = v;
  }
}

__device__ __forceinline__ float limit(float aph, float dhp, float dhm) {
  return fast::limit(aph, dhp, dhm);
}

// U'_j = Uhat_j - A_j + A_{j-1} on [0, n): A from Uhat (buffer U of
// [-2, n+2)) and the differences of the old state U^n.
__global__ void k_antidiffuse(SweepParams P, St s, int axis, Ext X, Ext U, const float* uh,
                              float eta, float* oq, float* orr) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= X.size()) return;
  int j;
  long long t;
  X.of(g, j, t);
  float b[5][5];  // U^n at j-2 .. j+2
#pragma unroll
  for (int k = 0; k < 5; ++k) load(P, s, t, j - 2 + k, axis, b[k]);
  float out[5];
#pragma unroll
  for (int f = 0; f < 5; ++f) {
    const float* h = uh + (long long)f * U.size();
    float hv[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) hv[k] = h[U.at(j - 2 + k, t)];
    float D[4], Dh[4];  // Delta and Delta-hat at j-2 .. j+1
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      D[k] = b[k + 1][f] - b[k][f];
      Dh[k] = hv[k + 1] - hv[k];
    }
    // A_{j-1} (index 1) and A_j (index 2)
    float A[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int m = i + 1;
      const float aph = eta * fmaf(-0.125f, D[m + 1] - 2.0f * D[m] + D[m - 1], Dh[m]);
      A[i] = limit(aph, Dh[m + 1], Dh[m - 1]);
    }
    out[f] = (hv[2] - A[1]) + A[0];
  }
  const long long c = cell0(P, t) + (long long)j * P.stride;
  *reinterpret_cast<float4*>(oq + 4 * c) = make_float4(out[0], out[1], out[2], out[3]);
  orr[c] = out[4];
}

unsigned blocks_for(long long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

}  // namespace

size_t split_scratch_floats(int nx, int ny, int nz) {
  // per axis: w, p on n+6 positions and Uhat on n+4, for every line
  const long long planes[3] = {(long long)ny * nz, (long long)nx * nz, (long long)nx * ny};
  const int ns[3] = {nx, ny, nz};
  long long most = 0;
  for (int a = 0; a < 3; ++a) {
    const long long need = planes[a] * (2LL * (ns[a] + 6) + 5LL * (ns[a] + 4));
    most = need > most ? need : most;
  }
  return (size_t)most;
}

cudaError_t launch_sweep_split(const SweepParams& P, int axis, int eos, float* scratch,
                               float* half_q, float* half_r, cudaStream_t s) {
  if (P.plane <= 0) return cudaSuccess;
  const bool along = P.stride == 1;
  const Ext W{P.plane, -3, P.n + 6, along};
  const Ext H{P.plane, -2, P.n + 4, along};
  const Ext I{P.plane, 0, P.n, along};
  float* w = scratch;
  float* p = w + W.plane * W.m;
  float* uh = p + W.plane * W.m;
  const St old{P.qin, P.rin};
  const St half{half_q, half_r};
  const long long nw = W.plane * W.m, nh = H.plane * H.m, ni = I.plane * I.m;
  for (int pass = 0; pass < 2; ++pass) {
    const St src = pass == 0 ? old : half;
    if (eos == EOS_BAG)
      k_recover<EOS_BAG><<<blocks_for(nw), kThreads, 0, s>>>(P, src, axis, W, w, p, pass == 0);
    else if (eos == EOS_TABLE)
      k_recover<EOS_TABLE><<<blocks_for(nw), kThreads, 0, s>>>(P, src, axis, W, w, p, pass == 0);
    else
      k_recover<EOS_IDEAL><<<blocks_for(nw), kThreads, 0, s>>>(P, src, axis, W, w, p, pass == 0);
    const float tau = float(pass == 0 ? P.tau_h : P.tau_f);
    const float htau = float(pass == 0 ? P.htau_h : P.htau_f);
    k_transport<<<blocks_for(nh), kThreads, 0, s>>>(P, old, axis, H, W, w, p, tau, htau, uh);
    k_antidiffuse<<<blocks_for(ni), kThreads, 0, s>>>(P, old, axis, I, H, uh, float(P.eta),
                                                      pass == 0 ? half_q : P.qout,
                                                      pass == 0 ? half_r : P.rout);
  }
  return cudaGetLastError();
}

}  // namespace shasta

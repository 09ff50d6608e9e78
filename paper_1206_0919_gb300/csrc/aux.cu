// aux.cu -- state conversion, primitive <-> conserved maps, input checks,
// deterministic totals and the frozen ghost store.  Built with -fmad=false
// and IEEE division / square root: these maps evaluate each expression of
// Sec. 2 in plain double precision, in source order.
#include <math.h>

#include "kernels.h"

namespace shasta {

namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(size_t n) {
  size_t b = (n + kThreads - 1) / kThreads;
  return (unsigned)(b > 65535u * 32u ? 65535u * 32u : (b == 0 ? 1 : b));
}

template <class T>
__global__ void k_from_f64(const double* __restrict__ src, T* __restrict__ dst, long long ds,
                           size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    dst[i * ds] = T(src[i]);
}

template <class T>
__global__ void k_to_f64(const T* __restrict__ src, long long ss, double* __restrict__ dst,
                         size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    dst[i] = double(src[i * ss]);
}

template <class T>
__device__ __forceinline__ T& fv(const FieldView& v, int k, size_t i) {
  return static_cast<T*>(v.p[k])[(long long)i * v.s[k]];
}

__device__ __forceinline__ double eos_p(const EosParams& q, double e) {
  if (q.kind == EOS_TABLE) return table_p64(q.tab, e);
  if (q.kind == EOS_BAG && e > q.ec) return (e - 4.0 * q.B) / 3.0;
  return e / 3.0;
}

struct Ptr5 {
  const double* in[5];
  FieldView out;
};

// Sec. 2: R = n gamma, M = (e + p) gamma^2 v, E = (e + p) gamma^2 - p.
template <class T>
__global__ void k_prim2cons(Ptr5 p, size_t n, EosParams q) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    double e = p.in[0][i], vx = p.in[1][i], vy = p.in[2][i], vz = p.in[3][i], nb = p.in[4][i];
    double v2 = (vx * vx + vy * vy) + vz * vz;
    double g2 = 1.0 / (1.0 - v2);
    double pr = eos_p(q, e);
    double w = (e + pr) * g2;
    fv<T>(p.out, 0, i) = T(w - pr);
    fv<T>(p.out, 1, i) = T(w * vx);
    fv<T>(p.out, 2, i) = T(w * vy);
    fv<T>(p.out, 3, i) = T(w * vz);
    fv<T>(p.out, 4, i) = T(nb * sqrt(g2));
  }
}

struct Rec6 {
  FieldView in;
  double* out[6];
};

// Sec. 3 phases 3-4 for every cell: e, v, n, p (double arithmetic).
template <class T>
__global__ void k_recover(Rec6 r, size_t n, EosParams q) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    double E = double(fv<T>(r.in, 0, i));
    double m[3] = {double(fv<T>(r.in, 1, i)), double(fv<T>(r.in, 2, i)),
                   double(fv<T>(r.in, 3, i))};
    double R = double(fv<T>(r.in, 4, i));
    double e = 0.0, v[3] = {0.0, 0.0, 0.0}, nb = 0.0, pp = 0.0;
    if (E > 0.0) {
      double M = sqrt((m[0] * m[0] + m[1] * m[1]) + m[2] * m[2]);
      double lim = q.omd * E;
      double scale = 1.0;
      if (M > lim) {
        scale = lim / M;
        M = lim;
      }
      if (q.kind == EOS_TABLE)
        eos_table_solve(E, M, q.tab, e, pp);
      else if (q.kind == EOS_BAG)
        eos_solve<double, EOS_BAG>(E, M, q.B, q.ec, e, pp);
      else
        eos_solve<double, EOS_IDEAL>(E, M, q.B, q.ec, e, pp);
      // v = M / (E + p) and n = R sqrt(1 - v^2) = R sqrt((e + p) / (E + p))
      // with one reciprocal of E + p (the quotients within an ulp of the
      // divisions; the state itself never depends on them)
      const double ih = 1.0 / (E + pp);
      for (int a = 0; a < 3; ++a) v[a] = ((scale == 1.0) ? m[a] : m[a] * scale) * ih;
      nb = R * sqrt((e + pp) * ih);
    }
    if (r.out[0]) r.out[0][i] = e;
    if (r.out[1]) r.out[1][i] = v[0];
    if (r.out[2]) r.out[2][i] = v[1];
    if (r.out[3]) r.out[3][i] = v[2];
    if (r.out[4]) r.out[4][i] = nb;
    if (r.out[5]) r.out[5][i] = pp;
  }
}

struct In5 {
  const double* f[5];
};

__global__ void k_check_cons(In5 p, size_t n, unsigned long long* count) {
  unsigned local = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    double E = p.f[0][i], x = p.f[1][i], y = p.f[2][i], z = p.f[3][i], R = p.f[4][i];
    bool fin = isfinite(E) && isfinite(x) && isfinite(y) && isfinite(z) && isfinite(R);
    double M2 = (x * x + y * y) + z * z;
    bool bad = !fin || E < 0.0 || (M2 >= E * E && M2 > 0.0);
    local += bad ? 1u : 0u;
  }
  if (local) atomicAdd(count, (unsigned long long)local);
}

__global__ void k_check_prims(In5 p, size_t n, unsigned long long* count) {
  unsigned local = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    double e = p.f[0][i], x = p.f[1][i], y = p.f[2][i], z = p.f[3][i], nb = p.f[4][i];
    bool fin = isfinite(e) && isfinite(x) && isfinite(y) && isfinite(z) && isfinite(nb);
    double v2 = (x * x + y * y) + z * z;
    bool bad = !fin || e < 0.0 || nb < 0.0 || v2 >= 1.0;
    local += bad ? 1u : 0u;
  }
  if (local) atomicAdd(count, (unsigned long long)local);
}

// Deterministic totals: block b sums its contiguous chunk in a fixed order
// (strided per thread, then a shared-memory tree), one block then sums the
// per-block partials the same way.  The result depends only on n.
constexpr int kTotThreads = 256;
constexpr int kTotMaxBlocks = 1024;

struct Tot5 {
  FieldView f;
};

template <class T>
__global__ void __launch_bounds__(kTotThreads) k_totals_partial(Tot5 p, size_t n, size_t chunk,
                                                                double* partials) {
  __shared__ double sh[5][kTotThreads];
  size_t lo = blockIdx.x * chunk;
  size_t hi = lo + chunk < n ? lo + chunk : n;
  double acc[5] = {0, 0, 0, 0, 0};
  for (size_t i = lo + threadIdx.x; i < hi; i += kTotThreads) {
#pragma unroll
    for (int k = 0; k < 5; ++k) acc[k] += double(fv<T>(p.f, k, i));
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int s = kTotThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
#pragma unroll
      for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x < 5) partials[threadIdx.x * gridDim.x + blockIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(kTotThreads) k_totals_final(const double* partials, int nb,
                                                              double* out) {
  __shared__ double sh[5][kTotThreads];
  double acc[5] = {0, 0, 0, 0, 0};
  for (int i = threadIdx.x; i < nb; i += kTotThreads) {
#pragma unroll
    for (int k = 0; k < 5; ++k) acc[k] += partials[k * nb + i];
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int s = kTotThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
#pragma unroll
      for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x < 5) out[threadIdx.x] = sh[threadIdx.x][0];
}

// Frozen ghost store: every ghost layer of a face holds the edge cell.
template <class T>
__global__ void k_frozen_capture(Tot5 p, T* frozen, int nx, int ny, int nz, size_t total) {
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total;
       g += (size_t)gridDim.x * blockDim.x) {
    size_t planes[3] = {(size_t)ny * nz, (size_t)nx * nz, (size_t)nx * ny};
    size_t off = 0;
    int axis = 0;
    for (; axis < 3; ++axis) {
      size_t sz = 2 * NG * 5 * planes[axis];
      if (g < off + sz) break;
      off += sz;
    }
    size_t r = g - off;
    size_t pl = planes[axis];
    size_t t = r % pl;
    size_t rest = r / pl;
    int field = (int)(rest % 5);
    int side = (int)((rest / 5) / NG);
    size_t base, stride;
    int n;
    if (axis == 0) {
      base = t * nx;
      stride = 1;
      n = nx;
    } else if (axis == 1) {
      base = (t % nx) + (size_t)nx * ny * (t / nx);
      stride = nx;
      n = ny;
    } else {
      base = t;
      stride = (size_t)nx * ny;
      n = nz;
    }
    size_t edge = base + (side == 0 ? 0 : (size_t)(n - 1) * stride);
    frozen[g] = fv<T>(p.f, field, edge);
  }
}

}  // namespace

cudaError_t launch_from_f64(const double* src, void* dst, long long dstride, size_t n, int is32,
                            cudaStream_t s) {
  if (!n) return cudaSuccess;
  if (is32)
    k_from_f64<float><<<grid_for(n), kThreads, 0, s>>>(src, (float*)dst, dstride, n);
  else
    k_from_f64<double><<<grid_for(n), kThreads, 0, s>>>(src, (double*)dst, dstride, n);
  return cudaGetLastError();
}

cudaError_t launch_to_f64(const void* src, long long sstride, double* dst, size_t n, int is32,
                          cudaStream_t s) {
  if (!n) return cudaSuccess;
  if (is32)
    k_to_f64<float><<<grid_for(n), kThreads, 0, s>>>((const float*)src, sstride, dst, n);
  else
    k_to_f64<double><<<grid_for(n), kThreads, 0, s>>>((const double*)src, sstride, dst, n);
  return cudaGetLastError();
}

cudaError_t launch_prim2cons(const double* const prim[5], const FieldView& cons, size_t n,
                             int is32, EosParams eos, cudaStream_t s) {
  if (!n) return cudaSuccess;
  Ptr5 p;
  for (int k = 0; k < 5; ++k) p.in[k] = prim[k];
  p.out = cons;
  if (is32)
    k_prim2cons<float><<<grid_for(n), kThreads, 0, s>>>(p, n, eos);
  else
    k_prim2cons<double><<<grid_for(n), kThreads, 0, s>>>(p, n, eos);
  return cudaGetLastError();
}

cudaError_t launch_recover(const FieldView& cons, double* const prim[6], size_t n, int is32,
                           EosParams eos, cudaStream_t s) {
  if (!n) return cudaSuccess;
  Rec6 r;
  r.in = cons;
  for (int k = 0; k < 6; ++k) r.out[k] = prim[k];
  if (is32)
    k_recover<float><<<grid_for(n), kThreads, 0, s>>>(r, n, eos);
  else
    k_recover<double><<<grid_for(n), kThreads, 0, s>>>(r, n, eos);
  return cudaGetLastError();
}

cudaError_t launch_check_cons(const double* const f[5], size_t n, unsigned long long* count,
                              cudaStream_t s) {
  if (!n) return cudaSuccess;
  In5 p;
  for (int k = 0; k < 5; ++k) p.f[k] = f[k];
  k_check_cons<<<grid_for(n), kThreads, 0, s>>>(p, n, count);
  return cudaGetLastError();
}

cudaError_t launch_check_prims(const double* const f[5], size_t n, unsigned long long* count,
                               cudaStream_t s) {
  if (!n) return cudaSuccess;
  In5 p;
  for (int k = 0; k < 5; ++k) p.f[k] = f[k];
  k_check_prims<<<grid_for(n), kThreads, 0, s>>>(p, n, count);
  return cudaGetLastError();
}

int totals_blocks(size_t n) {
  size_t b = (n + 8 * kTotThreads - 1) / (8 * kTotThreads);
  if (b < 1) b = 1;
  if (b > kTotMaxBlocks) b = kTotMaxBlocks;
  return (int)b;
}

cudaError_t launch_totals(const FieldView& f, size_t n, int is32, double* partials, double* out,
                          cudaStream_t s) {
  Tot5 p;
  p.f = f;
  int nb = totals_blocks(n);
  size_t chunk = (n + nb - 1) / nb;
  if (is32)
    k_totals_partial<float><<<nb, kTotThreads, 0, s>>>(p, n, chunk, partials);
  else
    k_totals_partial<double><<<nb, kTotThreads, 0, s>>>(p, n, chunk, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_totals_final<<<1, kTotThreads, 0, s>>>(partials, nb, out);
  return cudaGetLastError();
}

cudaError_t launch_totals_chunked(const FieldView& f, size_t n, int is32, size_t chunk, int nb,
                                  double* partials, double* out, cudaStream_t s) {
  Tot5 p;
  p.f = f;
  if (nb > 0) {
    if (is32)
      k_totals_partial<float><<<nb, kTotThreads, 0, s>>>(p, n, chunk, partials);
    else
      k_totals_partial<double><<<nb, kTotThreads, 0, s>>>(p, n, chunk, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_totals_final<<<1, kTotThreads, 0, s>>>(partials, nb, out);
  return cudaGetLastError();
}

size_t frozen_axis_offset(int nx, int ny, int nz, int axis) {
  size_t planes[3] = {(size_t)ny * nz, (size_t)nx * nz, (size_t)nx * ny};
  size_t off = 0;
  for (int a = 0; a < axis; ++a) off += 2 * NG * 5 * planes[a];
  return off;
}

size_t frozen_elems(int nx, int ny, int nz) { return frozen_axis_offset(nx, ny, nz, 3); }

cudaError_t launch_frozen_capture(const FieldView& f, void* frozen, int nx, int ny, int nz,
                                  int is32, cudaStream_t s) {
  size_t total = frozen_elems(nx, ny, nz);
  Tot5 p;
  p.f = f;
  if (is32)
    k_frozen_capture<float><<<grid_for(total), kThreads, 0, s>>>(p, (float*)frozen, nx, ny, nz,
                                                                 total);
  else
    k_frozen_capture<double><<<grid_for(total), kThreads, 0, s>>>(p, (double*)frozen, nx, ny, nz,
                                                                  total);
  return cudaGetLastError();
}

}  // namespace shasta

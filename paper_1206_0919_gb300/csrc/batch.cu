// batch.cu -- the C ABI of include/shasta_batch.h: many events in one device
// pool, advanced by one batched launch per (sweep slot, axis, EoS) group.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/shasta_batch.h"
#include "kernels.h"
#include "range_alloc.h"

using namespace shasta;

namespace {

thread_local std::string g_batch_create_error;

// Fixed permutation of the sweep axes, Sec. 3.1.4 (as in the single-event
// path).
const int kAxisTable[18] = {0, 1, 2, 0, 2, 1, 2, 0, 1, 2, 1, 0, 1, 2, 0, 1, 0, 2};

constexpr long long kAlign = 32;  // cells: every event starts on a 512-byte quad boundary
constexpr int kTotBlocks = 1024;  // partial sums of the totals reduction

struct Event {
  bool live = false;
  shasta_grid g{};
  double lambda = 0.4;
  shasta_eos eos{};
  long long off = 0;
  long long ncell = 0;
  int64_t steps = 0;
  void* frozen = nullptr;
};

// One batched launch of a plan: the events of list entries [idx_off, +nlist)
// of the device plan array, swept along `axis`.
struct LaunchRec {
  int axis = 0, eos = 0, nlist = 0;
  size_t idx_off = 0, pre_off = 0, gpre_off = 0;  // event indices, position / group prefixes
  long long items = 0;   // (line group, position) pairs
  long long groups = 0;  // line groups
};

}  // namespace

struct shasta_batch {
  int device = 0;
  shasta_batch_opts o{};
  bool mixed = false;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  long long cap = 0;
  void* pool = nullptr;
  unsigned long long* d_chk = nullptr;  // checked builds: refused accesses [count, code, index]
  float* quad[2] = {};
  float* rf[2] = {};
  int cur = 0;
  RangeAlloc cells{kAlign};
  std::vector<Event> ev;
  int nlive = 0;
  long long used = 0;
  EvDesc* d_desc = nullptr;
  unsigned long long* d_count = nullptr;  // per slot clamp counters; [max_events] check scratch
  int* d_plan = nullptr;
  size_t plan_cap = 0;  // ints
  // work-list uploads go through two pinned buffers used in turn, so that a
  // new list is written while the previous copy may still be queued behind
  // the steps (each buffer is reused only after its copy has run)
  EvDesc* h_desc[2] = {};
  int* h_plan[2] = {};
  size_t h_plan_cap[2] = {};
  cudaEvent_t up_done[2] = {};
  bool up_pending[2] = {};
  int up_next = 0;
  double* staging = nullptr;
  size_t staging_cells = 0;
  double* partials = nullptr;
  double* d_tot = nullptr;
  double* h_small = nullptr;  // pinned
  int sm_count = 152;
  int occ[3][3][2] = {};
  int wpb = 4;
  // launch choice per axis: register variant and positions per work range
  bool tuned = false;
  long long force_range = -1;  // >= 0: work range of every axis (environment override; 0 = line groups)
  int tune_var[3] = {0, 0, 0};
  long long tune_range[3] = {0, 0, 0};  // 0: whole line groups
  // work lists of six consecutive steps (index (steps - plan_base) mod 6)
  bool plan_valid = false;
  int64_t bsteps = 0, plan_base = 0;
  std::vector<LaunchRec> plan[6][3];
  cudaGraphExec_t graph = nullptr;
  int graph_r = -1, graph_cur = -1;
  int64_t graph_launches = 0;  // sweep launches in the graph
  // side streams: the launches of one sweep slot run concurrently, so that
  // the last wave of one overlaps the next (fork / join through events)
  static constexpr int kSide = 5;
  cudaStream_t side[kSide] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kSide] = {};
  int64_t launches = 0;        // sweep launches issued (graph replays included)
  std::string err;
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int now = -1;
    if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
  }
};

shasta_status fail(shasta_batch* b, shasta_status s, const std::string& msg) {
  if (b)
    b->err = msg;
  else
    g_batch_create_error = msg;
  return s;
}

shasta_status cuda_fail(shasta_batch* b, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return fail(b, e == cudaErrorMemoryAllocation ? SHASTA_ENOMEM : SHASTA_ECUDA, m);
}

#define CK(call, where)                                    \
  do {                                                     \
    cudaError_t _e = (call);                               \
    if (_e != cudaSuccess) return cuda_fail(b, _e, where); \
  } while (0)

int extent(const shasta_grid& g, int axis) { return axis == 0 ? g.nx : (axis == 1 ? g.ny : g.nz); }

long long plane_of(const shasta_grid& g, int axis) {
  return axis == 0 ? (long long)g.ny * g.nz
                   : (axis == 1 ? (long long)g.nx * g.nz : (long long)g.nx * g.ny);
}

long long groups_of(const Event& e, int axis) { return (plane_of(e.g, axis) + 31) / 32; }

// Resident warps of the machine for a launch choice.
long long warp_slots(const shasta_batch* b, int eos, int axis, int var) {
  const int w = b->occ[eos][axis][var];
  return (long long)b->sm_count * (w > 0 ? w : 1);
}

// Positions (line group x position pairs) of all live events along an axis.
long long total_positions(const shasta_batch* b, int axis) {
  long long t = 0;
  for (const Event& e : b->ev)
    if (e.live) t += groups_of(e, axis) * extent(e.g, axis);
  return t;
}

// Range length giving every resident warp `share` ranges (at least 24
// positions: each piece pays a 13-position halo and lag).
long long range_for(long long total, long long warps, double share) {
  const double want = (double)warps * share;
  long long len = (long long)((double)total / (want > 1.0 ? want : 1.0)) + 1;
  return len < 24 ? 24 : len;
}

long long total_groups(const shasta_batch* b, int axis) {
  long long t = 0;
  for (const Event& e : b->ev)
    if (e.live) t += groups_of(e, axis);
  return t;
}

// Model choice: variant 0; whole line groups (longest lines first, handed
// out round robin) when there are at least two per resident warp, else one
// range of positions per resident warp.
void model_choice(shasta_batch* b) {
  for (int a = 0; a < 3; ++a) {
    const long long warps = warp_slots(b, 0, a, 0);
    b->tune_var[a] = 0;
    b->tune_range[a] = total_groups(b, a) >= 2 * warps ? 0 : range_for(total_positions(b, a), warps, 1.0);
  }
}

FieldView view_of(const shasta_batch* b, const Event& e, int buf) {
  FieldView v;
  for (int k = 0; k < 4; ++k) {
    v.p[k] = b->quad[buf] + 4 * e.off + k;
    v.s[k] = 4;
  }
  v.p[4] = b->rf[buf] + e.off;
  v.s[4] = 1;
  return v;
}

EosParams eos_params(const shasta_batch* b, const Event& e) {
  EosParams q;
  q.kind = e.eos.kind;
  q.B = e.eos.B;
  q.ec = e.eos.e_c;
  q.omd = 1.0 - b->o.delta;
  return q;
}

// Descriptor of slot i.
EvDesc desc_of(const shasta_batch* b, int i) {
  const Event& e = b->ev[i];
  EvDesc d;
  memset(&d, 0, sizeof d);
  d.off = e.off;
  d.nx = e.g.nx;
  d.ny = e.g.ny;
  d.nz = e.g.nz;
  d.bc = e.g.bc;
  // the same double -> float conversions as the single-event launch
  const double tau_h = 0.5 * e.lambda, tau_f = e.lambda;
  d.tau_h = (float)tau_h;
  d.tau_f = (float)tau_f;
  d.htau_h = (float)(0.5 * tau_h);
  d.htau_f = (float)(0.5 * tau_f);
  d.bag_B = (float)e.eos.B;
  d.bag_ec = (float)e.eos.e_c;
  for (int a = 0; a < 3; ++a)
    d.frozen[a] = e.frozen ? (const float*)e.frozen +
                                 frozen_axis_offset(e.g.nx, e.g.ny, e.g.nz, a)
                           : nullptr;
  d.clamp_count = b->d_count + i;
  return d;
}

// Highest live slot + 1.
int slots_in_use(const shasta_batch* b) {
  int n = 0;
  for (int i = 0; i < (int)b->ev.size(); ++i)
    if (b->ev[i].live) n = i + 1;
  return n;
}

// Uploads the descriptors of all slots in use and the work lists `host`
// through the next pinned buffer pair; stream-ordered (the kernels already
// queued read the previous lists), no host wait unless that buffer pair's
// previous copy has not run yet.
shasta_status upload_lists(shasta_batch* b, const std::vector<int>& host) {
  const int i = b->up_next;
  b->up_next ^= 1;
  if (b->up_pending[i]) CK(cudaEventSynchronize(b->up_done[i]), "sync upload buffer");
  b->up_pending[i] = false;
  if (host.size() > b->plan_cap) {
    // the device lists grow (rare): no queued kernel may still read them
    CK(cudaStreamSynchronize(b->stream), "sync");
    cudaFree(b->d_plan);
    b->d_plan = nullptr;
    b->plan_cap = 0;
    size_t cap = std::max<size_t>(host.size() * 2, 4096);
    CK(cudaMalloc((void**)&b->d_plan, cap * sizeof(int)), "cudaMalloc plan");
    b->plan_cap = cap;
  }
  if (host.size() > b->h_plan_cap[i]) {
    cudaFreeHost(b->h_plan[i]);
    b->h_plan[i] = nullptr;
    b->h_plan_cap[i] = 0;
    size_t cap = std::max<size_t>(host.size() * 2, 4096);
    CK(cudaMallocHost((void**)&b->h_plan[i], cap * sizeof(int)), "cudaMallocHost plan");
    b->h_plan_cap[i] = cap;
  }
  const int n = slots_in_use(b);
  for (int k = 0; k < n; ++k)
    if (b->ev[k].live) b->h_desc[i][k] = desc_of(b, k);
  if (n)
    CK(cudaMemcpyAsync(b->d_desc, b->h_desc[i], n * sizeof(EvDesc), cudaMemcpyHostToDevice,
                       b->stream),
       "upload descriptors");
  if (!host.empty()) {
    memcpy(b->h_plan[i], host.data(), host.size() * sizeof(int));
    CK(cudaMemcpyAsync(b->d_plan, b->h_plan[i], host.size() * sizeof(int),
                       cudaMemcpyHostToDevice, b->stream),
       "upload plan");
  }
  CK(cudaEventRecord(b->up_done[i], b->stream), "record upload");
  b->up_pending[i] = true;
  return SHASTA_OK;
}

// Appends the work list of events `ids` along `axis` to the host plan
// array, longest lines first: event indices, the prefix of their positions
// and the prefix of their line groups.
LaunchRec make_list(const shasta_batch* b, std::vector<int> ids, int axis, int eos,
                    std::vector<int>& out) {
  std::stable_sort(ids.begin(), ids.end(), [&](int x, int y) {
    return extent(b->ev[x].g, axis) > extent(b->ev[y].g, axis);
  });
  LaunchRec L;
  L.axis = axis;
  L.eos = eos;
  L.nlist = (int)ids.size();
  L.idx_off = out.size();
  for (int i : ids) out.push_back(i);
  L.pre_off = out.size();
  long long acc = 0;
  for (int i : ids) {
    out.push_back((int)acc);
    acc += groups_of(b->ev[i], axis) * extent(b->ev[i].g, axis);
  }
  out.push_back((int)acc);
  L.items = acc;
  L.gpre_off = out.size();
  acc = 0;
  for (int i : ids) {
    out.push_back((int)acc);
    acc += groups_of(b->ev[i], axis);
  }
  out.push_back((int)acc);
  L.groups = acc;
  return L;
}

void drop_graph(shasta_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->graph_r = b->graph_cur = -1;
}

// Work lists of the next six steps: in step r and sweep slot s, event e
// sweeps along axis kAxisTable[3 ((steps_e + r) mod 6) + s]; the events of
// one (axis, EoS) share a launch.
shasta_status build_plan(shasta_batch* b) {
  std::vector<int> host;
  const int n = slots_in_use(b);
  for (int r = 0; r < 6; ++r)
    for (int s = 0; s < 3; ++s) {
      b->plan[r][s].clear();
      std::vector<int> groups[3][2];
      for (int i = 0; i < n; ++i) {
        const Event& e = b->ev[i];
        if (!e.live) continue;
        const int ph = (int)((e.steps + r) % 6);
        groups[kAxisTable[3 * ph + s]][e.eos.kind].push_back(i);
      }
      for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 2; ++k)
          if (!groups[a][k].empty())
            b->plan[r][s].push_back(make_list(b, groups[a][k], a, k, host));
    }
  shasta_status st = upload_lists(b, host);
  if (st != SHASTA_OK) return st;
  b->plan_base = b->bsteps;
  b->plan_valid = true;
  drop_graph(b);
  return SHASTA_OK;
}

SweepParams batch_params(const shasta_batch* b, const LaunchRec& L, int from, int variant,
                         long long range) {
  SweepParams P;
  memset(&P, 0, sizeof P);
  P.qin = b->quad[from];
  P.rin = b->rf[from];
  P.qout = b->quad[from ^ 1];
  P.rout = b->rf[from ^ 1];
  P.eta = b->o.eta;
  P.omd = 1.0 - b->o.delta;
  set_float_scalars(P);
  P.ncap = b->cap;
  P.chk = b->d_chk;  // null unless this is a checked build
  P.variant = variant;
  P.range_len = range < 1 ? 0 : range;
  P.plane = 1;
  // at most one wave of resident warps loops over the ranges (or groups)
  const long long wave = warp_slots(b, L.eos, L.axis, variant) / b->wpb;
  const long long ranges = range < 1 ? L.groups : (L.items + P.range_len - 1) / P.range_len;
  const long long need = (ranges + b->wpb - 1) / b->wpb;
  P.blocks = std::max(1LL, std::min(need, wave));
  return P;
}

cudaError_t launch_rec(shasta_batch* b, const LaunchRec& L, int from, int variant,
                       long long range, cudaStream_t st = nullptr) {
  if (!L.nlist || !L.items) return cudaSuccess;
  if (!st) st = b->stream;
  ++b->launches;
  const SweepParams P = batch_params(b, L, from, variant, range);
  BatchList BL;
  BL.ev = b->d_desc;
  BL.idx = b->d_plan + L.idx_off;
  BL.prefix = b->d_plan + (range < 1 ? L.gpre_off : L.pre_off);
  BL.nlist = L.nlist;
  return b->mixed ? launch_batch_mixed(P, BL, L.axis, L.eos, st)
                  : launch_batch_f32(P, BL, L.axis, L.eos, st);
}

// One step from plan index r: three sweep slots, each flipping the buffers.
cudaError_t launch_step(shasta_batch* b, int r) {
  for (int s = 0; s < 3; ++s) {
    const std::vector<LaunchRec>& V = b->plan[r][s];
    const int nside = std::min((int)V.size() - 1, shasta_batch::kSide);
    cudaError_t e = cudaSuccess;
    if (nside > 0) {
      e = cudaEventRecord(b->fork, b->stream);
      for (int i = 0; i < nside && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(b->side[i], b->fork, 0);
    }
    for (size_t i = 0; i < V.size() && e == cudaSuccess; ++i) {
      const int k = (int)i - 1;  // launch 0 on the batch stream, the others on side streams
      cudaStream_t st = k >= 0 && k < nside ? b->side[k] : b->stream;
      e = launch_rec(b, V[i], b->cur, b->tune_var[V[i].axis], b->tune_range[V[i].axis], st);
    }
    for (int i = 0; i < nside && e == cudaSuccess; ++i) {
      e = cudaEventRecord(b->join[i], b->side[i]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->join[i], 0);
    }
    if (e != cudaSuccess) return e;
    b->cur ^= 1;
  }
  return cudaSuccess;
}

// Times (variant, range length) per axis: every event sweeps along the
// axis from the current buffer into the other one (the state is not
// changed).  The launch choice does not change results.
shasta_status autotune(shasta_batch* b) {
  if (!b->nlive) return SHASTA_OK;
  static const double shares[] = {0.0, 0.5, 1.0, 2.0};
  const int64_t launches0 = b->launches;  // trial launches are not counted
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0), "cudaEventCreate");
  CK(cudaEventCreate(&e1), "cudaEventCreate");
  shasta_status st = SHASTA_OK;
  const int n = slots_in_use(b);
  for (int a = 0; a < 3 && st == SHASTA_OK; ++a) {
    std::vector<int> host;
    std::vector<LaunchRec> recs;
    for (int k = 0; k < 2; ++k) {
      std::vector<int> ids;
      for (int i = 0; i < n; ++i)
        if (b->ev[i].live && b->ev[i].eos.kind == k) ids.push_back(i);
      if (!ids.empty()) recs.push_back(make_list(b, ids, a, k, host));
    }
    st = upload_lists(b, host);
    if (st != SHASTA_OK) break;
    const long long total = total_positions(b, a);
    float best = 1e30f;
    int bv = 0;
    long long br = b->tune_range[a];
    for (int var = 0; var < 2 && st == SHASTA_OK; ++var)
      for (double sh : shares) {
        // share 0: whole line groups
        const long long range = sh > 0 ? range_for(total, warp_slots(b, 0, a, var), sh) : 0;
        cudaError_t ce = cudaSuccess;
        for (const LaunchRec& L : recs)
          if (ce == cudaSuccess) ce = launch_rec(b, L, b->cur, var, range);
        if (ce == cudaSuccess) ce = cudaEventRecord(e0, b->stream);
        for (int rep = 0; rep < 3 && ce == cudaSuccess; ++rep)
          for (const LaunchRec& L : recs)
            if (ce == cudaSuccess) ce = launch_rec(b, L, b->cur, var, range);
        if (ce == cudaSuccess) ce = cudaEventRecord(e1, b->stream);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
        float ms = 0;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
        if (ce != cudaSuccess) {
          st = cuda_fail(b, ce, "autotune");
          break;
        }
        if (ms < best) {
          best = ms;
          bv = var;
          br = range;
        }
      }
    b->tune_var[a] = bv;
    b->tune_range[a] = br;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->launches = launches0;
  b->plan_valid = false;
  if (st == SHASTA_OK) b->tuned = true;
  return st;
}

shasta_status ensure_staging(shasta_batch* b, long long cells) {
  if ((size_t)cells <= b->staging_cells) return SHASTA_OK;
  CK(cudaStreamSynchronize(b->stream), "sync");
  cudaFree(b->staging);
  b->staging = nullptr;
  b->staging_cells = 0;
  CK(cudaMalloc((void**)&b->staging, 6 * (size_t)cells * sizeof(double)), "cudaMalloc staging");
  b->staging_cells = (size_t)cells;
  return SHASTA_OK;
}

Event* find(shasta_batch* b, int id) {
  if (!b || id < 0 || id >= (int)b->ev.size() || !b->ev[id].live) return nullptr;
  return &b->ev[id];
}

void release(shasta_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graph(b);
  for (Event& e : b->ev) cudaFree(e.frozen);
  cudaFree(b->pool);
  cudaFree(b->d_desc);
  cudaFree(b->d_count);
  cudaFree(b->d_plan);
  for (int i = 0; i < 2; ++i) {
    cudaFreeHost(b->h_desc[i]);
    cudaFreeHost(b->h_plan[i]);
    if (b->up_done[i]) cudaEventDestroy(b->up_done[i]);
  }
  cudaFree(b->staging);
  cudaFree(b->partials);
  cudaFree(b->d_tot);
  cudaFree(b->d_chk);
  cudaFreeHost(b->h_small);
  for (int i = 0; i < shasta_batch::kSide; ++i) {
    if (b->side[i]) cudaStreamDestroy(b->side[i]);
    if (b->join[i]) cudaEventDestroy(b->join[i]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

}  // namespace

extern "C" {

void shasta_batch_default_opts(shasta_batch_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->precision = SHASTA_FP32;
  o->eta = 0.125;
  o->delta = 0.0;
  o->stream = nullptr;
  o->device = 0;
  o->check_input = 1;
  o->autotune = 1;
  o->use_graphs = 1;
  o->max_events = 1024;
  o->capacity_cells = 0;
}

shasta_status shasta_batch_create(const shasta_batch_opts* o, shasta_batch** out) {
  g_batch_create_error.clear();
  if (!out) return fail(nullptr, SHASTA_EINVAL, "out is NULL");
  *out = nullptr;
  if (!o) return fail(nullptr, SHASTA_EINVAL, "options are required (capacity_cells)");
  shasta_batch_opts opts = *o;
  if (opts.precision != SHASTA_FP32 && opts.precision != SHASTA_MIXED)
    return fail(nullptr, SHASTA_EINVAL, "a batch runs FP32 or MIXED");
  if (!(opts.eta >= 0.0 && opts.eta <= 0.5)) return fail(nullptr, SHASTA_EINVAL, "need 0 <= eta <= 0.5");
  if (!(opts.delta >= 0.0 && opts.delta < 0.5)) return fail(nullptr, SHASTA_EINVAL, "need 0 <= delta < 0.5");
  if (opts.delta == 0.0) opts.delta = 1e-6;
  if (opts.max_events < 1 || opts.max_events > 65536)
    return fail(nullptr, SHASTA_EINVAL, "max_events must be in 1..65536");
  if (opts.capacity_cells < 1 || opts.capacity_cells > (1LL << 31))
    return fail(nullptr, SHASTA_EINVAL, "capacity_cells must be in 1..2^31");
  int ndev = 0;
  cudaError_t ce = cudaGetDeviceCount(&ndev);
  if (ce != cudaSuccess || ndev < 1)
    return fail(nullptr, SHASTA_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(ce));
  if (opts.device < 0 || opts.device >= ndev) return fail(nullptr, SHASTA_EINVAL, "bad device ordinal");

  shasta_batch* b = new (std::nothrow) shasta_batch();
  if (!b) return fail(nullptr, SHASTA_ENOMEM, "host allocation failed");
  b->device = opts.device;
  DeviceGuard dg(b->device);
  b->o = opts;
  b->mixed = opts.precision == SHASTA_MIXED;
  b->cap = (opts.capacity_cells + kAlign - 1) / kAlign * kAlign;
  b->ev.resize(opts.max_events);
  b->cells.reset(b->cap);
  {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device) == cudaSuccess && sms > 0)
      b->sm_count = sms;
    const char* v = getenv("SHASTA_BATCH_RANGE");
    if (v && atoll(v) >= 0) b->force_range = atoll(v);
  }
  auto bail = [&](cudaError_t err, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(err);
    release(b);
    return fail(nullptr, err == cudaErrorMemoryAllocation ? SHASTA_ENOMEM : SHASTA_ECUDA, m);
  };
  const size_t qbytes = (size_t)b->cap * 16, rbytes = (size_t)b->cap * 4;
  cudaError_t err = cudaMalloc(&b->pool, 2 * (qbytes + rbytes));
  if (err != cudaSuccess) return bail(err, "cudaMalloc pool");
  for (int k = 0; k < 2; ++k) {
    b->quad[k] = (float*)((char*)b->pool + k * qbytes);
    b->rf[k] = (float*)((char*)b->pool + 2 * qbytes + k * rbytes);
  }
  err = cudaMalloc((void**)&b->d_desc, (size_t)opts.max_events * sizeof(EvDesc));
  if (err != cudaSuccess) return bail(err, "cudaMalloc descriptors");
  for (int i = 0; i < 2 && err == cudaSuccess; ++i) {
    err = cudaMallocHost((void**)&b->h_desc[i], (size_t)opts.max_events * sizeof(EvDesc));
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&b->up_done[i], cudaEventDisableTiming);
  }
  if (err != cudaSuccess) return bail(err, "pinned descriptors");
  err = cudaMalloc((void**)&b->d_count, ((size_t)opts.max_events + 1) * sizeof(unsigned long long));
  if (err != cudaSuccess) return bail(err, "cudaMalloc counters");
  err = cudaMemset(b->d_count, 0, ((size_t)opts.max_events + 1) * sizeof(unsigned long long));
  if (err != cudaSuccess) return bail(err, "cudaMemset counters");
  err = cudaMalloc((void**)&b->partials, 5 * kTotBlocks * sizeof(double));
  if (err != cudaSuccess) return bail(err, "cudaMalloc partials");
  err = cudaMalloc((void**)&b->d_tot, 8 * sizeof(double));
  if (err != cudaSuccess) return bail(err, "cudaMalloc totals");
#ifdef SHASTA_CHECKED
  err = cudaMalloc((void**)&b->d_chk, 4 * sizeof(unsigned long long));
  if (err == cudaSuccess) err = cudaMemset(b->d_chk, 0, 4 * sizeof(unsigned long long));
  if (err != cudaSuccess) return bail(err, "check record");
#endif
  err = cudaMallocHost((void**)&b->h_small, 16 * sizeof(double));
  if (err != cudaSuccess) return bail(err, "cudaMallocHost");
  err = b->mixed ? prepare_batch_mixed(b->occ) : prepare_batch_f32(b->occ);
  if (err != cudaSuccess) return bail(err, "prepare batched kernels");
  b->wpb = b->mixed ? sweep_warps_per_block_mixed() : sweep_warps_per_block_f32();
  if (opts.stream) {
    b->stream = (cudaStream_t)opts.stream;
  } else {
    err = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (err != cudaSuccess) return bail(err, "cudaStreamCreate");
    b->own_stream = true;
  }
  for (int i = 0; i < shasta_batch::kSide; ++i) {
    err = cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
    if (err != cudaSuccess) return bail(err, "side streams");
  }
  err = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (err != cudaSuccess) return bail(err, "fork event");
  *out = b;
  return SHASTA_OK;
}

shasta_status shasta_batch_destroy(shasta_batch* b) {
  if (!b) return SHASTA_OK;
  DeviceGuard dg(b->device);
  release(b);
  return SHASTA_OK;
}

}  // extern "C"

namespace {

// The add of shasta_batch_add.  check: scan the input (a host wait for the
// verdict); wait: return only when the state is in place (the inputs may
// then be reused at once).  Without either the add is only enqueued.
shasta_status add_impl(shasta_batch* b, const shasta_grid* g, double dx, double lambda,
                       const shasta_eos* eos, const double* const fields[5], int kind, int mem,
                       int* id, bool check, bool wait) {
  if (!b) return SHASTA_EINVAL;
  if (!id) return fail(b, SHASTA_EINVAL, "id is NULL");
  *id = -1;
  if (!g) return fail(b, SHASTA_EINVAL, "grid is NULL");
  if (g->nx < 1 || g->ny < 1 || g->nz < 1) return fail(b, SHASTA_EINVAL, "grid sizes must be >= 1");
  if (g->bc < SHASTA_BC_REFLECT || g->bc > SHASTA_BC_FROZEN)
    return fail(b, SHASTA_EINVAL, "unknown boundary rule");
  if (!(dx > 0) || !isfinite(dx)) return fail(b, SHASTA_EINVAL, "dx must be > 0");
  if (!(lambda > 0.0 && lambda <= 0.5)) return fail(b, SHASTA_EINVAL, "need 0 < lambda <= 0.5");
  shasta_eos e{SHASTA_EOS_IDEAL, 0.0, 0.0};
  if (eos) e = *eos;
  if (e.kind != SHASTA_EOS_IDEAL && e.kind != SHASTA_EOS_BAG) return fail(b, SHASTA_EINVAL, "unknown EoS");
  if (e.kind == SHASTA_EOS_BAG && !(e.B >= 0.0 && 4.0 * e.B <= e.e_c))
    return fail(b, SHASTA_EINVAL, "bag EoS needs 0 <= 4B <= e_c");
  if (!fields) return fail(b, SHASTA_EINVAL, "fields is NULL");
  for (int k = 0; k < 5; ++k)
    if (!fields[k]) return fail(b, SHASTA_EINVAL, "NULL field pointer");
  if (kind != SHASTA_STATE_CONSERVED && kind != SHASTA_STATE_PRIMITIVE)
    return fail(b, SHASTA_EINVAL, "bad state kind");
  if (mem != SHASTA_MEM_HOST && mem != SHASTA_MEM_DEVICE) return fail(b, SHASTA_EINVAL, "bad mem");
  const long long ncell = (long long)g->nx * g->ny * g->nz;
  if (ncell > b->cap) return fail(b, SHASTA_EINVAL, "grid larger than the pool");
  int slot = -1;
  for (int i = 0; i < (int)b->ev.size(); ++i)
    if (!b->ev[i].live) {
      slot = i;
      break;
    }
  if (slot < 0) return fail(b, SHASTA_EAGAIN, "no free event slot");
  DeviceGuard dg(b->device);
  const long long off = b->cells.alloc(ncell);
  if (off < 0) return fail(b, SHASTA_EAGAIN, "no contiguous room for the grid in the pool");
  Event ev;
  ev.g = *g;
  ev.lambda = lambda;
  ev.eos = e;
  ev.off = off;
  ev.ncell = ncell;
  auto undo = [&](shasta_status s) {
    cudaFree(ev.frozen);
    b->cells.release(off, ncell);
    return s;
  };
  if (g->bc == SHASTA_BC_FROZEN) {
    cudaError_t ce = cudaMalloc(&ev.frozen, frozen_elems(g->nx, g->ny, g->nz) * sizeof(float));
    if (ce != cudaSuccess) {
      ev.frozen = nullptr;
      return undo(cuda_fail(b, ce, "cudaMalloc frozen"));
    }
  }
  const double* d[5];
  if (mem == SHASTA_MEM_DEVICE) {
    for (int k = 0; k < 5; ++k) d[k] = fields[k];
  } else {
    shasta_status s = ensure_staging(b, ncell);
    if (s != SHASTA_OK) return undo(s);
    for (int k = 0; k < 5; ++k) {
      double* dd = b->staging + (size_t)k * ncell;
      cudaError_t ce = cudaMemcpyAsync(dd, fields[k], ncell * sizeof(double), cudaMemcpyHostToDevice,
                                       b->stream);
      if (ce != cudaSuccess) return undo(cuda_fail(b, ce, "cudaMemcpyAsync H2D"));
      d[k] = dd;
    }
  }
  unsigned long long* scratch = b->d_count + b->o.max_events;
  if (check) {
    cudaError_t ce = cudaMemsetAsync(scratch, 0, sizeof(unsigned long long), b->stream);
    if (ce == cudaSuccess)
      ce = kind == SHASTA_STATE_PRIMITIVE ? launch_check_prims(d, ncell, scratch, b->stream)
                                          : launch_check_cons(d, ncell, scratch, b->stream);
    unsigned long long* h = reinterpret_cast<unsigned long long*>(b->h_small + 8);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(h, scratch, sizeof *h, cudaMemcpyDeviceToHost, b->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(b->stream);
    if (ce != cudaSuccess) return undo(cuda_fail(b, ce, "input check"));
    if (*h) {
      char m[160];
      snprintf(m, sizeof m, "%llu cells are not physical (non-finite, %s)", *h,
               kind == SHASTA_STATE_PRIMITIVE ? "e < 0, n < 0 or |v| >= 1" : "E < 0 or |M| >= E");
      return undo(fail(b, SHASTA_EUNPHYSICAL, m));
    }
  }
  const FieldView v = view_of(b, ev, b->cur);
  cudaError_t ce = cudaSuccess;
  if (kind == SHASTA_STATE_PRIMITIVE) {
    ce = launch_prim2cons(d, v, ncell, 1, eos_params(b, ev), b->stream);
  } else {
    for (int k = 0; k < 5 && ce == cudaSuccess; ++k)
      ce = launch_from_f64(d[k], v.p[k], v.s[k], ncell, 1, b->stream);
  }
  if (ce == cudaSuccess && ev.frozen)
    ce = launch_frozen_capture(v, ev.frozen, g->nx, g->ny, g->nz, 1, b->stream);
  if (ce == cudaSuccess)
    ce = cudaMemsetAsync(b->d_count + slot, 0, sizeof(unsigned long long), b->stream);
  if (ce == cudaSuccess && (wait || mem == SHASTA_MEM_HOST)) ce = cudaStreamSynchronize(b->stream);
  if (ce != cudaSuccess) return undo(cuda_fail(b, ce, "set state"));
  ev.live = true;
  b->ev[slot] = ev;
  ++b->nlive;
  b->used += ncell;
  b->plan_valid = false;
  b->tuned = false;
  *id = slot;
  return SHASTA_OK;
}

// The remove of shasta_batch_remove; wait: first let the queued work finish.
// Without it the cells are reused in stream order (later kernels on the
// batch stream only); a frozen store is freed by cudaFree, which waits.
shasta_status remove_impl(shasta_batch* b, int id, bool wait) {
  Event* e = find(b, id);
  if (!e) return b ? fail(b, SHASTA_ENOTFOUND, "unknown event id") : SHASTA_EINVAL;
  DeviceGuard dg(b->device);
  if (wait) CK(cudaStreamSynchronize(b->stream), "sync");
  cudaFree(e->frozen);
  b->cells.release(e->off, e->ncell);
  b->used -= e->ncell;
  *e = Event();
  --b->nlive;
  b->plan_valid = false;
  b->tuned = false;
  return SHASTA_OK;
}

}  // namespace

namespace shasta {

shasta_status batch_add_enqueue(shasta_batch* b, const shasta_grid* g, double dx, double lambda,
                                const shasta_eos* eos, const double* const fields[5], int kind,
                                int* id) {
  return add_impl(b, g, dx, lambda, eos, fields, kind, SHASTA_MEM_DEVICE, id, false, false);
}

shasta_status batch_remove_enqueue(shasta_batch* b, int id) { return remove_impl(b, id, false); }

shasta_status batch_extract_enqueue(shasta_batch* b, int id, double* const prims[6],
                                    double* const cons[5], unsigned long long* counter) {
  Event* e = find(b, id);
  if (!e) return b ? fail(b, SHASTA_ENOTFOUND, "unknown event id") : SHASTA_EINVAL;
  DeviceGuard dg(b->device);
  const FieldView v = view_of(b, *e, b->cur);
  bool any = false;
  for (int k = 0; k < 6; ++k) any = any || prims[k];
  if (any) CK(launch_recover(v, prims, e->ncell, 1, eos_params(b, *e), b->stream), "recover");
  for (int k = 0; k < 5; ++k)
    if (cons[k]) CK(launch_to_f64(v.p[k], v.s[k], cons[k], e->ncell, 1, b->stream), "convert out");
  if (counter)
    CK(cudaMemcpyAsync(counter, b->d_count + id, sizeof *counter, cudaMemcpyDeviceToDevice,
                       b->stream),
       "copy counter");
  return SHASTA_OK;
}

}  // namespace shasta

extern "C" {

shasta_status shasta_batch_add(shasta_batch* b, const shasta_grid* g, double dx, double lambda,
                               const shasta_eos* eos, const double* const fields[5], int kind,
                               int mem, int* id) {
  return add_impl(b, g, dx, lambda, eos, fields, kind, mem, id, b && b->o.check_input, true);
}

shasta_status shasta_batch_remove(shasta_batch* b, int id) { return remove_impl(b, id, true); }

shasta_status shasta_batch_step(shasta_batch* b, int nsteps) {
  if (!b) return SHASTA_EINVAL;
  if (nsteps < 0) return fail(b, SHASTA_EINVAL, "nsteps < 0");
  if (!nsteps || !b->nlive) return SHASTA_OK;
  DeviceGuard dg(b->device);
  if (!b->tuned) {
    model_choice(b);
    if (b->o.autotune && b->force_range < 0) {
      shasta_status st = autotune(b);
      if (st != SHASTA_OK) return st;
    }
    if (b->force_range >= 0)
      for (int a = 0; a < 3; ++a) b->tune_range[a] = b->force_range;
    b->tuned = true;
    b->plan_valid = false;
  }
  if (!b->plan_valid) {
    shasta_status st = build_plan(b);
    if (st != SHASTA_OK) return st;
  }
  const int n = slots_in_use(b);
  while (nsteps > 0) {
    const int r = (int)((b->bsteps - b->plan_base) % 6);
    int done = 1;
    if (b->o.use_graphs && nsteps >= 6) {
      // six steps bring every event's phase and the buffer back: one graph
      if (!b->graph || b->graph_r != r || b->graph_cur != b->cur) {
        drop_graph(b);
        const int cur0 = b->cur;
        const int64_t l0 = b->launches;
        cudaGraph_t gr = nullptr;
        CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        cudaError_t ce = cudaSuccess;
        for (int k = 0; k < 6 && ce == cudaSuccess; ++k) ce = launch_step(b, (r + k) % 6);
        cudaError_t ce2 = cudaStreamEndCapture(b->stream, &gr);
        b->cur = cur0;
        b->graph_launches = b->launches - l0;
        b->launches = l0;
        if (ce != cudaSuccess || ce2 != cudaSuccess) {
          if (gr) cudaGraphDestroy(gr);
          return cuda_fail(b, ce != cudaSuccess ? ce : ce2, "capture six steps");
        }
        ce = cudaGraphInstantiate(&b->graph, gr, 0);
        cudaGraphDestroy(gr);
        if (ce != cudaSuccess) {
          b->graph = nullptr;
          return cuda_fail(b, ce, "cudaGraphInstantiate");
        }
        b->graph_r = r;
        b->graph_cur = cur0;
      }
      CK(cudaGraphLaunch(b->graph, b->stream), "cudaGraphLaunch");
      b->launches += b->graph_launches;
      done = 6;  // 18 buffer flips: cur unchanged
    } else {
      CK(launch_step(b, r), "batched sweep launch");
    }
    b->bsteps += done;
    for (int i = 0; i < n; ++i)
      if (b->ev[i].live) b->ev[i].steps += done;
    nsteps -= done;
  }
  return SHASTA_OK;
}

shasta_status shasta_batch_sync(shasta_batch* b) {
  if (!b) return SHASTA_EINVAL;
  DeviceGuard dg(b->device);
  CK(cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
  return SHASTA_OK;
}

shasta_status shasta_batch_autotune(shasta_batch* b) {
  if (!b) return SHASTA_EINVAL;
  DeviceGuard dg(b->device);
  model_choice(b);
  shasta_status st = autotune(b);
  return st;
}

shasta_status shasta_batch_get_conserved(shasta_batch* b, int id, double* const out[5], int mem) {
  Event* e = find(b, id);
  if (!e) return b ? fail(b, SHASTA_ENOTFOUND, "unknown event id") : SHASTA_EINVAL;
  if (!out) return fail(b, SHASTA_EINVAL, "out is NULL");
  if (mem != SHASTA_MEM_HOST && mem != SHASTA_MEM_DEVICE) return fail(b, SHASTA_EINVAL, "bad mem");
  DeviceGuard dg(b->device);
  if (mem == SHASTA_MEM_HOST) {
    shasta_status s = ensure_staging(b, e->ncell);
    if (s != SHASTA_OK) return s;
  }
  const FieldView v = view_of(b, *e, b->cur);
  for (int k = 0; k < 5; ++k) {
    if (!out[k]) continue;
    double* d = mem == SHASTA_MEM_DEVICE ? out[k] : b->staging + (size_t)k * e->ncell;
    CK(launch_to_f64(v.p[k], v.s[k], d, e->ncell, 1, b->stream), "convert out");
    if (mem == SHASTA_MEM_HOST)
      CK(cudaMemcpyAsync(out[k], d, e->ncell * sizeof(double), cudaMemcpyDeviceToHost, b->stream),
         "cudaMemcpyAsync D2H");
  }
  CK(cudaStreamSynchronize(b->stream), "sync");
  return SHASTA_OK;
}

shasta_status shasta_batch_get_primitives(shasta_batch* b, int id, double* const out[6], int mem) {
  Event* e = find(b, id);
  if (!e) return b ? fail(b, SHASTA_ENOTFOUND, "unknown event id") : SHASTA_EINVAL;
  if (!out) return fail(b, SHASTA_EINVAL, "out is NULL");
  if (mem != SHASTA_MEM_HOST && mem != SHASTA_MEM_DEVICE) return fail(b, SHASTA_EINVAL, "bad mem");
  DeviceGuard dg(b->device);
  if (mem == SHASTA_MEM_HOST) {
    shasta_status s = ensure_staging(b, e->ncell);
    if (s != SHASTA_OK) return s;
  }
  double* d[6];
  for (int k = 0; k < 6; ++k)
    d[k] = !out[k] ? nullptr : (mem == SHASTA_MEM_DEVICE ? out[k] : b->staging + (size_t)k * e->ncell);
  CK(launch_recover(view_of(b, *e, b->cur), d, e->ncell, 1, eos_params(b, *e), b->stream), "recover");
  if (mem == SHASTA_MEM_HOST)
    for (int k = 0; k < 6; ++k)
      if (out[k])
        CK(cudaMemcpyAsync(out[k], d[k], e->ncell * sizeof(double), cudaMemcpyDeviceToHost,
                           b->stream),
           "cudaMemcpyAsync D2H");
  CK(cudaStreamSynchronize(b->stream), "sync");
  return SHASTA_OK;
}

shasta_status shasta_batch_totals(shasta_batch* b, int id, double out[5]) {
  Event* e = find(b, id);
  if (!e) return b ? fail(b, SHASTA_ENOTFOUND, "unknown event id") : SHASTA_EINVAL;
  if (!out) return fail(b, SHASTA_EINVAL, "out is NULL");
  DeviceGuard dg(b->device);
  CK(launch_totals(view_of(b, *e, b->cur), e->ncell, 1, b->partials, b->d_tot, b->stream), "totals");
  CK(cudaMemcpyAsync(b->h_small, b->d_tot, 5 * sizeof(double), cudaMemcpyDeviceToHost, b->stream),
     "memcpy totals");
  CK(cudaStreamSynchronize(b->stream), "sync");
  for (int k = 0; k < 5; ++k) out[k] = b->h_small[k];
  return SHASTA_OK;
}

int64_t shasta_batch_steps_done(const shasta_batch* b, int id) {
  if (!b || id < 0 || id >= (int)b->ev.size() || !b->ev[id].live) return -1;
  return b->ev[id].steps;
}

shasta_status shasta_batch_set_step_counter(shasta_batch* b, int id, int64_t steps) {
  Event* e = find(b, id);
  if (!e) return b ? fail(b, SHASTA_ENOTFOUND, "unknown event id") : SHASTA_EINVAL;
  if (steps < 0) return fail(b, SHASTA_EINVAL, "negative step counter");
  if (steps != e->steps) {
    // the work lists follow every event's phase; the enqueued steps were
    // planned with the old one
    DeviceGuard dg(b->device);
    CK(cudaStreamSynchronize(b->stream), "sync");
    e->steps = steps;
    b->plan_valid = false;
  }
  return SHASTA_OK;
}

shasta_status shasta_batch_checked_report(shasta_batch* b, unsigned long long out[3]) {
  if (!b || !out) return SHASTA_EINVAL;
#ifdef SHASTA_CHECKED
  DeviceGuard dg(b->device);
  unsigned long long h[4] = {};
  CK(cudaDeviceSynchronize(), "sync");  // every side stream of the batch
  CK(cudaMemcpy(h, b->d_chk, sizeof h, cudaMemcpyDeviceToHost), "read the record");
  CK(cudaMemset(b->d_chk, 0, sizeof h), "clear the record");
  for (int k = 0; k < 3; ++k) out[k] = h[k];
  return SHASTA_OK;
#else
  return fail(b, SHASTA_EINVAL, "not a checked build (built without SHASTA_CHECKED)");
#endif
}

shasta_status shasta_batch_counters(shasta_batch* b, int id, int64_t out[1]) {
  Event* e = find(b, id);
  if (!e) return b ? fail(b, SHASTA_ENOTFOUND, "unknown event id") : SHASTA_EINVAL;
  if (!out) return fail(b, SHASTA_EINVAL, "out is NULL");
  DeviceGuard dg(b->device);
  unsigned long long* h = reinterpret_cast<unsigned long long*>(b->h_small + 9);
  CK(cudaMemcpyAsync(h, b->d_count + id, sizeof *h, cudaMemcpyDeviceToHost, b->stream),
     "memcpy counters");
  CK(cudaStreamSynchronize(b->stream), "sync");
  out[0] = (int64_t)*h;
  return SHASTA_OK;
}

shasta_status shasta_batch_info(shasta_batch* b, int64_t out[7]) {
  if (!b || !out) return SHASTA_EINVAL;
  out[0] = b->nlive;
  out[1] = b->used;
  out[2] = b->cap;
  out[3] = b->cells.largest();
  int64_t launches = 0, items = 0;
  if (b->plan_valid) {
    const int r = (int)((b->bsteps - b->plan_base) % 6);
    for (int s = 0; s < 3; ++s)
      for (const LaunchRec& L : b->plan[r][s]) {
        ++launches;
        items += L.items;
      }
  }
  out[4] = launches;
  out[5] = items;
  out[6] = b->launches;
  return SHASTA_OK;
}

void* shasta_batch_stream(const shasta_batch* b) { return b ? (void*)b->stream : nullptr; }

const char* shasta_batch_last_error(const shasta_batch* b) {
  return b ? b->err.c_str() : g_batch_create_error.c_str();
}

}  // extern "C"

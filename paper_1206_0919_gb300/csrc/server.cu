// server.cu -- the C ABI of include/shasta_serve.h: a worker thread that
// admits submitted events into one resident batch by device-memory
// footprint, advances them together and hands finished results back.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/shasta_serve.h"
#include "batch_internal.h"
#include "kernels.h"
#include "range_alloc.h"

using shasta::RangeAlloc;
using shasta::batch_add_enqueue;
using shasta::batch_extract_enqueue;
using shasta::batch_remove_enqueue;
using shasta::launch_check_cons;
using shasta::launch_check_prims;

namespace {

thread_local std::string g_server_create_error;

constexpr int kMaxStaged = 4;             // events copied in ahead of admission
constexpr long long kPoolAlign = 32;      // cells, as the batch pool
constexpr long long kStateBytes = 40;     // device bytes of state per cell (two buffers)
constexpr size_t kBounceHalf = 16u << 20; // bytes per half of a pinned bounce buffer

enum JobState { J_WAIT, J_STAGED, J_RESIDENT, J_OUT, J_DONE, J_FAILED };

struct Job {
  uint64_t ticket = 0;
  shasta_event ev{};
  long long ncell = 0;
  std::vector<double> in;  // the five input arrays, copied at submit
  JobState st = J_WAIT;
  shasta_status status = SHASTA_OK;
  double t_submit = 0, t_admit = 0, t_done = 0;
  int bid = -1;
  long long in_off = -1, out_off = -1, out_bytes = 0;
  cudaEvent_t in_ready = nullptr;   // inputs copied in and scanned
  cudaEvent_t out_ready = nullptr;  // results in output staging
  int chk = -1;                     // input-scan slot while staged
  int64_t steps_left = 0, steps = 0, clamps = 0;
};

using JobP = std::shared_ptr<Job>;

// Two pinned host buffers used in turn to bring results back to the
// callers' (pageable) arrays: the DMA into one half overlaps the CPU copy out
// of the other.  A device-to-pageable copy would be staged by the driver on
// the calling thread and measurably delays the worker thread's CUDA calls
// (the rounds' gaps between step launches); a copy into pinned memory is
// plain asynchronous DMA.
struct Bounce {
  char* buf = nullptr;  // 2 * kBounceHalf bytes
  cudaEvent_t done[2] = {};
};

cudaError_t bounce_init(Bounce& b) {
  cudaError_t e = cudaMallocHost((void**)&b.buf, 2 * kBounceHalf);
  if (e != cudaSuccess) {
    b.buf = nullptr;
    return e;
  }
  for (int h = 0; h < 2 && e == cudaSuccess; ++h)
    e = cudaEventCreateWithFlags(&b.done[h], cudaEventDisableTiming);
  return e;
}

void bounce_free(Bounce& b) {
  for (int h = 0; h < 2; ++h)
    if (b.done[h]) cudaEventDestroy(b.done[h]);
  if (b.buf) cudaFreeHost(b.buf);
  b = Bounce();
}

struct Piece {
  char* dst;
  const char* src;
  size_t len;
};

// Device -> host (pageable) for a list of pieces of at most kBounceHalf
// bytes, through `st`; returns when every piece is in place.
// Copies len bytes with kCopyThreads threads (the callers' arrays are often
// fresh: first-touch page faults dominate a single-threaded copy); falls
// back to one thread if no thread can be started.
constexpr int kCopyThreads = 4;
void par_copy(char* dst, const char* src, size_t len) {
  const size_t part = ((len + kCopyThreads - 1) / kCopyThreads + 4095) & ~(size_t)4095;
  std::thread th[kCopyThreads - 1];
  for (int t = 1; t < kCopyThreads; ++t) {
    const size_t o = (size_t)t * part;
    if (o >= len) break;
    const size_t n = std::min(part, len - o);
    try {
      th[t - 1] = std::thread([=] { memcpy(dst + o, src + o, n); });
    } catch (...) {
      memcpy(dst + o, src + o, n);
    }
  }
  memcpy(dst, src, std::min(part, len));
  for (auto& x : th)
    if (x.joinable()) x.join();
}

cudaError_t bounce_d2h(Bounce& b, const std::vector<Piece>& pcs, cudaStream_t st) {
  auto issue = [&](size_t k) {
    const int h = (int)(k & 1);
    cudaError_t e = cudaMemcpyAsync(b.buf + h * kBounceHalf, pcs[k].src, pcs[k].len,
                                    cudaMemcpyDeviceToHost, st);
    return e == cudaSuccess ? cudaEventRecord(b.done[h], st) : e;
  };
  cudaError_t e = pcs.empty() ? cudaSuccess : issue(0);
  for (size_t k = 0; k < pcs.size() && e == cudaSuccess; ++k) {
    if (k + 1 < pcs.size()) e = issue(k + 1);  // its half was emptied in step k - 1
    if (e == cudaSuccess) e = cudaEventSynchronize(b.done[k & 1]);
    if (e == cudaSuccess) par_copy(pcs[k].dst, b.buf + (k & 1) * kBounceHalf, pcs[k].len);
  }
  return e;
}

}  // namespace

struct shasta_server {
  shasta_server_opts o{};
  shasta_batch* batch = nullptr;
  cudaStream_t compute = nullptr, copy = nullptr, copy_out = nullptr;
  void* staging = nullptr;            // input half, then output half
  long long in_cap = 0, out_cap = 0;
  char* in_base = nullptr;
  char* out_base = nullptr;
  RangeAlloc in_arena{256}, out_arena{256};
  Bounce bounce;  // the deliverer's
  // input scans of staged events: device counters and their pinned copies
  unsigned long long* d_chk = nullptr;
  unsigned long long* h_chk = nullptr;
  bool chk_used[kMaxStaged] = {};
  // the worker runs at most two iterations ahead of the device: iteration i
  // waits for iteration i-2 (same parity), then releases the input staging
  // of the events that iteration admitted
  cudaEvent_t iter_done[2] = {};
  bool iter_pending[2] = {};
  std::vector<JobP> releasing[2];
  long long pool_cells = 0;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;  // guards the queue, the job table, out_arena, deliver and the counters
  std::condition_variable cv_work, cv_done, cv_deliver, cv_space;
  std::deque<JobP> queue;                      // waiting, first come first served
  std::unordered_map<uint64_t, JobP> jobs;     // every ticket not yet polled
  std::vector<JobP> staged, resident;          // owned by the worker
  std::deque<JobP> deliver;                    // results in output staging, for the deliverer
  uint64_t next_ticket = 1;
  bool stop = false;
  shasta_status fatal = SHASTA_OK;
  long long n_submitted = 0, n_done = 0, n_failed = 0, peak_resident = 0, batch_steps = 0;
  long long sweep_launches = 0;
  // worker time per phase (s): copy in, admit, harvest, step enqueue, copy
  // out, waiting for the steps, idle
  double t_phase[7] = {};
  std::string err;
  std::thread worker, deliverer;
};

namespace {

double now(const shasta_server* s) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

shasta_status fail(shasta_server* s, shasta_status st, const std::string& msg) {
  if (s) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->err = msg;
  } else {
    g_server_create_error = msg;
  }
  return st;
}

long long pool_need(long long ncell) { return (ncell + kPoolAlign - 1) / kPoolAlign * kPoolAlign; }

int n_outputs(const shasta_event& ev) {
  int k = 0;
  for (int i = 0; i < 6; ++i) k += ev.out_prims[i] != nullptr;
  for (int i = 0; i < 5; ++i) k += ev.out_cons[i] != nullptr;
  return k;
}

// Marks a job finished (or failed) and wakes pollers; called by the worker.
void finish(shasta_server* s, const JobP& j, shasta_status st) {
  std::lock_guard<std::mutex> lk(s->mu);
  j->status = st;
  j->st = st == SHASTA_OK ? J_DONE : J_FAILED;
  j->t_done = now(s);
  if (st == SHASTA_OK)
    ++s->n_done;
  else
    ++s->n_failed;
  s->cv_done.notify_all();
}

// A device error stops the server: every unfinished job fails.
void stop_all(shasta_server* s, const std::string& msg) {
  std::vector<JobP> all;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->fatal = SHASTA_ECUDA;
    s->err = msg;
    for (auto& kv : s->jobs)
      if (kv.second->st != J_DONE && kv.second->st != J_FAILED) all.push_back(kv.second);
    s->queue.clear();
  }
  for (auto& j : all) finish(s, j, SHASTA_ECUDA);
}

// Message of a failed batch call (worker thread only: the batch is its own).
std::string batch_msg(shasta_server* s, const char* where) {
  return std::string(where) + ": " + shasta_batch_last_error(s->batch);
}

bool cuda_ok(shasta_server* s, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return true;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->fatal = SHASTA_ECUDA;
  }
  stop_all(s, std::string(where) + " (" + cudaGetErrorString(e) + ")");
  return false;
}

// The deliverer thread: copies results from output staging into the
// callers' buffers (once the extraction queued by the worker has run) while
// the worker keeps the batch stepping.
void deliverer_main(shasta_server* s) {
  cudaSetDevice(s->o.device);
  for (;;) {
    JobP j;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      while (s->deliver.empty() && !s->stop) s->cv_deliver.wait_for(lk, std::chrono::milliseconds(20));
      if (s->stop) return;
      j = s->deliver.front();
      s->deliver.pop_front();
    }
    const double t0 = now(s);
    const char* base = s->out_base + j->out_off;
    const size_t bytes = (size_t)j->ncell * sizeof(double);
    std::vector<Piece> pcs;
    size_t k = 0;
    auto field = [&](double* dst) {
      for (size_t off = 0; off < bytes; off += kBounceHalf)
        pcs.push_back(Piece{(char*)dst + off, base + k * bytes + off, std::min(kBounceHalf, bytes - off)});
      ++k;
    };
    for (int i = 0; i < 6; ++i)
      if (j->ev.out_prims[i]) field(j->ev.out_prims[i]);
    for (int i = 0; i < 5; ++i)
      if (j->ev.out_cons[i]) field(j->ev.out_cons[i]);
    pcs.push_back(Piece{(char*)&j->clamps, base + k * bytes, sizeof(int64_t)});  // clamp counter
    cudaError_t e = cudaStreamWaitEvent(s->copy_out, j->out_ready, 0);
    if (e == cudaSuccess) e = bounce_d2h(s->bounce, pcs, s->copy_out);
    cudaEventDestroy(j->out_ready);
    j->out_ready = nullptr;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->out_arena.release(j->out_off, j->out_bytes);
      s->t_phase[4] += now(s) - t0;
      s->cv_space.notify_all();
    }
    if (e != cudaSuccess) {
      cuda_ok(s, e, "copy out");
      return;
    }
    finish(s, j, SHASTA_OK);
  }
}

// Events whose steps are all queued: their results (and clamp counter) are
// queued into output staging behind the steps, the event leaves the batch
// (its cells are reused only by later work), and the deliverer takes over.
bool harvest(shasta_server* s) {
  std::vector<JobP> keep;
  for (const JobP& j : s->resident) {
    if (j->steps_left > 0) {
      keep.push_back(j);
      continue;
    }
    const int nout = n_outputs(j->ev);
    j->out_bytes = ((long long)nout * j->ncell + 1) * (long long)sizeof(double);
    {
      // room in output staging: every job's outputs fit it, so waiting for
      // the deliverer to free some always ends
      std::unique_lock<std::mutex> lk(s->mu);
      while ((j->out_off = s->out_arena.alloc(j->out_bytes)) < 0) {
        if (s->stop || s->fatal != SHASTA_OK) return false;
        s->cv_space.wait_for(lk, std::chrono::milliseconds(20));
      }
    }
    double* pr[6] = {};
    double* cs[5] = {};
    int k = 0;
    double* base = (double*)(s->out_base + j->out_off);
    for (int i = 0; i < 6; ++i)
      if (j->ev.out_prims[i]) pr[i] = base + (size_t)(k++) * j->ncell;
    for (int i = 0; i < 5; ++i)
      if (j->ev.out_cons[i]) cs[i] = base + (size_t)(k++) * j->ncell;
    unsigned long long* cnt = (unsigned long long*)(base + (size_t)k * j->ncell);
    if (batch_extract_enqueue(s->batch, j->bid, pr, cs, cnt) != SHASTA_OK)
      return stop_all(s, batch_msg(s, "results")), false;
    if (!cuda_ok(s, cudaEventCreateWithFlags(&j->out_ready, cudaEventDisableTiming), "event") ||
        !cuda_ok(s, cudaEventRecord(j->out_ready, s->compute), "event"))
      return false;
    if (batch_remove_enqueue(s->batch, j->bid) != SHASTA_OK)
      return stop_all(s, batch_msg(s, "remove")), false;
    j->bid = -1;
    std::lock_guard<std::mutex> lk(s->mu);
    j->st = J_OUT;
    s->deliver.push_back(j);
    s->cv_deliver.notify_one();
  }
  s->resident.swap(keep);
  return true;
}

void release_input(shasta_server* s, const JobP& j) {
  if (j->in_ready) cudaEventDestroy(j->in_ready);
  j->in_ready = nullptr;
  if (j->chk >= 0) s->chk_used[j->chk] = false;
  j->chk = -1;
  if (j->in_off >= 0) s->in_arena.release(j->in_off, 5 * j->ncell * (long long)sizeof(double));
  j->in_off = -1;
  std::vector<double>().swap(j->in);
}

// Copies the next queue heads into input staging on the copy stream (first
// come first served, while slots, pool room and input staging allow) and
// scans them there for unphysical values.
bool stage(shasta_server* s) {
  std::vector<JobP> to_stage;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    // pool room: the largest free run less what staged events will take
    int64_t info[7] = {};
    shasta_batch_info(s->batch, info);
    long long room = info[3];
    for (const JobP& j : s->staged) room -= pool_need(j->ncell);
    int slots = s->o.max_resident - (int)s->resident.size() - (int)s->staged.size();
    while (!s->queue.empty() && (int)(s->staged.size() + to_stage.size()) < kMaxStaged &&
           slots > 0) {
      const JobP& j = s->queue.front();
      if (pool_need(j->ncell) > room) break;
      const long long off = s->in_arena.alloc(5 * j->ncell * (long long)sizeof(double));
      if (off < 0) break;
      j->in_off = off;
      j->st = J_STAGED;
      room -= pool_need(j->ncell);
      --slots;
      to_stage.push_back(j);
      s->queue.pop_front();
    }
  }
  for (const JobP& j : to_stage) {
    // a slot per staged job (at most kMaxStaged; freed when admission reads it)
    int c = 0;
    while (c < kMaxStaged && s->chk_used[c]) ++c;
    if (c == kMaxStaged) return stop_all(s, "no input-scan slot"), false;
    s->chk_used[c] = true;
    j->chk = c;
    double* d = (double*)(s->in_base + j->in_off);
    const double* f[5];
    for (int k = 0; k < 5; ++k) f[k] = d + (size_t)k * j->ncell;
    cudaError_t e = cudaEventCreateWithFlags(&j->in_ready, cudaEventDisableTiming);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d, j->in.data(), 5 * j->ncell * sizeof(double), cudaMemcpyHostToDevice,
                          s->copy);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_chk + c, 0, sizeof(unsigned long long), s->copy);
    if (e == cudaSuccess)
      e = j->ev.kind == SHASTA_STATE_PRIMITIVE
              ? launch_check_prims(f, (size_t)j->ncell, s->d_chk + c, s->copy)
              : launch_check_cons(f, (size_t)j->ncell, s->d_chk + c, s->copy);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s->h_chk + c, s->d_chk + c, sizeof(unsigned long long),
                          cudaMemcpyDeviceToHost, s->copy);
    if (e == cudaSuccess) e = cudaEventRecord(j->in_ready, s->copy);
    s->staged.push_back(j);
    if (!cuda_ok(s, e, "copy in")) return false;
  }
  return true;
}

// Admits staged jobs whose inputs are in and scanned, in order, while the
// pool has room; only at phase 0 of the resident events (so that they stay
// in step).  The conversion into the pool is queued on the batch stream;
// input staging is released once the iteration's work has run (`p`).
bool admit(shasta_server* s, int p) {
  if (!s->resident.empty() && s->resident.front()->steps % 6 != 0) return true;
  size_t i = 0;
  for (; i < s->staged.size(); ++i) {
    const JobP& j = s->staged[i];
    const cudaError_t q = cudaEventQuery(j->in_ready);
    if (q == cudaErrorNotReady) break;  // later, in order
    if (!cuda_ok(s, q, "copy in")) return false;
    const unsigned long long bad = s->h_chk[j->chk];
    s->chk_used[j->chk] = false;  // the scan's result is read
    j->chk = -1;
    if (bad) {
      char m[160];
      snprintf(m, sizeof m, "%llu cells are not physical (non-finite, %s)", bad,
               j->ev.kind == SHASTA_STATE_PRIMITIVE ? "e < 0, n < 0 or |v| >= 1" : "E < 0 or |M| >= E");
      release_input(s, j);
      {
        std::lock_guard<std::mutex> lk(s->mu);
        s->err = m;
      }
      finish(s, j, SHASTA_EUNPHYSICAL);
      continue;
    }
    if (!cuda_ok(s, cudaStreamWaitEvent(s->compute, j->in_ready, 0), "wait input")) return false;
    const double* base = (const double*)(s->in_base + j->in_off);
    const double* f[5];
    for (int k = 0; k < 5; ++k) f[k] = base + (size_t)k * j->ncell;
    int id = -1;
    shasta_status st = batch_add_enqueue(s->batch, &j->ev.grid, j->ev.dx, j->ev.lambda, &j->ev.eos,
                                         f, j->ev.kind, &id);
    if (st == SHASTA_EAGAIN) break;  // no contiguous room yet: retry in a later worker round
    if (st == SHASTA_ECUDA || st == SHASTA_ENOMEM) return stop_all(s, batch_msg(s, "admit")), false;
    if (st != SHASTA_OK) {
      release_input(s, j);
      {
        std::lock_guard<std::mutex> lk(s->mu);
        s->err = shasta_batch_last_error(s->batch);
      }
      finish(s, j, st);
      continue;
    }
    s->releasing[p].push_back(j);
    j->bid = id;
    j->steps_left = j->ev.nsteps;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      j->st = J_RESIDENT;
      j->t_admit = now(s);
      s->resident.push_back(j);
      s->peak_resident = std::max<long long>(s->peak_resident, (long long)s->resident.size());
    }
  }
  s->staged.erase(s->staged.begin(), s->staged.begin() + i);
  return true;
}

// The worker: iterations of (wait for the iteration before last, queue the
// next steps of the resident events, queue the results of the events that
// are through, copy and scan the next queue heads, admit the staged ones).
// Everything it queues on the device is stream-ordered, so the device
// always has the previous iteration's steps to run while the worker
// prepares the next one.
void worker_main(shasta_server* s) {
  cudaSetDevice(s->o.device);
  double tp[7] = {};  // [4] (copy out) is kept by the deliverer
  double mark = now(s);
  auto lap = [&](int k) {
    const double t = now(s);
    tp[k] += t - mark;
    mark = t;
  };
  for (int64_t iter = 0;; ++iter) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      for (int k = 0; k < 7; ++k)
        if (k != 4) s->t_phase[k] = tp[k];
      if (s->stop || s->fatal != SHASTA_OK) break;
      if (s->queue.empty() && s->staged.empty() && s->resident.empty() &&
          !s->iter_pending[0] && !s->iter_pending[1]) {
        s->cv_work.wait_for(lk, std::chrono::milliseconds(20));
        lk.unlock();
        lap(6);
        continue;
      }
    }
    const int p = (int)(iter & 1);
    if (s->iter_pending[p]) {
      if (!cuda_ok(s, cudaEventSynchronize(s->iter_done[p]), "wait")) break;
      s->iter_pending[p] = false;
      for (const JobP& j : s->releasing[p]) release_input(s, j);
      s->releasing[p].clear();
    }
    lap(5);
    bool queued = false;
    if (!s->resident.empty()) {
      // every resident event is at the same phase of the six-step axis
      // table (events join only at phase 0), so each sweep slot sweeps one
      // axis: one launch per EoS.  Rounds end on six-step boundaries.
      const int64_t phase = s->resident.front()->steps % 6;
      int64_t k = std::min<int64_t>(s->o.steps_per_round, 6 - phase);
      for (const JobP& j : s->resident) k = std::min(k, j->steps_left);
      if (shasta_batch_step(s->batch, (int)k) != SHASTA_OK) {
        stop_all(s, batch_msg(s, "step"));
        break;
      }
      for (const JobP& j : s->resident) {
        j->steps_left -= k;
        j->steps += k;
      }
      queued = queued || k > 0;
      int64_t info[7] = {};
      shasta_batch_info(s->batch, info);
      std::lock_guard<std::mutex> lk(s->mu);
      s->batch_steps += k;
      s->sweep_launches = info[6];
    }
    lap(3);
    const size_t out0 = s->resident.size();
    if (!harvest(s)) break;
    queued = queued || s->resident.size() != out0;
    lap(2);
    if (!stage(s)) break;
    lap(0);
    const size_t admitted0 = s->releasing[p].size();
    if (!admit(s, p)) break;
    lap(1);
    const bool admitted = s->releasing[p].size() != admitted0;
    if (queued || admitted) {
      if (!cuda_ok(s, cudaEventRecord(s->iter_done[p], s->compute), "record")) break;
      s->iter_pending[p] = true;
    }
    if (s->resident.empty() && !admitted && !s->staged.empty()) {
      // nothing to run: wait for the oldest copy in flight instead of spinning
      if (!cuda_ok(s, cudaEventSynchronize(s->staged.front()->in_ready), "wait input")) break;
      lap(6);
    }
  }
}

void release(shasta_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  s->cv_deliver.notify_all();
  s->cv_space.notify_all();
  if (s->worker.joinable()) s->worker.join();
  if (s->deliverer.joinable()) s->deliverer.join();
  if (s->batch) shasta_batch_destroy(s->batch);  // waits for the batch stream
  if (s->copy) cudaStreamSynchronize(s->copy);
  if (s->copy_out) cudaStreamSynchronize(s->copy_out);
  for (const JobP& j : s->staged)
    if (j->in_ready) cudaEventDestroy(j->in_ready);
  for (int p = 0; p < 2; ++p) {
    for (const JobP& j : s->releasing[p])
      if (j->in_ready) cudaEventDestroy(j->in_ready);
    if (s->iter_done[p]) cudaEventDestroy(s->iter_done[p]);
  }
  for (const JobP& j : s->deliver)
    if (j->out_ready) cudaEventDestroy(j->out_ready);
  cudaFree(s->staging);
  cudaFree(s->d_chk);
  cudaFreeHost(s->h_chk);
  bounce_free(s->bounce);
  if (s->compute) cudaStreamDestroy(s->compute);
  if (s->copy) cudaStreamDestroy(s->copy);
  if (s->copy_out) cudaStreamDestroy(s->copy_out);
  delete s;
}

}  // namespace

extern "C" {

void shasta_server_default_opts(shasta_server_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->precision = SHASTA_FP32;
  o->eta = 0.125;
  o->delta = 0.0;
  o->device = 0;
  o->hbm_budget_bytes = 0;
  o->staging_bytes = 0;
  o->max_resident = 256;
  o->max_queue = 4096;
  o->steps_per_round = 6;
}

shasta_status shasta_server_create(const shasta_server_opts* o, shasta_server** out) {
  g_server_create_error.clear();
  if (!out) return fail(nullptr, SHASTA_EINVAL, "out is NULL");
  *out = nullptr;
  if (!o) return fail(nullptr, SHASTA_EINVAL, "options are required (hbm_budget_bytes)");
  shasta_server_opts opts = *o;
  if (opts.staging_bytes == 0) opts.staging_bytes = opts.hbm_budget_bytes / 8;
  if (opts.hbm_budget_bytes <= 0 || opts.staging_bytes <= 0 ||
      opts.staging_bytes >= opts.hbm_budget_bytes)
    return fail(nullptr, SHASTA_EINVAL, "need 0 < staging_bytes < hbm_budget_bytes");
  if (opts.max_resident < 1 || opts.max_resident > 65536)
    return fail(nullptr, SHASTA_EINVAL, "max_resident must be in 1..65536");
  if (opts.max_queue < 1) return fail(nullptr, SHASTA_EINVAL, "max_queue must be >= 1");
  if (opts.steps_per_round < 1) return fail(nullptr, SHASTA_EINVAL, "steps_per_round must be >= 1");
  const long long cells = (opts.hbm_budget_bytes - opts.staging_bytes) / kStateBytes;
  if (cells < kPoolAlign) return fail(nullptr, SHASTA_EINVAL, "budget too small for any state");
  int ndev = 0;
  cudaError_t cd = cudaGetDeviceCount(&ndev);
  if (cd != cudaSuccess || ndev < 1)
    return fail(nullptr, SHASTA_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(cd));
  if (opts.device < 0 || opts.device >= ndev) return fail(nullptr, SHASTA_EINVAL, "bad device ordinal");
  shasta_server* s = new (std::nothrow) shasta_server();
  if (!s) return fail(nullptr, SHASTA_ENOMEM, "host allocation failed");
  s->o = opts;
  s->t0 = std::chrono::steady_clock::now();
  int prev = -1;
  cudaGetDevice(&prev);
  auto bail = [&](shasta_status st, const std::string& m) {
    release(s);
    if (prev >= 0) cudaSetDevice(prev);
    return fail(nullptr, st, m);
  };
  cudaError_t ce = cudaSetDevice(opts.device);
  if (ce != cudaSuccess) return bail(SHASTA_ECUDA, std::string("device: ") + cudaGetErrorString(ce));
  ce = cudaStreamCreateWithFlags(&s->compute, cudaStreamNonBlocking);
  if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking);
  if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&s->copy_out, cudaStreamNonBlocking);
  if (ce != cudaSuccess) return bail(SHASTA_ECUDA, std::string("streams: ") + cudaGetErrorString(ce));
  s->in_cap = s->out_cap = opts.staging_bytes / 512 * 256;
  ce = cudaMalloc(&s->staging, s->in_cap + s->out_cap);
  if (ce != cudaSuccess)
    return bail(ce == cudaErrorMemoryAllocation ? SHASTA_ENOMEM : SHASTA_ECUDA,
                std::string("staging: ") + cudaGetErrorString(ce));
  ce = bounce_init(s->bounce);
  if (ce == cudaSuccess) ce = cudaMalloc((void**)&s->d_chk, kMaxStaged * sizeof(unsigned long long));
  if (ce == cudaSuccess) ce = cudaMallocHost((void**)&s->h_chk, kMaxStaged * sizeof(unsigned long long));
  for (int p = 0; p < 2 && ce == cudaSuccess; ++p)
    ce = cudaEventCreateWithFlags(&s->iter_done[p], cudaEventDisableTiming);
  if (ce != cudaSuccess)
    return bail(SHASTA_ENOMEM, std::string("pinned host buffers: ") + cudaGetErrorString(ce));
  s->in_base = (char*)s->staging;
  s->out_base = (char*)s->staging + s->in_cap;
  s->in_arena.reset(s->in_cap);
  s->out_arena.reset(s->out_cap);
  shasta_batch_opts bo;
  shasta_batch_default_opts(&bo);
  bo.precision = opts.precision;
  bo.eta = opts.eta;
  bo.delta = opts.delta;
  bo.stream = s->compute;
  bo.device = opts.device;
  bo.check_input = 1;
  bo.autotune = 0;  // the set of events changes every few steps: the model picks
  bo.use_graphs = 0;  // and a graph would be captured again for almost every round
  bo.max_events = opts.max_resident;
  bo.capacity_cells = std::min<long long>(cells, 1LL << 31);
  shasta_status st = shasta_batch_create(&bo, &s->batch);
  if (st != SHASTA_OK) return bail(st, std::string("batch: ") + shasta_batch_last_error(nullptr));
  s->pool_cells = bo.capacity_cells;
  s->worker = std::thread(worker_main, s);
  s->deliverer = std::thread(deliverer_main, s);
  if (prev >= 0) cudaSetDevice(prev);
  *out = s;
  return SHASTA_OK;
}

shasta_status shasta_server_destroy(shasta_server* s) {
  if (!s) return SHASTA_OK;
  release(s);
  return SHASTA_OK;
}

shasta_status shasta_submit(shasta_server* s, const shasta_event* ev, uint64_t* ticket) {
  if (!s) return SHASTA_EINVAL;
  if (!ev || !ticket) return fail(s, SHASTA_EINVAL, "event or ticket is NULL");
  *ticket = 0;
  const shasta_grid& g = ev->grid;
  if (g.nx < 1 || g.ny < 1 || g.nz < 1) return fail(s, SHASTA_EINVAL, "grid sizes must be >= 1");
  if (g.bc < SHASTA_BC_REFLECT || g.bc > SHASTA_BC_FROZEN)
    return fail(s, SHASTA_EINVAL, "unknown boundary rule");
  if (!(ev->dx > 0) || !isfinite(ev->dx)) return fail(s, SHASTA_EINVAL, "dx must be > 0");
  if (!(ev->lambda > 0.0 && ev->lambda <= 0.5))
    return fail(s, SHASTA_EINVAL, "need 0 < lambda <= 0.5");
  if (ev->eos.kind != SHASTA_EOS_IDEAL && ev->eos.kind != SHASTA_EOS_BAG)
    return fail(s, SHASTA_EINVAL, "unknown EoS");
  if (ev->eos.kind == SHASTA_EOS_BAG && !(ev->eos.B >= 0.0 && 4.0 * ev->eos.B <= ev->eos.e_c))
    return fail(s, SHASTA_EINVAL, "bag EoS needs 0 <= 4B <= e_c");
  if (ev->kind != SHASTA_STATE_CONSERVED && ev->kind != SHASTA_STATE_PRIMITIVE)
    return fail(s, SHASTA_EINVAL, "bad state kind");
  if (ev->nsteps < 0) return fail(s, SHASTA_EINVAL, "nsteps < 0");
  for (int k = 0; k < 5; ++k)
    if (!ev->fields[k]) return fail(s, SHASTA_EINVAL, "NULL field pointer");
  const long long ncell = (long long)g.nx * g.ny * g.nz;
  if (pool_need(ncell) > s->pool_cells) return fail(s, SHASTA_EINVAL, "grid larger than the state pool");
  if (5 * ncell * (long long)sizeof(double) > s->in_cap ||
      (n_outputs(*ev) * ncell + 1) * (long long)sizeof(double) > s->out_cap)  // + clamp counter
    return fail(s, SHASTA_EINVAL, "grid larger than the staging memory");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->fatal != SHASTA_OK) return SHASTA_ECUDA;
    if ((int)s->queue.size() >= s->o.max_queue) {
      s->err = "queue full";
      return SHASTA_EAGAIN;
    }
  }
  JobP j = std::make_shared<Job>();
  j->ev = *ev;
  for (int k = 0; k < 5; ++k) j->ev.fields[k] = nullptr;
  j->ncell = ncell;
  try {
    j->in.resize(5 * (size_t)ncell);
  } catch (const std::bad_alloc&) {
    return fail(s, SHASTA_ENOMEM, "host copy of the input");
  }
  for (int k = 0; k < 5; ++k)
    memcpy(j->in.data() + (size_t)k * ncell, ev->fields[k], ncell * sizeof(double));
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->fatal != SHASTA_OK) return SHASTA_ECUDA;
    if ((int)s->queue.size() >= s->o.max_queue) {
      s->err = "queue full";
      return SHASTA_EAGAIN;
    }
    j->ticket = s->next_ticket++;
    j->t_submit = now(s);
    s->jobs[j->ticket] = j;
    s->queue.push_back(j);
    ++s->n_submitted;
  }
  s->cv_work.notify_one();
  *ticket = j->ticket;
  return SHASTA_OK;
}

shasta_status shasta_poll(shasta_server* s, uint64_t ticket, shasta_result* out) {
  if (!s) return SHASTA_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return SHASTA_ENOTFOUND;
  const JobP& j = it->second;
  if (j->st != J_DONE && j->st != J_FAILED) return SHASTA_EAGAIN;
  if (out) {
    out->t_submit = j->t_submit;
    out->t_admit = j->t_admit;
    out->t_done = j->t_done;
    out->steps = j->steps;
    out->clamp_count = j->clamps;
  }
  const shasta_status st = j->status;
  s->jobs.erase(it);
  return st;
}

shasta_status shasta_server_drain(shasta_server* s, double timeout_s) {
  if (!s) return SHASTA_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  const auto until = std::chrono::steady_clock::now() +
                     std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                         std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0));
  while (s->n_done + s->n_failed < s->n_submitted) {
    if (s->cv_done.wait_until(lk, until) == std::cv_status::timeout &&
        s->n_done + s->n_failed < s->n_submitted)
      return SHASTA_ETIMEOUT;
  }
  return s->fatal != SHASTA_OK ? s->fatal : SHASTA_OK;
}

shasta_status shasta_server_stats(shasta_server* s, double out[16]) {
  if (!s || !out) return SHASTA_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  out[0] = (double)s->n_submitted;
  out[1] = (double)s->n_done;
  out[2] = (double)s->n_failed;
  out[3] = (double)s->queue.size();
  out[4] = (double)(s->n_submitted - s->n_done - s->n_failed - (long long)s->queue.size());
  out[5] = (double)s->peak_resident;
  out[6] = (double)s->batch_steps;
  out[7] = (double)s->pool_cells;
  out[8] = (double)s->sweep_launches;
  for (int k = 0; k < 7; ++k) out[9 + k] = s->t_phase[k];
  return SHASTA_OK;
}

double shasta_server_clock(const shasta_server* s) { return s ? now(s) : 0.0; }

const char* shasta_server_last_error(const shasta_server* s) {
  if (!s) return g_server_create_error.c_str();
  // a copy per calling thread: the worker may set a new message meanwhile
  thread_local std::string copy;
  {
    std::lock_guard<std::mutex> lk(const_cast<shasta_server*>(s)->mu);
    copy = s->err;
  }
  return copy.c_str();
}

}  // extern "C"

// sk_serve.cu -- request server for left sketches: admission by an HBM
// budget, continuous batching into the persistent tensor-core kernel, two
// overlapping compute streams, per-request latency.
//
// One scheduler thread owns every CUDA call of the server except the event
// recorded at submission and the copy of a result out (sk_server_fetch).
// Request state lives in one map guarded by one mutex; the scheduler drops
// the mutex while it issues CUDA work and while it sleeps.  While a step is
// in flight the scheduler sleeps: a host function enqueued behind each step
// records the completion time and wakes it (without taking the mutex).
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sk_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

constexpr int64_t kItemStages = 512;  // batch default; every request sets its own
constexpr int kLanes = 2;             // compute streams with a step in flight each
constexpr size_t kMaxStepRequests = 256;
constexpr uint64_t kAlign = 256;

uint64_t round_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

// First-fit allocator over one device allocation.  Free ranges are kept by
// offset and merged with their neighbours on release.
class Pool {
 public:
  cudaError_t init(uint64_t bytes) {
    size_ = round_up(bytes, kAlign);
    const cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&base_), size_);
    if (e != cudaSuccess) {
      base_ = nullptr;
      return e;
    }
    free_[0] = size_;
    return cudaSuccess;
  }
  void destroy() {
    if (base_) cudaFree(base_);
    base_ = nullptr;
  }
  bool alloc(uint64_t bytes, uint64_t* off) {
    bytes = round_up(bytes, kAlign);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const uint64_t rest = it->second - bytes;
      const uint64_t roff = it->first + bytes;
      free_.erase(it);
      if (rest) free_[roff] = rest;
      in_use_ += bytes;
      peak_ = std::max(peak_, in_use_);
      return true;
    }
    return false;
  }
  void release(uint64_t off, uint64_t bytes) {
    bytes = round_up(bytes, kAlign);
    in_use_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  char* at(uint64_t off) const { return base_ + off; }
  uint64_t size() const { return size_; }
  uint64_t peak() const { return peak_; }
  void reset_peak() { peak_ = in_use_; }

 private:
  char* base_ = nullptr;
  uint64_t size_ = 0, in_use_ = 0, peak_ = 0;
  std::map<uint64_t, uint64_t> free_;
};

enum class State { Pending, Admitted, Running, Done, Failed, Fetching };

struct Request {
  sk::BatchMember mb{};     // A, Y and part point into the pool once admitted
  int prec = SK_FP32;
  const float* src = nullptr;
  const float* src_dev = nullptr;  // device-accessible address of src, or null
  int64_t src_ld = 0;
  cudaEvent_t src_ready = nullptr;  // recorded on the producer's stream at submission
  int64_t ldp = 0;          // row stride of the pool copies of A and Y
  // work block: [copy of A (a_bytes; none when a BF16 request is split
  // straight from its source)][workspace (ws_bytes): the BF16 split and the
  // partials, or the SIMT partials]
  uint64_t a_bytes = 0, ws_bytes = 0, work_bytes = 0, y_bytes = 0;
  uint64_t work_off = 0, y_off = 0;
  bool has_work = false, has_y = false;
  State state = State::Pending;
  bool release_when_done = false;
  sk_status err = SK_OK;
  Clock::time_point t_arrival, t_launch, t_done;
};

// A copy of one admitted request's A into the pool.
struct AdmitCopy {
  int64_t ticket;
  float* dst;
  int64_t ldd;
  const float* src;      // as submitted
  const float* src_dev;  // device-accessible address of src, or null (pageable host)
  int64_t lds, m, n;
  void* split;           // non-null: write the BF16 split here instead of copying A
  cudaEvent_t ready;     // the producer's event, returned to the free list after use
};

// One request of a step, copied out of the request table.
struct StepItem {
  int64_t ticket;
  sk::BatchMember mb;
  int prec;
  float* simt_part;
  uint64_t simt_bytes;
};

struct Lane {
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
  sk::BatchArena arena;
  int* h_status = nullptr;  // pinned copy of the lane's status word
  bool busy = false;
  std::vector<int64_t> tickets;
  // completion signal of the step in flight: a host function enqueued after
  // the step records when it ran and wakes the scheduler.  It takes no lock
  // (a thread holding mu may be inside a CUDA call that waits for the CUDA
  // thread running host functions), so these fields are atomics.
  std::atomic<uint64_t> seq{0};            // steps launched on this lane
  std::atomic<uint64_t> signalled_seq{0};  // the step whose host function ran
  std::atomic<int64_t> t_signal_ns{0};     // when it ran (steady clock)
  Clock::time_point t_launch;              // when the step was taken (under mu)
};

}  // namespace

struct sk_server {
  int device = 0;
  int num_sms = 1;
  int max_slots = 1;
  Pool pool;
  Lane lanes[kLanes];
  cudaStream_t copy_st = nullptr;
  cudaEvent_t copy_ev = nullptr;
  // GPU-clock reference for completion times: ref_ev completed at about
  // host time ref_host (recorded on an idle stream and synchronised on), so a
  // step's Y-ready event maps to ref_host + elapsed(ref_ev, done)
  cudaEvent_t ref_ev = nullptr;
  Clock::time_point ref_host;
  bool ref_valid = false;
  void calibrate_clock();
  bool copy_recorded = false;
  std::vector<cudaEvent_t> free_events;  // submission events not in use (under mu)
  std::vector<cudaEvent_t> all_events;

  std::mutex mu;
  std::condition_variable work_cv;  // scheduler: new work, releases, stop
  std::condition_variable done_cv;  // waiters: completions
  bool stop = false;
  std::thread thread;

  std::unordered_map<int64_t, Request> reqs;
  std::deque<int64_t> pending;
  std::vector<int64_t> admitted;  // admitted, not launched
  int64_t next_ticket = 1;
  int64_t resident = 0;

  // statistics of finished requests
  int64_t submitted = 0, completed = 0, failed = 0, steps = 0, max_step = 0;
  std::vector<double> latencies;
  double wait_sum_ms = 0.0, flops = 0.0;
  bool have_first = false;
  Clock::time_point first_arrival, last_done;

  void scheduler();
  bool retire_lanes(std::unique_lock<std::mutex>& lk);
  std::vector<AdmitCopy> admit_locked();
  std::vector<StepItem> take_step_locked(Lane* ln);
  cudaError_t launch_items(Lane* ln, const std::vector<StepItem>& items);
  cudaError_t issue_copy(const AdmitCopy& c);
  void finish(int64_t ticket, sk_status err, Clock::time_point now);
  void free_work(Request& r);
  void free_y(Request& r);
};

namespace {

// Argument of the completion host function of one step.
struct StepSignal {
  sk_server* s;
  Lane* ln;
  uint64_t seq;
};

// Runs on a CUDA runtime thread once everything enqueued before it on the
// lane's stream has finished (no CUDA calls here).  Records the time for the
// step it belongs to and wakes the scheduler, which otherwise sleeps while a
// step is in flight.
void CUDART_CB step_done_host_fn(void* p) {
  StepSignal* sg = static_cast<StepSignal*>(p);
  if (sg->ln->seq.load() == sg->seq) {
    sg->ln->t_signal_ns.store(Clock::now().time_since_epoch().count());
    sg->ln->signalled_seq.store(sg->seq);
  }
  // no lock: a wake-up that slips in between the scheduler's last look at
  // the signals and its wait is caught by the wait's short timeout
  sg->s->work_cv.notify_one();
  delete sg;
}

}  // namespace

// Copy A[m x n] (row stride lds) into the pool (row stride ldd): one warp
// per row, consecutive lanes on consecutive columns.  The source may be
// device memory or mapped pinned host memory read through its device
// address; rows of any alignment are read with 4-byte loads.
__global__ void k_admit_copy(const float* __restrict__ src, int64_t lds,
                             float* __restrict__ dst, int64_t ldd, int64_t m, int64_t n) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  for (int64_t r = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
       r < m; r += warps) {
    const float* s = src + r * lds;
    float* d = dst + r * ldd;
    for (int64_t c = lane; c < n; c += 32) d[c] = s[c];
  }
}

cudaError_t sk_server::issue_copy(const AdmitCopy& c) {
  const cudaError_t we = cudaStreamWaitEvent(copy_st, c.ready, 0);
  if (we != cudaSuccess) return we;
  if (c.split != nullptr) return sk::split_rows(c.src_dev, c.lds, c.m, c.n, c.split, copy_st);
  if (c.src_dev == nullptr)  // pageable host memory: the copy engine stages it
    return cudaMemcpy2DAsync(c.dst, c.ldd * sizeof(float), c.src, c.lds * sizeof(float),
                             c.n * sizeof(float), c.m, cudaMemcpyDefault, copy_st);
  const int threads = 256;
  const int64_t rows_per_block = threads / 32;
  const int64_t blocks = std::min<int64_t>((c.m + rows_per_block - 1) / rows_per_block,
                                           static_cast<int64_t>(num_sms) * 8);
  k_admit_copy<<<static_cast<unsigned>(blocks), threads, 0, copy_st>>>(c.src_dev, c.lds, c.dst,
                                                                      c.ldd, c.m, c.n);
  sk::count_launches(1);
  return cudaGetLastError();
}

// Record ref_ev on the idle copy stream and note when it completed.  Called
// without mu while no step is in flight (at creation and then at most once a
// second when the lanes are idle), which bounds the drift between the GPU
// and host clocks to what accumulates in about a second.
void sk_server::calibrate_clock() {
  if (cudaEventRecord(ref_ev, copy_st) != cudaSuccess ||
      cudaEventSynchronize(ref_ev) != cudaSuccess) {
    cudaGetLastError();
    ref_valid = false;
    return;
  }
  ref_host = Clock::now();
  ref_valid = true;
}

void sk_server::free_work(Request& r) {
  if (r.has_work) pool.release(r.work_off, r.work_bytes);
  r.has_work = false;
}

void sk_server::free_y(Request& r) {
  if (r.has_y) pool.release(r.y_off, r.y_bytes);
  r.has_y = false;
}

// Mark one request finished (done or failed) at `now`; caller holds mu.
void sk_server::finish(int64_t ticket, sk_status err, Clock::time_point now) {
  auto it = reqs.find(ticket);
  if (it == reqs.end()) return;
  Request& r = it->second;
  r.t_done = now;
  r.err = err;
  free_work(r);
  if (err == SK_OK) {
    r.state = State::Done;
    ++completed;
    latencies.push_back(ms_between(r.t_arrival, now));
    wait_sum_ms += ms_between(r.t_arrival, r.t_launch);
    flops += 2.0 * static_cast<double>(r.mb.k) * static_cast<double>(r.mb.m) *
             static_cast<double>(r.mb.n);
    last_done = now;
  } else {
    r.state = State::Failed;
    ++failed;
  }
  if (r.release_when_done) {
    free_y(r);
    --resident;
    reqs.erase(it);
  }
}

// Complete the steps whose events have fired; returns whether any did.
bool sk_server::retire_lanes(std::unique_lock<std::mutex>&) {
  bool any = false;
  for (Lane& ln : lanes) {
    if (!ln.busy) continue;
    const cudaError_t q = cudaEventQuery(ln.done);
    if (q == cudaErrorNotReady) continue;
    // a request's latency ends when its step's Y-ready event completed: the
    // event's GPU time mapped to the host clock (or, without a reference,
    // when the step's host function ran, or now)
    const Clock::time_point seen = Clock::now();
    Clock::time_point now =
        ln.signalled_seq.load() == ln.seq.load()
            ? Clock::time_point(Clock::duration(ln.t_signal_ns.load()))
            : seen;
    float ev_ms = 0.0f;
    if (q == cudaSuccess && ref_valid && cudaEventElapsedTime(&ev_ms, ref_ev, ln.done) == cudaSuccess)
      now = std::max(ln.t_launch,
                     std::min(seen, ref_host + std::chrono::duration_cast<Clock::duration>(
                                                   std::chrono::duration<double, std::milli>(ev_ms))));
    else
      cudaGetLastError();
    sk_status err = SK_OK;
    if (q != cudaSuccess) {
      err = sk::status_from_cuda(q);
    } else if (*ln.h_status != 0) {
      err = static_cast<sk_status>(*ln.h_status);
      // clear the device word for the lane's next step (stream order)
      *ln.h_status = 0;
      cudaMemsetAsync(ln.arena.d_status, 0, sizeof(int) * 4, ln.st);
    }
    for (int64_t t : ln.tickets) finish(t, err, now);
    ln.tickets.clear();
    ln.busy = false;
    any = true;
  }
  if (any) done_cv.notify_all();
  return any;
}

// Admit pending requests in arrival order: pool memory now, the copy of A is
// returned for the caller to issue without the lock.  Caller holds mu.
std::vector<AdmitCopy> sk_server::admit_locked() {
  std::vector<AdmitCopy> copies;
  while (!pending.empty() && resident < max_slots) {
    const int64_t t = pending.front();
    Request& r = reqs.at(t);
    uint64_t woff = 0, yoff = 0;
    if (!pool.alloc(r.work_bytes, &woff)) break;
    if (!pool.alloc(r.y_bytes, &yoff)) {
      pool.release(woff, r.work_bytes);
      break;
    }
    pending.pop_front();
    ++resident;
    r.work_off = woff;
    r.y_off = yoff;
    r.has_work = r.has_y = true;
    void* wsp = pool.at(woff + r.a_bytes);
    r.mb.A = r.a_bytes ? reinterpret_cast<const float*>(pool.at(woff)) : nullptr;
    r.mb.Y = reinterpret_cast<float*>(pool.at(yoff));
    r.mb.lda = r.ldp;
    r.mb.ldy = r.ldp;
    if (r.prec == SK_BF16X2) {
      r.mb.ws = wsp;
      r.mb.split_ready = r.a_bytes == 0;
    }
    r.state = State::Admitted;
    admitted.push_back(t);
    AdmitCopy c;
    c.ticket = t;
    c.dst = const_cast<float*>(r.mb.A);
    c.ldd = r.ldp;
    c.split = r.a_bytes == 0 ? wsp : nullptr;
    c.src = r.src;
    c.src_dev = r.src_dev;
    c.lds = r.src_ld;
    c.m = r.mb.m;
    c.n = r.mb.n;
    c.ready = r.src_ready;
    r.src_ready = nullptr;
    copies.push_back(c);
  }
  return copies;
}

// Take up to kMaxStepRequests admitted requests for lane `ln`.  Caller
// holds mu.
std::vector<StepItem> sk_server::take_step_locked(Lane* ln) {
  std::vector<StepItem> items;
  const size_t take = std::min<size_t>(admitted.size(), kMaxStepRequests);
  const Clock::time_point now = Clock::now();
  for (size_t i = 0; i < take; ++i) {
    const int64_t t = admitted[i];
    Request& r = reqs.at(t);
    r.state = State::Running;
    r.t_launch = now;
    items.push_back({t, r.mb, r.prec,
                     reinterpret_cast<float*>(pool.at(r.work_off + r.a_bytes)), r.ws_bytes});
    ln->tickets.push_back(t);
  }
  admitted.erase(admitted.begin(), admitted.begin() + take);
  ln->busy = true;
  ln->t_launch = now;
  ln->seq.fetch_add(1);
  ++steps;
  max_step = std::max<int64_t>(max_step, static_cast<int64_t>(take));
  return items;
}

// Enqueue one step on `ln`.  No lock held.
cudaError_t sk_server::launch_items(Lane* ln, const std::vector<StepItem>& items) {
  std::vector<sk::BatchMember> tc;
  for (const StepItem& it : items)
    if (it.prec == SK_BF16X2) tc.push_back(it.mb);
  cudaEvent_t ready = copy_recorded ? copy_ev : nullptr;
  cudaError_t e = cudaSuccess;
  if (!tc.empty())
    e = sk::batch_launch_members(tc.data(), tc.size(), kItemStages, &ln->arena, ready, ln->st);
  else if (ready)
    e = cudaStreamWaitEvent(ln->st, ready, 0);
  for (size_t i = 0; i < items.size() && e == cudaSuccess; ++i) {
    const StepItem& it = items[i];
    if (it.prec == SK_BF16X2) continue;
    sk_sketch h;
    memset(&h, 0, sizeof(h));
    h.seed = it.mb.seed;
    h.dist = it.mb.dist;
    h.k = it.mb.k;
    h.prec = SK_FP32;
    h.scale = it.mb.scale;
    h.device = device;
    h.d_status = ln->arena.d_status;
    h.wait_limit_ns = sk::kDefaultWaitLimitNs;
    h.stall_stage = -1;
    sk::GemmShape s;
    s.left = true;
    s.P = it.mb.k;
    s.Q = it.mb.n;
    s.L = it.mb.m;
    e = sk::simt_sketch(&h, s, it.mb.A, it.mb.lda, it.mb.Y, it.mb.ldy, it.simt_part,
                        it.simt_bytes, ln->st);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ln->h_status, ln->arena.d_status, sizeof(int), cudaMemcpyDeviceToHost,
                        ln->st);
  if (e == cudaSuccess) e = cudaEventRecord(ln->done, ln->st);
  if (e == cudaSuccess) {
    // wake the scheduler when the step has finished; if this cannot be
    // enqueued the scheduler still polls the event, at a slower cadence
    StepSignal* sg = new (std::nothrow) StepSignal;
    if (sg != nullptr) {
      *sg = StepSignal{this, ln, ln->seq.load()};  // seq is written by this thread only
      if (cudaLaunchHostFunc(ln->st, step_done_host_fn, sg) != cudaSuccess) {
        cudaGetLastError();
        delete sg;
      }
    }
  }
  return e;
}

void sk_server::scheduler() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    if (stop) break;
    const bool retired = retire_lanes(lk);
    std::vector<AdmitCopy> copies = admit_locked();
    Lane* ln = nullptr;
    std::vector<StepItem> items;
    if (!admitted.empty())
      for (Lane& l : lanes)
        if (!l.busy) {
          ln = &l;
          items = take_step_locked(ln);
          break;
        }
    if (copies.empty() && items.empty()) {
      if (retired) continue;
      bool busy = false;
      for (const Lane& l : lanes) busy |= l.busy;
      if (busy) {
        // a step is in flight: sleep until its host function (or new work)
        // wakes the scheduler, unless one has signalled already; the short
        // timeout bounds the cost of a wake-up that arrived between this
        // check and the wait (the host function takes no lock)
        bool signalled = false;
        for (const Lane& l : lanes)
          signalled |= l.busy && l.signalled_seq.load() == l.seq.load();
        if (!signalled) work_cv.wait_for(lk, std::chrono::microseconds(200));
      } else {
        // idle: refresh the clock reference if it is a second old
        if (!ref_valid || Clock::now() - ref_host > std::chrono::seconds(1)) {
          lk.unlock();
          calibrate_clock();
          lk.lock();
          continue;
        }
        work_cv.wait_for(lk, std::chrono::seconds(1));
      }
      continue;
    }
    // CUDA work without the lock: copies of A first, then the step that
    // waits for them
    lk.unlock();
    std::vector<std::pair<int64_t, cudaError_t>> copy_failed;
    for (const AdmitCopy& c : copies) {
      const cudaError_t e = issue_copy(c);
      if (e != cudaSuccess) copy_failed.push_back({c.ticket, e});
    }
    if (!copies.empty()) {
      cudaEventRecord(copy_ev, copy_st);
      copy_recorded = true;
    }
    if (!copy_failed.empty() && !items.empty()) {
      std::vector<StepItem> keep;
      for (const StepItem& it : items) {
        bool bad = false;
        for (const auto& f : copy_failed) bad |= f.first == it.ticket;
        if (!bad) keep.push_back(it);
      }
      items.swap(keep);
    }
    cudaError_t le = cudaSuccess;
    if (ln) {
      le = launch_items(ln, items);
      if (le != cudaSuccess) cudaStreamSynchronize(ln->st);
    }
    lk.lock();
    // the waits on the producers' events are enqueued: the events may be
    // recorded again by later submissions
    for (const AdmitCopy& c : copies) free_events.push_back(c.ready);
    const Clock::time_point now = Clock::now();
    for (const auto& f : copy_failed) {
      admitted.erase(std::remove(admitted.begin(), admitted.end(), f.first), admitted.end());
      if (ln)
        ln->tickets.erase(std::remove(ln->tickets.begin(), ln->tickets.end(), f.first),
                          ln->tickets.end());
      finish(f.first, sk::status_from_cuda(f.second), now);
    }
    if (ln && le != cudaSuccess) {
      const sk_status err = sk::status_from_cuda(le);
      for (int64_t t : ln->tickets) finish(t, err, now);
      ln->tickets.clear();
      ln->busy = false;
    } else if (ln && ln->tickets.empty()) {
      ln->busy = false;  // every request of the step failed its copy
    }
    if (!copy_failed.empty() || le != cudaSuccess) done_cv.notify_all();
  }
  // shutdown: cancel what has not been launched, drain what has
  const Clock::time_point now = Clock::now();
  for (int64_t t : pending) {
    Request& r = reqs.at(t);
    if (r.src_ready) free_events.push_back(r.src_ready);
    r.src_ready = nullptr;
    r.state = State::Failed;
    r.err = SK_ECANCELLED;
    r.t_done = now;
  }
  pending.clear();
  for (int64_t t : admitted) finish(t, SK_ECANCELLED, now);
  admitted.clear();
  for (Lane& l : lanes)
    if (l.busy) {
      lk.unlock();
      cudaEventSynchronize(l.done);
      lk.lock();
    }
  retire_lanes(lk);
  // the completion host functions take mu: wait for them without it
  lk.unlock();
  for (Lane& l : lanes) cudaStreamSynchronize(l.st);
  lk.lock();
  cudaStreamSynchronize(copy_st);
  done_cv.notify_all();
}

namespace {

void destroy_resources(sk_server* s) {
  for (Lane& l : s->lanes) {
    if (l.done) cudaEventDestroy(l.done);
    if (l.st) cudaStreamDestroy(l.st);
    if (l.h_status) cudaFreeHost(l.h_status);
    if (l.arena.d_buf) cudaFree(l.arena.d_buf);
    if (l.arena.ws) cudaFree(l.arena.ws);
    if (l.arena.d_status) cudaFree(l.arena.d_status);
    if (l.arena.h_stage) cudaFreeHost(l.arena.h_stage);
  }
  if (s->copy_ev) cudaEventDestroy(s->copy_ev);
  if (s->ref_ev) cudaEventDestroy(s->ref_ev);
  if (s->copy_st) cudaStreamDestroy(s->copy_st);
  for (cudaEvent_t ev : s->all_events) cudaEventDestroy(ev);
  s->pool.destroy();
}

sk_status poll_locked(sk_server* s, int64_t ticket, double* latency_ms) {
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return SK_EINVAL;
  const Request& r = it->second;
  switch (r.state) {
    case State::Done:
    case State::Fetching:
      if (latency_ms) *latency_ms = ms_between(r.t_arrival, r.t_done);
      return SK_OK;
    case State::Failed:
      return r.err;
    default:
      return SK_EBUSY;
  }
}

}  // namespace

extern "C" {

sk_status sk_server_create(uint64_t hbm_budget_bytes, int32_t max_slots, sk_server_handle* out) {
  if (!out || hbm_budget_bytes == 0 || max_slots < 1) return SK_EINVAL;
  *out = nullptr;
  sk_server* s = new (std::nothrow) sk_server;
  if (!s) return SK_ENOMEM;
  s->max_slots = max_slots;
  cudaError_t e = cudaGetDevice(&s->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device);
  if (e == cudaSuccess) e = s->pool.init(hbm_budget_bytes);
  for (Lane& l : s->lanes) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&l.st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&l.done, cudaEventDefault);  // timed
    if (e == cudaSuccess)
      e = cudaHostAlloc(reinterpret_cast<void**>(&l.h_status), sizeof(int) * 4,
                        cudaHostAllocDefault);
    if (e == cudaSuccess)
      e = cudaMalloc(reinterpret_cast<void**>(&l.arena.d_status), sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMemset(l.arena.d_status, 0, sizeof(int) * 4);
    l.arena.async_upload = true;  // a lane is reused only after its step finished
    if (e == cudaSuccess) memset(l.h_status, 0, sizeof(int) * 4);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy_st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->copy_ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ref_ev, cudaEventDefault);
  if (e == cudaSuccess) s->calibrate_clock();
  if (e != cudaSuccess) {
    const sk_status st = sk::status_from_cuda(e);
    destroy_resources(s);
    delete s;
    return st;
  }
  s->thread = std::thread([s] { s->scheduler(); });
  *out = s;
  return SK_OK;
}

sk_status sk_server_submit(sk_server_handle s, sk_handle h, const float* A, int64_t m,
                           int64_t n, int64_t lda, void* stream, int64_t* ticket) {
  const Clock::time_point arrival = Clock::now();
  if (!s || !h || !A || !ticket || m <= 0 || n <= 0 || lda < n) return SK_EINVAL;
  if (m >= (1LL << 31) - 64) return SK_EINVAL;
  if (h->prec != SK_BF16X2 && h->prec != SK_FP32) return SK_EUNSUPPORTED;
  Request r;
  r.prec = h->prec;
  r.src = A;
  r.src_ld = lda;
  r.ldp = (n + 3) / 4 * 4;
  r.mb.seed = h->seed;
  r.mb.dist = h->dist;
  r.mb.k = h->k;
  r.mb.scale = h->scale;
  r.mb.m = m;
  r.mb.n = n;
  sk::GemmShape sh;
  sh.left = true;
  sh.P = h->k;
  sh.Q = n;
  sh.L = m;
  // device memory, managed memory and mapped pinned host memory are read by
  // the admission kernels; anything else goes through the copy engine
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, A) == cudaSuccess) {
    if (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged ||
        pa.type == cudaMemoryTypeHost) {
      if (pa.type != cudaMemoryTypeHost || pa.device == s->device)
        r.src_dev = static_cast<const float*>(pa.devicePointer);
      if (pa.type == cudaMemoryTypeDevice && pa.device != s->device) return SK_EINVAL;
    }
  } else {
    cudaGetLastError();
  }
  const uint64_t a_copy = round_up(static_cast<uint64_t>(m) * r.ldp * sizeof(float), kAlign);
  if (r.prec == SK_BF16X2) {
    // pool addresses are 256-byte aligned and the strides multiples of 4
    const sk_status cs = sk::tc_check(sh, reinterpret_cast<const float*>(kAlign), r.ldp,
                                      reinterpret_cast<const float*>(kAlign), r.ldp);
    if (cs != SK_OK) return cs;
    // items sized so that a request alone spreads over the whole GPU; the
    // length depends on the request's shape only
    r.mb.item_stages = sk::spread_item_stages(r.mb);
    r.ws_bytes = round_up(sk::batch_member_workspace(r.mb, r.mb.item_stages), kAlign);
    // a readable source is split on admission; a pageable one is copied first
    r.a_bytes = r.src_dev ? 0 : a_copy;
  } else {
    r.ws_bytes = round_up(sk::simt_workspace_bytes(sh), kAlign);
    r.a_bytes = a_copy;
  }
  r.work_bytes = r.a_bytes + r.ws_bytes;
  r.y_bytes = round_up(static_cast<uint64_t>(h->k) * r.ldp * sizeof(float), kAlign);
  r.t_arrival = arrival;
  std::lock_guard<std::mutex> g(s->mu);
  if (s->stop) return SK_ECANCELLED;
  if (r.work_bytes + r.y_bytes > s->pool.size()) return SK_EBUDGET;
  if (s->free_events.empty()) {
    cudaEvent_t ev = nullptr;
    const cudaError_t ce = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (ce != cudaSuccess) return sk::status_from_cuda(ce);
    s->all_events.push_back(ev);
    s->free_events.push_back(ev);
  }
  r.src_ready = s->free_events.back();
  const cudaError_t re = cudaEventRecord(r.src_ready, static_cast<cudaStream_t>(stream));
  if (re != cudaSuccess) {
    r.src_ready = nullptr;
    return sk::status_from_cuda(re);
  }
  s->free_events.pop_back();
  const int64_t t = s->next_ticket++;
  s->reqs.emplace(t, r);
  s->pending.push_back(t);
  ++s->submitted;
  if (!s->have_first) {
    s->have_first = true;
    s->first_arrival = arrival;
  }
  *ticket = t;
  s->work_cv.notify_one();
  return SK_OK;
}

sk_status sk_server_poll(sk_server_handle s, int64_t ticket, double* latency_ms) {
  if (!s) return SK_EINVAL;
  std::lock_guard<std::mutex> g(s->mu);
  return poll_locked(s, ticket, latency_ms);
}

sk_status sk_server_wait(sk_server_handle s, int64_t ticket, double timeout_s,
                         double* latency_ms) {
  if (!s || !(timeout_s >= 0.0)) return SK_EINVAL;
  const auto deadline =
      Clock::now() + std::chrono::duration_cast<Clock::duration>(
                         std::chrono::duration<double>(std::min(timeout_s, 1e7)));
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    const sk_status st = poll_locked(s, ticket, latency_ms);
    if (st != SK_EBUSY) return st;
    if (s->done_cv.wait_until(lk, deadline) == std::cv_status::timeout)
      return poll_locked(s, ticket, latency_ms);
  }
}

sk_status sk_server_fetch(sk_server_handle s, int64_t ticket, float* Y, int64_t ldy,
                          void* stream) {
  if (!s || !Y) return SK_EINVAL;
  const float* src = nullptr;
  int64_t rows = 0, cols = 0, ldp = 0;
  {
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return SK_EINVAL;
    Request& r = it->second;
    if (r.state == State::Failed) {
      const sk_status err = r.err;
      if (r.has_y || r.has_work) --s->resident;
      s->free_work(r);
      s->free_y(r);
      s->reqs.erase(it);
      s->work_cv.notify_one();
      return err;
    }
    if (r.state != State::Done) return r.state == State::Fetching ? SK_EINVAL : SK_EBUSY;
    if (ldy < r.mb.n) return SK_EINVAL;
    r.state = State::Fetching;
    src = r.mb.Y;
    rows = r.mb.k;
    cols = r.mb.n;
    ldp = r.ldp;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpy2DAsync(Y, ldy * sizeof(float), src, ldp * sizeof(float),
                                    cols * sizeof(float), rows, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->reqs.find(ticket);
  Request& r = it->second;
  if (e != cudaSuccess) {
    r.state = State::Done;  // the result is still there; the caller may retry
    return sk::status_from_cuda(e);
  }
  s->free_y(r);
  --s->resident;
  s->reqs.erase(it);
  s->work_cv.notify_one();
  return SK_OK;
}

sk_status sk_server_release(sk_server_handle s, int64_t ticket) {
  if (!s) return SK_EINVAL;
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return SK_EINVAL;
  Request& r = it->second;
  switch (r.state) {
    case State::Pending:
    case State::Admitted:
    case State::Running:
      r.release_when_done = true;
      break;
    case State::Fetching:
      return SK_EINVAL;
    case State::Done:
    case State::Failed:
      if (r.has_y || r.has_work) --s->resident;
      s->free_work(r);
      s->free_y(r);
      s->reqs.erase(it);
      break;
  }
  s->work_cv.notify_one();
  return SK_OK;
}

sk_status sk_server_stats_get(sk_server_handle s, sk_server_stats* out) {
  if (!s || !out) return SK_EINVAL;
  std::vector<double> lat;
  {
    std::lock_guard<std::mutex> g(s->mu);
    memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->pending = static_cast<int64_t>(s->pending.size());
    out->resident = s->resident;
    out->steps = s->steps;
    out->max_step_requests = s->max_step;
    out->flops = s->flops;
    out->pool_bytes = s->pool.size();
    out->peak_bytes = s->pool.peak();
    if (s->completed > 0) out->mean_wait_ms = s->wait_sum_ms / s->completed;
    if (s->have_first && s->completed > 0)
      out->busy_s = ms_between(s->first_arrival, s->last_done) * 1e-3;
    lat = s->latencies;
  }
  if (!lat.empty()) {
    std::sort(lat.begin(), lat.end());
    // nearest-rank percentiles
    auto pct = [&](double p) {
      size_t r = static_cast<size_t>(std::ceil(p / 100.0 * lat.size()));
      return lat[std::min(lat.size(), std::max<size_t>(r, 1)) - 1];
    };
    out->p50_ms = pct(50.0);
    out->p99_ms = pct(99.0);
    double sum = 0.0;
    for (double v : lat) sum += v;
    out->mean_ms = sum / lat.size();
    out->max_ms = lat.back();
  }
  return SK_OK;
}

sk_status sk_server_reset_stats(sk_server_handle s) {
  if (!s) return SK_EINVAL;
  std::lock_guard<std::mutex> g(s->mu);
  s->submitted = static_cast<int64_t>(s->pending.size());
  s->completed = s->failed = s->steps = s->max_step = 0;
  s->latencies.clear();
  s->wait_sum_ms = s->flops = 0.0;
  s->have_first = false;
  for (const auto& kv : s->reqs) {
    const Request& r = kv.second;
    if (r.state == State::Pending || r.state == State::Admitted || r.state == State::Running) {
      if (!s->have_first || r.t_arrival < s->first_arrival) s->first_arrival = r.t_arrival;
      s->have_first = true;
    }
  }
  s->pool.reset_peak();
  return SK_OK;
}

sk_status sk_server_destroy(sk_server_handle s) {
  if (!s) return SK_EINVAL;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
  }
  s->work_cv.notify_all();
  if (s->thread.joinable()) s->thread.join();
  destroy_resources(s);
  delete s;
  return SK_OK;
}

}  // extern "C"

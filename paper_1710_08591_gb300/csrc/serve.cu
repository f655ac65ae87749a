// Continuous-batching server: voltage frames from many independent streams, each one
// window (n_int samples) of one of a few lattices, transformed as they arrive.
//
// A scheduler thread owns the device side:
//   admission  a frame is admitted when a device slot is free; slots are fixed-size
//              regions (frame bytes + its beams) carved from one allocation of the HBM
//              budget, so admission is bounded by that budget;
//   staging    admitted frames are copied host -> slot on a copy stream (one event each);
//   ticks      whenever frames are staged and fewer than kTicks launches are in flight,
//              every staged frame (up to 64) goes into ONE persistent launch of the batch
//              kernel (one job per frame) on the next tick stream, which waits for the
//              frames' copy events; the beams are copied back to the caller's buffers on
//              the same stream. Frames that arrive while ticks run join the next tick, so
//              work from different arrivals overlaps on the device.
//   completion ticks are polled by event; a frame's latency is completion - submission
//              (host steady clock, read before the submitting thread takes the lock),
//              and its slot returns to the free list.
// The scheduler holds the server's lock only to move frames between its queues and to
// publish completions; every CUDA call (copies, event records and queries, launches) is
// issued with the lock released, so submitters and waiters never wait behind the GPU.
// Completion is tracked as a watermark (every ticket below it is done) plus the set of
// tickets done out of order above it, and latencies in a bounded reservoir, so a
// long-running server's bookkeeping stays small.
// A frame's beams depend only on the frame (the batch kernel's summation order is fixed
// per work item), so they are bit-identical alone and in any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <random>
#include <set>
#include <thread>
#include <vector>

#include "internal.cuh"

namespace fftbf {
namespace {

using Clock = std::chrono::steady_clock;
constexpr int kTicks = 2;        // launches in flight
constexpr int kJobsPerTick = 64;
constexpr size_t kReservoir = 1 << 16;   // latency samples kept (exact below this count)

struct Frame {
  int64_t ticket = 0;
  int lattice = 0;
  const uint8_t* host_in = nullptr;
  float* host_out = nullptr;
  Clock::time_point t_submit;
  int slot = -1;
  cudaEvent_t copied = nullptr;
};

// Owned by the scheduler thread alone (no lock needed).
struct Tick {
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
  BatchJob* d_jobs = nullptr;
  unsigned long long* d_counter = nullptr;
  std::vector<Frame> frames;
  bool busy = false;
};

}  // namespace
}  // namespace fftbf

using namespace fftbf;

struct fftbf_server {
  int device = 0;
  std::vector<fftbf_plan*> lattices;
  fftbf_batch* tuner = nullptr;          // owns the tuned tile per lattice
  std::vector<int> S;
  std::vector<int> V;                    // tuned variant per lattice (generic or warp path)
  size_t smem = 0;
  int grid = 0;
  size_t slot_bytes = 0, frame_off = 0;
  std::vector<size_t> in_bytes, out_bytes;
  unsigned char* arena = nullptr;
  std::vector<cudaEvent_t> slot_events;
  cudaStream_t copy_st = nullptr;
  Tick ticks[kTicks];                    // scheduler thread only
  int next_tick = 0;                     // scheduler thread only

  // ---- shared state, under mu
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::vector<int> free_slots;
  std::deque<Frame> pending;             // submitted, not yet admitted
  std::deque<Frame> staged;              // copy issued, waiting for a launch
  int64_t done_below = 0;                // every ticket < done_below has completed
  std::set<int64_t> done_above;          // completed tickets >= done_below
  int64_t next_ticket = 0, completed = 0, launches = 0, frames_launched = 0;
  int64_t max_frames_launch = 0, max_items_launch = 0;
  int64_t inflight = 0, peak_inflight = 0;
  std::vector<double> lat_res;           // reservoir sample of latencies (ms)
  int64_t lat_seen = 0;
  double lat_sum = 0.0, lat_max = 0.0;
  std::mt19937_64 lat_rng{0x5eed};
  int error = FFTBF_OK;
  bool hold = false;
  bool stop = false;
  std::thread worker;
};

namespace {

void record_done(fftbf_server* sv, int64_t ticket, double ms) {
  if (ticket == sv->done_below) {
    ++sv->done_below;
    while (!sv->done_above.empty() && *sv->done_above.begin() == sv->done_below) {
      sv->done_above.erase(sv->done_above.begin());
      ++sv->done_below;
    }
  } else {
    sv->done_above.insert(ticket);
  }
  ++sv->lat_seen;
  sv->lat_sum += ms;
  sv->lat_max = std::max(sv->lat_max, ms);
  if (sv->lat_res.size() < kReservoir) {
    sv->lat_res.push_back(ms);
  } else {
    const uint64_t j = sv->lat_rng() % (uint64_t)sv->lat_seen;   // Algorithm R
    if (j < kReservoir) sv->lat_res[j] = ms;
  }
}

void fail(fftbf_server* sv, int rc) {
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->error == FFTBF_OK) sv->error = rc;
  sv->cv_done.notify_all();
}

// Issue one launch over `frames` on tick `tk` (lock not held).
int launch_tick(fftbf_server* sv, Tick& tk, int64_t* items_out) {
  NvtxRange nvtx("serve tick");
  const int n = (int)tk.frames.size();
  std::vector<BatchJob> jobs(n);
  int64_t total = 0;
  for (int k = 0; k < n; ++k) {
    const Frame& f = tk.frames[k];
    const fftbf_plan* p = sv->lattices[f.lattice];
    BatchJob& J = jobs[k];
    batch_fill_args(p, J.a);
    J.a.S = sv->S[f.lattice];
    unsigned char* slot = sv->arena + (size_t)f.slot * sv->slot_bytes;
    J.a.volts = slot;
    J.a.beams = reinterpret_cast<float*>(slot + sv->frame_off);
    J.a.nwin = 1;
    J.variant = sv->V[f.lattice];
    J.nitems = p->nfreq;
    J.item0 = total;
    total += J.nitems;
    if (cudaStreamWaitEvent(tk.st, f.copied, 0) != cudaSuccess) return FFTBF_ECUDA;
  }
  *items_out = total;
  int rc = batch_launch_jobs(jobs.data(), n, tk.d_jobs, tk.d_counter, sv->smem, sv->grid, tk.st);
  for (int k = 0; k < n && rc == FFTBF_OK; ++k) {
    const Frame& f = tk.frames[k];
    unsigned char* slot = sv->arena + (size_t)f.slot * sv->slot_bytes;
    if (cudaMemcpyAsync(f.host_out, slot + sv->frame_off, sv->out_bytes[f.lattice],
                        cudaMemcpyDeviceToHost, tk.st) != cudaSuccess)
      rc = FFTBF_ECUDA;
  }
  if (rc == FFTBF_OK && cudaEventRecord(tk.done, tk.st) != cudaSuccess) rc = FFTBF_ECUDA;
  return rc;
}

void run_scheduler(fftbf_server* sv) {
  cudaSetDevice(sv->device);
  std::vector<Frame> admitted;
  bool deferred = false;
  while (true) {
    bool any_busy = false;
    for (const Tick& t : sv->ticks) any_busy = any_busy || t.busy;
    // ---- admission: frames get free slots (under the lock)
    admitted.clear();
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      auto has_work = [&]() {
        return (sv->stop && !any_busy) || (!sv->pending.empty() && !sv->free_slots.empty()) ||
               (!sv->staged.empty() && !sv->hold && !sv->ticks[sv->next_tick].busy);
      };
      if (!has_work()) {
        // busy ticks are polled every 20 us; otherwise sleep until a submission
        sv->cv_work.wait_for(lk, any_busy ? std::chrono::microseconds(20) : std::chrono::milliseconds(5),
                             has_work);
      }
      if (sv->stop && sv->pending.empty() && sv->staged.empty() && !any_busy) break;
      while (!sv->pending.empty() && !sv->free_slots.empty()) {
        Frame f = sv->pending.front();
        sv->pending.pop_front();
        f.slot = sv->free_slots.back();
        sv->free_slots.pop_back();
        f.copied = sv->slot_events[f.slot];
        admitted.push_back(f);
        ++sv->inflight;
        sv->peak_inflight = std::max(sv->peak_inflight, sv->inflight);
      }
    }
    // ---- staging: host -> slot copies (lock released)
    int rc = FFTBF_OK;
    for (const Frame& f : admitted) {
      unsigned char* dst = sv->arena + (size_t)f.slot * sv->slot_bytes;
      cudaError_t e = cudaMemcpyAsync(dst, f.host_in, sv->in_bytes[f.lattice],
                                      cudaMemcpyHostToDevice, sv->copy_st);
      if (e == cudaSuccess) e = cudaEventRecord(f.copied, sv->copy_st);
      if (e != cudaSuccess) rc = FFTBF_ECUDA;
    }
    if (rc != FFTBF_OK) fail(sv, rc);
    // ---- pick a launch: every staged frame (up to kJobsPerTick) on the next free tick
    Tick& tk = sv->ticks[sv->next_tick];
    bool launch = false;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      for (const Frame& f : admitted) sv->staged.push_back(f);
      // frames that can still be admitted go into this launch too: admit them first (for
      // one round at most, so that a steady stream of arrivals cannot hold a launch back)
      const bool admissible = !sv->pending.empty() && !sv->free_slots.empty();
      if (!sv->staged.empty() && !sv->hold && !tk.busy && admissible && !deferred) {
        deferred = true;
      } else if (!sv->staged.empty() && !sv->hold && !tk.busy) {
        deferred = false;
        const int n = (int)std::min<size_t>(sv->staged.size(), kJobsPerTick);
        tk.frames.assign(sv->staged.begin(), sv->staged.begin() + n);
        sv->staged.erase(sv->staged.begin(), sv->staged.begin() + n);
        launch = true;
      }
    }
    if (launch) {
      int64_t items = 0;
      rc = launch_tick(sv, tk, &items);
      tk.busy = true;
      sv->next_tick = (sv->next_tick + 1) % kTicks;
      std::lock_guard<std::mutex> lk(sv->mu);
      if (rc != FFTBF_OK && sv->error == FFTBF_OK) sv->error = rc;
      ++sv->launches;
      sv->frames_launched += (int64_t)tk.frames.size();
      sv->max_frames_launch = std::max(sv->max_frames_launch, (int64_t)tk.frames.size());
      sv->max_items_launch = std::max(sv->max_items_launch, items);
    }
    // ---- completions: query unlocked, publish under the lock
    for (Tick& k : sv->ticks) {
      if (!k.busy) continue;
      const cudaError_t q = cudaEventQuery(k.done);
      if (q == cudaErrorNotReady) continue;
      const auto now = Clock::now();
      std::lock_guard<std::mutex> lk(sv->mu);
      if (q != cudaSuccess && sv->error == FFTBF_OK) sv->error = FFTBF_ECUDA;
      for (const Frame& f : k.frames) {
        record_done(sv, f.ticket, std::chrono::duration<double, std::milli>(now - f.t_submit).count());
        sv->free_slots.push_back(f.slot);
        --sv->inflight;
        ++sv->completed;
      }
      k.frames.clear();
      k.busy = false;
      sv->cv_done.notify_all();
    }
  }
}

}  // namespace

extern "C" {

fftbf_server* fftbf_server_create(fftbf_plan* const* lattices, int n, int64_t hbm_budget_bytes) {
  if (!lattices || n < 1 || n > 64 || hbm_budget_bytes <= 0) {
    set_error(FFTBF_EINVAL, "need 1..64 lattice plans and a positive HBM budget");
    return nullptr;
  }
  fftbf_server* sv = new (std::nothrow) fftbf_server();
  if (!sv) { set_error(FFTBF_ENOMEM, "cannot allocate server"); return nullptr; }
  sv->lattices.assign(lattices, lattices + n);
  sv->device = lattices[0]->device;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(sv->device);
  sv->tuner = fftbf_batch_create(lattices, n);
  if (!sv->tuner) { delete sv; cudaSetDevice(prev); return nullptr; }
  for (int i = 0; i < n; ++i) {
    sv->S.push_back(fftbf_batch_tuned_steps(sv->tuner, i));
    sv->V.push_back(fftbf_batch_tuned_variant(sv->tuner, i));
  }
  sv->smem = fftbf_batch_smem(sv->tuner);
  sv->grid = fftbf_batch_grid(sv->tuner);
  size_t max_in = 0, max_out = 0;
  for (auto* p : sv->lattices) {
    sv->in_bytes.push_back((size_t)p->n_int * p->nfreq * p->npol * p->nx * p->ny);
    sv->out_bytes.push_back((size_t)p->nfreq * p->mx * p->my * sizeof(float));
    max_in = std::max(max_in, sv->in_bytes.back());
    max_out = std::max(max_out, sv->out_bytes.back());
  }
  sv->frame_off = (max_in + 255) & ~(size_t)255;
  sv->slot_bytes = (sv->frame_off + max_out + 255) & ~(size_t)255;
  const int64_t nslots = std::min<int64_t>(hbm_budget_bytes / (int64_t)sv->slot_bytes, 1 << 16);
  cudaError_t e = cudaSuccess;
  if (nslots < 1) {
    set_error(FFTBF_EINVAL, "HBM budget %lld below one frame slot (%zu bytes)",
              (long long)hbm_budget_bytes, sv->slot_bytes);
    fftbf_server_destroy(sv);
    cudaSetDevice(prev);
    return nullptr;
  }
  e = cudaMalloc(&sv->arena, (size_t)nslots * sv->slot_bytes);
  for (int64_t i = 0; i < nslots && e == cudaSuccess; ++i) {
    cudaEvent_t ev;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) {
      sv->slot_events.push_back(ev);
      sv->free_slots.push_back((int)(nslots - 1 - i));
    }
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->copy_st, cudaStreamNonBlocking);
  for (int t = 0; t < kTicks && e == cudaSuccess; ++t) {
    e = cudaStreamCreateWithFlags(&sv->ticks[t].st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sv->ticks[t].done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&sv->ticks[t].d_jobs, sizeof(BatchJob) * kJobsPerTick);
    if (e == cudaSuccess) e = cudaMalloc(&sv->ticks[t].d_counter, sizeof(unsigned long long));
  }
  if (e != cudaSuccess) {
    cuda_error(e, "fftbf_server_create");
    fftbf_server_destroy(sv);
    cudaSetDevice(prev);
    return nullptr;
  }
  sv->worker = std::thread(run_scheduler, sv);
  cudaSetDevice(prev);
  return sv;
}

int64_t fftbf_server_submit(fftbf_server* sv, int lattice, const uint8_t* frame_host,
                            float* beams_host) {
  const auto t_submit = Clock::now();       // before the lock: waiting for it is latency
  if (!sv) return set_error(FFTBF_EINVAL, "null server");
  if (lattice < 0 || lattice >= (int)sv->lattices.size())
    return set_error(FFTBF_EINVAL, "lattice %d out of range", lattice);
  if (!frame_host || !beams_host) return set_error(FFTBF_EINVAL, "null frame or beam buffer");
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->error != FFTBF_OK) return set_error(sv->error, "server stopped after a CUDA error");
  Frame f;
  f.ticket = sv->next_ticket++;
  f.lattice = lattice;
  f.host_in = frame_host;
  f.host_out = beams_host;
  f.t_submit = t_submit;
  sv->pending.push_back(f);
  sv->cv_work.notify_one();
  return f.ticket;
}

int fftbf_server_hold(fftbf_server* sv, int hold) {
  if (!sv) return set_error(FFTBF_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->hold = hold != 0;
  sv->cv_work.notify_one();
  return FFTBF_OK;
}

int fftbf_server_wait(fftbf_server* sv, int64_t ticket, double timeout_s) {
  if (!sv) return set_error(FFTBF_EINVAL, "null server");
  std::unique_lock<std::mutex> lk(sv->mu);
  if (ticket >= sv->next_ticket)
    return set_error(FFTBF_EINVAL, "ticket %lld was never issued", (long long)ticket);
  const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s);
  auto done = [&]() {
    if (sv->error != FFTBF_OK) return true;
    if (ticket < 0) return sv->completed == sv->next_ticket;
    return ticket < sv->done_below || sv->done_above.count(ticket) != 0;
  };
  if (!sv->cv_done.wait_until(lk, deadline, done))
    return set_error(FFTBF_ETIMEOUT, "frame %lld not complete within %.3f s", (long long)ticket, timeout_s);
  if (sv->error != FFTBF_OK) return set_error(sv->error, "server stopped after a CUDA error");
  return FFTBF_OK;
}

int fftbf_server_stats(fftbf_server* sv, fftbf_server_stats_t* out) {
  if (!sv || !out) return set_error(FFTBF_EINVAL, "null argument");
  std::vector<double> l;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    l = sv->lat_res;
    out->submitted = sv->next_ticket;
    out->completed = sv->completed;
    out->launches = sv->launches;
    out->frames_per_launch = sv->launches ? (double)sv->frames_launched / (double)sv->launches : 0.0;
    out->max_frames_per_launch = sv->max_frames_launch;
    out->max_items_per_launch = sv->max_items_launch;
    out->grid = sv->grid;
    out->peak_inflight = sv->peak_inflight;
    out->slots = (int64_t)sv->slot_events.size();
    out->max_ms = sv->lat_max;
    out->mean_ms = sv->lat_seen ? sv->lat_sum / (double)sv->lat_seen : 0.0;
  }
  std::sort(l.begin(), l.end());
  auto pct = [&](double q) {
    if (l.empty()) return 0.0;
    const size_t i = std::min(l.size() - 1, (size_t)(q * (double)(l.size() - 1) + 0.5));
    return l[i];
  };
  out->p50_ms = pct(0.50);
  out->p99_ms = pct(0.99);
  std::lock_guard<std::mutex> lk(sv->mu);
  return sv->error;
}

void fftbf_server_destroy(fftbf_server* sv) {
  if (!sv) return;
  if (sv->worker.joinable()) {
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->stop = true;
      sv->hold = false;                 // held frames still run before the server stops
      sv->cv_work.notify_one();
    }
    sv->worker.join();
  }
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(sv->device);
  for (auto& t : sv->ticks) {
    if (t.st) cudaStreamSynchronize(t.st);
    if (t.done) cudaEventDestroy(t.done);
    cudaFree(t.d_jobs);
    cudaFree(t.d_counter);
    if (t.st) cudaStreamDestroy(t.st);
  }
  if (sv->copy_st) {
    cudaStreamSynchronize(sv->copy_st);
    cudaStreamDestroy(sv->copy_st);
  }
  for (auto ev : sv->slot_events) cudaEventDestroy(ev);
  cudaFree(sv->arena);
  fftbf_batch_destroy(sv->tuner);
  cudaSetDevice(prev);
  delete sv;
}

}  // extern "C"

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
//              (host steady clock), and its slot returns to the free list.
// A frame's beams depend only on the frame (the batch kernel's summation order is fixed
// per work item), so they are bit-identical alone and in any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "internal.cuh"

namespace fftbf {
namespace {

using Clock = std::chrono::steady_clock;
constexpr int kTicks = 2;        // launches in flight
constexpr int kJobsPerTick = 64;

struct Frame {
  int64_t ticket = 0;
  int lattice = 0;
  const uint8_t* host_in = nullptr;
  float* host_out = nullptr;
  Clock::time_point t_submit;
  int slot = -1;
  cudaEvent_t copied = nullptr;
};

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
  std::vector<int> free_slots;
  std::vector<cudaEvent_t> slot_events;
  cudaStream_t copy_st = nullptr;
  Tick ticks[kTicks];
  int next_tick = 0;

  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Frame> pending;             // submitted, not yet admitted
  std::deque<Frame> staged;              // copy issued, waiting for a tick
  std::vector<int64_t> done_tickets;     // sorted insert not needed: checked by scan
  int64_t next_ticket = 0, completed = 0, launches = 0, frames_launched = 0;
  int64_t inflight = 0, peak_inflight = 0;
  std::vector<double> latencies_ms;
  int error = FFTBF_OK;
  bool stop = false;
  std::thread worker;
};

namespace {

void run_scheduler(fftbf_server* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  while (true) {
    bool progressed = false;
    // ---- admission + staging
    while (!sv->pending.empty() && !sv->free_slots.empty()) {
      Frame f = sv->pending.front();
      sv->pending.pop_front();
      f.slot = sv->free_slots.back();
      sv->free_slots.pop_back();
      f.copied = sv->slot_events[f.slot];
      unsigned char* dst = sv->arena + (size_t)f.slot * sv->slot_bytes;
      cudaError_t e = cudaMemcpyAsync(dst, f.host_in, sv->in_bytes[f.lattice],
                                      cudaMemcpyHostToDevice, sv->copy_st);
      if (e == cudaSuccess) e = cudaEventRecord(f.copied, sv->copy_st);
      if (e != cudaSuccess && sv->error == FFTBF_OK) sv->error = FFTBF_ECUDA;
      sv->staged.push_back(f);
      ++sv->inflight;
      sv->peak_inflight = std::max(sv->peak_inflight, sv->inflight);
      progressed = true;
    }
    // ---- launch a tick over everything staged
    Tick& tk = sv->ticks[sv->next_tick];
    if (!sv->staged.empty() && !tk.busy) {
      NvtxRange nvtx("serve tick");
      const int n = (int)std::min<size_t>(sv->staged.size(), kJobsPerTick);
      tk.frames.assign(sv->staged.begin(), sv->staged.begin() + n);
      sv->staged.erase(sv->staged.begin(), sv->staged.begin() + n);
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
        cudaStreamWaitEvent(tk.st, f.copied, 0);
      }
      int rc = batch_launch_jobs(jobs.data(), n, tk.d_jobs, tk.d_counter, sv->smem, sv->grid, tk.st);
      for (int k = 0; k < n && rc == FFTBF_OK; ++k) {
        const Frame& f = tk.frames[k];
        unsigned char* slot = sv->arena + (size_t)f.slot * sv->slot_bytes;
        if (cudaMemcpyAsync(f.host_out, slot + sv->frame_off, sv->out_bytes[f.lattice],
                            cudaMemcpyDeviceToHost, tk.st) != cudaSuccess)
          rc = FFTBF_ECUDA;
      }
      if (rc == FFTBF_OK && cudaEventRecord(tk.done, tk.st) != cudaSuccess) rc = FFTBF_ECUDA;
      if (rc != FFTBF_OK && sv->error == FFTBF_OK) sv->error = rc;
      tk.busy = true;
      ++sv->launches;
      sv->frames_launched += n;
      sv->next_tick = (sv->next_tick + 1) % kTicks;
      progressed = true;
    }
    // ---- completions
    for (int t = 0; t < kTicks; ++t) {
      Tick& k = sv->ticks[t];
      if (!k.busy) continue;
      const cudaError_t q = cudaEventQuery(k.done);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess && sv->error == FFTBF_OK) sv->error = FFTBF_ECUDA;
      const auto now = Clock::now();
      for (const Frame& f : k.frames) {
        sv->latencies_ms.push_back(std::chrono::duration<double, std::milli>(now - f.t_submit).count());
        sv->done_tickets.push_back(f.ticket);
        sv->free_slots.push_back(f.slot);
        --sv->inflight;
        ++sv->completed;
      }
      k.frames.clear();
      k.busy = false;
      progressed = true;
      sv->cv_done.notify_all();
    }
    if (sv->stop && sv->pending.empty() && sv->staged.empty() && !sv->ticks[0].busy &&
        !sv->ticks[1].busy)
      break;
    if (!progressed) {
      // nothing to do right now: sleep until a submission or a short poll interval
      sv->cv_work.wait_for(lk, std::chrono::microseconds(20));
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
  f.t_submit = Clock::now();
  sv->pending.push_back(f);
  sv->cv_work.notify_one();
  return f.ticket;
}

int fftbf_server_wait(fftbf_server* sv, int64_t ticket, double timeout_s) {
  if (!sv) return set_error(FFTBF_EINVAL, "null server");
  std::unique_lock<std::mutex> lk(sv->mu);
  const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s);
  auto done = [&]() {
    if (sv->error != FFTBF_OK) return true;
    if (ticket < 0) return sv->completed == sv->next_ticket;
    return std::find(sv->done_tickets.begin(), sv->done_tickets.end(), ticket) != sv->done_tickets.end();
  };
  if (!sv->cv_done.wait_until(lk, deadline, done))
    return set_error(FFTBF_ETIMEOUT, "frame %lld not complete within %.3f s", (long long)ticket, timeout_s);
  if (sv->error != FFTBF_OK) return set_error(sv->error, "server stopped after a CUDA error");
  return FFTBF_OK;
}

int fftbf_server_stats(fftbf_server* sv, fftbf_server_stats_t* out) {
  if (!sv || !out) return set_error(FFTBF_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  std::vector<double> l = sv->latencies_ms;
  std::sort(l.begin(), l.end());
  auto pct = [&](double q) {
    if (l.empty()) return 0.0;
    const size_t i = std::min(l.size() - 1, (size_t)(q * (double)(l.size() - 1) + 0.5));
    return l[i];
  };
  out->submitted = sv->next_ticket;
  out->completed = sv->completed;
  out->launches = sv->launches;
  out->frames_per_launch = sv->launches ? (double)sv->frames_launched / (double)sv->launches : 0.0;
  out->peak_inflight = sv->peak_inflight;
  out->slots = (int64_t)sv->slot_events.size();
  out->p50_ms = pct(0.50);
  out->p99_ms = pct(0.99);
  out->max_ms = l.empty() ? 0.0 : l.back();
  double sum = 0.0;
  for (double x : l) sum += x;
  out->mean_ms = l.empty() ? 0.0 : sum / (double)l.size();
  return sv->error;
}

void fftbf_server_destroy(fftbf_server* sv) {
  if (!sv) return;
  if (sv->worker.joinable()) {
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->stop = true;
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

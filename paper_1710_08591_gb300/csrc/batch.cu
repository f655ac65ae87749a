// Batched uneven lattices: many plans (arrays of different sizes) in one persistent
// launch of the FP32 form.
//
// Every (array, window, channel) is a work item. CTAs take items from a global atomic
// counter (costliest arrays first, so the tail is made of cheap items), look up their
// array in a job table held in shared memory and run the transform of that array's shape
// through a compile-time dispatch table of (E-W size, log2 N-S length) variants. A
// variant is the generic Stockham path of the FP32 form (unpack x weight, E-W DFT, padded
// N-S FFT, detect, integrate), processing S snapshots per step; S is picked per array by
// an autotuner that times the candidates on the device when the batch is created. Each
// item's accumulation order depends only on the item, so an array's beams are
// bit-identical alone and in any mix. The launch (counter reset + kernel) is captured in
// a CUDA graph and replayed while the batch's buffers stay the same.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "beam_fp32.cuh"
#include "beam_fp32_warp.cuh"

namespace fftbf {

namespace bt {
constexpr int kMaxJobs = 64;
struct Variant { int mx, log2n; };
// Shapes compiled into the batch kernel: the lattices of the batched workload.
constexpr Variant kVariants[] = {{4, 9}, {8, 7}, {16, 5}, {2, 10}, {1, 11}, {3, 8}};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);
// Warp-per-transform variants of the same shapes (E-W size, N-S length), used when the
// N-S axis is at least 2x zero-padded; ids kNumVariants + index. 2048 beams take a warp
// pair per transform, 32 beams x 16 E-W beams a lane per transform.
struct WarpVariant { int mx, my; };
constexpr WarpVariant kWarpVariants[] = {{4, 512}, {8, 128}, {2, 1024}, {3, 256}, {1, 2048}, {16, 32}};
constexpr int kNumWarpVariants = sizeof(kWarpVariants) / sizeof(kWarpVariants[0]);
}  // namespace bt

// Each warp-path item runs the constant-size instance when its lattice is exactly the
// variant's shape with 2x N-S padding (warp_full), the runtime-size one otherwise.
template <int MX, int R>
__device__ __noinline__ void batch_warp_item(const BeamArgs& a, int64_t item, unsigned char* smem,
                                             bool load_tables) {
  if (warp_full(a, 16 * R))
    warp_item<MX, R, true>(a, item, smem, load_tables);
  else
    warp_item<MX, R>(a, item, smem, load_tables);
}
__device__ __noinline__ void batch_warp2_item(const BeamArgs& a, int64_t item, unsigned char* smem,
                                              bool load_tables) {
  if (warp_full(a, 1024))
    warp2_item<1, true>(a, item, smem, load_tables);
  else
    warp2_item<1>(a, item, smem, load_tables);
}
__device__ __noinline__ void batch_lane16_item(const BeamArgs& a, int64_t item, unsigned char* smem,
                                               bool load_tables) {
  if (warp_full(a, 16))
    lane_item16<true>(a, item, smem, load_tables);
  else
    lane_item16(a, item, smem, load_tables);
}


// One work item of one job: all its snapshots, S per step, bytes double-buffered.
template <int MX, int LOG2N>
__device__ __noinline__ void batch_item(const BeamArgs& a, int64_t item, unsigned char* smem,
                                           bool load_tables) {
  using P = FftPlan<LOG2N>;
  constexpr int N = P::N;
  constexpr int TS = Tstride<N>::v;
  const int nant = a.nx * a.ny;
  const int rawsz = (a.S * nant + 15) & ~15;
  float2* wsm = reinterpret_cast<float2*>(smem + 2 * rawsz);
  float2* exsm = wsm + nant;
  float2* twsm = exsm + MX * a.nx;
  float2* buf = twsm + N;
  const int ntr = a.S * MX;
  const int nsnap = a.n_int * a.npol;
  const int niter = (nsnap + a.S - 1) / a.S;
  const bool vec16 = ((nant & 15) == 0) && ((reinterpret_cast<uintptr_t>(a.volts) & 15) == 0);
  const bool prune = (P::R0 > 1) && (2 * a.nyf <= N);
  if (load_tables) {
    for (int i = threadIdx.x; i < nant; i += kThreads) wsm[i] = a.w[i];
    for (int i = threadIdx.x; i < MX * a.nx; i += kThreads) exsm[i] = a.ex[i];
    for (int i = threadIdx.x; i < N; i += kThreads) twsm[i] = a.tw[i];
  }
  constexpr int NACC = kMaxElems / kThreads;
  float acc[NACC];
#pragma unroll
  for (int i = 0; i < NACC; ++i) acc[i] = 0.f;
  const uint8_t* ivol = item_volts(a, item, nant);
  stage_bytes(a, smem, ivol, 0, nsnap, nant, vec16);
  cp_async_commit();
  for (int it = 0; it < niter; ++it) {
    if (it + 1 < niter) stage_bytes(a, smem + ((it + 1) & 1) * rawsz, ivol, it + 1, nsnap, nant, vec16);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    const uint8_t* raw = smem + (it & 1) * rawsz;
    const int ncol = a.S * a.nyf;
    for (int c = threadIdx.x; c < ncol; c += kThreads) {
      const int s = c / a.nyf;
      const int iyf = c - s * a.nyf;
      float2 z[MX];
#pragma unroll
      for (int A = 0; A < MX; ++A) z[A] = czero();
      if (it * a.S + s < nsnap) {
        const uint8_t* rs = raw + s * nant;
        if constexpr (MX == 1 || MX == 2 || MX == 4 || MX == 8 || MX == 16) {
          if (a.ew_dft) {
#pragma unroll
            for (int ix = 0; ix < MX; ++ix) {
              float2 col = czero();
              for (int iy = iyf; iy < a.ny; iy += N)
                col = cadd(col, cmul(wsm[ix * a.ny + iy], unpack_byte(rs[ix * a.ny + iy])));
              z[ix] = col;
            }
            Dft<MX>::run(z);
          }
        }
        if (!a.ew_dft) {
          for (int ix = 0; ix < a.nx; ++ix) {
            float2 col = czero();
            for (int iy = iyf; iy < a.ny; iy += N)
              col = cadd(col, cmul(wsm[ix * a.ny + iy], unpack_byte(rs[ix * a.ny + iy])));
#pragma unroll
            for (int A = 0; A < MX; ++A) z[A] = cadd(z[A], cmul(exsm[A * a.nx + ix], col));
          }
        }
      }
#pragma unroll
      for (int A = 0; A < MX; ++A) buf[(s * MX + A) * TS + pad16(iyf)] = z[A];
    }
    __syncthreads();
    fft_all<LOG2N>(buf, ntr, a.nyf, prune, twsm, acc);
  }
  // add the S partial sums in a fixed order and write the item's beams once
  __syncthreads();
  float* red = reinterpret_cast<float*>(buf);
  constexpr int RL = P::RL, LRL = P::LRL;
  constexpr int LOG2BPT = LOG2N - LRL;
  const int tot = ntr << LOG2BPT;
#pragma unroll
  for (int e = 0; e < NACC; ++e) {
    const int b = threadIdx.x + (e / RL) * kThreads;
    if (e / RL < kMaxElems / kThreads / RL && b < tot) {
      const int t = b >> LOG2BPT;
      const int j = b & ((1 << LOG2BPT) - 1);
      red[(t << LOG2N) + j + ((e % RL) << LOG2BPT)] = acc[e];
    }
  }
  __syncthreads();
  const int nout = MX * N;
  float* dst = a.beams + item * (int64_t)nout;
  for (int o = threadIdx.x; o < nout; o += kThreads) {
    float sum = 0.f;
    for (int q = 0; q < a.S; ++q) sum += red[q * nout + o];
    dst[o] = sum;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads, 2) batch_kernel(const BatchJob* __restrict__ jobs,
                                                            int njobs, int64_t total,
                                                            unsigned long long* counter) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ BatchJob js[bt::kMaxJobs];
  __shared__ long long s_item;
  __shared__ int s_job;
  for (int i = threadIdx.x; i < njobs; i += kThreads) js[i] = jobs[i];
  int last_job = -1;
  __syncthreads();
  while (true) {
    if (threadIdx.x == 0) {
      const long long g = (long long)atomicAdd(counter, 1ull);
      int j = 0;
      while (j + 1 < njobs && g >= js[j + 1].item0) ++j;
      s_item = g;
      s_job = j;
    }
    __syncthreads();
    const long long g = s_item;
    const int j = s_job;
    __syncthreads();
    if (g >= total) break;
    const BatchJob& J = js[j];
    const int64_t item = g - J.item0;
    const bool load = j != last_job;
    last_job = j;
    switch (J.variant) {
      case 0: batch_item<4, 9>(J.a, item, smem, load); break;
      case 1: batch_item<8, 7>(J.a, item, smem, load); break;
      case 2: batch_item<16, 5>(J.a, item, smem, load); break;
      case 3: batch_item<2, 10>(J.a, item, smem, load); break;
      case 4: batch_item<1, 11>(J.a, item, smem, load); break;
      case 5: batch_item<3, 8>(J.a, item, smem, load); break;
      case bt::kNumVariants + 0: batch_warp_item<4, 16>(J.a, item, smem, load); break;
      case bt::kNumVariants + 1: batch_warp_item<8, 4>(J.a, item, smem, load); break;
      case bt::kNumVariants + 2: batch_warp_item<2, 32>(J.a, item, smem, load); break;
      case bt::kNumVariants + 3: batch_warp_item<3, 8>(J.a, item, smem, load); break;
      case bt::kNumVariants + 4: batch_warp2_item(J.a, item, smem, load); break;
      case bt::kNumVariants + 5: batch_lane16_item(J.a, item, smem, load); break;
      default: break;
    }
  }
}

// Tuned snapshots-per-step per lattice shape, shared by every batch of the process, so a
// plan gets the same tile (and hence bit-identical sums) in any batch.
struct TuneKey {
  int nx, ny, mx, my, npol, n_int;
  bool operator==(const TuneKey& o) const {
    return nx == o.nx && ny == o.ny && mx == o.mx && my == o.my && npol == o.npol && n_int == o.n_int;
  }
};
struct Tuned { int variant, S; };
static std::mutex g_tune_mu;
static std::vector<std::pair<TuneKey, Tuned>> g_tuned;

static int variant_of(int mx, int my) {
  for (int v = 0; v < bt::kNumVariants; ++v)
    if (bt::kVariants[v].mx == mx && (1 << bt::kVariants[v].log2n) == my) return v;
  return -1;
}
// warp variant of a shape (needs the N-S input to fill at most half of the transform)
static int warp_variant_of(int mx, int my, int nyf) {
  for (int v = 0; v < bt::kNumWarpVariants; ++v)
    if (bt::kWarpVariants[v].mx == mx && bt::kWarpVariants[v].my == my && 2 * nyf <= my)
      return bt::kNumVariants + v;
  return -1;
}
static bool is_warp(int variant) { return variant >= bt::kNumVariants; }
// snapshots per step of a warp variant (fixed by its layout)
static int warp_variant_S(int variant) {
  const bt::WarpVariant& w = bt::kWarpVariants[variant - bt::kNumVariants];
  if (w.my == 2048) return 4 / w.mx;
  if (w.my == 32) return kLaneS;
  return wt::kWarps / wt::gcd8(w.mx);
}

static size_t item_smem(const BeamArgs& a, int variant) {
  if (is_warp(variant)) {
    const bt::WarpVariant& w = bt::kWarpVariants[variant - bt::kNumVariants];
    if (w.my == 2048) return warp2_item_smem(a.S, a.mx, a.nx, a.ny);
    if (w.my == 32) return lane_item_smem(a.nx, a.ny);
    return warp_item_smem(a.S, a.mx, a.nx, a.ny, w.my / 32);
  }
  const int nant = a.nx * a.ny;
  const size_t rawsz = ((size_t)a.S * nant + 15) & ~(size_t)15;
  return 2 * rawsz + sizeof(float2) * ((size_t)nant + (size_t)a.mx * a.nx + a.my +
                                       (size_t)a.S * a.mx * (a.my + (a.my >> 4)));
}

int batch_variant(int mx, int my) { return variant_of(mx, my); }

void batch_fill_args(const fftbf_plan* p, BeamArgs& a);

int batch_launch_jobs(const BatchJob* h_jobs, int njobs, BatchJob* d_jobs,
                      unsigned long long* d_counter, size_t smem, int grid, cudaStream_t st) {
  if (njobs < 1 || njobs > bt::kMaxJobs) return set_error(FFTBF_EINVAL, "1..%d jobs per launch", bt::kMaxJobs);
  int64_t total = 0;
  for (int i = 0; i < njobs; ++i) total += h_jobs[i].nitems;
  FFTBF_CUDA_TRY(cudaMemcpyAsync(d_jobs, h_jobs, sizeof(BatchJob) * njobs, cudaMemcpyHostToDevice, st));
  FFTBF_CUDA_TRY(cudaMemsetAsync(d_counter, 0, sizeof(unsigned long long), st));
  const int64_t g = total < grid ? total : grid;
  batch_kernel<<<(unsigned)g, kThreads, smem, st>>>(d_jobs, njobs, total, d_counter);
  FFTBF_CUDA_TRY(cudaGetLastError());
  return FFTBF_OK;
}

size_t batch_item_smem(const BeamArgs& a, int variant) { return item_smem(a, variant); }

}  // namespace fftbf

using namespace fftbf;

struct fftbf_batch {
  int device = 0, nsm = 0;
  std::vector<fftbf_plan*> plans;
  std::vector<int> order;          // job order: costliest items first
  std::vector<int> S;              // tuned snapshots per step, per plan
  std::vector<int> V;              // tuned variant (generic or warp path), per plan
  std::vector<BatchJob> jobs;
  BatchJob* d_jobs = nullptr;
  unsigned long long* d_counter = nullptr;
  size_t smem = 0;
  int grid_per_sm = 2;
  // graph of (counter reset + kernel) for the current job table
  cudaGraphExec_t exec = nullptr;
  cudaStream_t exec_stream = nullptr;
  int64_t exec_T = -1;
  std::vector<const void*> exec_ptrs;
};

static void fill_args(const fftbf_plan* p, BeamArgs& a);
void fftbf::batch_fill_args(const fftbf_plan* p, BeamArgs& a) { fill_args(p, a); }

static void fill_args(const fftbf_plan* p, BeamArgs& a) {
  a = BeamArgs{};
  a.w = p->d_w;
  a.ex = p->d_ex;
  a.tw = p->d_tw;
  a.nx = p->nx; a.ny = p->ny; a.mx = p->mx; a.my = p->my;
  a.npol = p->npol; a.nfreq = p->nfreq; a.n_int = p->n_int;
  a.nyf = std::min(p->ny, p->my);
  a.ew_dft = (p->mx == p->nx) && (p->mx & (p->mx - 1)) == 0 && p->mx <= 16;
  a.real_w = p->real_w ? 1 : 0;
}

static int launch_jobs(fftbf_batch* bb, int64_t total, cudaStream_t st) {
  FFTBF_CUDA_TRY(cudaMemsetAsync(bb->d_counter, 0, sizeof(unsigned long long), st));
  const int64_t grid = std::min<int64_t>(total, (int64_t)bb->nsm * bb->grid_per_sm);
  batch_kernel<<<(unsigned)grid, kThreads, bb->smem, st>>>(bb->d_jobs, (int)bb->jobs.size(),
                                                           total, bb->d_counter);
  FFTBF_CUDA_TRY(cudaGetLastError());
  return FFTBF_OK;
}

// Time one single-job batch launch of plan p with S snapshots per step on `nwin`
// windows of zero bytes (the kernel has no data-dependent control flow).
static float time_candidate(fftbf_batch* bb, const fftbf_plan* p, int variant, int S, int64_t nwin,
                            const uint8_t* dv, float* db, cudaStream_t st) {
  BatchJob J{};
  fill_args(p, J.a);
  J.a.S = S;
  J.a.volts = dv;
  J.a.beams = db;
  J.a.nwin = nwin;
  J.variant = variant;
  J.item0 = 0;
  J.nitems = nwin * p->nfreq;
  if (cudaMemcpyAsync(bb->d_jobs, &J, sizeof(J), cudaMemcpyHostToDevice, st) != cudaSuccess) return 1e30f;
  const size_t need = item_smem(J.a, variant);
  if (need > bb->smem) return 1e30f;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaMemsetAsync(bb->d_counter, 0, sizeof(unsigned long long), st);
    cudaEventRecord(e0, st);
    batch_kernel<<<(unsigned)std::min<int64_t>(J.nitems, (int64_t)bb->nsm * bb->grid_per_sm), kThreads,
                   bb->smem, st>>>(bb->d_jobs, 1, J.nitems, bb->d_counter);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cudaGetLastError() != cudaSuccess) return 1e30f;
  return best;
}

extern "C" {

fftbf_batch* fftbf_batch_create(fftbf_plan* const* plans, int n) {
  NvtxRange nvtx("fftbf_batch_create (autotune)");
  if (!plans || n < 1 || n > bt::kMaxJobs) {
    set_error(FFTBF_EINVAL, "need 1..%d plans", bt::kMaxJobs);
    return nullptr;
  }
  for (int i = 0; i < n; ++i) {
    if (!plans[i]) { set_error(FFTBF_EINVAL, "plan %d is null", i); return nullptr; }
    if (plans[i]->device != plans[0]->device) { set_error(FFTBF_EINVAL, "plans on different devices"); return nullptr; }
    if (variant_of(plans[i]->mx, plans[i]->my) < 0 || plans[i]->ny > plans[i]->my) {
      set_error(FFTBF_EUNSUPPORTED,
                "plan %d (pad_x=%d pad_y=%d, ny=%d): the batch kernel holds the shapes 4x512, "
                "8x128, 16x32, 2x1024, 1x2048, 3x256 with pad_y >= ny", i, plans[i]->mx,
                plans[i]->my, plans[i]->ny);
      return nullptr;
    }
  }
  fftbf_batch* bb = new (std::nothrow) fftbf_batch();
  if (!bb) { set_error(FFTBF_ENOMEM, "cannot allocate batch"); return nullptr; }
  bb->device = plans[0]->device;
  bb->nsm = plans[0]->nsm;
  bb->plans.assign(plans, plans + n);
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(bb->device);
  cudaError_t e = cudaMalloc(&bb->d_jobs, sizeof(BatchJob) * bt::kMaxJobs);
  if (e == cudaSuccess) e = cudaMalloc(&bb->d_counter, sizeof(unsigned long long));
  // shared memory: the largest item footprint over the plans and their S candidates
  bb->smem = 200 * 1024;
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bb->smem);
  cudaStream_t st = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  // ---- autotune S per plan on a small sample
  uint8_t* dv = nullptr;
  float* db = nullptr;
  size_t vbytes = 0, bbytes = 0;
  for (auto* p : bb->plans) {
    vbytes = std::max(vbytes, (size_t)2 * p->n_int * p->nfreq * p->npol * p->nx * p->ny);
    bbytes = std::max(bbytes, (size_t)2 * p->nfreq * p->mx * p->my * sizeof(float));
  }
  if (e == cudaSuccess) e = cudaMalloc(&dv, vbytes);
  if (e == cudaSuccess) e = cudaMalloc(&db, bbytes);
  if (e == cudaSuccess) e = cudaMemset(dv, 0, vbytes);
  size_t max_smem = 0;
  if (e == cudaSuccess) {
    for (auto* p : bb->plans) {
      const TuneKey key{p->nx, p->ny, p->mx, p->my, p->npol, p->n_int};
      // FFTBF_BATCH_PATH=generic|warp restricts the candidates (a test hook; bypasses the
      // process-wide cache)
      const char* force = std::getenv("FFTBF_BATCH_PATH");
      const bool only_generic = force && std::strcmp(force, "generic") == 0;
      const bool only_warp = force && std::strcmp(force, "warp") == 0;
      Tuned best_t{-1, 0};
      if (!force) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        for (auto& kv : g_tuned)
          if (kv.first == key) best_t = kv.second;
      }
      if (best_t.S == 0) {
        // candidates: the generic path at S = 1, 2, 4, ... snapshots per step, and the
        // warp-per-transform path (its S is fixed by the E-W size)
        const int nsnap = p->n_int * p->npol;
        const int gv = variant_of(p->mx, p->my);
        float best = 1e30f;
        best_t = {gv, 1};
        BeamArgs aw;
        fill_args(p, aw);
        const int wv = only_generic ? -1 : warp_variant_of(p->mx, p->my, aw.nyf);
        for (int S = 1; S <= nsnap && S * p->mx * p->my <= kMaxElems && !(only_warp && wv >= 0); S *= 2) {
          BeamArgs a;
          fill_args(p, a);
          a.S = S;
          if (item_smem(a, gv) > bb->smem) break;
          const float ms = time_candidate(bb, p, gv, S, 2, dv, db, st);
          if (ms < best) { best = ms; best_t = {gv, S}; }
        }
        if (wv >= 0) {
          aw.S = warp_variant_S(wv);
          if (item_smem(aw, wv) <= bb->smem) {
            const float ms = time_candidate(bb, p, wv, aw.S, 2, dv, db, st);
            if (ms < best || only_warp) { best = ms; best_t = {wv, aw.S}; }
          }
        }
        if (!force) {
          std::lock_guard<std::mutex> lock(g_tune_mu);
          g_tuned.push_back({key, best_t});
        }
      }
      bb->S.push_back(best_t.S);
      bb->V.push_back(best_t.variant);
      BeamArgs a;
      fill_args(p, a);
      a.S = best_t.S;
      max_smem = std::max(max_smem, item_smem(a, best_t.variant));
    }
    e = cudaGetLastError();
  }
  cudaFree(dv);
  cudaFree(db);
  if (st) cudaStreamDestroy(st);
  if (e != cudaSuccess) {
    cuda_error(e, "fftbf_batch_create");
    fftbf_batch_destroy(bb);
    cudaSetDevice(prev);
    return nullptr;
  }
  bb->smem = std::max<size_t>(max_smem, 16);
  cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bb->smem);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel, kThreads, bb->smem);
  bb->grid_per_sm = std::max(1, per_sm);
  // costliest items first: snapshots per item x transform work per snapshot
  bb->order.resize(n);
  for (int i = 0; i < n; ++i) bb->order[i] = i;
  auto cost = [&](int i) {
    const fftbf_plan* p = bb->plans[i];
    return (double)p->n_int * p->npol * p->mx * p->my * std::log2((double)p->my + 1.0);
  };
  std::stable_sort(bb->order.begin(), bb->order.end(), [&](int x, int y) { return cost(x) > cost(y); });
  cudaSetDevice(prev);
  return bb;
}

int fftbf_batch_execute(fftbf_batch* bb, const uint8_t* const* volts_dev, int64_t T,
                        float* const* beams_dev, void* stream) {
  NvtxRange nvtx("fftbf_batch_execute");
  if (!bb) return set_error(FFTBF_EINVAL, "null batch");
  if (!volts_dev || !beams_dev) return set_error(FFTBF_EINVAL, "null pointer array");
  const int n = (int)bb->plans.size();
  for (int i = 0; i < n; ++i) {
    if (T < 0 || T % bb->plans[i]->n_int != 0)
      return set_error(FFTBF_EINVAL, "T = %lld is not a multiple of plan %d's n_int = %d",
                       (long long)T, i, bb->plans[i]->n_int);
    if (T > 0 && (!volts_dev[i] || !beams_dev[i])) return set_error(FFTBF_EINVAL, "null buffer of plan %d", i);
  }
  if (T == 0) return FFTBF_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != bb->device) cudaSetDevice(bb->device);
  struct Restore { int d; ~Restore() { cudaSetDevice(d); } } restore{prev};
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  std::vector<BatchJob> jobs(n);
  std::vector<const void*> ptrs;
  int64_t total = 0;
  for (int k = 0; k < n; ++k) {
    const int i = bb->order[k];
    BatchJob& J = jobs[k];
    fill_args(bb->plans[i], J.a);
    J.a.S = bb->S[i];
    J.a.volts = volts_dev[i];
    J.a.beams = beams_dev[i];
    J.a.nwin = T / bb->plans[i]->n_int;
    J.variant = bb->V[i];
    J.nitems = J.a.nwin * bb->plans[i]->nfreq;
    J.item0 = total;
    total += J.nitems;
    ptrs.push_back(volts_dev[i]);
    ptrs.push_back(beams_dev[i]);
  }
  if (st == nullptr) {
    // the legacy default stream cannot be captured: upload the table and launch directly
    if (bb->exec) { cudaGraphExecDestroy(bb->exec); bb->exec = nullptr; }
    bb->jobs = jobs;
    FFTBF_CUDA_TRY(cudaMemcpyAsync(bb->d_jobs, bb->jobs.data(), sizeof(BatchJob) * n,
                                   cudaMemcpyHostToDevice, st));
    return launch_jobs(bb, total, st);
  }
  const bool same = bb->exec && bb->exec_stream == st && bb->exec_T == T && bb->exec_ptrs == ptrs;
  if (!same) {
    // new job table: upload it and capture (counter reset + kernel) as a graph
    if (bb->exec) { cudaGraphExecDestroy(bb->exec); bb->exec = nullptr; }
    bb->jobs = jobs;
    FFTBF_CUDA_TRY(cudaMemcpyAsync(bb->d_jobs, bb->jobs.data(), sizeof(BatchJob) * n,
                                   cudaMemcpyHostToDevice, st));
    cudaGraph_t g = nullptr;
    FFTBF_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const int rc = launch_jobs(bb, total, st);
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (rc != FFTBF_OK) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return cuda_error(e, "batch graph capture");
    e = cudaGraphInstantiate(&bb->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { bb->exec = nullptr; return cuda_error(e, "batch graph instantiate"); }
    bb->exec_stream = st;
    bb->exec_T = T;
    bb->exec_ptrs = ptrs;
  }
  FFTBF_CUDA_TRY(cudaGraphLaunch(bb->exec, st));
  return FFTBF_OK;
}

int fftbf_batch_grid(const fftbf_batch* bb) { return bb->nsm * bb->grid_per_sm; }
size_t fftbf_batch_smem(const fftbf_batch* bb) { return bb->smem; }

int fftbf_batch_tuned_steps(const fftbf_batch* bb, int i) {
  if (!bb || i < 0 || i >= (int)bb->plans.size()) return set_error(FFTBF_EINVAL, "bad batch index");
  return bb->S[i];
}

int fftbf_batch_tuned_variant(const fftbf_batch* bb, int i) {
  if (!bb || i < 0 || i >= (int)bb->plans.size()) return set_error(FFTBF_EINVAL, "bad batch index");
  return bb->V[i];
}

void fftbf_batch_destroy(fftbf_batch* bb) {
  if (!bb) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(bb->device);
  if (bb->exec_stream) cudaStreamSynchronize(bb->exec_stream);
  if (bb->exec) cudaGraphExecDestroy(bb->exec);
  cudaFree(bb->d_jobs);
  cudaFree(bb->d_counter);
  cudaSetDevice(prev);
  delete bb;
}

}  // extern "C"

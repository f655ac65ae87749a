// Tied-array beams on the tensor cores (Eq. bp_max_arbitrary as a GEMM) when the E-W axis
// is on the FFT-beam grid (pad_x < 2 nx - 1, at most 4 E-W beams): per channel f,
//   out[j, s] = sum_B wx[s, A_s] wy[s, B] P[j, f, A_s, B],
// a [pointings x beams] x [beams x windows] product for each E-W beam A. Operands are
// split FP16 pairs, x = 2^-e (hi + lo) with hi = fp16(2^e x), lo = fp16(2^e x - hi), and
// each K step accumulates hi*hi + hi*lo + lo*hi in FP32 (tcgen05.mma kind::f16, TMEM), which
// keeps FP32 accuracy; e scales every weight row and every beam row so that its largest
// magnitude lies in [2^14, 2^15) (inside the FP16 range, with the residuals normal), and the
// epilogue divides by 2^(e_s + e_j) exactly. Both split operands are stored in global
// memory already cut into 16 KB tiles (128 rows x 64 beams, the canonical K-major layout,
// zero rows past the ends). A CTA computes 128 pointings x 128 windows of one channel: one
// thread stages each K chunk as four bulk copies completing on a full-mbarrier (three
// stages), issues its MMAs and commits them to the stage's empty-mbarrier; one TMEM
// accumulator of 128 columns per E-W beam used by the tile's pointings, and each pointing
// (TMEM lane) reads its own beam's accumulator. Every wait is bounded; a timeout sets the
// plan's error word.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>

#include "internal.cuh"
#include "tc_ptx.cuh"

namespace fftbf {

namespace ttc {
constexpr int TM = 128, TN = 128, KC = 64;     // pointings, windows, beams per K chunk
constexpr int LBO = 128, SBO = 1024;           // canonical K-major tile: 8 K blocks per row group
constexpr int TILE = TM * KC * 2;              // bytes of one 128 x 64 FP16 tile
constexpr int STAGE = 4 * TILE;                // W hi, W lo, P hi, P lo
constexpr int NT = 256;                        // warps w and w + 4 share TMEM lane quarter w % 4
constexpr int NS = 3;                          // staging buffers
constexpr int MAXA = 4;                        // E-W beams (one accumulator each)
constexpr uint32_t TMEM_COLS = 512;
constexpr uint64_t WAIT_NS = 1000000000ull;
}  // namespace ttc

// e such that 2^e m lies in [2^14, 2^15) (0 for a zero row)
__device__ __forceinline__ int split_exp(float m) { return m > 0.f ? 14 - ilogbf(m) : 0; }

// Half offset of element (row r < 128, k) of a row tile: tile (k / 64) of the row tile's
// chunks, canonical K-major layout inside.
__device__ __forceinline__ int64_t tiled_off(int64_t tile0, int r, int k) {
  return (tile0 + (k >> 6)) * (ttc::TILE / 2) +
         (int64_t)(tc::kmajor_off(r, k & 63, ttc::LBO, ttc::SBO) >> 1);
}

// Split one row x (one warp): hi and lo written at tiled_off(tile0, r, k), the row exponent
// returned; a null x writes a zero row.
__device__ __forceinline__ int split_row_tiled(const float* x, float scale_in, int n, __half* hi,
                                               __half* lo, int64_t tile0, int r, int lane) {
  float m = 0.f;
  if (x)
    for (int b = lane; b < n; b += 32) m = fmaxf(m, fabsf(scale_in * x[b]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  const int e = split_exp(m);
  for (int b = lane; b < n; b += 32) {
    const float v = x ? ldexpf(scale_in * x[b], e) : 0.f;
    const __half h = __float2half_rn(v);
    const int64_t o = tiled_off(tile0, r, b);
    hi[o] = h;
    lo[o] = __float2half_rn(v - __half2float(h));
  }
  return e;
}

// Weight tables in tiles: per channel, pointing tiles of 128 sorted slots (zero rows past
// n_tied), each [my / 64] chunks of 128 x 64. Also the row's E-W beam A_s (the largest
// |wx|) and exponent; the row is wx[s, A_s] wy[s, :].
__global__ void tied_tc_table_kernel(const float* __restrict__ wx, const float* __restrict__ wy,
                                     int nfreq, int n_tied, int mx, int my, __half* wyh,
                                     __half* wyl, int* wye, int* wa) {
  const int lane = threadIdx.x & 31;
  const int nts = (n_tied + ttc::TM - 1) / ttc::TM, kcs = my / ttc::KC;
  const int64_t nrows = (int64_t)nfreq * nts * ttc::TM;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t rp = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); rp < nrows; rp += nw) {
    const int f = (int)(rp / ((int64_t)nts * ttc::TM));
    const int slot = (int)(rp - (int64_t)f * nts * ttc::TM);
    const int64_t tile0 = ((int64_t)f * nts + (slot >> 7)) * kcs;
    if (slot >= n_tied) {
      split_row_tiled(nullptr, 0.f, my, wyh, wyl, tile0, slot & 127, lane);
      continue;
    }
    const int64_t r = (int64_t)f * n_tied + slot;
    int A = 0;
    float best = -1.f;
    for (int a = 0; a < mx; ++a) {
      const float v = fabsf(wx[r * mx + a]);
      if (v > best) { best = v; A = a; }
    }
    const int e = split_row_tiled(wy + r * my, wx[r * mx + A], my, wyh, wyl, tile0, slot & 127, lane);
    if (lane == 0) {
      wye[r] = e;
      wa[r] = A;
    }
  }
}

// Beam rows P[j, f, A, :] split the same way (per call), in tiles per (channel, E-W beam) of
// 128 windows (zero rows past nwin); exponents at pe[(j nfreq + f) mx + A].
__global__ void tied_tc_prep_kernel(const float* __restrict__ P, int64_t nwin, int nfreq, int mx,
                                    int my, __half* ph, __half* pl, int* pe) {
  const int lane = threadIdx.x & 31;
  const int ntj = (int)((nwin + ttc::TN - 1) / ttc::TN), kcs = my / ttc::KC;
  const int64_t per_fa = (int64_t)ntj * ttc::TN;
  const int64_t nrows = (int64_t)nfreq * mx * per_fa;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t rp = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); rp < nrows; rp += nw) {
    const int64_t fa = rp / per_fa;                 // f mx + A
    const int64_t j = rp - fa * per_fa;
    const int f = (int)(fa / mx), A = (int)(fa - (int64_t)f * mx);
    const int64_t tile0 = (fa * ntj + (j >> 7)) * kcs;
    const float* x = j < nwin ? P + ((j * nfreq + f) * mx + A) * my : nullptr;
    const int e = split_row_tiled(x, 1.f, my, ph, pl, tile0, (int)(j & 127), lane);
    if (x && lane == 0) pe[(j * nfreq + f) * mx + A] = e;
  }
}

__global__ void __launch_bounds__(ttc::NT, 1) tied_tc_kernel(
    const __half* __restrict__ wyh, const __half* __restrict__ wyl, const int* __restrict__ wye,
    const int* __restrict__ wa, const int* __restrict__ perm, const __half* __restrict__ ph,
    const __half* __restrict__ pl, const int* __restrict__ pe, float* __restrict__ out,
    int64_t nwin, int nfreq, int n_tied, int mx, int my, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_t[];
  __shared__ uint64_t full[ttc::NS], empty[ttc::NS];
  __shared__ uint32_t taddr;
  __shared__ int s_mask;
  __shared__ int s_pe[ttc::MAXA][ttc::TN];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int f = blockIdx.z;
  const int s0 = blockIdx.x * ttc::TM;
  const int64_t j0 = (int64_t)blockIdx.y * ttc::TN;
  const int64_t fs0 = (int64_t)f * n_tied;
  if (warp == 0) {
    tc::tmem_alloc(&taddr, ttc::TMEM_COLS);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    for (int i = 0; i < ttc::NS; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&empty[i], 1);
    }
    tc::mbar_init_fence();
    s_mask = 0;
  }
  __syncthreads();
  const int row = tid & (ttc::TM - 1);           // TMEM lane / pointing of this thread
  const int s = s0 + row;
  const bool srow = s < n_tied;
  const int my_a = srow ? wa[fs0 + s] : 0;
  const int my_e = srow ? wye[fs0 + s] : 0;
  if (srow && tid < ttc::TM) atomicOr(&s_mask, 1 << my_a);
  __syncthreads();
  const int mask = s_mask;
  int nact = 0, my_ai = 0;
  for (int A = 0; A < mx; ++A)
    if ((mask >> A) & 1) {
      if (A == my_a) my_ai = nact;
      ++nact;
    }
  // exponents of the tile's windows, per E-W beam in use
  for (int i = tid; i < nact * ttc::TN; i += ttc::NT) {
    const int ai = i / ttc::TN, jj = i - ai * ttc::TN;
    int A = 0;
    for (int a = 0, c = -1; a < mx; ++a)
      if ((mask >> a) & 1 && ++c == ai) A = a;
    const int64_t j = j0 + jj;
    s_pe[ai][jj] = j < nwin ? pe[(j * nfreq + f) * mx + A] : 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = taddr;
  const int kcs = my / ttc::KC;
  const int total = nact * kcs;
  const uint32_t idesc = tc::idesc_f16(ttc::TM, ttc::TN, false);
  // Thread 0 runs the pipeline: chunk t = (E-W beam in use number t / kcs, K chunk t % kcs)
  // goes to stage t % NS as four 16 KB bulk copies completing on full[stage]; its MMAs
  // commit to empty[stage], after which the stage takes chunk t + NS. The other threads wait
  // at the CTA barrier. Every wait is bounded.
  __shared__ int s_ok;
  if (tid == 0) {
    bool ok = true;
    const int nts = (n_tied + ttc::TM - 1) / ttc::TM;
    const int ntj = (int)((nwin + ttc::TN - 1) / ttc::TN);
    const int64_t wt0 = ((int64_t)f * nts + blockIdx.x) * kcs;   // first weight tile
    auto issue = [&](int t) {
      const int st = t % ttc::NS;
      unsigned char* stg = smem_t + st * ttc::STAGE;
      const int ai = t / kcs, kc = t - ai * kcs;
      int A = 0;
      for (int a = 0, c = -1; a < mx; ++a)
        if ((mask >> a) & 1 && ++c == ai) A = a;
      const int64_t pt = (((int64_t)f * mx + A) * ntj + blockIdx.y) * kcs + kc;
      const int64_t wt = wt0 + kc;
      tc::mbar_arrive_expect_tx(&full[st], (uint32_t)ttc::STAGE);
      tc::bulk_g2s(stg, wyh + wt * (ttc::TILE / 2), ttc::TILE, &full[st]);
      tc::bulk_g2s(stg + ttc::TILE, wyl + wt * (ttc::TILE / 2), ttc::TILE, &full[st]);
      tc::bulk_g2s(stg + 2 * ttc::TILE, ph + pt * (ttc::TILE / 2), ttc::TILE, &full[st]);
      tc::bulk_g2s(stg + 3 * ttc::TILE, pl + pt * (ttc::TILE / 2), ttc::TILE, &full[st]);
    };
    for (int t = 0; t < ttc::NS && t < total; ++t) issue(t);
    for (int t = 0; t < total && ok; ++t) {
      const int st = t % ttc::NS;
      const uint32_t par = (uint32_t)((t / ttc::NS) & 1);
      ok = tc::mbar_wait(&full[st], par, ttc::WAIT_NS);
      if (!ok) break;
      tc::fence_after_sync();
      const uint32_t sa = tc::smem_u32(smem_t + st * ttc::STAGE);
      const uint32_t d = tbase + (uint32_t)((t / kcs) * ttc::TN);
      const int kc = t % kcs;
#pragma unroll
      for (int ks = 0; ks < ttc::KC / 16; ++ks) {
        const uint32_t ko = (uint32_t)(ks * 2 * ttc::LBO);
        const uint64_t dwh = tc::smem_desc(sa + ko, ttc::LBO, ttc::SBO);
        const uint64_t dwl = tc::smem_desc(sa + ttc::TILE + ko, ttc::LBO, ttc::SBO);
        const uint64_t dph = tc::smem_desc(sa + 2 * ttc::TILE + ko, ttc::LBO, ttc::SBO);
        const uint64_t dpl = tc::smem_desc(sa + 3 * ttc::TILE + ko, ttc::LBO, ttc::SBO);
        tc::mma_f16(d, dwh, dph, idesc, (kc > 0 || ks > 0) ? 1u : 0u);
        tc::mma_f16(d, dwh, dpl, idesc, 1u);
        tc::mma_f16(d, dwl, dph, idesc, 1u);
      }
      tc::mma_commit(&empty[st]);
      // refill the stage of chunk t - 1 once its MMAs are done
      const int tp = t - 1;
      if (tp >= 0 && tp + ttc::NS < total) {
        ok = tc::mbar_wait(&empty[tp % ttc::NS], (uint32_t)((tp / ttc::NS) & 1), ttc::WAIT_NS);
        if (ok) issue(tp + ttc::NS);
      }
    }
    if (ok && total > 0) {                          // the last commit covers every MMA
      const int tl = total - 1;
      ok = tc::mbar_wait(&empty[tl % ttc::NS], (uint32_t)((tl / ttc::NS) & 1), ttc::WAIT_NS);
    }
    s_ok = ok ? 1 : 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  const bool ok = s_ok != 0;
  tc::fence_after_sync();
  if (ok && total > 0) {
    // warp w reads TMEM lanes 32 (w % 4) .. + 31 (its pointings) and windows 64 (w / 4) .. + 63
    const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
    const int dst_s = srow ? perm[fs0 + s] : 0;
    for (int c = 2 * (warp >> 2); c < 2 * (warp >> 2) + 2; ++c) {
      for (int a2 = 0; a2 < nact; ++a2) {
        uint32_t r[32];
        tc::tmem_ld32(tbase + lane_off + (uint32_t)(a2 * ttc::TN + 32 * c), r);
        tc::tmem_wait_ld();
        if (a2 == my_ai && srow) {
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            const int64_t j = j0 + 32 * c + q;
            if (j < nwin) {
              // D 2^-E: a power-of-two product (exact) while 2^-E is a normal float
              const int E = my_e + s_pe[a2][32 * c + q];
              const float d = __uint_as_float(r[q]);
              out[(j * nfreq + f) * (int64_t)n_tied + dst_s] =
                  (E > -127 && E < 127) ? d * __int_as_float((127 - E) << 23) : ldexpf(d, -E);
            }
          }
        }
      }
    }
  } else if (!ok && tid == 0) {
    atomicExch(err, FFTBF_ETIMEOUT);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, ttc::TMEM_COLS);
}

// ------------------------------------------------------------------------------ host --
bool tied_tc_eligible(bool dense_x, int mx, int my) {
  const char* env = getenv("FFTBF_TIED_TC");
  if (env && env[0] == '0') return false;
  return !dense_x && mx <= ttc::MAXA && my >= ttc::KC && my % ttc::KC == 0;
}

int tied_tc_build(TiedTables& tt, int64_t nuv, int mx, int my, cudaStream_t st) {
  cudaFree(tt.wyh);
  cudaFree(tt.wyl);
  cudaFree(tt.wye);
  cudaFree(tt.wa);
  tt.wyh = tt.wyl = nullptr;
  tt.wye = tt.wa = nullptr;
  const int n_tied = tt.tc_n_tied;
  const int nfreq = (int)(nuv / n_tied);
  const int64_t nts = (n_tied + ttc::TM - 1) / ttc::TM;
  const size_t halves = (size_t)nfreq * nts * ttc::TM * my;      // padded to whole tiles
  // test hook: FFTBF_TEST_TIED_TC_NOMEM=1 makes the split tables look unallocatable, so
  // that the fallback to the CUDA-core GEMM can be exercised without exhausting the device
  const char* nomem = getenv("FFTBF_TEST_TIED_TC_NOMEM");
  if (nomem && nomem[0] == '1') return set_error(FFTBF_ENOMEM, "split tied-beam tables (test hook)");
  bool ok = cudaMalloc(&tt.wyh, halves * sizeof(__half)) == cudaSuccess &&
            cudaMalloc(&tt.wyl, halves * sizeof(__half)) == cudaSuccess &&
            cudaMalloc(&tt.wye, nuv * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&tt.wa, nuv * sizeof(int)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    cudaFree(tt.wyh);
    cudaFree(tt.wyl);
    cudaFree(tt.wye);
    cudaFree(tt.wa);
    tt.wyh = tt.wyl = nullptr;
    tt.wye = tt.wa = nullptr;
    return set_error(FFTBF_ENOMEM, "cannot allocate the split tied-beam tables");
  }
  const int64_t rows = (int64_t)nfreq * nts * ttc::TM;
  const unsigned blocks = (unsigned)std::min<int64_t>((rows + 7) / 8, 1 << 20);
  tied_tc_table_kernel<<<blocks, 256, 0, st>>>(tt.wx, tt.wy, nfreq, n_tied, mx, my,
                                               reinterpret_cast<__half*>(tt.wyh),
                                               reinterpret_cast<__half*>(tt.wyl), tt.wye, tt.wa);
  FFTBF_CUDA_TRY(cudaGetLastError());
  tt.tc = 1;
  return FFTBF_OK;
}

int tied_tc_launch(TiedTables& tt, const float* beams, int64_t nwin, int nfreq, int mx, int my,
                   float* out, cudaStream_t st) {
  const int64_t ntj = (nwin + ttc::TN - 1) / ttc::TN;
  if (ntj > 65535 || nfreq > 65535)
    return set_error(FFTBF_EUNSUPPORTED, "tied beams: too many windows or channels per call");
  const int64_t prow = (int64_t)nfreq * mx * ntj * ttc::TN;        // padded beam rows
  const int64_t erow = nwin * nfreq * mx;                           // exponents
  if ((size_t)prow > tt.p_cap) {
    cudaStreamSynchronize(st);                  // the old scratch may still be read
    cudaFree(tt.ph);
    cudaFree(tt.pl);
    cudaFree(tt.pe);
    tt.ph = tt.pl = nullptr;
    tt.pe = nullptr;
    tt.p_cap = 0;
    bool ok = cudaMalloc(&tt.ph, prow * my * sizeof(__half)) == cudaSuccess &&
              cudaMalloc(&tt.pl, prow * my * sizeof(__half)) == cudaSuccess &&
              cudaMalloc(&tt.pe, std::max<int64_t>(erow, prow) * sizeof(int)) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      cudaFree(tt.ph);
      cudaFree(tt.pl);
      cudaFree(tt.pe);
      tt.ph = tt.pl = nullptr;
      tt.pe = nullptr;
      return set_error(FFTBF_ENOMEM, "cannot allocate the split beam scratch");
    }
    tt.p_cap = (size_t)prow;
  }
  const unsigned pblocks = (unsigned)std::min<int64_t>((prow + 7) / 8, 1 << 20);
  tied_tc_prep_kernel<<<pblocks, 256, 0, st>>>(beams, nwin, nfreq, mx, my,
                                               reinterpret_cast<__half*>(tt.ph),
                                               reinterpret_cast<__half*>(tt.pl), tt.pe);
  FFTBF_CUDA_TRY(cudaGetLastError());
  const size_t smem = ttc::NS * (size_t)ttc::STAGE;
  FFTBF_CUDA_TRY(cudaFuncSetAttribute(tied_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
  dim3 grid((tt.n_tied + ttc::TM - 1) / ttc::TM, (unsigned)ntj, nfreq);
  tied_tc_kernel<<<grid, ttc::NT, smem, st>>>(
      reinterpret_cast<const __half*>(tt.wyh), reinterpret_cast<const __half*>(tt.wyl), tt.wye,
      tt.wa, tt.perm, reinterpret_cast<const __half*>(tt.ph), reinterpret_cast<const __half*>(tt.pl),
      tt.pe, out, nwin, nfreq, tt.n_tied, mx, my, tt.err);
  FFTBF_CUDA_TRY(cudaGetLastError());
  return FFTBF_OK;
}

}  // namespace fftbf

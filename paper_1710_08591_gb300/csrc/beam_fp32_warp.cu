// Standalone launches of the warp-per-transform FP32 path (beam_fp32_warp.cuh) for
// fftbf_execute: E-W sizes 1, 2, 3, 4, 8 x N-S lengths 128, 256, 512, 1024.
#include <cuda_runtime.h>

#include "beam_fp32_warp.cuh"

namespace fftbf {

template <int MX, int R, bool FULL>
__global__ void __launch_bounds__(kThreads, 2) beams_fp32_warp_kernel(const BeamArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int64_t nitems = a.nwin * a.nfreq;
  bool load = true;
  for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
    warp_item<MX, R, FULL>(a, item, smem, load);
    load = false;
  }
}

template <int MX, int R>
static int launch_warp(const BeamArgs& a0, int nsm, cudaStream_t st) {
  BeamArgs a = a0;
  a.S = WarpCfg<MX, R>::S;
  const size_t smem = warp_item_smem(a.S, a.mx, a.nx, a.ny, R);
  auto kern = warp_full(a, 16 * R) ? beams_fp32_warp_kernel<MX, R, true>
                                    : beams_fp32_warp_kernel<MX, R, false>;
  FFTBF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  FFTBF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      cudaSharedmemCarveoutMaxShared));
  int per_sm = 0;
  FFTBF_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
  if (per_sm < 1) return set_error(FFTBF_EUNSUPPORTED, "warp FFT kernel does not fit on an SM");
  const int64_t items = a.nwin * a.nfreq;
  const int64_t grid = items < (int64_t)nsm * per_sm ? items : (int64_t)nsm * per_sm;
  kern<<<(unsigned)grid, kThreads, smem, st>>>(a);
  FFTBF_CUDA_TRY(cudaGetLastError());
  return FFTBF_OK;
}

template <int MX, bool FULL>
__global__ void __launch_bounds__(kThreads, 2) beams_fp32_warp2_kernel(const BeamArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int64_t nitems = a.nwin * a.nfreq;
  bool load = true;
  for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
    warp2_item<MX, FULL>(a, item, smem, load);
    load = false;
  }
}

template <bool FULL>
__global__ void __launch_bounds__(kThreads, 2) beams_fp32_lane16_kernel(const BeamArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int64_t nitems = a.nwin * a.nfreq;
  bool load = true;
  for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
    lane_item16<FULL>(a, item, smem, load);
    load = false;
  }
}

template <typename K>
static int launch_item_kernel(K kern, const BeamArgs& a, size_t smem, int nsm, cudaStream_t st) {
  FFTBF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  FFTBF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      cudaSharedmemCarveoutMaxShared));
  int per_sm = 0;
  FFTBF_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
  if (per_sm < 1) return set_error(FFTBF_EUNSUPPORTED, "FFT kernel does not fit on an SM");
  const int64_t items = a.nwin * a.nfreq;
  const int64_t grid = items < (int64_t)nsm * per_sm ? items : (int64_t)nsm * per_sm;
  kern<<<(unsigned)grid, kThreads, smem, st>>>(a);
  FFTBF_CUDA_TRY(cudaGetLastError());
  return FFTBF_OK;
}

static int warp_r(int my) {
  switch (my) {
    case 128: return 4;
    case 256: return 8;
    case 512: return 16;
    case 1024: return 32;
    default: return 0;
  }
}

bool fp32_warp_supported(const BeamArgs& a) {
  if (a.my == 2048)
    return (a.mx == 1 || a.mx == 2) && 2 * a.nyf <= a.my &&
           warp2_item_smem(4 / a.mx, a.mx, a.nx, a.ny) <= 112 * 1024;
  if (a.my == 32) return a.mx == 16 && a.nyf <= 16 && lane_item_smem(a.nx, a.ny) <= 112 * 1024;
  const int R = warp_r(a.my);
  // E-W size 3 keeps three transforms per warp: its accumulators fit up to 256 beams
  const bool mx_ok = a.mx == 1 || a.mx == 2 || (a.mx == 3 && R <= 8) || a.mx == 4 || a.mx == 8;
  if (!R || !mx_ok || 2 * a.nyf > a.my) return false;
  const int S = wt::kWarps / wt::gcd8(a.mx);
  return warp_item_smem(S, a.mx, a.nx, a.ny, R) <= 112 * 1024;
}

template <int MX>
static int launch_warp_mx(const BeamArgs& a, int nsm, cudaStream_t st) {
  switch (warp_r(a.my)) {
    case 4: return launch_warp<MX, 4>(a, nsm, st);
    case 8: return launch_warp<MX, 8>(a, nsm, st);
    case 16: if constexpr (MX != 3) return launch_warp<MX, 16>(a, nsm, st); break;
    case 32: if constexpr (MX != 3) return launch_warp<MX, 32>(a, nsm, st); break;
    default: break;
  }
  return set_error(FFTBF_EUNSUPPORTED, "warp FFT kernel: E-W %d x N-S %d", a.mx, a.my);
}

int launch_beams_fp32_warp(const BeamArgs& a0, int nsm, cudaStream_t st) {
  if (a0.my == 2048) {
    BeamArgs a = a0;
    a.S = 4 / a.mx;
    const size_t smem = warp2_item_smem(a.S, a.mx, a.nx, a.ny);
    const bool full = warp_full(a, 1024);
    if (a.mx == 1)
      return launch_item_kernel(full ? beams_fp32_warp2_kernel<1, true> : beams_fp32_warp2_kernel<1, false>,
                                a, smem, nsm, st);
    return launch_item_kernel(full ? beams_fp32_warp2_kernel<2, true> : beams_fp32_warp2_kernel<2, false>,
                              a, smem, nsm, st);
  }
  if (a0.my == 32) {
    BeamArgs a = a0;
    a.S = kLaneS;
    return launch_item_kernel(warp_full(a, 16) ? beams_fp32_lane16_kernel<true>
                                               : beams_fp32_lane16_kernel<false>,
                              a, lane_item_smem(a.nx, a.ny), nsm, st);
  }
  const BeamArgs& a = a0;
  switch (a.mx) {
    case 1: return launch_warp_mx<1>(a, nsm, st);
    case 2: return launch_warp_mx<2>(a, nsm, st);
    case 3: return launch_warp_mx<3>(a, nsm, st);
    case 4: return launch_warp_mx<4>(a, nsm, st);
    case 8: return launch_warp_mx<8>(a, nsm, st);
    default: return set_error(FFTBF_EUNSUPPORTED, "warp FFT kernel: E-W size %d", a.mx);
  }
}

}  // namespace fftbf

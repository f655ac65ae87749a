// FP32 throughput probe: the measured FP32 peak that the FP32 form's roofline is judged
// against, for scalar FFMA and for the packed two-lane FFMA2 (fma.rn.f32x2) of sm_100 and
// later. Each thread runs NCHAIN independent multiply-add chains (enough to cover the FMA
// latency at full occupancy) for `iters` steps; the result is folded into one store per
// thread so that nothing is dead code. 2 flops per FMA, 4 per FFMA2.
#include <cuda_runtime.h>

#include "internal.cuh"

namespace fftbf {
namespace {

constexpr int NCHAIN = 8;

__global__ void __launch_bounds__(256) ffma_probe_kernel(int64_t iters, float b, float c, float* out) {
  float a[NCHAIN];
#pragma unroll
  for (int k = 0; k < NCHAIN; ++k) a[k] = (float)(threadIdx.x + k);
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < NCHAIN; ++k) a[k] = fmaf(a[k], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < NCHAIN; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) ffma2_probe_kernel(int64_t iters, float b, float c, float* out) {
  float2 a[NCHAIN];
  const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
#pragma unroll
  for (int k = 0; k < NCHAIN; ++k) a[k] = make_float2((float)(threadIdx.x + k), (float)(k - (int)threadIdx.x));
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < NCHAIN; ++k) a[k] = __ffma2_rn(a[k], b2, c2);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < NCHAIN; ++k) s += a[k].x + a[k].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace fftbf

using namespace fftbf;

extern "C" int fftbf_probe_fp32(int packed, int64_t iters, int blocks, float* out_dev,
                                double* flops_out, void* stream) {
  if (iters < 1 || blocks < 1 || !out_dev || !flops_out)
    return set_error(FFTBF_EINVAL, "probe: iters and blocks >= 1, non-null pointers");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // b slightly below 1 and c small keep every chain finite for any iteration count
  if (packed)
    ffma2_probe_kernel<<<blocks, 256, 0, st>>>(iters, 0.999999f, 1e-3f, out_dev);
  else
    ffma_probe_kernel<<<blocks, 256, 0, st>>>(iters, 0.999999f, 1e-3f, out_dev);
  FFTBF_CUDA_TRY(cudaGetLastError());
  *flops_out = (double)blocks * 256.0 * (double)iters * NCHAIN * (packed ? 4.0 : 2.0);
  return FFTBF_OK;
}

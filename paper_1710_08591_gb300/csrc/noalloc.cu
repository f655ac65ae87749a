// fftbf_execute_noalloc: the FP32 beam pass for callers that cannot allocate device
// memory. The plan tables live in a statically reserved device array instead of
// cudaMalloc'd buffers; the transform kernels are the ones fftbf_execute launches.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.cuh"

namespace fftbf {
namespace {

// Table space for one call: E-W DFT matrix, N-S twiddles and (optionally) unit weights.
static __device__ __align__(256) unsigned char g_noalloc_scratch[FFTBF_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_dev[kMaxDevices];   // device address of g_noalloc_scratch, per device

// Device address of the array on the current device `dev`. In host code the symbol
// name is only a host-side handle, so the address must be looked up (once per device).
int scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices)
    return set_error(FFTBF_EUNSUPPORTED, "device ordinal %d beyond %d", dev, kMaxDevices);
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(noalloc scratch)");
    g_scratch_dev[dev] = p;
  }
  *out = g_scratch_dev[dev];
  return FFTBF_OK;
}

__global__ void fill_unit_weights(float2* w, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    w[i] = make_float2(1.f, 0.f);
}

}  // namespace
}  // namespace fftbf

using namespace fftbf;

extern "C" int fftbf_execute_noalloc(int nx, int ny, int pad_x, int pad_y, int npol,
                                     int nfreq, int n_int, const float* weights_dev,
                                     const uint8_t* volts_dev, int64_t T, float* beams_dev,
                                     void* stream) {
  if (nx < 1 || ny < 1 || pad_x < 1 || pad_y < 1 || npol < 1 || nfreq < 1 || n_int < 1)
    return set_error(FFTBF_EINVAL, "sizes must all be >= 1");
  if ((int64_t)nx * ny > 65536 || pad_x > 64 || pad_y > 65536)
    return set_error(FFTBF_EUNSUPPORTED, "lattice limits: nx*ny <= 65536, pad_x <= 64, pad_y <= 65536");
  if (T < 0 || T % n_int != 0)
    return set_error(FFTBF_EINVAL, "T = %lld is not a non-negative multiple of n_int = %d",
                     (long long)T, n_int);
  const size_t need = sizeof(float2) * ((size_t)pad_x * nx + (size_t)pad_y +
                                        (weights_dev ? 0 : (size_t)nx * ny));
  if (need > FFTBF_NOALLOC_SCRATCH_BYTES)
    return set_error(FFTBF_EINVAL,
                     "tables need %zu bytes, above the %d-byte static scratch of "
                     "fftbf_execute_noalloc (use a plan for this lattice)",
                     need, FFTBF_NOALLOC_SCRATCH_BYTES);
  if (T == 0) return FFTBF_OK;
  if (!volts_dev || !beams_dev) return set_error(FFTBF_EINVAL, "null voltage or beam pointer");
  if (reinterpret_cast<uintptr_t>(weights_dev) & 7)
    return set_error(FFTBF_EINVAL, "weights_dev must be 8-byte aligned");
  int dev = 0;
  FFTBF_CUDA_TRY(cudaGetDevice(&dev));
  void* base = nullptr;
  int rc = scratch_address(dev, &base);
  if (rc != FFTBF_OK) return rc;
  int nsm = 0;
  FFTBF_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  float2* ex = static_cast<float2*>(base);
  float2* tw = ex + (size_t)pad_x * nx;
  float2* w = weights_dev ? reinterpret_cast<float2*>(const_cast<float*>(weights_dev)) : tw + pad_y;
  rc = build_tables(nx, pad_x, pad_y, ex, tw, st);
  if (rc != FFTBF_OK) return rc;
  if (!weights_dev) {
    fill_unit_weights<<<(nx * ny + 255) / 256, 256, 0, st>>>(w, nx * ny);
    FFTBF_CUDA_TRY(cudaGetLastError());
  }

  BeamArgs a{};
  a.volts = volts_dev;
  a.beams = beams_dev;
  a.w = w;
  a.ex = ex;
  a.tw = tw;
  a.nx = nx; a.ny = ny; a.mx = pad_x; a.my = pad_y;
  a.npol = npol; a.nfreq = nfreq; a.n_int = n_int;
  a.nyf = ny < pad_y ? ny : pad_y;
  a.nwin = T / n_int;
  a.ew_dft = (pad_x == nx) && (pad_x & (pad_x - 1)) == 0 && pad_x <= 16;
  a.real_w = weights_dev ? 0 : 1;      // the unit weights written above are real
  const int nsnap = n_int * npol;
  int S = kMaxElems / (pad_x * pad_y);
  if (S < 1) S = 1;
  if (S > nsnap) S = nsnap;
  a.S = S;
  if (fp32_fft_supported(pad_x, pad_y)) {
    // radix plan of the Stockham kernel: 2 or 4 first, then radix 8
    int l = 0;
    while ((1 << l) < pad_y) ++l;
    a.r0 = pad_y == 1 ? 1 : (l % 3 == 1) ? 2 : (l % 3 == 2) ? 4 : 8;
    a.nst = pad_y == 1 ? 1 : (l % 3 == 0 ? l / 3 : l / 3 + 1);
  }
  return launch_beams_fp32(a, nsm, st);
}

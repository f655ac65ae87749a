// FP32 beam path: dispatch to the fused FFT kernels, the direct-DFT fallback for other
// shapes, the unpack test hook and the FP64 plan-table builder.
#include <cuda_runtime.h>

#include <cstdlib>

#include "beam_fp32.cuh"
#include "beam_fp32_warp.cuh"

namespace fftbf {

// Test hook: FFTBF_FP32_GENERIC=1 routes every shape to the generic kernels, so the
// parity tests can cover both paths on the same inputs.
static bool getenv_flag(const char* name) {
  const char* v = getenv(name);
  return v && v[0] && v[0] != '0';
}

// ------------------------------------------------------ direct-DFT fallback kernel --
// Any mx, my (e.g. the M = 2n - 1 minimum padding). One snapshot at a time; thread-owned
// accumulators in shared memory keep the summation order fixed.
__global__ void __launch_bounds__(kThreads) beams_direct_kernel(const BeamArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int nant = a.nx * a.ny;
  const int mx = a.mx, my = a.my, nyf = a.nyf;
  float2* z = reinterpret_cast<float2*>(smem);                    // [mx][nyf]
  float* accs = reinterpret_cast<float*>(z + mx * nyf);           // [mx][my]
  uint8_t* raw = reinterpret_cast<uint8_t*>(accs + mx * my);      // [nant]
  const int nsnap = a.n_int * a.npol;
  const int64_t nitems = a.nwin * a.nfreq;
  for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int64_t jw = item / a.nfreq;
    const int f = (int)(item - jw * a.nfreq);
    for (int o = threadIdx.x; o < mx * my; o += kThreads) accs[o] = 0.f;
    for (int g = 0; g < nsnap; ++g) {
      const int64_t t = jw * a.n_int + g / a.npol;
      const int p = g % a.npol;
      const uint8_t* src = a.volts + ((t * a.nfreq + f) * a.npol + p) * (int64_t)nant;
      __syncthreads();
      for (int q = threadIdx.x; q < nant; q += kThreads) raw[q] = src[q];
      __syncthreads();
      for (int c = threadIdx.x; c < mx * nyf; c += kThreads) {
        const int A = c / nyf, iyf = c - A * nyf;
        float2 zz = czero();
        for (int ix = 0; ix < a.nx; ++ix) {
          float2 col = czero();
          for (int iy = iyf; iy < a.ny; iy += my)
            col = cadd(col, cmul(a.w[ix * a.ny + iy], unpack_byte(raw[ix * a.ny + iy])));
          zz = cadd(zz, cmul(a.ex[A * a.nx + ix], col));
        }
        z[c] = zz;
      }
      __syncthreads();
      for (int o = threadIdx.x; o < mx * my; o += kThreads) {
        const int A = o / my, B = o - A * my;
        float2 y = czero();
        for (int iy = 0; iy < nyf; ++iy)
          y = cadd(y, cmul(z[A * nyf + iy], a.tw[(int)(((int64_t)B * iy) % my)]));
        accs[o] = fmaf(y.x, y.x, fmaf(y.y, y.y, accs[o]));
      }
    }
    __syncthreads();
    float* dst = a.beams + item * (int64_t)(mx * my);
    for (int o = threadIdx.x; o < mx * my; o += kThreads) dst[o] = accs[o];
  }
}

// -------------------------------------------------------------------- launchers --
static size_t direct_smem_bytes(const BeamArgs& a) {
  return sizeof(float2) * (size_t)a.mx * a.nyf + sizeof(float) * (size_t)a.mx * a.my +
         (size_t)a.nx * a.ny + 16;
}

bool fp32_fft_supported(int mx, int my) {
  const bool mx_ok = mx == 1 || mx == 2 || mx == 3 || mx == 4 || mx == 8 || mx == 16;
  const bool pow2 = my >= 1 && (my & (my - 1)) == 0;
  return mx_ok && pow2 && (int64_t)mx * my <= kMaxElems;
}

extern template int launch_fft_mx<1>(const BeamArgs&, int, int, cudaStream_t);
extern template int launch_fft_mx<2>(const BeamArgs&, int, int, cudaStream_t);
extern template int launch_fft_mx<3>(const BeamArgs&, int, int, cudaStream_t);
extern template int launch_fft_mx<4>(const BeamArgs&, int, int, cudaStream_t);
extern template int launch_fft_mx<8>(const BeamArgs&, int, int, cudaStream_t);
extern template int launch_fft_mx<16>(const BeamArgs&, int, int, cudaStream_t);

int launch_beams_fp32(const BeamArgs& a, int nsm, cudaStream_t st) {
  if (a.nwin <= 0) return FFTBF_OK;
  if (fp32_n512_supported(a) && !getenv_flag("FFTBF_FP32_GENERIC"))
    return launch_beams_fp32_n512(a, nsm, st);
  if (fp32_warp_supported(a) && !getenv_flag("FFTBF_FP32_GENERIC"))
    return launch_beams_fp32_warp(a, nsm, st);
  if (fp32_fft_supported(a.mx, a.my) && fft_smem_bytes(a) <= 200 * 1024) {
    int log2n = 0;
    while ((1 << log2n) < a.my) ++log2n;
    switch (a.mx) {
      case 1: return launch_fft_mx<1>(a, log2n, nsm, st);
      case 2: return launch_fft_mx<2>(a, log2n, nsm, st);
      case 3: return launch_fft_mx<3>(a, log2n, nsm, st);
      case 4: return launch_fft_mx<4>(a, log2n, nsm, st);
      case 8: return launch_fft_mx<8>(a, log2n, nsm, st);
      case 16: return launch_fft_mx<16>(a, log2n, nsm, st);
      default: break;
    }
  }
  const size_t smem = direct_smem_bytes(a);
  if (smem > 220 * 1024)
    return set_error(FFTBF_EUNSUPPORTED, "lattice too large for the direct-DFT kernel");
  FFTBF_CUDA_TRY(cudaFuncSetAttribute(beams_direct_kernel,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  FFTBF_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, beams_direct_kernel,
                                                               kThreads, smem));
  if (per_sm < 1) per_sm = 1;
  const int64_t items = a.nwin * a.nfreq;
  const int64_t grid = items < (int64_t)nsm * per_sm ? items : (int64_t)nsm * per_sm;
  beams_direct_kernel<<<(unsigned)grid, kThreads, smem, st>>>(a);
  FFTBF_CUDA_TRY(cudaGetLastError());
  return FFTBF_OK;
}

// ------------------------------------------------------------------ unpack hook --
__global__ void debug_unpack_kernel(const uint8_t* in, int64_t n, float* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = unpack_byte(in[i]);
    out[2 * i] = v.x;
    out[2 * i + 1] = v.y;
  }
}

int launch_debug_unpack(const uint8_t* in, int64_t n, float* out, cudaStream_t st) {
  if (n <= 0) return FFTBF_OK;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 65535) blocks = 65535;
  debug_unpack_kernel<<<(unsigned)blocks, 256, 0, st>>>(in, n, out);
  FFTBF_CUDA_TRY(cudaGetLastError());
  return FFTBF_OK;
}

// ------------------------------------------------------------- FP64 plan tables --
__global__ void tables_kernel(int nx, int mx, int my, float2* ex, float2* tw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < my) {
    double s, c;
    sincospi(2.0 * (double)i / (double)my, &s, &c);
    tw[i] = make_float2((float)c, (float)-s);
  }
  if (i < mx * nx) {
    const int A = i / nx, ix = i - (i / nx) * nx;
    const int m = (int)(((int64_t)A * ix) % mx);
    double s, c;
    sincospi(2.0 * (double)m / (double)mx, &s, &c);
    ex[i] = make_float2((float)c, (float)-s);
  }
}

int build_tables(int nx, int mx, int my, float2* ex, float2* tw, cudaStream_t st) {
  const int n = my > mx * nx ? my : mx * nx;
  tables_kernel<<<(n + 255) / 256, 256, 0, st>>>(nx, mx, my, ex, tw);
  FFTBF_CUDA_TRY(cudaGetLastError());
  return FFTBF_OK;
}

}  // namespace fftbf

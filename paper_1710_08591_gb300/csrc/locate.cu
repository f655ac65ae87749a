// Localisation of a point source from its integrated FFT-beam intensities (Section 4.3),
// one warp per (window, channel):
//   start at the strongest FFT beam (first maximum in FP32);
//   on each axis with M >= 2n - 1 and n > 1, n_iter Newton steps
//       y <- y + T'(y) n^2 / (4 pi^2 MOI T(y)),   MOI = sum_delta delta^2 (n - |delta|),
//   where T and T' are the pointed beam and its derivative regridded from the FFT beams
//   (Eq. bp_max_arbitrary and its derivative), the curvature taken at the maximum
//   (Eq. baseline_MOI) and the sums truncated to the n_taps beams nearest the estimate;
//   an axis with M < 2n - 1 keeps the beam position A/M.
// Weights and sums in FP64 (the FFT beams are FP32); output (y_x, y_y, T(y)) with T
// regridded from every FFT beam.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace fftbf {

// Dirichlet regridding weight and its derivative at e = y - A/M (reduced to [-1/2, 1/2)).
__device__ __forceinline__ void dirichlet_wd(int n, int M, double y, int A, double* w, double* dw) {
  double e = y - (double)A / (double)M;
  e -= rint(e);
  const double L = 2.0 * n - 1.0;
  if (fabs(e) < 1e-7) {
    *w = L / M;
    *dw = -(M_PI * M_PI * L * (L * L - 1.0) / (3.0 * M)) * e;
    return;
  }
  double sL, cL, s1, c1;
  sincospi(L * e, &sL, &cL);
  sincospi(e, &s1, &c1);
  *w = sL / (s1 * M);
  *dw = (M_PI / M) * (L * cL * s1 - sL * c1) / (s1 * s1);
}

__device__ __forceinline__ int first_near(int M, double y, int k) {
  long long f0 = (long long)floor(y * (double)M - 0.5 * (k - 1) + 0.5);
  f0 %= M;
  if (f0 < 0) f0 += M;
  return (int)f0;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(256) localise_kernel(const float* __restrict__ P,
                                                       float* __restrict__ out, int64_t items,
                                                       int nx, int ny, int mx, int my,
                                                       int fit_x, int fit_y, int n_iter,
                                                       int taps_x, int taps_y, double moi_x,
                                                       double moi_y) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t item = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); item < items;
       item += warps) {
    const float* tile = P + item * (int64_t)(mx * my);
    // first maximum
    float best = -INFINITY;
    int bi = 0x7fffffff;
    for (int i = lane; i < mx * my; i += 32) {
      const float v = tile[i];
      if (v > best) { best = v; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (bi >= mx * my) bi = 0;                      // a tile with no ordered value (NaN)
    const int a0 = bi / my, b0 = bi - (bi / my) * my;
    double yx = (double)a0 / mx, yy = (double)b0 / my;
    const int kx = fit_x ? taps_x : 1, ky = fit_y ? taps_y : 1;
    for (int it = 0; it < n_iter; ++it) {
      const int fx = fit_x ? first_near(mx, yx, kx) : a0;
      const int fy = fit_y ? first_near(my, yy, ky) : b0;
      double T = 0.0, Dx = 0.0, Dy = 0.0;
      for (int q = lane; q < kx * ky; q += 32) {
        const int tx = q / ky, ty = q - (q / ky) * ky;
        const int A = (fx + tx) % mx, B = (fy + ty) % my;
        double wx = 1.0, dwx = 0.0, wy = 1.0, dwy = 0.0;
        if (fit_x) dirichlet_wd(nx, mx, yx, A, &wx, &dwx);
        if (fit_y) dirichlet_wd(ny, my, yy, B, &wy, &dwy);
        const double p = (double)tile[A * my + B];
        T += wx * wy * p;
        Dx += dwx * wy * p;
        Dy += wx * dwy * p;
      }
      T = warp_sum(T);
      Dx = warp_sum(Dx);
      Dy = warp_sum(Dy);
      const double fourpi2 = 4.0 * M_PI * M_PI;
      if (fit_x) yx += Dx * (double)nx * nx / (fourpi2 * moi_x * T);
      if (fit_y) yy += Dy * (double)ny * ny / (fourpi2 * moi_y * T);
    }
    // the pointed beam at the estimate, from every FFT beam
    double T = 0.0;
    for (int i = lane; i < mx * my; i += 32) {
      const int A = i / my, B = i - (i / my) * my;
      double wx = (A == a0) ? 1.0 : 0.0, wy = (B == b0) ? 1.0 : 0.0, d;
      if (fit_x) dirichlet_wd(nx, mx, yx, A, &wx, &d);
      if (fit_y) dirichlet_wd(ny, my, yy, B, &wy, &d);
      T += wx * wy * (double)tile[i];
    }
    T = warp_sum(T);
    if (lane == 0) {
      out[3 * item] = (float)(yx - floor(yx));
      out[3 * item + 1] = (float)(yy - floor(yy));
      out[3 * item + 2] = (float)T;
    }
  }
}

}  // namespace fftbf

using namespace fftbf;

extern "C" int fftbf_localise(fftbf_plan* p, const float* beams_dev, int64_t n_windows,
                              int n_iter, int n_taps, float* out_dev, void* stream) {
  if (!p) return set_error(FFTBF_EINVAL, "null plan");
  if (n_windows < 0 || n_iter < 0 || n_taps < 1)
    return set_error(FFTBF_EINVAL, "need n_windows >= 0, n_iter >= 0, n_taps >= 1");
  if (n_windows == 0) return FFTBF_OK;
  if (!beams_dev || !out_dev) return set_error(FFTBF_EINVAL, "null buffer");
  const int fit_x = p->mx >= 2 * p->nx - 1 && p->nx > 1;
  const int fit_y = p->my >= 2 * p->ny - 1 && p->ny > 1;
  auto moi = [](int n) {
    double s = 0.0;
    for (int d = -(n - 1); d < n; ++d) s += (double)d * d * (n - (d < 0 ? -d : d));
    return s;
  };
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != p->device) cudaSetDevice(p->device);
  const int64_t items = n_windows * p->nfreq;
  const int64_t blocks = std::min<int64_t>((items + 7) / 8, (int64_t)p->nsm * 16);
  localise_kernel<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      beams_dev, out_dev, items, p->nx, p->ny, p->mx, p->my, fit_x, fit_y, n_iter,
      std::min(n_taps, p->mx), std::min(n_taps, p->my), moi(p->nx), moi(p->ny));
  const cudaError_t e = cudaGetLastError();
  if (prev != p->device) cudaSetDevice(prev);
  if (e != cudaSuccess) return cuda_error(e, "fftbf_localise");
  return FFTBF_OK;
}

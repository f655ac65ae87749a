// Localisation of a point source from its integrated FFT-beam intensities (Section 4.3),
// one warp per (window, channel):
//   start at the strongest FFT beam (first maximum in FP32);
//   on each axis with M >= 2n - 1 and n > 1, n_iter Newton steps
//       y <- y + T'(y) n^2 / (4 pi^2 MOI T(y)),   MOI = sum_delta delta^2 (n - |delta|),
//   where T and T' are the pointed beam and its derivative regridded from the FFT beams
//   (Eq. bp_max_arbitrary and its derivative), the curvature taken at the maximum
//   (Eq. baseline_MOI) and the sums truncated to the n_taps beams nearest the estimate;
//   an axis with M < 2n - 1 keeps the beam position A/M.
// Output (y_x, y_y, T(y)) with T regridded from every FFT beam.
//
// Numerics: a position is kept as y M = ih + fr (integer ih, FP32 fraction fr in [0, 1)),
// so that the distance to FFT beam B, e M = (ih - B) + fr, and the Dirichlet phase
// (2n - 1) e mod 2 = [((2n - 1)(ih - B) mod 2M) + (2n - 1) fr] / M are formed from exact
// integers plus one FP32 term; the weights w = sin((2n-1) pi e) / (M sin(pi e)) and their
// derivative then come from FP32 sinpi/cospi, with a series near e = 0. The final sum of
// the pointed beam is accumulated in FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace fftbf {

constexpr int kLocTaps = 64;          // most taps per axis
constexpr int kLocWarps = 8;

struct LocAxis {
  int n, M, fit;
  int pow2;                           // M is a power of two: residues by masks
  float invM, newton;                 // newton = n^2 / (4 pi^2 MOI)
};

// k mod M in [0, M)
__device__ __forceinline__ int mod_m(const LocAxis& ax, int k) {
  if (ax.pow2) return k & (ax.M - 1);
  const int r = k % ax.M;
  return r < 0 ? r + ax.M : r;
}

// Dirichlet regridding weight of FFT beam B at the position (ih, fr), and its y-derivative.
__device__ __forceinline__ void dir_weight(const LocAxis& ax, int ih, float fr, int B, float* w,
                                           float* dw) {
  const int M = ax.M, L = 2 * ax.n - 1;
  int d = mod_m(ax, ih - B);                          // e M = d + fr, reduced to [-M/2, M/2)
  if ((float)d + fr >= 0.5f * M) d -= M;
  const float r = (float)d + fr;
  const float e = r * ax.invM;
  // (2n - 1) d mod 2M, any representative: |L d| <= M^2 / 2 + M fits 32 bits for M <= 32768
  const int m2 = ax.pow2 ? ((L * d) & (2 * M - 1))
                         : (M <= 32768 ? (L * d) % (2 * M) : (int)(((long long)L * d) % (2LL * M)));
  float ph = ((float)m2 + (float)L * fr) * ax.invM;   // (2n - 1) e  (mod 2)
  ph -= 2.f * rintf(0.5f * ph);
  float sL, cL, s1, c1;
  sincospif(ph, &sL, &cL);
  sincospif(e, &s1, &c1);
  const float Le = (float)L * e;
  if (fabsf(Le) < 0.05f) {
    // f(x) = sin(Lx)/sin(x) = L[1 + x^2 (1 - L^2)/6 + x^4 (7/360 - L^2/36 + L^4/120)] + ...
    const float x = 3.14159265358979f * e, x2 = x * x, L2 = (float)L * (float)L;
    const float c2 = (1.f - L2) * (1.f / 6.f);
    const float c4 = 7.f / 360.f - L2 * (1.f / 36.f) + L2 * L2 * (1.f / 120.f);
    *w = (float)L * (1.f + x2 * (c2 + x2 * c4)) * ax.invM;
    *dw = 3.14159265358979f * (float)L * x * (2.f * c2 + 4.f * c4 * x2) * ax.invM;
  } else {
    *w = sL / (s1 * (float)M);
    *dw = 3.14159265358979f * ax.invM * ((float)L * cL * s1 - sL * c1) / (s1 * s1);
  }
}

// first of the k taps nearest y M = ih + fr: floor(y M - (k - 1)/2 + 1/2), mod M
__device__ __forceinline__ int first_tap(const LocAxis& ax, int ih, float fr, int k) {
  return mod_m(ax, ih + (int)floorf(fr + 0.5f - 0.5f * (float)(k - 1)));
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// Compensated FP32 summation (Neumaier): s + c carries the sum of the added terms with an
// error of about one rounding of the result, independent of the number of terms.
struct CSum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = s + x;
    c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
    s = t;
  }
};
// Error-free sum of two floats (Knuth's TwoSum): a + b = t + e exactly.
__device__ __forceinline__ float two_sum(float a, float b, float* e) {
  const float t = a + b;
  const float bp = t - a;
  *e = (a - (t - bp)) + (b - bp);
  return t;
}
// Warp sum of compensated partial sums: every level adds exactly (TwoSum) and keeps the
// rounding errors in the compensation term.
__device__ __forceinline__ float warp_sum_c(CSum v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float os = __shfl_xor_sync(0xffffffffu, v.s, o);
    const float oc = __shfl_xor_sync(0xffffffffu, v.c, o);
    float e;
    v.s = two_sum(v.s, os, &e);
    v.c = (v.c + oc) + e;
  }
  return v.s + v.c;
}

// advance a position by dy (in units of y) and renormalise fr into [0, 1), ih into [0, M)
__device__ __forceinline__ void move(const LocAxis& ax, int* ih, float* fr, float dyM) {
  float f = *fr + dyM;
  const float k = floorf(f);
  f -= k;
  if (f >= 1.f) f = 0.f;                               // rounding of f - k at the top end
  *ih = mod_m(ax, *ih + (int)k);
  *fr = f;
}

__global__ void __launch_bounds__(32 * kLocWarps, 4) localise_kernel(
    const float* __restrict__ P, float* __restrict__ out, int64_t items, LocAxis axx,
    LocAxis axy, int n_iter, int taps_x, int taps_y, int vec4) {
  __shared__ float sw[kLocWarps][4][kLocTaps];         // wx, dwx, wy, dwy of the taps
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float* wx = sw[wib][0];
  float* dwx = sw[wib][1];
  float* wy = sw[wib][2];
  float* dwy = sw[wib][3];
  const int mx = axx.M, my = axy.M, nel = mx * my;
  const int64_t warps = (int64_t)gridDim.x * kLocWarps;
  for (int64_t item = (int64_t)blockIdx.x * kLocWarps + wib; item < items; item += warps) {
    const float* tile = P + item * (int64_t)nel;
    // first maximum
    float best = -INFINITY;
    int bi = 0x7fffffff;
    if (vec4) {
      const float4* t4 = reinterpret_cast<const float4*>(tile);
      for (int i = lane; i < (nel >> 2); i += 32) {
        const float4 v = t4[i];
        if (v.x > best) { best = v.x; bi = 4 * i; }
        if (v.y > best) { best = v.y; bi = 4 * i + 1; }
        if (v.z > best) { best = v.z; bi = 4 * i + 2; }
        if (v.w > best) { best = v.w; bi = 4 * i + 3; }
      }
    } else {
      for (int i = lane; i < nel; i += 32) {
        const float v = tile[i];
        if (v > best) { best = v; bi = i; }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (bi >= nel) bi = 0;                             // a tile with no ordered value (NaN)
    const int a0 = bi / my, b0 = bi - (bi / my) * my;
    int ihx = a0, ihy = b0;
    float frx = 0.f, fry = 0.f;
    const int kx = axx.fit ? taps_x : 1, ky = axy.fit ? taps_y : 1;
    // this lane's first tap pair (tx, ty) of the k_x k_y products, and the step for q += 32
    const int tx0 = lane / ky, ty0 = lane - tx0 * ky;
    const int stx = 32 / ky, sty = 32 - stx * ky;
    for (int it = 0; it < n_iter; ++it) {
      const int fx = axx.fit ? first_tap(axx, ihx, frx, kx) : a0;
      const int fy = axy.fit ? first_tap(axy, ihy, fry, ky) : b0;
      for (int t = lane; t < kx; t += 32) {
        float w = 1.f, d = 0.f;
        if (axx.fit) dir_weight(axx, ihx, frx, mod_m(axx, fx + t), &w, &d);
        wx[t] = w;
        dwx[t] = d;
      }
      for (int t = lane; t < ky; t += 32) {
        float w = 1.f, d = 0.f;
        if (axy.fit) dir_weight(axy, ihy, fry, mod_m(axy, fy + t), &w, &d);
        wy[t] = w;
        dwy[t] = d;
      }
      __syncwarp();
      float T = 0.f, Dx = 0.f, Dy = 0.f;
      for (int q = lane, tx = tx0, ty = ty0; q < kx * ky; q += 32) {
        const float p = tile[mod_m(axx, fx + tx) * my + mod_m(axy, fy + ty)];
        T = fmaf(wx[tx] * wy[ty], p, T);
        Dx = fmaf(dwx[tx] * wy[ty], p, Dx);
        Dy = fmaf(wx[tx] * dwy[ty], p, Dy);
        tx += stx;                                       // q += 32
        ty += sty;
        if (ty >= ky) { ty -= ky; ++tx; }
      }
      T = warp_sum_f(T);
      Dx = warp_sum_f(Dx);
      Dy = warp_sum_f(Dy);
      __syncwarp();
      if (axx.fit) move(axx, &ihx, &frx, Dx * axx.newton / T * (float)mx);
      if (axy.fit) move(axy, &ihy, &fry, Dy * axy.newton / T * (float)my);
    }
    // the pointed beam at the estimate, from every FFT beam: sum_B w^B sum_A w^A P[A, B]
    // (regridding weights of both signs: compensated FP32 sums keep the cancellation exact
    // to about one rounding)
    CSum T;
    if (axx.fit) {
      for (int c = 0; c < mx; c += kLocTaps) {
        for (int t = lane; t < kLocTaps && c + t < mx; t += 32) {
          float w, d;
          dir_weight(axx, ihx, frx, c + t, &w, &d);
          wx[t] = w;
        }
        __syncwarp();
        const int na = mx - c < kLocTaps ? mx - c : kLocTaps;
        for (int B = lane; B < my; B += 32) {
          float wB = 1.f, d;
          if (axy.fit) dir_weight(axy, ihy, fry, B, &wB, &d);
          else if (B != b0) continue;
          float s = 0.f;
          for (int A = 0; A < na; ++A) s = fmaf(wx[A], tile[(c + A) * my + B], s);
          T.add(wB * s);
        }
        __syncwarp();
      }
    } else {
      for (int B = lane; B < my; B += 32) {
        float wB = 1.f, d;
        if (axy.fit) dir_weight(axy, ihy, fry, B, &wB, &d);
        else if (B != b0) continue;
        T.add(wB * tile[a0 * my + B]);
      }
    }
    const float Tsum = warp_sum_c(T);
    if (lane == 0) {
      out[3 * item] = fmaf(frx, axx.invM, (float)ihx * axx.invM);
      out[3 * item + 1] = fmaf(fry, axy.invM, (float)ihy * axy.invM);
      out[3 * item + 2] = Tsum;
    }
  }
}

}  // namespace fftbf

using namespace fftbf;

extern "C" int fftbf_localise(fftbf_plan* p, const float* beams_dev, int64_t n_windows,
                              int n_iter, int n_taps, float* out_dev, void* stream) {
  NvtxRange nvtx("fftbf_localise");
  if (!p) return set_error(FFTBF_EINVAL, "null plan");
  if (n_windows < 0 || n_iter < 0 || n_taps < 1 || n_taps > kLocTaps)
    return set_error(FFTBF_EINVAL, "need n_windows >= 0, n_iter >= 0, 1 <= n_taps <= %d",
                     kLocTaps);
  if (n_windows == 0) return FFTBF_OK;
  if (!beams_dev || !out_dev) return set_error(FFTBF_EINVAL, "null buffer");
  auto axis = [](int n, int M) {
    LocAxis a;
    a.n = n;
    a.M = M;
    a.fit = M >= 2 * n - 1 && n > 1;
    a.pow2 = (M & (M - 1)) == 0;
    a.invM = (float)(1.0 / M);
    double moi = 0.0;
    for (int d = -(n - 1); d < n; ++d) moi += (double)d * d * (n - (d < 0 ? -d : d));
    a.newton = moi > 0.0 ? (float)((double)n * n / (4.0 * M_PI * M_PI * moi)) : 0.f;
    return a;
  };
  const LocAxis ax = axis(p->nx, p->mx), ay = axis(p->ny, p->my);
  const int vec4 = ((p->mx * p->my) % 4 == 0) && ((reinterpret_cast<uintptr_t>(beams_dev) & 15) == 0);
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != p->device) cudaSetDevice(p->device);
  const int64_t items = n_windows * p->nfreq;
  const int64_t blocks = std::min<int64_t>((items + kLocWarps - 1) / kLocWarps, (int64_t)p->nsm * 4);
  localise_kernel<<<(unsigned)blocks, 32 * kLocWarps, 0, static_cast<cudaStream_t>(stream)>>>(
      beams_dev, out_dev, items, ax, ay, n_iter, std::min(n_taps, p->mx), std::min(n_taps, p->my),
      vec4);
  const cudaError_t e = cudaGetLastError();
  if (prev != p->device) cudaSetDevice(prev);
  if (e != cudaSuccess) return cuda_error(e, "fftbf_localise");
  return FFTBF_OK;
}

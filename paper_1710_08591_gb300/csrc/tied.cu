// Tied-array beams regridded from FFT-beam intensities (K4; Eq. bp_max_arbitrary).
//
//   tied[j,f,s] = sum_A wx[f,s,A] sum_B wy[f,s,B] P[j,f,A,B]
//
// Per axis the weight is the Dirichlet regridding kernel
//   w^A(y) = (1/M) sin[(2n-1) pi (y - A/M)] / sin[pi (y - A/M)]       (M >= 2n - 1)
// or, on an axis padded below 2n - 1, the FFT beam at A = y M (y M must be an integer).
// The tables are generated in FP64 on the device and rounded to FP32 once per set of
// pointings. Pointings are sorted by their dominant E-W beam so that a tile of pointings
// touches one E-W column when that axis is a one-hot selection; the regridding is then
// a per-frequency FP32 GEMM over B with the intensities as the shared operand.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.cuh"

namespace fftbf {

// Axis modes: 0 = Dirichlet kernel (M >= 2n-1), 1 = the FFT beam itself (M < 2n-1, on
// grid), 2 = optimal windowed kernel from lag coefficients g (M >= 2n-1).
// FP64 regridding weight of beam k on an axis of n feeds and M beams for pointing y.
__device__ __forceinline__ double regrid_weight(int n, int M, int mode, const double* g,
                                                double y, int k) {
  if (mode == 0) {
    double e = y - (double)k / (double)M;
    e -= rint(e);                          // the kernel has period 1 in y
    const double L = 2.0 * n - 1.0;
    if (fabs(e) < 1e-9) return L / M;      // limit at y - k/M integer (error ~ n^2 e^2)
    return sinpi(L * e) / (sinpi(e) * (double)M);
  }
  if (mode == 1) {
    long long k0 = llrint(y * (double)M) % M;
    if (k0 < 0) k0 += M;
    return k0 == k ? 1.0 : 0.0;
  }
  // (1/M) sum_delta g_delta exp(-2 pi i delta e): powers of z = exp(-2 pi i e) by rotation
  double e = y - (double)k / (double)M;
  e -= rint(e);
  double zs, zc;
  sincospi(-2.0 * e, &zs, &zc);
  double pr = 1.0, pi = 0.0, acc = g[n - 1];
  for (int d = 1; d < n; ++d) {
    const double r = pr * zc - pi * zs;
    pi = pr * zs + pi * zc;
    pr = r;
    acc += (g[n - 1 + d] + g[n - 1 - d]) * pr;   // real, symmetric lag weights
  }
  return acc / M;
}

// First kept beam of a truncated kernel of `k` taps (k nearest beams to y M).
__device__ __forceinline__ int first_tap(int M, int mode, double y, int k) {
  long long f0;
  if (mode == 1) f0 = llrint(y * (double)M);
  else f0 = (long long)floor(y * (double)M - 0.5 * (k - 1) + 0.5);
  f0 %= M;
  if (f0 < 0) f0 += M;
  return (int)f0;
}

__global__ void tied_table_kernel(int n, int M, int mode, const double* g, int trunc,
                                  int nfreq, int n_tied, const double* y, const int* perm,
                                  float* out) {
  const int64_t total = (int64_t)nfreq * n_tied * M;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(i % M);
    const int64_t fs = i / M;                         // f * n_tied + sorted slot
    const int f = (int)(fs / n_tied);
    const int s = perm[fs];
    const double yv = y[(int64_t)f * n_tied + s];
    double w = regrid_weight(n, M, mode, g, yv, k);
    if (trunc > 0 && mode != 1) {
      const int rel = (k - first_tap(M, mode, yv, trunc) + M) % M;
      if (rel >= trunc) w = 0.0;
    }
    out[i] = (float)w;
  }
}

// Dirichlet tables (mode 0), one CTA per (f, pointing) row at a time, by angle addition:
// with e = y - k/M and L = 2n - 1,
//   sin(L pi e) = sin(L pi y) cos(L pi k/M) - cos(L pi y) sin(L pi k/M),
//   sin(pi e)   = sin(pi y) cos(pi k/M) - cos(pi y) sin(pi k/M),
// from FP64 sines of the row (two sincospi per row) and of the beams (a shared-memory table,
// L k reduced modulo 2M in integers), so a weight costs a few FP64 multiply-adds instead of
// two sincospi and a division (FP64 is slow on this part); the ratio of the two FP64 sines
// is taken in FP32, the precision of the table. Limit L/M for |e| < 1e-9.
__global__ void __launch_bounds__(256) tied_dirichlet_table_kernel(int n, int M, int trunc, int nfreq,
                                                                   int n_tied, const double* y,
                                                                   const int* perm, float* out) {
  extern __shared__ double2 dtab[];      // [M][2]: (cos, sin)(pi k/M), (cos, sin)(L pi k/M)
  __shared__ double row[5];              // sin, cos of pi y and L pi y; y
  const int L = 2 * n - 1;
  const double invM = 1.0 / (double)M;
  const float invMf = (float)invM;
  for (int k = threadIdx.x; k < M; k += blockDim.x) {
    double s1, c1, sL, cL;
    sincospi((double)k / (double)M, &s1, &c1);
    sincospi((double)(((long long)L * k) % (2LL * M)) / (double)M, &sL, &cL);
    dtab[2 * k] = make_double2(c1, s1);
    dtab[2 * k + 1] = make_double2(cL, sL);
  }
  const int64_t rows = (int64_t)nfreq * n_tied;
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
    __syncthreads();                     // tables ready; previous row's values consumed
    if (threadIdx.x == 0) {
      const int f = (int)(r / n_tied);
      const double yv = y[(int64_t)f * n_tied + perm[r]];
      sincospi(yv, &row[0], &row[1]);
      sincospi((double)L * yv, &row[2], &row[3]);
      row[4] = yv;
    }
    __syncthreads();
    const double sy = row[0], cy = row[1], sLy = row[2], cLy = row[3], yv = row[4];
    const int first = trunc > 0 ? first_tap(M, 0, yv, trunc) : 0;
    for (int k = threadIdx.x; k < M; k += blockDim.x) {
      double e = fma(-(double)k, invM, yv);
      e -= rint(e);
      float w;
      if (fabs(e) < 1e-9) {
        w = (float)L * invMf;
      } else {
        const double2 t1 = dtab[2 * k], tL = dtab[2 * k + 1];
        const double num = sLy * tL.x - cLy * tL.y;
        const double den = sy * t1.x - cy * t1.y;
        w = (float)num / (float)den * invMf;     // FP64 sines, their ratio in FP32
      }
      if (trunc > 0 && (k - first + M) % M >= trunc) w = 0.f;
      out[r * M + k] = w;
    }
  }
}

// Windowed tables (mode 2) for a power-of-two M, one CTA per row at a time: the kernel is a
// trigonometric polynomial of degree n - 1, sampled at the M beams,
//   w(y - j/M) = (1/M) Re sum_{d < n} a_d exp(-2 pi i d y) exp(+2 pi i d j / M),
// a_0 = g_0, a_d = 2 g_d (real symmetric lags), i.e. one inverse DFT of length M per
// pointing: radix-2 Stockham in FP64 in shared memory, O(M log M) per row instead of the
// O(M n) direct sums.
__global__ void __launch_bounds__(256) tied_window_table_kernel(int n, int M, const double* g,
                                                                int trunc, int nfreq, int n_tied,
                                                                const double* y, const int* perm,
                                                                float* out) {
  extern __shared__ double2 wsm2[];
  const int half = M >> 1;
  double2* twp = wsm2;                   // [M/2] exp(+2 pi i m / M)
  double2* b0 = twp + half;              // [M]
  double2* b1 = b0 + M;                  // [M]
  __shared__ double rowy;
  __shared__ double2 zlo[16], zhi[128];  // exp(-2 pi i d y) = zlo[d mod 16] zhi[d / 16], n <= 2048
  for (int m = threadIdx.x; m < half; m += blockDim.x) {
    double s, c;
    sincospi(2.0 * (double)m / (double)M, &s, &c);
    twp[m] = make_double2(c, s);
  }
  const int64_t rows = (int64_t)nfreq * n_tied;
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
    __syncthreads();
    if (threadIdx.x == 0) rowy = y[(int64_t)(r / n_tied) * n_tied + perm[r]];
    __syncthreads();
    const double yv = rowy;
    // the phases of the row: 16 + n/16 sincospi instead of n
    {
      const int t = threadIdx.x;
      const int m = t < 16 ? t : 16 * (t - 16);
      if (t < 16 + (n + 15) / 16) {
        double ph = (double)m * yv;
        ph -= rint(ph);
        double sn, cs;
        sincospi(-2.0 * ph, &sn, &cs);
        if (t < 16) zlo[t] = make_double2(cs, sn);
        else zhi[t - 16] = make_double2(cs, sn);
      }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < M; d += blockDim.x) {
      double2 v = make_double2(0.0, 0.0);
      if (d < n) {
        const double2 p = zlo[d & 15], q = zhi[d >> 4];
        const double a = d == 0 ? g[n - 1] : 2.0 * g[n - 1 + d];
        v = make_double2(a * (p.x * q.x - p.y * q.y), a * (p.x * q.y + p.y * q.x));
      }
      b0[d] = v;
    }
    __syncthreads();
    double2* src = b0;
    double2* dst = b1;
    for (int ns = 1; ns < M; ns <<= 1) {
      for (int j = threadIdx.x; j < half; j += blockDim.x) {
        const int k = j & (ns - 1);
        const double2 w = twp[k * (half / ns)];
        const double2 a = src[j], c = src[j + half];
        const double2 b = make_double2(c.x * w.x - c.y * w.y, c.x * w.y + c.y * w.x);
        const int d = ((j - k) << 1) + k;
        dst[d] = make_double2(a.x + b.x, a.y + b.y);
        dst[d + ns] = make_double2(a.x - b.x, a.y - b.y);
      }
      __syncthreads();
      double2* t = src; src = dst; dst = t;
    }
    const int first = trunc > 0 ? first_tap(M, 2, yv, trunc) : 0;
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
      double w = src[j].x / (double)M;
      if (trunc > 0 && (j - first + M) % M >= trunc) w = 0.0;
      out[r * M + j] = (float)w;
    }
  }
}

// Compact tables: per (f, pointing) the first kept beam of each axis and the kx + ky tap
// weights (caller's pointing order).
__global__ void tied_compact_table_kernel(int nx, int ny, int mx, int my, int mode_x,
                                          int mode_y, const double* gx, const double* gy,
                                          int kx, int ky, int nfreq, int n_tied,
                                          const double* u, const double* v, int* first,
                                          float* cw) {
  const int64_t total = (int64_t)nfreq * n_tied;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int fx = first_tap(mx, mode_x, u[i], kx), fy = first_tap(my, mode_y, v[i], ky);
    first[2 * i] = fx;
    first[2 * i + 1] = fy;
    float* c = cw + i * (kx + ky);
    for (int t = 0; t < kx; ++t) c[t] = (float)regrid_weight(nx, mx, mode_x, gx, u[i], (fx + t) % mx);
    for (int t = 0; t < ky; ++t) c[kx + t] = (float)regrid_weight(ny, my, mode_y, gy, v[i], (fy + t) % my);
  }
}

// out[j,f,s] = sum_{tx<kx, ty<ky} cx[tx] cy[ty] P[j,f,(fx+tx) mod Mx,(fy+ty) mod My]: a
// thread per (channel, pointing), pointings fastest, looping over windows (grid z), so the
// pointing's taps and weights are fetched once and no index needs a division.
__global__ void __launch_bounds__(256) tied_compact_kernel(const float* __restrict__ P,
                                                            const int* __restrict__ first,
                                                            const float* __restrict__ cw,
                                                            float* __restrict__ out, int64_t nwin,
                                                            int nfreq, int n_tied, int mx,
                                                            int my, int kx, int ky) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_tied) return;
  for (int f = blockIdx.y; f < nfreq; f += gridDim.y) {
    const int64_t fs = (int64_t)f * n_tied + s;
    const float* c = cw + fs * (kx + ky);
    const int fx = first[2 * fs], fy = first[2 * fs + 1];
    for (int64_t j = blockIdx.z; j < nwin; j += gridDim.z) {
      const int64_t jf = j * nfreq + f;
      const float* Pj = P + jf * (int64_t)(mx * my);
      float acc = 0.f;
      int rx = fx;                                    // (fx + tx) mod Mx, fx < Mx, kx <= Mx
      for (int tx = 0; tx < kx; ++tx) {
        const float* row = Pj + rx * my;
        float racc = 0.f;
        int cy = fy;                                  // (fy + ty) mod My
        for (int ty = 0; ty < ky; ++ty) {
          racc = fmaf(c[kx + ty], __ldg(row + cy), racc);
          if (++cy == my) cy = 0;
        }
        acc = fmaf(c[tx], racc, acc);
        if (++rx == mx) rx = 0;
      }
      out[jf * n_tied + s] = acc;
    }
  }
}

constexpr int TS = 64, TJ = 64, TK = 16;

// Regridding GEMM with 128 pointings x 128 windows per CTA (256 threads, 8 x 8 outputs
// each: rows 4 tm .. + 3 and 64 + 4 tm .. + 3, the same for columns, so the float4 reads
// of a k-step fall in distinct banks), K steps of 16 FFT beams double-buffered through
// registers (the next step's global loads are in flight while this one is multiplied).
// The K loop runs over the E-W beams A that some pointing of the tile weights (one or two
// for a one-hot E-W axis, the pointings being sorted by it) and the N-S beams B:
//   out[j, f, perm(s)] = sum_A sum_B wx[f, s, A] wy[f, s, B] P[j, f, A, B].
#ifndef FFTBF_TIED_GK
#define FFTBF_TIED_GK 16          // FFT beams per K step of the GEMM (8 or 16)
#endif
constexpr int GM = 128, GN = 128, GK = FFTBF_TIED_GK;
constexpr int GEPT = GK / 2;      // staged elements per thread and operand per K step
#ifndef FFTBF_TIED_MIN_BLOCKS
#define FFTBF_TIED_MIN_BLOCKS 2   // CTAs per SM the register budget of the GEMM targets
#endif

__global__ void __launch_bounds__(256, FFTBF_TIED_MIN_BLOCKS) tied_gemm128_kernel(const float* __restrict__ P,
                                                              const float* __restrict__ wx,
                                                              const float* __restrict__ wy,
                                                              const int* __restrict__ perm,
                                                              float* __restrict__ out,
                                                              int64_t nwin, int nfreq, int n_tied,
                                                              int mx, int my) {
  __shared__ __align__(16) float As[2][GK][GM + 4];
  __shared__ __align__(16) float Bs[2][GK][GN + 4];
  __shared__ unsigned long long s_active;
  const int f = blockIdx.z;
  const int s0 = blockIdx.x * GM;
  const int64_t j0 = (int64_t)blockIdx.y * GN;
  const int tid = threadIdx.x, tm = tid >> 4, tn = tid & 15;
  const int64_t fs0 = (int64_t)f * n_tied;
  const int64_t prow = (int64_t)nfreq * mx * my;
  // E-W beams used by this tile's pointings (mx <= 64)
  if (tid == 0) s_active = 0ull;
  __syncthreads();
  for (int i = tid; i < GM * mx; i += blockDim.x) {
    const int r = i / mx, A = i - (i / mx) * mx;
    if (s0 + r < n_tied && wx[(fs0 + s0 + r) * mx + A] != 0.f) atomicOr(&s_active, 1ull << A);
  }
  __syncthreads();
  const unsigned long long active = s_active;
  const int kb = (my + GK - 1) / GK;
  // load mapping: row (pointing / window) = tid >> 1, GK / 2 consecutive k from
  // (tid & 1) * GK / 2 (float4 loads when the rows are 16-byte aligned)
  const int lr = tid >> 1, lk = (tid & 1) * GEPT;
  const int gs = s0 + lr;
  const int64_t gj = j0 + lr;
  const bool vec = (my & 3) == 0;
  float ra[GEPT], rb[GEPT];
  auto load = [&](int A, int b0) {
    const float w = gs < n_tied ? wx[(fs0 + gs) * mx + A] : 0.f;
    const float* wrow = wy + (fs0 + gs) * my + b0 + lk;
    const float* prow_p = P + gj * prow + (int64_t)f * mx * my + (int64_t)A * my + b0 + lk;
    const bool rin = gs < n_tied, pin = gj < nwin;
    if (vec && b0 + lk + GEPT <= my) {
#pragma unroll
      for (int h = 0; h < GEPT / 4; ++h) {
        const float4 a = rin ? *reinterpret_cast<const float4*>(wrow + 4 * h) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 p = pin ? *reinterpret_cast<const float4*>(prow_p + 4 * h) : make_float4(0.f, 0.f, 0.f, 0.f);
        ra[4 * h] = w * a.x; ra[4 * h + 1] = w * a.y; ra[4 * h + 2] = w * a.z; ra[4 * h + 3] = w * a.w;
        rb[4 * h] = p.x; rb[4 * h + 1] = p.y; rb[4 * h + 2] = p.z; rb[4 * h + 3] = p.w;
      }
    } else {
#pragma unroll
      for (int i = 0; i < GEPT; ++i) {
        const bool kin = b0 + lk + i < my;
        ra[i] = (rin && kin) ? w * wrow[i] : 0.f;
        rb[i] = (pin && kin) ? prow_p[i] : 0.f;
      }
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int i = 0; i < GEPT; ++i) {
      As[buf][lk + i][lr] = ra[i];
      Bs[buf][lk + i][lr] = rb[i];
    }
  };
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[i][q] = 0.f;
  // the (A, b0) steps in order
  int A = 0;
  while (A < mx && !((active >> A) & 1ull)) ++A;
  if (A < mx) {
    int b = 0, buf = 0;
    load(A, 0);
    store(0);
    __syncthreads();
    while (true) {
      // next step
      int nA = A, nb = b + 1;
      if (nb == kb) {
        nb = 0;
        ++nA;
        while (nA < mx && !((active >> nA) & 1ull)) ++nA;
      }
      const bool more = nA < mx;
      if (more) load(nA, nb * GK);
#pragma unroll
      for (int k = 0; k < GK; ++k) {
        const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][k][4 * tm]);
        const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][k][64 + 4 * tm]);
        const float4 b0v = *reinterpret_cast<const float4*>(&Bs[buf][k][4 * tn]);
        const float4 b1v = *reinterpret_cast<const float4*>(&Bs[buf][k][64 + 4 * tn]);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float bv[8] = {b0v.x, b0v.y, b0v.z, b0v.w, b1v.x, b1v.y, b1v.z, b1v.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int q = 0; q < 8; ++q) acc[i][q] = fmaf(av[i], bv[q], acc[i][q]);
      }
      if (!more) break;
      store(buf ^ 1);
      __syncthreads();
      buf ^= 1;
      A = nA;
      b = nb;
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int s = s0 + (i < 4 ? 4 * tm + i : 64 + 4 * tm + i - 4);
    if (s >= n_tied) continue;
    const int dst = perm[fs0 + s];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int64_t j = j0 + (q < 4 ? 4 * tn + q : 64 + 4 * tn + q - 4);
      if (j < nwin) out[(j * nfreq + f) * (int64_t)n_tied + dst] = acc[i][q];
    }
  }
}

__global__ void __launch_bounds__(256) tied_gemm_kernel(const float* __restrict__ P,
                                                         const float* __restrict__ wx,
                                                         const float* __restrict__ wy,
                                                         const int* __restrict__ perm,
                                                         float* __restrict__ out,
                                                         int64_t nwin, int nfreq, int n_tied,
                                                         int mx, int my) {
  __shared__ __align__(16) float Ws[TK][TS + 4];
  __shared__ __align__(16) float Ps[TK][TJ + 4];
  __shared__ float wxs[TS];
  const int f = blockIdx.z;
  const int s0 = blockIdx.x * TS;
  const int64_t j0 = (int64_t)blockIdx.y * TJ;
  const int tx = threadIdx.x & 15;   // window direction
  const int ty = threadIdx.x >> 4;   // pointing direction
  const int64_t fs0 = (int64_t)f * n_tied;
  const int64_t prow = (int64_t)nfreq * mx * my;   // stride of P between windows
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[i][q] = 0.f;

  for (int A = 0; A < mx; ++A) {
    __syncthreads();
    if (threadIdx.x < TS) {
      const int s = s0 + threadIdx.x;
      wxs[threadIdx.x] = s < n_tied ? wx[(fs0 + s) * mx + A] : 0.f;
    }
    const int any = __syncthreads_or(threadIdx.x < TS && wxs[threadIdx.x] != 0.f);
    if (!any) continue;
    const float* Pa = P + (int64_t)f * mx * my + (int64_t)A * my;
    for (int b0 = 0; b0 < my; b0 += TK) {
#pragma unroll
      for (int q = 0; q < (TS * TK) / 256; ++q) {
        const int e = threadIdx.x + q * 256;
        const int s = e >> 4, k = e & 15;
        const int gs = s0 + s, gb = b0 + k;
        Ws[k][s] = (gs < n_tied && gb < my) ? wxs[s] * wy[(fs0 + gs) * my + gb] : 0.f;
        const int64_t gj = j0 + s;
        Ps[k][s] = (gj < nwin && gb < my) ? Pa[gj * prow + gb] : 0.f;
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < TK; ++k) {
        const float4 a = *reinterpret_cast<const float4*>(&Ws[k][ty * 4]);
        const float4 b = *reinterpret_cast<const float4*>(&Ps[k][tx * 4]);
        const float av[4] = {a.x, a.y, a.z, a.w};
        const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[i][q] = fmaf(av[i], bv[q], acc[i][q]);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int s = s0 + ty * 4 + i;
    if (s >= n_tied) continue;
    const int dst = perm[fs0 + s];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t j = j0 + tx * 4 + q;
      if (j < nwin) out[(j * nfreq + f) * (int64_t)n_tied + dst] = acc[i][q];
    }
  }
}

void tied_free(TiedTables& tt) {
  cudaFree(tt.wyh);
  cudaFree(tt.wyl);
  cudaFree(tt.wye);
  cudaFree(tt.wa);
  cudaFree(tt.ph);
  cudaFree(tt.pl);
  cudaFree(tt.pe);
  cudaFree(tt.wx);
  cudaFree(tt.wy);
  cudaFree(tt.perm);
  cudaFree(tt.duv);
  cudaFree(tt.d_g);
  cudaFree(tt.first);
  cudaFree(tt.cw);
  tt = TiedTables();
}

// multiprocessors of the current device (grid sizing of the row kernels)
static int tt_sms(cudaStream_t) {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

int tied_prepare(TiedTables& tt, int nx, int ny, int mx, int my, int nfreq, int n_tied,
                 const double* u, const double* v, cudaStream_t st) {
  const size_t nuv = (size_t)nfreq * n_tied;
  if (tt.n_tied == n_tied && tt.u.size() == nuv && tt.built_version == tt.version &&
      std::memcmp(tt.u.data(), u, nuv * sizeof(double)) == 0 &&
      std::memcmp(tt.v.data(), v, nuv * sizeof(double)) == 0)
    return FFTBF_OK;                                  // same pointings: tables are current

  const bool dense_x = mx >= 2 * nx - 1, dense_y = my >= 2 * ny - 1;
  const int mode_x = !dense_x ? 1 : (tt.win_x.g.empty() ? 0 : 2);
  const int mode_y = !dense_y ? 1 : (tt.win_y.g.empty() ? 0 : 2);
  // compact path when both axes use a few taps: a grid axis (1 tap) or a truncated kernel
  const int kx = mode_x == 1 ? 1 : tt.win_x.trunc, ky = mode_y == 1 ? 1 : tt.win_y.trunc;
  const bool compact = kx > 0 && ky > 0;
  for (size_t i = 0; i < nuv; ++i) {
    if (!std::isfinite(u[i]) || !std::isfinite(v[i]))
      return set_error(FFTBF_EINVAL, "tied pointing %zu is not finite", i);
    if (!dense_x && std::fabs(u[i] * mx - std::nearbyint(u[i] * mx)) > 1e-9)
      return set_error(FFTBF_EINVAL,
                       "pointing %zu: u*pad_x = %.12g is off the FFT-beam grid and pad_x < "
                       "2nx-1, so no regridding kernel exists on that axis", i, u[i] * mx);
    if (!dense_y && std::fabs(v[i] * my - std::nearbyint(v[i] * my)) > 1e-9)
      return set_error(FFTBF_EINVAL,
                       "pointing %zu: v*pad_y = %.12g is off the FFT-beam grid and pad_y < "
                       "2ny-1, so no regridding kernel exists on that axis", i, v[i] * my);
  }
  // Sort each frequency's pointings by E-W beam (one-hot axis) so tiles skip columns: a
  // stable counting sort on the pad_x possible beams.
  std::vector<int> perm(nuv);
  std::vector<int> key(dense_x ? 0 : n_tied), count(dense_x ? 0 : mx + 1);
  for (int f = 0; f < nfreq; ++f) {
    int* p = perm.data() + (size_t)f * n_tied;
    if (dense_x) {
      for (int s = 0; s < n_tied; ++s) p[s] = s;
      continue;
    }
    const double* uf = u + (size_t)f * n_tied;
    std::fill(count.begin(), count.end(), 0);
    for (int s = 0; s < n_tied; ++s) {
      key[s] = (int)(((llrint(uf[s] * mx) % mx) + mx) % mx);
      ++count[key[s] + 1];
    }
    for (int k = 0; k < mx; ++k) count[k + 1] += count[k];
    for (int s = 0; s < n_tied; ++s) p[count[key[s]]++] = s;
  }
  // (re)allocate the tables of the path in use
  cudaFree(tt.wx);
  cudaFree(tt.wy);
  cudaFree(tt.perm);
  cudaFree(tt.duv);
  cudaFree(tt.d_g);
  cudaFree(tt.first);
  cudaFree(tt.cw);
  tt.wx = tt.wy = tt.cw = nullptr;
  tt.perm = tt.first = nullptr;
  tt.duv = tt.d_g = nullptr;
  tt.cap_tied = 0;
  tt.tc = 0;
  const size_t ng = tt.win_x.g.size() + tt.win_y.g.size();
  bool ok = cudaMalloc(&tt.perm, nuv * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&tt.duv, 2 * nuv * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&tt.d_g, (ng ? ng : 1) * sizeof(double)) == cudaSuccess;
  if (ok && compact)
    ok = cudaMalloc(&tt.first, 2 * nuv * sizeof(int)) == cudaSuccess &&
         cudaMalloc(&tt.cw, nuv * (kx + ky) * sizeof(float)) == cudaSuccess;
  if (ok && !compact)
    ok = cudaMalloc(&tt.wx, nuv * mx * sizeof(float)) == cudaSuccess &&
         cudaMalloc(&tt.wy, nuv * my * sizeof(float)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    tied_free(tt);
    return set_error(FFTBF_ENOMEM, "cannot allocate tied-beam tables (%zu pointings)", nuv);
  }
  tt.cap_tied = nuv;
  tt.kx = compact ? kx : 0;
  tt.ky = compact ? ky : 0;
  // The plan keeps host copies of the pointings (to detect a repeat) and of the order;
  // the uploads read those plan-owned buffers, never the caller's.
  tt.n_tied = 0;
  tt.u.assign(u, u + nuv);
  tt.v.assign(v, v + nuv);
  tt.hperm.swap(perm);
  FFTBF_CUDA_TRY(cudaMemcpyAsync(tt.duv, tt.u.data(), nuv * sizeof(double), cudaMemcpyHostToDevice, st));
  FFTBF_CUDA_TRY(cudaMemcpyAsync(tt.duv + nuv, tt.v.data(), nuv * sizeof(double), cudaMemcpyHostToDevice, st));
  FFTBF_CUDA_TRY(cudaMemcpyAsync(tt.perm, tt.hperm.data(), nuv * sizeof(int), cudaMemcpyHostToDevice, st));
  tt.hg.assign(tt.win_x.g.begin(), tt.win_x.g.end());
  tt.hg.insert(tt.hg.end(), tt.win_y.g.begin(), tt.win_y.g.end());
  if (!tt.hg.empty())
    FFTBF_CUDA_TRY(cudaMemcpyAsync(tt.d_g, tt.hg.data(), tt.hg.size() * sizeof(double),
                                   cudaMemcpyHostToDevice, st));
  const double* gx = tt.d_g;
  const double* gy = tt.d_g + tt.win_x.g.size();
  const int threads = 256;
  auto blocks = [&](int64_t n) { return (unsigned)std::min<int64_t>((n + threads - 1) / threads, 1 << 20); };
  if (compact) {
    tied_compact_table_kernel<<<blocks((int64_t)nuv), threads, 0, st>>>(
        nx, ny, mx, my, mode_x, mode_y, gx, gy, kx, ky, nfreq, n_tied, tt.duv, tt.duv + nuv,
        tt.first, tt.cw);
    FFTBF_CUDA_TRY(cudaGetLastError());
  } else {
    // per axis: the row kernels for the Dirichlet and (power-of-two M) windowed tables,
    // else the per-weight kernel
    auto axis_table = [&](int n, int M, int mode, const double* g, int trunc, const double* yy,
                          float* out) -> int {
      const int grid = (int)std::min<int64_t>((int64_t)nuv, (int64_t)tt_sms(st) * 4);
      if (mode == 0 && M <= 4096) {
        const size_t sm = sizeof(double2) * 2 * (size_t)M;
        FFTBF_CUDA_TRY(cudaFuncSetAttribute(tied_dirichlet_table_kernel,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        tied_dirichlet_table_kernel<<<grid, threads, sm, st>>>(n, M, trunc, nfreq, n_tied, yy,
                                                               tt.perm, out);
      } else if (mode == 2 && M <= 4096 && (M & (M - 1)) == 0 && M >= 2 && n <= 2048) {
        const size_t sm = sizeof(double2) * ((size_t)M / 2 + 2 * (size_t)M);
        FFTBF_CUDA_TRY(cudaFuncSetAttribute(tied_window_table_kernel,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        tied_window_table_kernel<<<grid, threads, sm, st>>>(n, M, g, trunc, nfreq, n_tied, yy,
                                                            tt.perm, out);
      } else {
        tied_table_kernel<<<blocks((int64_t)nuv * M), threads, 0, st>>>(n, M, mode, g, trunc, nfreq,
                                                                        n_tied, yy, tt.perm, out);
      }
      FFTBF_CUDA_TRY(cudaGetLastError());
      return FFTBF_OK;
    };
    int rc = axis_table(nx, mx, mode_x, gx, tt.win_x.trunc, tt.duv, tt.wx);
    if (rc == FFTBF_OK) rc = axis_table(ny, my, mode_y, gy, tt.win_y.trunc, tt.duv + nuv, tt.wy);
    if (rc != FFTBF_OK) return rc;
    tt.tc = 0;
    if (tied_tc_eligible(dense_x, mx, my)) {
      tt.tc_n_tied = n_tied;
      // without room for the split tables the CUDA-core GEMM serves (its tables are
      // built); any other failure is the call's error
      const int trc = tied_tc_build(tt, (int64_t)nuv, mx, my, st);
      if (trc == FFTBF_ENOMEM) {
        tt.tc = 0;
        clear_error();
      } else if (trc != FFTBF_OK) {
        return trc;
      }
    }
  }
  tt.built_version = tt.version;
  tt.n_tied = n_tied;
  return FFTBF_OK;
}

int tied_launch(TiedTables& tt, const float* beams, int64_t nwin, int nfreq, int mx,
                int my, float* out, cudaStream_t st) {
  if (nwin <= 0) return FFTBF_OK;
  if (tt.tc && tt.kx == 0) {
    const int rc = tied_tc_launch(tt, beams, nwin, nfreq, mx, my, out, st);
    if (rc != FFTBF_ENOMEM) return rc;
    clear_error();                               // no room for the beam split: CUDA-core GEMM
  }
  if (tt.kx > 0 && tt.ky > 0) {
    dim3 grid((tt.n_tied + 255) / 256, (unsigned)std::min(nfreq, 65535),
              (unsigned)std::min<int64_t>(nwin, 16));
    tied_compact_kernel<<<grid, 256, 0, st>>>(beams, tt.first, tt.cw, out, nwin, nfreq,
                                              tt.n_tied, mx, my, tt.kx, tt.ky);
    FFTBF_CUDA_TRY(cudaGetLastError());
    return FFTBF_OK;
  }
  if (mx <= 64 && nwin >= 64) {
    const int64_t jt = (nwin + GN - 1) / GN;
    if (jt > 65535 || nfreq > 65535)
      return set_error(FFTBF_EUNSUPPORTED, "tied beams: too many windows or channels per call");
    dim3 grid((tt.n_tied + GM - 1) / GM, (unsigned)jt, nfreq);
    tied_gemm128_kernel<<<grid, 256, 0, st>>>(beams, tt.wx, tt.wy, tt.perm, out, nwin, nfreq,
                                              tt.n_tied, mx, my);
    FFTBF_CUDA_TRY(cudaGetLastError());
    return FFTBF_OK;
  }
  const int64_t jt = (nwin + TJ - 1) / TJ;
  if (jt > 65535 || nfreq > 65535)
    return set_error(FFTBF_EUNSUPPORTED, "tied beams: too many windows or channels per call");
  dim3 grid((tt.n_tied + TS - 1) / TS, (unsigned)jt, nfreq);
  tied_gemm_kernel<<<grid, 256, 0, st>>>(beams, tt.wx, tt.wy, tt.perm, out, nwin, nfreq,
                                         tt.n_tied, mx, my);
  FFTBF_CUDA_TRY(cudaGetLastError());
  return FFTBF_OK;
}

}  // namespace fftbf

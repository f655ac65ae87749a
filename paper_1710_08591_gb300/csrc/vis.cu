// Redundancy-stacked visibilities recovered from integrated FFT-beam intensities
// (Eq. inv_b2n-1): per axis with pad M >= 2n - 1,
//   V~_delta = (1/M) sum_A exp(+2 pi i delta A / M) P_A ,  |delta| < n,
// the inverse of Eq. b2n-1 (the FFT beams hold the same information as V~_delta); on an
// axis with M < 2n - 1 the FFT-beam index is kept. Direct route, one CTA per (window, channel): the
// N-S step reads the beam tile from shared memory and a table of exp(+2 pi i k / My), the
// E-W step (if any) combines the Mx rows. FP32 sums of FP32 twiddles (from FP64).
#include <cuda_runtime.h>

#include "beam_fp32.cuh"

namespace fftbf {

__global__ void __launch_bounds__(256) stacked_vis_kernel(const float* __restrict__ P,
                                                          float2* __restrict__ out,
                                                          const float2* __restrict__ tw_y,
                                                          int64_t nitems, int nx, int ny,
                                                          int mx, int my, int inv_x,
                                                          int inv_y) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int dx_n = inv_x ? 2 * nx - 1 : mx;
  const int dy_n = inv_y ? 2 * ny - 1 : my;
  float* ps = reinterpret_cast<float*>(smem);                       // [mx][my]
  float2* tys = reinterpret_cast<float2*>(ps + ((mx * my + 1) & ~1)); // [my] exp(+2 pi i k/My)
  float2* txs = tys + my;                                            // [mx] exp(+2 pi i k/Mx)
  float2* q = txs + mx;                                              // [mx][dy_n]
  for (int i = threadIdx.x; i < my; i += blockDim.x) {
    const float2 t = tw_y[i];
    tys[i] = make_float2(t.x, -t.y);
  }
  for (int i = threadIdx.x; i < mx; i += blockDim.x) {
    double s, c;
    sincospi(2.0 * (double)i / (double)mx, &s, &c);
    txs[i] = make_float2((float)c, (float)s);
  }
  const float iny = 1.0f / (float)my, inx = 1.0f / (float)mx;
  for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
    __syncthreads();
    const float* src = P + item * (int64_t)(mx * my);
    for (int i = threadIdx.x; i < mx * my; i += blockDim.x) ps[i] = src[i];
    __syncthreads();
    // N-S: q[A][d] = (1/My) sum_B exp(+2 pi i lag B / My) P[A][B]   (or q = P)
    for (int o = threadIdx.x; o < mx * dy_n; o += blockDim.x) {
      const int A = o / dy_n, d = o - A * dy_n;
      float2 acc = make_float2(0.f, 0.f);
      if (inv_y) {
        const int lag = d - (ny - 1);
        const unsigned lm = (unsigned)(((lag % my) + my) % my);
        const float* row = ps + A * my;
        unsigned idx = 0;
        for (int B = 0; B < my; ++B) {
          const float2 t = tys[idx];
          acc.x = fmaf(t.x, row[B], acc.x);
          acc.y = fmaf(t.y, row[B], acc.y);
          idx += lm;
          if (idx >= (unsigned)my) idx -= my;
        }
        acc.x *= iny;
        acc.y *= iny;
      } else {
        acc.x = ps[A * my + d];
      }
      q[o] = acc;
    }
    __syncthreads();
    // E-W: V[dx][d] = (1/Mx) sum_A exp(+2 pi i lag A / Mx) q[A][d]   (or V = q)
    float2* dst = out + item * (int64_t)(dx_n * dy_n);
    for (int o = threadIdx.x; o < dx_n * dy_n; o += blockDim.x) {
      const int e = o / dy_n, d = o - e * dy_n;
      float2 v;
      if (inv_x) {
        const int lag = e - (nx - 1);
        const int lm = ((lag % mx) + mx) % mx;
        v = make_float2(0.f, 0.f);
        int idx = 0;
        for (int A = 0; A < mx; ++A) {
          const float2 t = txs[idx], z = q[A * dy_n + d];
          v.x = fmaf(t.x, z.x, fmaf(-t.y, z.y, v.x));
          v.y = fmaf(t.x, z.y, fmaf(t.y, z.x, v.y));
          idx += lm;
          if (idx >= mx) idx -= mx;
        }
        v.x *= inx;
        v.y *= inx;
      } else {
        v = q[e * dy_n + d];
      }
      dst[o] = v;
    }
  }
}

// The same N-S inversion by FFT when My is a power of two: two beam rows a, b share one
// complex transform z = P_a + i P_b, Z[k] = sum_B z_B exp(+2 pi i k B / My) (radix-2
// Stockham in shared memory), and the rows separate by Hermitian symmetry,
//   X_a[k] = (Z[k] + conj Z[My-k]) / 2,   X_b[k] = (Z[k] - conj Z[My-k]) / 2i,
// with V~_delta = X[delta] / My for delta >= 0 and conj(X[-delta]) / My below. All row
// pairs of a (window, channel) go through the same stage loop (one barrier per stage for
// the whole tile), whose first stage reads the raw rows; the next (window, channel) tile
// is fetched with cp.async meanwhile. The E-W step (when Mx >= 2nx - 1) is the direct one
// above.
__global__ void __launch_bounds__(256) stacked_vis_fft_kernel(const float* __restrict__ P,
                                                              float2* __restrict__ out,
                                                              const float2* __restrict__ tw_y,
                                                              int64_t nitems, int nx, int ny,
                                                              int mx, int my, int inv_x) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int half = my >> 1, dy_n = 2 * ny - 1, dx_n = inv_x ? 2 * nx - 1 : mx;
  const int np = (mx + 1) >> 1;                    // row pairs, transformed together
  const int lh = __ffs(half) - 1;                  // log2(My/2)
  const int tsz = mx * my;                         // floats per beam tile
  float* tiles = reinterpret_cast<float*>(smem);   // [2][Mx * My] raw tiles, next one in flight
  float2* twp = reinterpret_cast<float2*>(tiles + 2 * ((tsz + 3) & ~3));   // [My/2] exp(+2 pi i k / My)
  float2* buf0 = twp + half;                       // [np][My]
  float2* buf1 = buf0 + np * my;                   // [np][My]
  float2* q = buf1 + np * my;                      // [Mx][dy_n] when inverting E-W
  float2* txs = q + (inv_x ? mx * dy_n : 0);       // [Mx] exp(+2 pi i k / Mx)
  for (int i = threadIdx.x; i < half; i += blockDim.x) {
    const float2 t = tw_y[i];
    twp[i] = make_float2(t.x, -t.y);
  }
  if (inv_x)
    for (int i = threadIdx.x; i < mx; i += blockDim.x) {
      double s, c;
      sincospi(2.0 * (double)i / (double)mx, &s, &c);
      txs[i] = make_float2((float)c, (float)s);
    }
  const float iny = 1.0f / (float)my, inx = 1.0f / (float)mx;
  // tiles are fetched with 16-byte cp.async when they start on 16-byte boundaries
  const bool vec = (tsz & 3) == 0 && (reinterpret_cast<uintptr_t>(P) & 15) == 0;
  auto fetch = [&](int64_t itm, float* dst) {
    if (itm >= nitems) return;
    const float* src = P + itm * (int64_t)tsz;
    if (vec) {
      for (int i = threadIdx.x; i < (tsz >> 2); i += blockDim.x) cp_async16(dst + 4 * i, src + 4 * i);
    } else {
      for (int i = threadIdx.x; i < tsz; i += blockDim.x) dst[i] = src[i];
    }
  };
  int cur = 0;
  fetch(blockIdx.x, tiles);
  cp_async_commit();
  for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
    float2* dst = out + item * (int64_t)(dx_n * dy_n);
    __syncthreads();                               // the other tile buffer is free again
    fetch(item + gridDim.x, tiles + (cur ^ 1) * ((tsz + 3) & ~3));
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();                               // this item's tile is in shared memory
    const float* tile = tiles + cur * ((tsz + 3) & ~3);
    // first stage (Ns = 1, unit twiddle) straight from the rows: z = P_a + i P_b
    for (int jj = threadIdx.x; jj < np * half; jj += blockDim.x) {
      const int pr = jj >> lh, j = jj & (half - 1);
      const int r = 2 * pr;
      const float* ra = tile + r * my;
      const bool two = r + 1 < mx;
      const float2 a = make_float2(ra[j], two ? ra[my + j] : 0.f);
      const float2 b = make_float2(ra[j + half], two ? ra[my + j + half] : 0.f);
      float2* dp = buf0 + pr * my;
      dp[2 * j] = make_float2(a.x + b.x, a.y + b.y);
      dp[2 * j + 1] = make_float2(a.x - b.x, a.y - b.y);
    }
    __syncthreads();
    float2* src = buf0;
    float2* dsb = buf1;
    for (int ns = 2, ls = 1; ns < my; ns <<= 1, ++ls) {
      for (int jj = threadIdx.x; jj < np * half; jj += blockDim.x) {
        const int pr = jj >> lh, j = jj & (half - 1);
        const float2* sp = src + pr * my;
        float2* dp = dsb + pr * my;
        const int k = j & (ns - 1);
        const float2 w = twp[k << (lh - ls)];
        const float2 a = sp[j], b0 = sp[j + half];
        const float2 b = make_float2(b0.x * w.x - b0.y * w.y, b0.x * w.y + b0.y * w.x);
        const int d = ((j - k) << 1) + k;
        dp[d] = make_float2(a.x + b.x, a.y + b.y);
        dp[d + ns] = make_float2(a.x - b.x, a.y - b.y);
      }
      __syncthreads();
      float2* t = src; src = dsb; dsb = t;
    }
    for (int A = 0; A < mx; ++A) {
      const int row = A & 1;
      const float2* z = src + (A >> 1) * my;
      for (int d = threadIdx.x; d < dy_n; d += blockDim.x) {
        const int lag = d - (ny - 1), k = lag < 0 ? -lag : lag;
        const float2 zk = z[k], zm = z[(my - k) & (my - 1)];
        float2 x = row == 0 ? make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y))
                            : make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
        if (lag < 0) x.y = -x.y;
        x.x *= iny;
        x.y *= iny;
        if (inv_x) q[A * dy_n + d] = x;
        else dst[A * dy_n + d] = x;
      }
    }
    if (inv_x) {
      __syncthreads();
      for (int o = threadIdx.x; o < dx_n * dy_n; o += blockDim.x) {
        const int e = o / dy_n, d = o - e * dy_n;
        const int lag = e - (nx - 1);
        const int lm = ((lag % mx) + mx) % mx;
        float2 v = make_float2(0.f, 0.f);
        int idx = 0;
        for (int A = 0; A < mx; ++A) {
          const float2 t = txs[idx], z = q[A * dy_n + d];
          v.x = fmaf(t.x, z.x, fmaf(-t.y, z.y, v.x));
          v.y = fmaf(t.x, z.y, fmaf(t.y, z.x, v.y));
          idx += lm;
          if (idx >= mx) idx -= mx;
        }
        dst[o] = make_float2(v.x * inx, v.y * inx);
      }
    }
    cur ^= 1;
  }
  cp_async_wait<0>();
}


// Warp route for My = 512 when the E-W index is kept (Mx < 2nx - 1, at most 4 row pairs):
// one warp per row pair, no CTA barrier inside the transform. The pair is transformed
// forward on the conjugate, Zc = DFT(P_a - i P_b), so Z = conj Zc, split N = 16 x 32 as in
// the 512-beam kernel (n = n2 + 16 n1, k = k1 + 32 k2): pass 1, lane (n2, h), is the
// 16-point DFT of (x[n1] + (-1)^h x[n1 + 16]) W32^(h n1), i.e. the outputs k1 = 2m + h of
// the 32-point DFT over n1, times W512^(n2 k1), stored transposed (row stride 17); pass 2,
// lane k1, is the 16-point DFT over n2. Zc goes to the warp's region and the two rows
// separate from Zc[k] and Zc[512 - k]:
//   X_a[k] = (conj Zc[k] + Zc[N-k]) / 2,   X_b[k] = (conj Zc[k] - Zc[N-k]) / 2i.
// A CTA of 8 warps takes 8 / pairs (window, channel) tiles per step; the tiles of the next
// step are fetched with cp.async meanwhile.
namespace vw {
constexpr int N = 512, NW = 8, REG = 32 * 17;
}

__global__ void __launch_bounds__(vw::NW * 32, 2)
stacked_vis_warp_kernel(const float* __restrict__ P, float2* __restrict__ out,
                        const float2* __restrict__ tw_y, int64_t nitems, int ny, int mx) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int N = vw::N;
  const int np = (mx + 1) >> 1;                    // row pairs per tile (1, 2 or 4)
  const int G = vw::NW / np;                       // tiles per step
  const int tsz = mx * N;                          // floats per tile
  const int dy_n = 2 * ny - 1;
  float* tiles = reinterpret_cast<float*>(smem);   // [2][G][Mx * N]
  float2* tw512 = reinterpret_cast<float2*>(tiles + 2 * G * tsz);   // [32 k1][16 n2] W512^(n2 k1)
  float2* tw32 = tw512 + 512;                      // [2 h][16 n1] W32^(h n1)
  float2* regs = tw32 + 32;                        // [NW][REG]
  for (int i = threadIdx.x; i < 512; i += blockDim.x) tw512[i] = tw_y[(i & 15) * (i >> 4)];
  for (int i = threadIdx.x; i < 32; i += blockDim.x) tw32[i] = tw_y[16 * (i >> 4) * (i & 15)];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int slot = warp / np, pair = warp - slot * np;
  float2* rg = regs + warp * vw::REG;
  const float inv = 1.0f / (float)N;
  const int64_t ngroups = (nitems + G - 1) / G;
  // tiles g*G .. g*G + G - 1 (those < nitems), 16-byte copies (the tiles are 2 KB multiples)
  auto fetch = [&](int64_t g, float* dst) {
    if (g >= ngroups) return;
    const int64_t i0 = g * G;
    const int ntile = (int)(nitems - i0 < G ? nitems - i0 : G);
    const float* src = P + i0 * (int64_t)tsz;
    for (int i = threadIdx.x; i < (ntile * tsz) >> 2; i += blockDim.x) cp_async16(dst + 4 * i, src + 4 * i);
  };
  int cur = 0;
  fetch(blockIdx.x, tiles);
  cp_async_commit();
  for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
    __syncthreads();                               // the other buffer is free again
    fetch(g + gridDim.x, tiles + (cur ^ 1) * G * tsz);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();                               // this step's tiles are in shared memory
    const int64_t item = g * G + slot;
    if (item < nitems) {
      const float* ra = tiles + cur * G * tsz + slot * tsz + 2 * pair * N;
      const bool two = 2 * pair + 1 < mx;
      // ---- pass 1: lane (n2, h)
      const int n2 = lane & 15, h = lane >> 4;
      const float sg = h ? -1.f : 1.f;
      float2 x[16];
#pragma unroll
      for (int n1 = 0; n1 < 16; ++n1) {
        const int i0 = n2 + 16 * n1, i1 = i0 + 256;
        const float2 u = make_float2(ra[i0], two ? -ra[N + i0] : 0.f);
        const float2 v = make_float2(ra[i1], two ? -ra[N + i1] : 0.f);
        x[n1] = cmul(make_float2(fmaf(sg, v.x, u.x), fmaf(sg, v.y, u.y)), tw32[h * 16 + n1]);
      }
      Dft<16>::run(x);
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const int k1 = 2 * m + h;
        rg[k1 * 17 + n2] = cmul(x[m], tw512[k1 * 16 + n2]);
      }
      __syncwarp();
      // ---- pass 2: lane k1; Zc[k1 + 32 k2] back into the region
      float2 y[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) y[q] = rg[lane * 17 + q];
      Dft<16>::run(y);
      __syncwarp();
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) rg[lane + 32 * k2] = y[k2];
      __syncwarp();
      // ---- separate the rows, lags -(ny-1) .. ny-1
      float2* da = out + item * (int64_t)(mx * dy_n) + (2 * pair) * dy_n;
      for (int d = lane; d < dy_n; d += 32) {
        const int lag = d - (ny - 1), k = lag < 0 ? -lag : lag;
        const float2 zk = rg[k], zm = rg[(N - k) & (N - 1)];
        float2 xa = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zm.y - zk.y));
        if (lag < 0) xa.y = -xa.y;
        da[d] = make_float2(xa.x * inv, xa.y * inv);
        if (two) {
          float2 xb = make_float2(-0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
          if (lag < 0) xb.y = -xb.y;
          da[dy_n + d] = make_float2(xb.x * inv, xb.y * inv);
        }
      }
    }
    cur ^= 1;
  }
  cp_async_wait<0>();
}

static size_t vis_warp_smem(int mx) {
  const int np = (mx + 1) >> 1, G = vw::NW / np;
  return sizeof(float) * 2 * (size_t)G * mx * vw::N + sizeof(float2) * (512 + 32 + (size_t)vw::NW * vw::REG);
}

}  // namespace fftbf

using namespace fftbf;

extern "C" {

int fftbf_stacked_shape(const fftbf_plan* p, int* dx, int* dy) {
  if (!p || !dx || !dy) return set_error(FFTBF_EINVAL, "null argument");
  *dx = p->mx >= 2 * p->nx - 1 ? 2 * p->nx - 1 : p->mx;
  *dy = p->my >= 2 * p->ny - 1 ? 2 * p->ny - 1 : p->my;
  return FFTBF_OK;
}

int fftbf_stacked_visibilities(fftbf_plan* p, const float* beams_dev, int64_t n_windows,
                               float* vis_dev, void* stream) {
  NvtxRange nvtx("fftbf_stacked_visibilities");
  if (!p) return set_error(FFTBF_EINVAL, "null plan");
  if (n_windows < 0) return set_error(FFTBF_EINVAL, "n_windows < 0");
  if (n_windows == 0) return FFTBF_OK;
  if (!beams_dev || !vis_dev) return set_error(FFTBF_EINVAL, "null buffer");
  const int inv_x = p->mx >= 2 * p->nx - 1, inv_y = p->my >= 2 * p->ny - 1;
  int dx = 0, dy = 0;
  fftbf_stacked_shape(p, &dx, &dy);
  // FFT route: N-S invertible and My a power of two (>= 2)
  const bool fft = inv_y && p->my >= 2 && (p->my & (p->my - 1)) == 0;
  const size_t smem_fft = sizeof(float) * 2 * (((size_t)p->mx * p->my + 3) & ~(size_t)3) +
                          sizeof(float2) * ((size_t)p->my / 2 + 2 * (size_t)((p->mx + 1) / 2) * p->my +
                                            (inv_x ? (size_t)p->mx * dy + p->mx : 0));
  const size_t smem = sizeof(float) * (((size_t)p->mx * p->my + 1) & ~(size_t)1) +
                      sizeof(float2) * ((size_t)p->my + p->mx + (size_t)p->mx * dy);
  const bool use_fft = fft && smem_fft <= 200 * 1024;
  // warp route: 512 N-S beams, E-W index kept, 1, 2 or 4 row pairs, 16-byte aligned beams
  const int np = (p->mx + 1) / 2;
  const bool use_warp = inv_y && !inv_x && p->my == 512 && (np == 1 || np == 2 || np == 4) &&
                        (reinterpret_cast<uintptr_t>(beams_dev) & 15) == 0 &&
                        vis_warp_smem(p->mx) <= 200 * 1024;
  if (!use_fft && smem > 200 * 1024)
    return set_error(FFTBF_EUNSUPPORTED, "beam tile too large for the stacking kernel");
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != p->device) cudaSetDevice(p->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t items = n_windows * p->nfreq;
  cudaError_t e;
  if (use_warp) {
    const size_t sm = vis_warp_smem(p->mx);
    e = cudaFuncSetAttribute(stacked_vis_warp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int per_sm = 0;
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stacked_vis_warp_kernel, vw::NW * 32, sm);
    if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
    const int64_t groups = (items + vw::NW / np - 1) / (vw::NW / np);
    const int64_t cap = (int64_t)p->nsm * per_sm;
    const int64_t grid = groups < cap ? groups : cap;
    if (e == cudaSuccess) {
      stacked_vis_warp_kernel<<<(unsigned)grid, vw::NW * 32, sm, st>>>(
          beams_dev, reinterpret_cast<float2*>(vis_dev), p->d_tw, items, p->ny, p->mx);
      e = cudaGetLastError();
    }
  } else if (use_fft) {
    e = cudaFuncSetAttribute(stacked_vis_fft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_fft);
    // resident CTAs per SM from shared memory (256 threads each, at most 8 by threads)
    int per_sm = (int)((200 * 1024) / (smem_fft + 1024));
    per_sm = per_sm < 1 ? 1 : (per_sm > 8 ? 8 : per_sm);
    const int64_t cap = (int64_t)p->nsm * per_sm;
    const int64_t grid = items < cap ? items : cap;
    if (e == cudaSuccess) {
      stacked_vis_fft_kernel<<<(unsigned)grid, 256, smem_fft, st>>>(
          beams_dev, reinterpret_cast<float2*>(vis_dev), p->d_tw, items, p->nx, p->ny, p->mx,
          p->my, inv_x);
      e = cudaGetLastError();
    }
  } else {
    e = cudaFuncSetAttribute(stacked_vis_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int64_t grid = items < (int64_t)p->nsm * 4 ? items : (int64_t)p->nsm * 4;
    if (e == cudaSuccess) {
      stacked_vis_kernel<<<(unsigned)grid, 256, smem, st>>>(beams_dev, reinterpret_cast<float2*>(vis_dev),
                                                            p->d_tw, items, p->nx, p->ny, p->mx,
                                                            p->my, inv_x, inv_y);
      e = cudaGetLastError();
    }
  }
  if (prev != p->device) cudaSetDevice(prev);
  if (e != cudaSuccess) return cuda_error(e, "fftbf_stacked_visibilities");
  return FFTBF_OK;
}

}  // extern "C"

// FP32 form, one warp per N-S transform, for N = 32 R beams (R = 4, 8, 16, 32, i.e. 128 to
// 1024 beams) over at most N/2 feeds (the zero padding of Eq. b2n-1), any E-W size up to
// 8. It generalises the 512-beam kernel: N = 32 x R Cooley-Tukey with n = n2 + R n1 and
// k = k1 + 32 k2, inputs with n1 >= 16 being the padding.
//   pass 1: X1[n2][k1] = sum_{n1 < 16} x[n2 + R n1] W32^(n1 k1). The 32 outputs k1 of one
//     n2 split into H = 32 / D classes k1 = H m + h, D = min(R, 16): class h is a D-point
//     DFT of the inputs pre-twiddled by W32^(n1 h) and folded modulo D. A lane owns one
//     (n2, h) pair (R <= 16) or both classes of one n2 (R = 32). Then X1 *= W_N^(n2 k1)
//     and the tile is stored transposed, [k1][n2] with row stride R + 1.
//   pass 2: lane k1, an R-point DFT over n2 gives X[k1 + 32 k2]; its |.|^2 goes into
//     per-lane accumulators (Eq. bf), so no complex beam leaves the SM.
// A CTA has 8 warps and runs S snapshots per step (S MX a multiple of 8, so each warp
// owns the same J = S MX / 8 transforms every step); at the end of a window the partial
// sums of the S snapshot slots are added in a fixed order. Only warp-level
// synchronisation inside the transforms; two CTA barriers per step.
#pragma once

#include "beam_fp32.cuh"

namespace fftbf {

// W32^k = exp(-2 pi i k / 32), k < 16.
__device__ __forceinline__ float2 w32c(int k) {
  const float2 w[16] = {
      {1.000000000e+00f, -0.000000000e+00f}, {9.807852804e-01f, -1.950903220e-01f},
      {9.238795325e-01f, -3.826834324e-01f}, {8.314696123e-01f, -5.555702330e-01f},
      {7.071067812e-01f, -7.071067812e-01f}, {5.555702330e-01f, -8.314696123e-01f},
      {3.826834324e-01f, -9.238795325e-01f}, {1.950903220e-01f, -9.807852804e-01f},
      {0.000000000e+00f, -1.000000000e+00f}, {-1.950903220e-01f, -9.807852804e-01f},
      {-3.826834324e-01f, -9.238795325e-01f}, {-5.555702330e-01f, -8.314696123e-01f},
      {-7.071067812e-01f, -7.071067812e-01f}, {-8.314696123e-01f, -5.555702330e-01f},
      {-9.238795325e-01f, -3.826834324e-01f}, {-9.807852804e-01f, -1.950903220e-01f}};
  return w[k];
}

// 32-point DFT as two 16-point DFTs and one radix-2 combination.
template <> struct Dft<32> {
  __device__ __forceinline__ static void run(float2* v) {
    float2 e[16], o[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      e[k] = v[2 * k];
      o[k] = v[2 * k + 1];
    }
    Dft<16>::run(e);
    Dft<16>::run(o);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const float2 t = k == 0 ? o[0] : (k == 8 ? mul_mi(o[8]) : cmul(o[k], w32c(k)));
      v[k] = cadd(e[k], t);
      v[k + 16] = csub(e[k], t);
    }
  }
};

namespace wt {
constexpr int kWarps = 8;
__host__ __device__ constexpr int gcd8(int m) {
  return m % 8 == 0 ? 8 : (m % 4 == 0 ? 4 : (m % 2 == 0 ? 2 : 1));
}
}  // namespace wt

template <int MX, int R> struct WarpCfg {
  static constexpr int N = 32 * R;
  static constexpr int S = wt::kWarps / wt::gcd8(MX);   // snapshots per step
  static constexpr int J = MX / wt::gcd8(MX);           // transforms per warp per step
  static constexpr int REG = 32 * (R + 1);              // float2 slots per transform region
  static constexpr int D = R < 16 ? R : 16;             // pass-1 DFT length
  static constexpr int H = 32 / D;                      // k1 classes per n2
};

// Physical row of tile row x (x < 32) in a transform region of rows of R complex values:
// for R <= 8 a warp's stores cover 32 / R consecutive rows (E-W stage: input rows n1;
// pass 1: rows k1 = H m + h of one m), which the row stride R + 1 would put in shared
// banks; x / (32 / R) + R (x mod 32 / R) spreads them so that every bank takes two words.
// Pass 2 then reads physical row `lane`, which holds k1 = prow_inv(lane).
template <int R>
__device__ __forceinline__ int prow(int x) {
  if constexpr (R <= 8) return x / (32 / R) + R * (x % (32 / R));
  else return x;
}
template <int R>
__device__ __forceinline__ int prow_inv(int y) {
  if constexpr (R <= 8) return (32 / R) * (y % R) + y / R;
  else return y;
}

// FULL: the lattice is MX x NH feeds, all live, with an MX-point E-W DFT (the radix-3
// butterfly for MX = 3) and 16-byte aligned voltages, i.e. exactly 2x N-S padding: its
// sizes are compile-time constants.
__host__ __device__ inline bool warp_full(const BeamArgs& a, int nh) {
  return a.nx == a.mx && a.ny == nh && a.nyf == nh && (a.ew_dft || a.mx == 3) &&
         (reinterpret_cast<uintptr_t>(a.volts) & 15) == 0;
}

// Weight x unpacked byte; real weights in one packed multiply of both parts (the same
// roundings as the complex product with a zero imaginary part).
__device__ __forceinline__ float2 weigh(bool real_w, float2 w, uint8_t b) {
  const float2 x = unpack_byte(b);
  return real_w ? __fmul2_rn(make_float2(w.x, w.x), x) : cmul(w, x);
}

// Unpack x weight and E-W transform of S snapshots into per-transform regions:
// region (s MX + A), slot (iy mod R) + stride (iy / R), for the feeds iy < NH (zeros
// past nyf and past the last snapshot).
template <int MX, int R, int NH, bool FULL = false>
__device__ __forceinline__ void warp_ew_stage(const BeamArgs& a, const uint8_t* raw, int S, int it,
                                              int nsnap, int nant, const float2* wsm,
                                              const float2* exsm, float2* regs, int reg,
                                              int stride) {
  const int ny = FULL ? NH : a.ny;
  const int nyf = FULL ? NH : a.nyf;
  const bool rw = a.real_w != 0;
  if constexpr (FULL && MX <= 4 && R >= 2) {
    // two adjacent feeds per thread: one 16-bit byte load and one 128-bit load of two
    // weights per E-W row; the pair lands in adjacent slots (iy even, rows of R >= 2)
    auto ew = [&](float2* z) {
      if constexpr (MX == 3) {
        // 3-point DFT: X_{1,2} = z0 - (z1 + z2)/2 -/+ i (sqrt(3)/2)(z1 - z2)
        const float2 z0 = z[0], sm = cadd(z[1], z[2]), df = csub(z[1], z[2]);
        const float h3 = 0.86602540378443865f;
        const float2 m = make_float2(z0.x - 0.5f * sm.x, z0.y - 0.5f * sm.y);
        const float2 t = make_float2(h3 * df.y, -h3 * df.x);
        z[0] = cadd(z0, sm);
        z[1] = cadd(m, t);
        z[2] = csub(m, t);
      } else {
        Dft<MX>::run(z);
      }
    };
    for (int c = threadIdx.x; c < S * (NH / 2); c += kThreads) {
      const int s = c / (NH / 2), iy = 2 * (c - s * (NH / 2));
      float2 z0[MX], z1[MX];
#pragma unroll
      for (int A = 0; A < MX; ++A) z0[A] = z1[A] = czero();
      if (it * S + s < nsnap) {
        const uint8_t* rs = raw + s * nant;
#pragma unroll
        for (int ix = 0; ix < MX; ++ix) {
          const unsigned v = *reinterpret_cast<const uint16_t*>(rs + ix * NH + iy);
          const float4 w = *reinterpret_cast<const float4*>(wsm + ix * NH + iy);
          z0[ix] = weigh(rw, make_float2(w.x, w.y), (uint8_t)(v & 255u));
          z1[ix] = weigh(rw, make_float2(w.z, w.w), (uint8_t)(v >> 8));
        }
        ew(z0);
        ew(z1);
      }
      const int slot = (iy % R) + stride * prow<R>(iy / R);
#pragma unroll
      for (int A = 0; A < MX; ++A) {
        regs[(s * MX + A) * reg + slot] = z0[A];
        regs[(s * MX + A) * reg + slot + 1] = z1[A];
      }
    }
    return;
  }
  for (int c = threadIdx.x; c < S * NH; c += kThreads) {
    const int s = c / NH, iy = c - s * NH;
    float2 z[MX];
#pragma unroll
    for (int A = 0; A < MX; ++A) z[A] = czero();
    if (iy < nyf && it * S + s < nsnap) {
      const uint8_t* rs = raw + s * nant;
      if constexpr (MX == 1 || MX == 2 || MX == 4 || MX == 8 || MX == 16) {
        if (FULL || a.ew_dft) {
#pragma unroll
          for (int ix = 0; ix < MX; ++ix) z[ix] = weigh(rw, wsm[ix * ny + iy], rs[ix * ny + iy]);
          Dft<MX>::run(z);
        }
      }
      bool done = false;
      if constexpr (MX == 3) {
        if (FULL || a.nx == 3) {
          // 3-point DFT: X_{1,2} = z0 - (z1 + z2)/2 -/+ i (sqrt(3)/2)(z1 - z2)
          const float2 z0 = weigh(rw, wsm[iy], rs[iy]);
          const float2 z1 = weigh(rw, wsm[ny + iy], rs[ny + iy]);
          const float2 z2 = weigh(rw, wsm[2 * ny + iy], rs[2 * ny + iy]);
          const float2 sm = cadd(z1, z2), df = csub(z1, z2);
          const float h3 = 0.86602540378443865f;
          const float2 m = make_float2(z0.x - 0.5f * sm.x, z0.y - 0.5f * sm.y);
          const float2 t = make_float2(h3 * df.y, -h3 * df.x);
          z[0] = cadd(z0, sm);
          z[1] = cadd(m, t);
          z[2] = csub(m, t);
          done = true;
        }
      }
      if (!FULL && !a.ew_dft && !done) {
        for (int ix = 0; ix < a.nx; ++ix) {
          const float2 col = cmul(wsm[ix * ny + iy], unpack_byte(rs[ix * ny + iy]));
#pragma unroll
          for (int A = 0; A < MX; ++A) z[A] = cadd(z[A], cmul(exsm[A * a.nx + ix], col));
        }
      }
    }
    const int slot = (iy % R) + stride * prow<R>(iy / R);
#pragma unroll
    for (int A = 0; A < MX; ++A) regs[(s * MX + A) * reg + slot] = z[A];
  }
}

// Shared-memory bytes of one item of the warp path.
__host__ __device__ inline size_t warp_item_smem(int S, int mx, int nx, int ny, int R) {
  const size_t nant = (size_t)nx * ny;
  const size_t rawsz = ((size_t)S * nant + 15) & ~(size_t)15;
  return 2 * rawsz + sizeof(float2) * (nant + (size_t)mx * nx + 32 * (size_t)R + 32 +
                                       (size_t)S * mx * 32 * (R + 1));
}

// One work item (window, channel): all its snapshots, S per step, bytes double-buffered
// through cp.async. 256 threads. a.S must be WarpCfg<MX, R>::S and a.nyf <= N/2; FULL
// only where warp_full(a, N/2) holds.
template <int MX, int R, bool FULL = false>
__device__ __forceinline__ void warp_item(const BeamArgs& a, int64_t item, unsigned char* smem,
                                          bool load_tables) {
  using C = WarpCfg<MX, R>;
  constexpr int N = C::N, S = C::S, J = C::J, REG = C::REG, D = C::D, H = C::H;
  const int nant = FULL ? MX * (N / 2) : a.nx * a.ny;
  const int rawsz = (S * nant + 15) & ~15;
  float2* wsm = reinterpret_cast<float2*>(smem + 2 * rawsz);
  float2* exsm = wsm + nant;
  float2* twk = exsm + MX * a.nx;          // [k1 32][n2 R] W_N^(n2 k1)
  float2* w32 = twk + 32 * R;              // [32] W32^m
  float2* regs = w32 + 32;                 // [S * MX][REG]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nsnap = a.n_int * a.npol;
  const int niter = (nsnap + S - 1) / S;
  const bool vec16 =
      FULL || (((nant & 15) == 0) && ((reinterpret_cast<uintptr_t>(a.volts) & 15) == 0));
  if (load_tables) {
    for (int i = threadIdx.x; i < nant; i += kThreads) wsm[i] = a.w[i];
    for (int i = threadIdx.x; i < MX * a.nx; i += kThreads) exsm[i] = a.ex[i];
    for (int i = threadIdx.x; i < 32 * R; i += kThreads) twk[i] = a.tw[(i % R) * (i / R)];
    for (int i = threadIdx.x; i < 32; i += kThreads) w32[i] = a.tw[i * R];
  }
  float acc[J][R];
#pragma unroll
  for (int j = 0; j < J; ++j)
#pragma unroll
    for (int k = 0; k < R; ++k) acc[j][k] = 0.f;

  const uint8_t* ivol = item_volts(a, item, nant);
  stage_bytes(a, smem, ivol, 0, nsnap, nant, vec16);
  cp_async_commit();
  for (int it = 0; it < niter; ++it) {
    if (it + 1 < niter) stage_bytes(a, smem + ((it + 1) & 1) * rawsz, ivol, it + 1, nsnap, nant, vec16);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();                                  // bytes of `it` visible; regions free
    // ---- unpack x weight, E-W transform -> region (s MX + A), slot (iy mod R) + (R+1)(iy / R)
    warp_ew_stage<MX, R, N / 2, FULL>(a, smem + (it & 1) * rawsz, S, it, nsnap, nant, wsm, exsm, regs,
                                REG, R + 1);
    __syncthreads();                                  // regions written
#pragma unroll
    for (int j = 0; j < J; ++j) {
      float2* rg = regs + (warp + wt::kWarps * j) * REG;
      // ---- pass 1
      if constexpr (R <= 16) {
        const int n2 = lane % R, h = lane / R;
        float2 y[D];
#pragma unroll
        for (int q = 0; q < D; ++q) y[q] = czero();
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1)
          y[n1 % D] = cadd(y[n1 % D], cmul(rg[n2 + (R + 1) * prow<R>(n1)], w32[(n1 * h) & 31]));
        Dft<D>::run(y);
        __syncwarp();
#pragma unroll
        for (int m = 0; m < D; ++m) {
          const int k1 = H * m + h;
          rg[prow<R>(k1) * (R + 1) + n2] = cmul(y[m], twk[k1 * R + n2]);
        }
      } else {
        const int n2 = lane;
        float2 x[16];
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) x[n1] = rg[n2 + (R + 1) * n1];
        __syncwarp();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float2 y[16];
#pragma unroll
          for (int n1 = 0; n1 < 16; ++n1) y[n1] = h ? cmul(x[n1], w32[n1]) : x[n1];
          Dft<16>::run(y);
#pragma unroll
          for (int m = 0; m < 16; ++m) {
            const int k1 = 2 * m + h;
            rg[k1 * (R + 1) + n2] = cmul(y[m], twk[k1 * R + n2]);
          }
        }
      }
      __syncwarp();
      // ---- pass 2: lane k1
      {
        float2 v[R];
#pragma unroll
        for (int q = 0; q < R; ++q) v[q] = rg[lane * (R + 1) + q];
        Dft<R>::run(v);
#pragma unroll
        for (int k2 = 0; k2 < R; ++k2) acc[j][k2] = fmaf(v[k2].x, v[k2].x, fmaf(v[k2].y, v[k2].y, acc[j][k2]));
      }
    }
  }
  // ---- window complete: add the S snapshot slots of each E-W beam in order, write once
  float* dst = a.beams + item * (int64_t)(MX * N);
  const int k1o = prow_inv<R>(lane);              // the k1 this lane's pass 2 produced
  if constexpr (S == 1 && J == 1) {
#pragma unroll
    for (int k2 = 0; k2 < R; ++k2) dst[warp * N + k1o + 32 * k2] = acc[0][k2];
    __syncthreads();
  } else {
    __syncthreads();
    float* red = reinterpret_cast<float*>(regs);
#pragma unroll
    for (int j = 0; j < J; ++j)
#pragma unroll
      for (int k2 = 0; k2 < R; ++k2) red[(warp + wt::kWarps * j) * N + k1o + 32 * k2] = acc[j][k2];
    __syncthreads();
    for (int o = threadIdx.x; o < MX * N; o += kThreads) {
      const int A = o / N, k = o - A * N;
      float sum = 0.f;
#pragma unroll
      for (int s = 0; s < S; ++s) sum += red[(s * MX + A) * N + k];
      dst[o] = sum;
    }
    __syncthreads();
  }
}

// ---- 2048 beams (N = 32 x 64): two warps per transform --------------------------------
// Warp g of a pair runs pass 1 for n2 = 32 g + lane (both classes h of a 16-point DFT over
// the 16 nonzero n1), the pair meets on a named barrier, and in pass 2 warp g takes the
// outputs k2 = 2 m + g: X[k1 + 32 k2] = sum_{n2 < 32} u_g[n2] W32^(n2 m) with
// u_0 = T[n2] + T[n2 + 32] and u_1 = (T[n2] - T[n2 + 32]) W64^n2 (a radix-2 split of the
// 64-point DFT over n2), so each lane keeps 32 accumulators.
template <int MX> struct Warp2Cfg {
  static constexpr int N = 2048, R = 64, S = 4 / MX, REG = 32 * (R + 1);
};
__host__ __device__ inline size_t warp2_item_smem(int S, int mx, int nx, int ny) {
  const size_t nant = (size_t)nx * ny;
  const size_t rawsz = ((size_t)S * nant + 15) & ~(size_t)15;
  return 2 * rawsz + sizeof(float2) * (nant + (size_t)mx * nx + 32 * 64 + 32 + 32 +
                                       (size_t)S * mx * 32 * 65);
}

template <int MX, bool FULL = false>
__device__ __forceinline__ void warp2_item(const BeamArgs& a, int64_t item, unsigned char* smem,
                                           bool load_tables) {
  using C = Warp2Cfg<MX>;
  constexpr int N = C::N, R = C::R, S = C::S, REG = C::REG;
  const int nant = FULL ? MX * 1024 : a.nx * a.ny;
  const int rawsz = (S * nant + 15) & ~15;
  float2* wsm = reinterpret_cast<float2*>(smem + 2 * rawsz);
  float2* exsm = wsm + nant;
  float2* twk = exsm + MX * a.nx;          // [k1 32][n2 64] W_N^(n2 k1)
  float2* w32 = twk + 32 * R;              // [32] W32^m
  float2* w64 = w32 + 32;                  // [32] W64^n
  float2* regs = w64 + 32;                 // [S * MX][REG]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int pair = warp >> 1, g = warp & 1;
  const int nsnap = a.n_int * a.npol;
  const int niter = (nsnap + S - 1) / S;
  const bool vec16 =
      FULL || (((nant & 15) == 0) && ((reinterpret_cast<uintptr_t>(a.volts) & 15) == 0));
  if (load_tables) {
    for (int i = threadIdx.x; i < nant; i += kThreads) wsm[i] = a.w[i];
    for (int i = threadIdx.x; i < MX * a.nx; i += kThreads) exsm[i] = a.ex[i];
    for (int i = threadIdx.x; i < 32 * R; i += kThreads) twk[i] = a.tw[(i % R) * (i / R)];
    for (int i = threadIdx.x; i < 32; i += kThreads) {
      w32[i] = a.tw[i * 64];
      w64[i] = a.tw[i * 32];
    }
  }
  float acc[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) acc[k] = 0.f;
  const uint8_t* ivol = item_volts(a, item, nant);
  stage_bytes(a, smem, ivol, 0, nsnap, nant, vec16);
  cp_async_commit();
  for (int it = 0; it < niter; ++it) {
    if (it + 1 < niter) stage_bytes(a, smem + ((it + 1) & 1) * rawsz, ivol, it + 1, nsnap, nant, vec16);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    warp_ew_stage<MX, R, N / 2, FULL>(a, smem + (it & 1) * rawsz, S, it, nsnap, nant, wsm, exsm, regs,
                                REG, R + 1);
    __syncthreads();
    float2* rg = regs + pair * REG;          // transform `pair` of this step
    {
      const int n2 = 32 * g + lane;
      float2 x[16];
#pragma unroll
      for (int n1 = 0; n1 < 16; ++n1) x[n1] = rg[n2 + (R + 1) * n1];
      __syncwarp();
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float2 y[16];
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) y[n1] = h ? cmul(x[n1], w32[n1]) : x[n1];
        Dft<16>::run(y);
#pragma unroll
        for (int m = 0; m < 16; ++m) {
          const int k1 = 2 * m + h;
          rg[k1 * (R + 1) + n2] = cmul(y[m], twk[k1 * R + n2]);
        }
      }
    }
    asm volatile("bar.sync %0, %1;\n" ::"r"(1 + pair), "r"(64) : "memory");
    {
      float2 u[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const float2 lo = rg[lane * (R + 1) + q], hi = rg[lane * (R + 1) + q + 32];
        u[q] = g == 0 ? cadd(lo, hi) : cmul(csub(lo, hi), w64[q]);
      }
      Dft<32>::run(u);
#pragma unroll
      for (int m = 0; m < 32; ++m) acc[m] = fmaf(u[m].x, u[m].x, fmaf(u[m].y, u[m].y, acc[m]));
    }
  }
  // ---- window complete: slot (pair) holds (s, A) = (pair / MX, pair % MX)
  __syncthreads();
  float* red = reinterpret_cast<float*>(regs);
#pragma unroll
  for (int m = 0; m < 32; ++m) red[pair * N + lane + 32 * (2 * m + g)] = acc[m];
  __syncthreads();
  float* dst = a.beams + item * (int64_t)(MX * N);
  for (int o = threadIdx.x; o < MX * N; o += kThreads) {
    const int A = o / N, k = o - A * N;
    float sum = 0.f;
#pragma unroll
    for (int s = 0; s < S; ++s) sum += red[(s * MX + A) * N + k];
    dst[o] = sum;
  }
  __syncthreads();
}

// ---- 32 beams over at most 16 feeds, 16 E-W beams: one lane per transform ------------
// 256 transforms per step (S = 16 snapshots x 16 E-W beams); lane t reads its 16 inputs
// (row stride 17) and forms the 32 outputs as two 16-point DFTs (inputs x and x W32^n),
// squaring them into 32 accumulators.
constexpr int kLaneS = 16;
__host__ __device__ inline size_t lane_item_smem(int nx, int ny) {
  const size_t nant = (size_t)nx * ny;
  const size_t rawsz = ((size_t)kLaneS * nant + 15) & ~(size_t)15;
  return 2 * rawsz + sizeof(float2) * (nant + (size_t)16 * nx + (size_t)kLaneS * 16 * 17);
}

template <bool FULL = false>
__device__ __forceinline__ void lane_item16(const BeamArgs& a, int64_t item, unsigned char* smem,
                                            bool load_tables) {
  constexpr int MX = 16, N = 32, S = kLaneS, REG = 17;
  const int nant = FULL ? 256 : a.nx * a.ny;
  const int rawsz = (S * nant + 15) & ~15;
  float2* wsm = reinterpret_cast<float2*>(smem + 2 * rawsz);
  float2* exsm = wsm + nant;
  float2* regs = exsm + MX * a.nx;         // [S * MX][17]
  const int t = threadIdx.x;               // transform (s, A) = (t / 16, t % 16)
  const int nsnap = a.n_int * a.npol;
  const int niter = (nsnap + S - 1) / S;
  const bool vec16 =
      FULL || (((nant & 15) == 0) && ((reinterpret_cast<uintptr_t>(a.volts) & 15) == 0));
  if (load_tables) {
    for (int i = threadIdx.x; i < nant; i += kThreads) wsm[i] = a.w[i];
    for (int i = threadIdx.x; i < MX * a.nx; i += kThreads) exsm[i] = a.ex[i];
  }
  float acc[N];
#pragma unroll
  for (int k = 0; k < N; ++k) acc[k] = 0.f;
  const uint8_t* ivol = item_volts(a, item, nant);
  stage_bytes(a, smem, ivol, 0, nsnap, nant, vec16);
  cp_async_commit();
  for (int it = 0; it < niter; ++it) {
    if (it + 1 < niter) stage_bytes(a, smem + ((it + 1) & 1) * rawsz, ivol, it + 1, nsnap, nant, vec16);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    warp_ew_stage<MX, 16, 16, FULL>(a, smem + (it & 1) * rawsz, S, it, nsnap, nant, wsm, exsm, regs, REG, 17);
    __syncthreads();
    float2 x[16];
#pragma unroll
    for (int n = 0; n < 16; ++n) x[n] = regs[t * REG + n];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float2 y[16];
#pragma unroll
      for (int n = 0; n < 16; ++n) y[n] = h ? cmul(x[n], w32c(n)) : x[n];
      Dft<16>::run(y);
#pragma unroll
      for (int m = 0; m < 16; ++m)
        acc[2 * m + h] = fmaf(y[m].x, y[m].x, fmaf(y[m].y, y[m].y, acc[2 * m + h]));
    }
  }
  __syncthreads();
  float* red = reinterpret_cast<float*>(regs);
#pragma unroll
  for (int k = 0; k < N; ++k) red[t * N + k] = acc[k];
  __syncthreads();
  float* dst = a.beams + item * (int64_t)(MX * N);
  for (int o = threadIdx.x; o < MX * N; o += kThreads) {
    const int A = o / N, k = o - A * N;
    float sum = 0.f;
#pragma unroll
    for (int s = 0; s < S; ++s) sum += red[(s * MX + A) * N + k];
    dst[o] = sum;
  }
  __syncthreads();
}

// Standalone launch for fftbf_execute (beam_fp32_warp.cu): 128..1024 beams (one warp per
// transform), 2048 beams (a warp pair per transform), 32 beams x 16 E-W (a lane each).
bool fp32_warp_supported(const BeamArgs& a);
int launch_beams_fp32_warp(const BeamArgs& a, int nsm, cudaStream_t st);

}  // namespace fftbf

// FP32 CUDA-core form of the FFT-beam hot path (K1 unpack + K2 fused transform).
//
// One CTA owns one (window j, frequency f) work item at a time and loops over its
// n_int * npol snapshots, S snapshots per iteration:
//   1. the bytes of the next iteration are staged into shared memory with cp.async
//      (16-byte copies, double-buffered) while the current one is transformed;
//   2. unpack (exact nibble decode) x apodisation weight, cyclic N-S fold if my < ny,
//      and the E-W transform of each column (a radix butterfly when mx == nx is a power
//      of two, else the folded DFT matrix) -> Z[s][A][iy] in shared memory;
//   3. N-S transform of length my = 2^LOG2N as mixed-radix Stockham stages in shared
//      memory, the first stage pruned when half of its inputs are zero padding
//      (Section 3.2);
//   4. the last stage keeps its outputs in registers, squares them and adds them to
//      per-thread accumulators (Eq. bf): no complex beam leaves the SM.
// At the end of the window the S partial sums are added in a fixed order and written
// once. The accumulation order depends only on the work item, so results are
// bit-identical whatever else runs in the same launch.
//
// The radix plan is a compile-time function of LOG2N, so every index of every stage is
// static and the accumulators stay in registers.
#pragma once

#include <cuda_runtime.h>

#include "internal.cuh"

namespace fftbf {

// ---------------------------------------------------------------- complex helpers --
// Packed two-lane FP32 (add / fma .f32x2 of sm_100 and later): one instruction per complex
// add; a - b as fma(b, -1, a), which rounds exactly as the subtraction does, so the sums are
// bit-identical to scalar code while taking half the issue slots.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }  // * (-i)
__device__ __forceinline__ float2 czero() { return make_float2(0.f, 0.f); }

// Exact int4 -> float: 2^23 + (n ^ 8) is representable, subtracting 2^23 + 8 leaves the
// two's-complement value of the nibble n.
__device__ __forceinline__ float nib(unsigned n) {
  return __int_as_float(0x4B000000u | (n ^ 8u)) - 8388616.0f;
}
__device__ __forceinline__ float2 unpack_byte(unsigned b) {
  // both nibbles' subtractions as one packed add (the same roundings: exact)
  return __fadd2_rn(make_float2(__int_as_float(0x4B000000u | (((b >> 4) & 15u) ^ 8u)),
                                __int_as_float(0x4B000000u | ((b & 15u) ^ 8u))),
                    make_float2(-8388616.0f, -8388616.0f));
}

// ------------------------------------------------------ forward DFTs in registers --
// v[k] <- sum_r v[r] exp(-2 pi i r k / R).
template <int R> struct Dft;
template <> struct Dft<1> { __device__ __forceinline__ static void run(float2*) {} };
template <> struct Dft<2> {
  __device__ __forceinline__ static void run(float2* v) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};
template <> struct Dft<4> {
  __device__ __forceinline__ static void run(float2* v) {
    // d = v1 - v3; v1' = d02 - i d = d02 + (d.y, -d.x), v3' = d02 + (-d.y, d.x): one fma
    // each on the swapped pair (d.y, d.x), exact multiplies by +-1
    float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    float2 s13 = cadd(v[1], v[3]), d = csub(v[1], v[3]);
    const float2 dsw = make_float2(d.y, d.x);
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    v[1] = __ffma2_rn(dsw, make_float2(1.f, -1.f), d02);
    v[3] = __ffma2_rn(dsw, make_float2(-1.f, 1.f), d02);
  }
};
constexpr float kRs2 = 0.70710678118654752440f;
__device__ __forceinline__ float2 mul_w8(float2 a) {   // * exp(-i pi/4)
  return make_float2((a.x + a.y) * kRs2, (a.y - a.x) * kRs2);
}
__device__ __forceinline__ float2 mul_w83(float2 a) {  // * exp(-3i pi/4)
  return make_float2((a.y - a.x) * kRs2, -(a.x + a.y) * kRs2);
}
template <> struct Dft<8> {
  __device__ __forceinline__ static void run(float2* v) {
    float2 e[4] = {v[0], v[2], v[4], v[6]};
    float2 o[4] = {v[1], v[3], v[5], v[7]};
    Dft<4>::run(e);
    Dft<4>::run(o);
    o[1] = mul_w8(o[1]);
    o[2] = mul_mi(o[2]);
    o[3] = mul_w83(o[3]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[k] = cadd(e[k], o[k]);
      v[k + 4] = csub(e[k], o[k]);
    }
  }
};
template <> struct Dft<16> {
  __device__ __forceinline__ static void run(float2* v) {
    // 16 = 4 x 4: inner DFT4 over n1 (stride 4), twiddle W16^(n2 k1), outer DFT4 over n2.
    const float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f;
    float2 a[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
#pragma unroll
      for (int n1 = 0; n1 < 4; ++n1) a[n2][n1] = v[4 * n1 + n2];
      Dft<4>::run(a[n2]);
    }
    const float2 w[10] = {{1.f, 0.f}, {c1, -s1}, {kRs2, -kRs2}, {s1, -c1}, {0.f, -1.f},
                          {-s1, -c1}, {-kRs2, -kRs2}, {-c1, -s1}, {-1.f, 0.f}, {-c1, s1}};
    // W16^4 = -i is a swap (the complex multiply by (0, -1) gives the same values up to the
    // sign of a zero, which no later sum or square can turn into a different magnitude)
#pragma unroll
    for (int n2 = 1; n2 < 4; ++n2)
#pragma unroll
      for (int k1 = 1; k1 < 4; ++k1)
        a[n2][k1] = n2 * k1 == 4 ? mul_mi(a[n2][k1]) : cmul(a[n2][k1], w[n2 * k1]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      float2 b[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
      Dft<4>::run(b);
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = b[k2];
    }
  }
};

// DFT of length R whose inputs r >= R/2 are zero (first stage of a 2x zero-padded axis).
template <int R> struct DftHalf;
template <> struct DftHalf<1> { __device__ __forceinline__ static void run(float2*) {} };
template <> struct DftHalf<2> {
  __device__ __forceinline__ static void run(float2* v) { v[1] = v[0]; }
};
template <> struct DftHalf<4> {
  __device__ __forceinline__ static void run(float2* v) {
    float2 x0 = v[0], x1 = v[1], mi = mul_mi(x1);
    v[0] = cadd(x0, x1);
    v[2] = csub(x0, x1);
    v[1] = cadd(x0, mi);
    v[3] = csub(x0, mi);
  }
};
template <> struct DftHalf<8> {
  __device__ __forceinline__ static void run(float2* v) {
    // y[k] = a[k mod 4] + W8^k b[k mod 4], a_k = x0 + (-i)^k x2, b_k = x1 + (-i)^k x3
    float2 a[4], b[4];
    float2 m2 = mul_mi(v[2]), m3 = mul_mi(v[3]);
    a[0] = cadd(v[0], v[2]); a[2] = csub(v[0], v[2]);
    a[1] = cadd(v[0], m2);   a[3] = csub(v[0], m2);
    b[0] = cadd(v[1], v[3]); b[2] = csub(v[1], v[3]);
    b[1] = cadd(v[1], m3);   b[3] = csub(v[1], m3);
    b[1] = mul_w8(b[1]);
    b[2] = mul_mi(b[2]);
    b[3] = mul_w83(b[3]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[k] = cadd(a[k], b[k]);
      v[k + 4] = csub(a[k], b[k]);
    }
  }
};

// Shared-memory layout of a transform: one float2 of padding after every 16, so the
// stride-R writes of the first Stockham stage and the stride-16 reads of the next stages
// fall in distinct banks. A transform of length N occupies N + N/16 slots.
__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }
template <int N> struct Tstride { static constexpr int v = N + (N >> 4); };

// ------------------------------------------------------------ static radix plan --
// N = 2^LOG2N; the small radix (2 or 4) goes first so the last stage is radix 8.
template <int LOG2N> struct FftPlan {
  static constexpr int N = 1 << LOG2N;
  static constexpr int NST = LOG2N == 0 ? 1 : (LOG2N + 2) / 3;
  static constexpr int LR0 = LOG2N == 0 ? 0 : (LOG2N % 3 == 0 ? 3 : LOG2N % 3);
  static constexpr int R0 = 1 << LR0;
  static constexpr int RL = NST == 1 ? R0 : 8;
  static constexpr int LRL = NST == 1 ? LR0 : 3;
};

// ----------------------------------------------------------- Stockham FFT stages --
// One radix-R stage over `ntr` transforms of length N stored back to back in buf.
// Butterfly j of a transform reads in[j + r N/R], applies W_N^(r k N/(Ns R)) with
// k = j mod Ns, runs the radix-R DFT and writes out[(j/Ns) Ns R + k + r Ns]; the
// register round trip makes the stage in-place. FIRST: Ns = 1, inputs past nyf read as
// zero. PRUNE: FIRST with nyf <= N/2. LAST: outputs are squared into acc instead.
template <int R, int LR, bool FIRST, bool PRUNE, bool LAST, int LOG2N, int LOG2NS>
__device__ __forceinline__ void fft_stage(float2* buf, int ntr, int nyf, const float2* tw,
                                          float* acc) {
  constexpr int MAXB = kMaxElems / kThreads / R;
  constexpr int LOG2BPT = LOG2N - LR;              // butterflies per transform = N / R
  constexpr int STEP = LOG2N - LOG2NS - LR;        // twiddle W_N^(r k 2^STEP)
  constexpr int TS = Tstride<(1 << LOG2N)>::v;
  const int total = ntr << LOG2BPT;
  float2 v[MAXB][R];
#pragma unroll
  for (int i = 0; i < MAXB; ++i) {
    const int b = threadIdx.x + i * kThreads;
    if (b < total) {
      const int t = b >> LOG2BPT;
      const int j = b & ((1 << LOG2BPT) - 1);
      const float2* in = buf + t * TS;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int idx = j + (r << LOG2BPT);
        if (FIRST) {
          if (PRUNE && r >= R / 2) v[i][r] = czero();
          else v[i][r] = idx < nyf ? in[pad16(idx)] : czero();
        } else {
          v[i][r] = in[pad16(idx)];
        }
      }
      if (!FIRST) {
        const int k = j & ((1 << LOG2NS) - 1);
#pragma unroll
        for (int r = 1; r < R; ++r) v[i][r] = cmul(v[i][r], tw[(r * k) << STEP]);
      }
      if (PRUNE) DftHalf<R>::run(v[i]);
      else Dft<R>::run(v[i]);
    }
  }
  if (LAST) {
#pragma unroll
    for (int i = 0; i < MAXB; ++i) {
      if (threadIdx.x + i * kThreads < total) {
#pragma unroll
        for (int r = 0; r < R; ++r)
          acc[i * R + r] = fmaf(v[i][r].x, v[i][r].x, fmaf(v[i][r].y, v[i][r].y, acc[i * R + r]));
      }
    }
    return;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < MAXB; ++i) {
    const int b = threadIdx.x + i * kThreads;
    if (b < total) {
      const int t = b >> LOG2BPT;
      const int j = b & ((1 << LOG2BPT) - 1);
      const int k = j & ((1 << LOG2NS) - 1);
      const int d = ((j >> LOG2NS) << (LOG2NS + LR)) + k;
      float2* out = buf + t * TS;
#pragma unroll
      for (int r = 0; r < R; ++r) out[pad16(d + (r << LOG2NS))] = v[i][r];
    }
  }
  __syncthreads();
}

template <int LOG2N>
__device__ __forceinline__ void fft_all(float2* buf, int ntr, int nyf, bool prune,
                                        const float2* tw, float* acc) {
  using P = FftPlan<LOG2N>;
  if constexpr (P::NST == 1) {
    if (prune) fft_stage<P::R0, P::LR0, true, true, true, LOG2N, 0>(buf, ntr, nyf, tw, acc);
    else fft_stage<P::R0, P::LR0, true, false, true, LOG2N, 0>(buf, ntr, nyf, tw, acc);
  } else {
    if (prune) fft_stage<P::R0, P::LR0, true, true, false, LOG2N, 0>(buf, ntr, nyf, tw, acc);
    else fft_stage<P::R0, P::LR0, true, false, false, LOG2N, 0>(buf, ntr, nyf, tw, acc);
    if constexpr (P::NST >= 3)
      fft_stage<8, 3, false, false, false, LOG2N, P::LR0>(buf, ntr, nyf, tw, acc);
    if constexpr (P::NST >= 4)
      fft_stage<8, 3, false, false, false, LOG2N, P::LR0 + 3>(buf, ntr, nyf, tw, acc);
    static_assert(P::NST <= 4, "N-S length above 4096");
    fft_stage<8, 3, false, false, true, LOG2N, P::LR0 + 3 * (P::NST - 2)>(buf, ntr, nyf, tw, acc);
  }
}

// ----------------------------------------------------------------- byte staging --
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Voltages are [t][f][p][feed]. First byte of work item `item` (window jw = item / nfreq,
// channel f): snapshot 0 of time jw n_int. One 64-bit division per work item.
__device__ __forceinline__ const uint8_t* item_volts(const BeamArgs& a, int64_t item, int nant) {
  const int64_t jw = item / a.nfreq;
  const int f = (int)(item - jw * a.nfreq);
  return a.volts + ((jw * a.n_int * a.nfreq + f) * a.npol) * (int64_t)nant;
}
// Offset of snapshot g (time g / npol, pol g % npol) from the first byte of its work item.
__device__ __forceinline__ int64_t snap_offset(const BeamArgs& a, int g, int nant) {
  int tt, p;
  if (a.npol == 2) {
    tt = g >> 1;
    p = g & 1;
  } else if (a.npol == 1) {
    tt = g;
    p = 0;
  } else {
    tt = g / a.npol;
    p = g - tt * a.npol;
  }
  return ((int64_t)tt * a.nfreq * a.npol + p) * (int64_t)nant;
}

// Stage the bytes of snapshots it*S .. it*S+S-1 of the work item starting at ivol into raw.
__device__ __forceinline__ void stage_bytes(const BeamArgs& a, uint8_t* raw, const uint8_t* ivol,
                                            int it, int nsnap, int nant, bool vec16) {
  if (vec16) {
    const int cps = nant >> 4;              // 16-byte chunks per snapshot
    const int nchunk = a.S * cps;
    const bool pow2 = (cps & (cps - 1)) == 0;
    const int lcps = __ffs(cps) - 1;
    for (int q = threadIdx.x; q < nchunk; q += kThreads) {
      const int s = pow2 ? q >> lcps : q / cps;
      const int g = it * a.S + s;
      if (g < nsnap) {
        const uint8_t* src = ivol + snap_offset(a, g, nant);
        cp_async16(raw + s * nant + ((q - s * cps) << 4), src + ((q - s * cps) << 4));
      }
    }
  } else {
    const int nb = a.S * nant;
    for (int q = threadIdx.x; q < nb; q += kThreads) {
      const int s = q / nant;
      const int g = it * a.S + s;
      if (g < nsnap) raw[q] = ivol[snap_offset(a, g, nant) + (q - s * nant)];
    }
  }
}

// ------------------------------------------------------------ fused FFT kernel --
template <int MX, int LOG2N>
__global__ void __launch_bounds__(kThreads, FFTBF_FP32_MIN_BLOCKS) beams_fp32_kernel(const BeamArgs a) {
  using P = FftPlan<LOG2N>;
  constexpr int N = P::N;
  constexpr int TS = Tstride<N>::v;
  extern __shared__ __align__(16) unsigned char smem[];
  const int nant = a.nx * a.ny;
  const int rawsz = (a.S * nant + 15) & ~15;
  float2* wsm = reinterpret_cast<float2*>(smem + 2 * rawsz);
  float2* exsm = wsm + nant;
  float2* twsm = exsm + MX * a.nx;
  float2* buf = twsm + N;
  const int ntr = a.S * MX;
  const int nsnap = a.n_int * a.npol;
  const int niter = (nsnap + a.S - 1) / a.S;
  const int64_t nitems = a.nwin * a.nfreq;
  const bool vec16 = ((nant & 15) == 0) && ((reinterpret_cast<uintptr_t>(a.volts) & 15) == 0);
  const bool prune = (P::R0 > 1) && (2 * a.nyf <= N);

  for (int i = threadIdx.x; i < nant; i += kThreads) wsm[i] = a.w[i];
  for (int i = threadIdx.x; i < MX * a.nx; i += kThreads) exsm[i] = a.ex[i];
  for (int i = threadIdx.x; i < N; i += kThreads) twsm[i] = a.tw[i];

  int64_t item = blockIdx.x;
  if (item >= nitems) return;
  int it = 0, cur = 0;
  const uint8_t* ivol = item_volts(a, item, nant);
  stage_bytes(a, smem, ivol, 0, nsnap, nant, vec16);
  cp_async_commit();

  constexpr int NACC = kMaxElems / kThreads;
  float acc[NACC];
#pragma unroll
  for (int i = 0; i < NACC; ++i) acc[i] = 0.f;

  while (true) {
    int64_t nitem = item;
    int nit = it + 1;
    if (nit == niter) { nitem = item + gridDim.x; nit = 0; }
    const bool has_next = nitem < nitems;
    const uint8_t* nvol = nit == 0 && has_next ? item_volts(a, nitem, nant) : ivol;
    if (has_next) stage_bytes(a, smem + (cur ^ 1) * rawsz, nvol, nit, nsnap, nant, vec16);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();

    // ---- unpack x weight, N-S fold, E-W transform -> Z[s][A][iyf] in buf
    const uint8_t* raw = smem + cur * rawsz;
    // columns (s, iyf); no integer division when a row of columns spans the CTA
    const bool rows = a.nyf >= kThreads;
    const int ncol = rows ? a.S * kThreads : a.S * a.nyf;
    for (int c = threadIdx.x; c < ncol; c += kThreads) {
      int s, iyf0, iystep;
      if (rows) { s = c / kThreads; iyf0 = c - s * kThreads; iystep = kThreads; }
      else { s = c / a.nyf; iyf0 = c - s * a.nyf; iystep = a.nyf; }
      const bool live = it * a.S + s < nsnap;
      const uint8_t* rs = raw + s * nant;
      for (int iyf = iyf0; iyf < a.nyf; iyf += iystep) {
        float2 z[MX];
#pragma unroll
        for (int A = 0; A < MX; ++A) z[A] = czero();
        if (live) {
          if constexpr (MX == 1 || MX == 2 || MX == 4 || MX == 8 || MX == 16) {
            if (a.ew_dft) {
#pragma unroll
              for (int ix = 0; ix < MX; ++ix) {
                float2 col = czero();
                for (int iy = iyf; iy < a.ny; iy += N)
                  col = cadd(col, cmul(wsm[ix * a.ny + iy], unpack_byte(rs[ix * a.ny + iy])));
                z[ix] = col;
              }
              Dft<MX>::run(z);
            }
          }
          if (!a.ew_dft) {
            for (int ix = 0; ix < a.nx; ++ix) {
              float2 col = czero();
              for (int iy = iyf; iy < a.ny; iy += N)
                col = cadd(col, cmul(wsm[ix * a.ny + iy], unpack_byte(rs[ix * a.ny + iy])));
#pragma unroll
              for (int A = 0; A < MX; ++A) z[A] = cadd(z[A], cmul(exsm[A * a.nx + ix], col));
            }
          }
        }
#pragma unroll
        for (int A = 0; A < MX; ++A) buf[(s * MX + A) * TS + pad16(iyf)] = z[A];
        if (!rows) break;
      }
    }
    __syncthreads();

    // ---- N-S transform; the last stage squares and accumulates
    fft_all<LOG2N>(buf, ntr, a.nyf, prune, twsm, acc);

    if (it == niter - 1) {
      // ---- window complete: add the S partial sums in a fixed order, write once
      __syncthreads();
      float* red = reinterpret_cast<float*>(buf);
      constexpr int RL = P::RL, LRL = P::LRL;
      constexpr int LOG2BPT = LOG2N - LRL;
      const int tot = ntr << LOG2BPT;                  // last-stage butterflies in the CTA
#pragma unroll
      for (int e = 0; e < NACC; ++e) {                 // acc[e]: butterfly e / RL, leg e % RL
        const int b = threadIdx.x + (e / RL) * kThreads;
        if (e / RL < kMaxElems / kThreads / RL && b < tot) {
          const int t = b >> LOG2BPT;
          const int j = b & ((1 << LOG2BPT) - 1);
          red[(t << LOG2N) + j + ((e % RL) << LOG2BPT)] = acc[e];   // unpadded
        }
        acc[e] = 0.f;
      }
      __syncthreads();
      const int nout = MX * N;
      float* dst = a.beams + item * (int64_t)nout;
      for (int o = threadIdx.x; o < nout; o += kThreads) {
        float sum = 0.f;
        for (int q = 0; q < a.S; ++q) sum += red[q * nout + o];
        dst[o] = sum;
      }
    }
    if (!has_next) break;
    item = nitem;
    ivol = nvol;
    it = nit;
    cur ^= 1;
  }
  cp_async_wait<0>();
}

inline size_t fft_smem_bytes(const BeamArgs& a) {
  const int nant = a.nx * a.ny;
  const size_t rawsz = ((size_t)a.S * nant + 15) & ~(size_t)15;
  const size_t ts = (size_t)a.my + (a.my >> 4);
  return 2 * rawsz + sizeof(float2) * ((size_t)nant + (size_t)a.mx * a.nx + a.my +
                                       (size_t)a.S * a.mx * ts);
}

template <int MX, int LOG2N>
int launch_fft_one(const BeamArgs& a, int nsm, cudaStream_t st) {
  const size_t smem = fft_smem_bytes(a);
  auto kern = beams_fp32_kernel<MX, LOG2N>;
  FFTBF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  FFTBF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      cudaSharedmemCarveoutMaxShared));
  int per_sm = 0;
  FFTBF_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
  if (per_sm < 1) return set_error(FFTBF_EUNSUPPORTED, "FP32 beam kernel does not fit on an SM");
  const int64_t items = a.nwin * a.nfreq;
  const int64_t grid = items < (int64_t)nsm * per_sm ? items : (int64_t)nsm * per_sm;
  kern<<<(unsigned)grid, kThreads, smem, st>>>(a);
  FFTBF_CUDA_TRY(cudaGetLastError());
  return FFTBF_OK;
}

// Dispatch on log2(my) for a fixed E-W size; MX * 2^LOG2N <= kMaxElems.
template <int MX>
int launch_fft_mx(const BeamArgs& a, int log2n, int nsm, cudaStream_t st) {
#define FFTBF_CASE(L) \
  case L:             \
    if constexpr (MX * (1 << L) <= kMaxElems) return launch_fft_one<MX, L>(a, nsm, st); \
    break;
  switch (log2n) {
    FFTBF_CASE(0) FFTBF_CASE(1) FFTBF_CASE(2) FFTBF_CASE(3) FFTBF_CASE(4) FFTBF_CASE(5)
    FFTBF_CASE(6) FFTBF_CASE(7) FFTBF_CASE(8) FFTBF_CASE(9) FFTBF_CASE(10) FFTBF_CASE(11)
    FFTBF_CASE(12)
    default: break;
  }
#undef FFTBF_CASE
  return set_error(FFTBF_EUNSUPPORTED, "no FP32 FFT kernel for mx=%d my=2^%d", MX, log2n);
}

}  // namespace fftbf

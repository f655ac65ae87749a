// Tensor-core form of the FFT-beam hot path for 4 E-W beams x 512 N-S beams over at most
// 256 N-S feeds (the 4x256 lattice padded N-S to 2n, Eq. b2n-1).
//
// The zero-padded 512-point N-S transform of each (snapshot, E-W beam) is split as
// 512 = 32 x 16 (n = n2 + 16 n1, k = k1 + 32 k2; inputs with n1 >= 16 are the padding):
//   stage 1 (tcgen05.mma, M=128 N=64 K=32): rows (snapshot, E-W beam A, n2), the pruned
//     32-point DFT X1[k1] = sum_{n1<16} x[n2 + 16 n1] W32^(n1 k1) as a real-embedded GEMM
//     (complex values interleaved (re, im) along K and N);
//   twiddle on the CUDA cores while draining TMEM: X1 *= W512^(n2 k1) in FP32, rounded
//     to 16 bits and written transposed as the stage-2 operand;
//   stage 2 (tcgen05.mma, M=128 N=32 K=32): rows (A, k1) of one snapshot, a 16-point DFT
//     over n2 giving X[k1 + 32 k2]; warp A, lane k1 of the CTA read their own TMEM row,
//     square it and add it to 16 register accumulators (Eq. bf), so integration over time
//     and polarisation needs no cross-lane reduction.
// Operands are FP16 or BF16 (the 4-bit inputs are exact in both), accumulation is FP32.
// BF16 form: unpacking, apodisation and the 4-point E-W DFT run in FP32 on the CUDA cores,
// as in the FP32 form, and are rounded to 16 bits once (times a plan scale). FP16 form:
// the same steps in packed-half arithmetic (nibbles decoded exactly into half2 through
// the mantissa of 1024, weight x scale pre-rounded to FP16, the E-W butterflies in half2)
// and the twiddle between the stages as a half2 complex multiply; this roughly halves the
// CUDA-core instructions per snapshot at about 1.3x the FP16 rounding error.
// A CTA (4 warps, 64 TMEM columns: stage 2 reuses the columns of stage 1 once they are
// drained; the stage-1 operand likewise overlays the stage-2 operand in shared memory)
// processes the two polarisations of one time sample (two snapshots) per iteration; five
// CTAs per SM (registers and shared memory), 320 of the 512 TMEM columns. Every wait on
// the tensor core is bounded by device time; on timeout the kernel records an error word
// (FFTBF_ETIMEOUT at fftbf_plan_sync), frees its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdlib>

#include "beam_fp32.cuh"
#include "tc_ptx.cuh"

namespace fftbf {

namespace tcl {
constexpr int NT = 128;
constexpr int A1_LBO = 128, A1_SBO = 512, A1_BYTES = 16 * 512;     // 128 rows x K 32
constexpr int A2_LBO = 144, A2_SBO = 592, A2_BYTES = 16 * 592;     // padded: conflict-free stores
constexpr int B_LBO = 128, B_SBO = 512;
constexpr int B1_BYTES = 8 * 512, B2_BYTES = 4 * 512;              // 64 and 32 rows x K 32
constexpr uint32_t TMEM_COLS = 64;     // D1: cols 0-63; D2 (two snapshots, after D1 is
                                       // drained): 0-31, 32-63
constexpr uint64_t WAIT_NS = 1000000000ull;
}  // namespace tcl

template <bool BF16>
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  if constexpr (BF16) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
  } else {
    __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
  }
}

// ---- packed-half helpers of the FP16 form ------------------------------------------------
__device__ __forceinline__ __half2 u2h(uint32_t v) { return *reinterpret_cast<__half2*>(&v); }
__device__ __forceinline__ uint32_t h2u(__half2 v) { return *reinterpret_cast<uint32_t*>(&v); }

// Byte k of `w` (bits 7..4 real, 3..0 imaginary, two's complement) as the exact half2
// (16 re, im): the nibbles are placed in the mantissas of 1024 (0x6400), the real one four
// bits up, with their sign bits flipped, which gives (1152 + 16 re, 1032 + im).
__device__ __forceinline__ __half2 unpack16(uint32_t w, int k) {
  const uint32_t t = __byte_perm(w, 0u, 0x4040u | (uint32_t)k | ((uint32_t)k << 8));
  const uint32_t u = (t & 0x000F00F0u) ^ 0x64086480u;
  return __hsub2(u2h(u), u2h(0x64086480u));           // (1152, 1032) as half2
}

// 4-point forward DFT of packed-half complex values, v[A] <- sum_ix v[ix] (-i)^(A ix).
__device__ __forceinline__ void dft4_h2(__half2* v) {
  const __half2 a = __hadd2(v[0], v[2]), b = __hsub2(v[0], v[2]);
  const __half2 c = __hadd2(v[1], v[3]), d = __hsub2(v[1], v[3]);
  const __half2 dsw = __lowhigh2highlow(d);            // (d.im, d.re)
  v[0] = __hadd2(a, c);
  v[2] = __hsub2(a, c);
  v[1] = __hfma2(dsw, u2h(0xBC003C00u), b);            // b - i d: (1, -1)
  v[3] = __hfma2(dsw, u2h(0x3C00BC00u), b);            // b + i d: (-1, 1)
}

// Slot of N-S feed iy within its row of the 4-byte weight table: bit 6 of iy is XORed
// into bit 4 when rows hold a multiple of 32 feeds (a permutation of each aligned block of
// 128), so that feeds 64 apart, read by the two half-warps of the input stage at the same
// time, sit 16 banks apart.
__device__ __forceinline__ int w4_pos(int iy, int ny) {
  return (ny & 31) == 0 ? iy ^ ((iy & 64) >> 2) : iy;
}

// FP16 form, stage-1 operand of one snapshot pair: A1[(s, A, n2)][(n1, c)] = scale x the
// E-W DFT of w x over the feeds iy = n2 + 16 n1. Thread (s, j, n2) forms n1 = 4j .. 4j + 3,
// so each E-W beam A is one 16-byte core-matrix row (one store), lanes run over n2 (the
// stores of a warp fill all banks) and the weights [ix][iy] are read 128 bytes at a time.
// Feeds iy >= ny and a missing second snapshot (odd n_int * npol) give zeros.
// REALW: real weights, one half2 (scale w / 16, scale w) per feed and one HMUL2.
template <bool REALW = false>
__device__ __forceinline__ void input_stage16(unsigned char* a1, const unsigned char* raw,
                                              const void* wtab, int nant, int ny, int tid,
                                              bool snap1_ok, int lbo, int sbo) {
  const uint2* w16 = reinterpret_cast<const uint2*>(wtab);
  const uint32_t* w16r = reinterpret_cast<const uint32_t*>(wtab);
  const int s = tid >> 6, j = (tid >> 4) & 3, n2 = tid & 15;
  const bool sok = s == 0 || snap1_ok;
  const unsigned char* rs = raw + s * nant;
  // w4_pos(iy) = iy ^ wsw: bit 6 of iy = n2 + 64 j + 16 kk is the low bit of j
  const int wsw = (ny & 31) == 0 ? (j & 1) << 4 : 0;
  uint32_t o[4][4];
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    const int iy = n2 + 64 * j + 16 * kk;
    __half2 z[4];
#pragma unroll
    for (int A = 0; A < 4; ++A) z[A] = u2h(0u);
    if (sok && iy < ny) {
#pragma unroll
      for (int ix = 0; ix < 4; ++ix) {
        const __half2 x = unpack16((uint32_t)rs[ix * ny + iy], 0);
        if constexpr (REALW) {
          // _rn: the product is rounded before the E-W adds (no fusing into them), as in
          // the complex-weight path, so both paths give bit-identical results
          z[ix] = __hmul2_rn(x, u2h(w16r[ix * ny + (iy ^ wsw)]));
        } else {
          const uint2 wv = w16[ix * ny + iy];
          z[ix] = __hfma2(__high2half2(x), u2h(wv.y), __hmul2(__low2half2(x), u2h(wv.x)));
        }
      }
      dft4_h2(z);
    }
#pragma unroll
    for (int A = 0; A < 4; ++A) o[A][kk] = h2u(z[A]);
  }
#pragma unroll
  for (int A = 0; A < 4; ++A)
    *reinterpret_cast<uint4*>(a1 + tc::kmajor_off(s * 64 + A * 16 + n2, 8 * j, lbo, sbo)) =
        make_uint4(o[A][0], o[A][1], o[A][2], o[A][3]);
}

struct TcSmem {
  int a1, a2, b1, b2, tw, w, raw, bars, taddr, total;
};
// split: hi and lo halves of every operand (A1 lo at a1 + A1_BYTES, A2 lo of snapshot s
// at a2 + (2 + s) A2_BYTES, B lo right after B hi).
__host__ __device__ inline TcSmem tc_smem_layout(int nant, bool split = false, bool w4 = false) {
  TcSmem L;
  int o = 0;
  auto take = [&](int bytes) { int r = o; o += (bytes + 127) & ~127; return r; };
  // A1 overlays the first bytes of A2: A1 is consumed by stage 1 before A2 is written,
  // and A2 by stage 2 before the next A1 is written
  L.a2 = take((split ? 4 : 2) * tcl::A2_BYTES);
  L.a1 = L.a2;
  L.b1 = take((split ? 2 : 1) * tcl::B1_BYTES);
  L.b2 = take((split ? 2 : 1) * tcl::B2_BYTES);
  L.tw = take(16 * 32 * 8);
  L.w = take(nant * (w4 ? 4 : 8));            // 4 bytes per feed: real FP16-form weights
  L.raw = take(2 * ((2 * nant + 15) & ~15));
  L.bars = take(16);
  L.taddr = take(16);
  L.total = o;
  return L;
}

// Copy a row-major [rows][32] 16-bit matrix into the canonical K-major layout.
__device__ __forceinline__ void load_kmajor(unsigned char* dst, const uint16_t* src, int rows,
                                           int lbo, int sbo, int tid, int nt) {
  for (int i = tid; i < rows * 16; i += nt) {         // pairs of 16-bit values
    const int m = i >> 4, k = (i & 15) * 2;
    const uint32_t v = (uint32_t)src[m * 32 + k] | ((uint32_t)src[m * 32 + k + 1] << 16);
    *reinterpret_cast<uint32_t*>(dst + tc::kmajor_off(m, k, lbo, sbo)) = v;
  }
}

// SPLIT (FP16 only): every operand is an FP16 value and its FP16 residual, and each stage
// is hi*hi + hi*lo + lo*hi accumulated in FP32, which gives the result FP32 accuracy.
// NY256 (the 4x256 lattice with a 4-point E-W DFT and 16-byte aligned voltages; for the
// FP16 form also real weights): the lattice sizes and the input-stage path are constants.
#ifndef FFTBF_TC16_MIN_BLOCKS
#define FFTBF_TC16_MIN_BLOCKS 6     // CTAs per SM the FP16 form's register budget targets
#endif
template <bool BF16, bool SPLIT = false, bool NY256 = false>
__global__ void __launch_bounds__(tcl::NT, SPLIT ? 3 : (BF16 ? 5 : FFTBF_TC16_MIN_BLOCKS))
beams_tc_kernel(const TcArgs ta) {
  const BeamArgs& a = ta.b;
  extern __shared__ __align__(1024) unsigned char smem_tc[];
  unsigned char* smem = smem_tc;
  const int ny = NY256 ? 256 : a.ny;
  const int nyf = NY256 ? 256 : a.nyf;
  const int nant = NY256 ? 1024 : a.nx * a.ny;
  constexpr bool FP16W4 = NY256 && !BF16 && !SPLIT;
  const bool w4 = FP16W4 || ta.w4 != 0;
  const TcSmem L = tc_smem_layout(nant, SPLIT, w4);
  unsigned char* a1 = smem + L.a1;
  unsigned char* a2 = smem + L.a2;
  unsigned char* b1s = smem + L.b1;
  unsigned char* b2s = smem + L.b2;
  float2* twsm = reinterpret_cast<float2*>(smem + L.tw);     // [k1 32][n2 16] W512^(n2 k1)
  float2* wsm = reinterpret_cast<float2*>(smem + L.w);
  unsigned char* raw0 = smem + L.raw;
  const int rawsz = (2 * nant + 15) & ~15;
  uint64_t* bar1 = reinterpret_cast<uint64_t*>(smem + L.bars);
  uint64_t* bar2 = bar1 + 1;
  uint32_t* taddr_sm = reinterpret_cast<uint32_t*>(smem + L.taddr);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t nitems = a.nwin * a.nfreq;
  const int nsnap = a.n_int * a.npol;
  const int niter = (nsnap + 1) / 2;

  if ((int64_t)blockIdx.x >= nitems) return;

  // ---- set-up: TMEM, barriers, constant operands, tables
  if (warp == 0) {
    tc::tmem_alloc(taddr_sm, tcl::TMEM_COLS);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(bar1, 1);
    tc::mbar_init(bar2, 1);
    tc::mbar_init_fence();
  }
  load_kmajor(b1s, ta.b1, 64, tcl::B_LBO, tcl::B_SBO, tid, tcl::NT);
  load_kmajor(b2s, ta.b2, 32, tcl::B_LBO, tcl::B_SBO, tid, tcl::NT);
  if constexpr (SPLIT) {
    load_kmajor(b1s + tcl::B1_BYTES, ta.b1lo, 64, tcl::B_LBO, tcl::B_SBO, tid, tcl::NT);
    load_kmajor(b2s + tcl::B2_BYTES, ta.b2lo, 32, tcl::B_LBO, tcl::B_SBO, tid, tcl::NT);
  }
  // FP16 form: packed-half input stage when the E-W axis is a plain 4-point DFT over
  // groups of four N-S feeds (4-byte words), and packed-half twiddles between the stages.
  const bool fast16 =
      FP16W4 || (!BF16 && !SPLIT && a.ew_dft && a.nx == 4 && (a.ny & 3) == 0 && a.nyf == a.ny);
  if constexpr (!BF16 && !SPLIT) {
    uint2* tw16 = reinterpret_cast<uint2*>(twsm);      // [k1][n2] {(c, d), (-d, c)}
    for (int i = tid; i < 512; i += tcl::NT) {
      const float2 t = a.tw[(i >> 4) * (i & 15)];
      tw16[i] = make_uint2(pack2<false>(t.x, t.y), pack2<false>(-t.y, t.x));
    }
  } else {
    for (int i = tid; i < 512; i += tcl::NT) twsm[i] = a.tw[(i >> 4) * (i & 15)];
  }
  if (fast16 && w4) {
    // real weights: per feed (scale w / 16, scale w), (16 re, im) -> scale (re + i im) w
    uint32_t* w16r = reinterpret_cast<uint32_t*>(wsm);
    const float sc = ta.scale;
    for (int i = tid; i < nant; i += tcl::NT) {
      const float w = a.w[i].x;
      const int ix = i / ny, iy = i - ix * ny;
      w16r[ix * ny + w4_pos(iy, ny)] = pack2<false>(w * sc * 0.0625f, w * sc);
    }
  } else if (fast16) {
    // per feed {scale w / 16, scale i w}: (16 re, im) -> scale (re + i im) w
    uint2* w16 = reinterpret_cast<uint2*>(wsm);
    const float sc = ta.scale;
    for (int i = tid; i < nant; i += tcl::NT) {
      const float2 w = a.w[i];
      w16[i] = make_uint2(pack2<false>(w.x * sc * 0.0625f, w.y * sc * 0.0625f),
                          pack2<false>(-w.y * sc, w.x * sc));
    }
  } else {
    for (int i = tid; i < nant; i += tcl::NT) wsm[i] = a.w[i];
  }
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *taddr_sm;
  const uint32_t tlane = (uint32_t)(32 * warp) << 16;        // this warp's TMEM lane quarter
  const bool vec16 =
      NY256 || (((nant & 15) == 0) && ((reinterpret_cast<uintptr_t>(a.volts) & 15) == 0));
  const uint32_t id1 = tc::idesc_f16(128, 64, BF16);
  const uint32_t id2 = tc::idesc_f16(128, 32, BF16);
  const float inv_s2 = 1.0f / (ta.scale * ta.scale);

  // bytes of snapshot pair `it` of the work item starting at ivol
  auto stage = [&](const uint8_t* ivol, int it, unsigned char* raw) {
    if (vec16) {
      const int cps = nant >> 4;
      for (int q = tid; q < 2 * cps; q += tcl::NT) {
        const int s = q >= cps ? 1 : 0, g = 2 * it + s;      // q < 2 cps
        if (g < nsnap) {
          const uint8_t* src = ivol + snap_offset(a, g, nant);
          cp_async16(raw + s * nant + ((q - s * cps) << 4), src + ((q - s * cps) << 4));
        }
      }
    } else {
      for (int q = tid; q < 2 * nant; q += tcl::NT) {
        const int s = q / nant, g = 2 * it + s;
        if (g < nsnap) raw[q] = ivol[snap_offset(a, g, nant) + (q - s * nant)];
      }
    }
  };

  int64_t item = blockIdx.x;
  int it = 0, cur = 0;
  uint32_t phase = 0;
  bool ok = true;
  float acc[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] = 0.f;
  const uint8_t* ivol = item_volts(a, item, nant);
  stage(ivol, 0, raw0);
  cp_async_commit();

  while (true) {
    int64_t nitem = item;
    int nit = it + 1;
    if (nit == niter) { nitem = item + gridDim.x; nit = 0; }
    const bool has_next = nitem < nitems;
    const uint8_t* nvol = nit == 0 && has_next ? item_volts(a, nitem, nant) : ivol;
    cp_async_wait<0>();
    __syncthreads();                                            // (S1)
    if (has_next) stage(nvol, nit, raw0 + (cur ^ 1) * rawsz);
    cp_async_commit();

    // ---- unpack x weight, E-W DFT, scale, round: stage-1 operand A1[(s,A,n2)][(n1,c)]
    const unsigned char* raw = raw0 + cur * rawsz;
    if (fast16) {
      if (w4)
        input_stage16<true>(a1, raw, wsm, nant, ny, tid, 2 * it + 1 < nsnap, tcl::A1_LBO,
                            tcl::A1_SBO);
      else
        input_stage16<false>(a1, raw, wsm, nant, ny, tid, 2 * it + 1 < nsnap, tcl::A1_LBO,
                             tcl::A1_SBO);
    } else
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = tid + q * tcl::NT;
      const int s = c >> 8, iy = c & 255;
      float2 z[4] = {czero(), czero(), czero(), czero()};
      if (iy < nyf && 2 * it + s < nsnap) {
        const unsigned char* rs = raw + s * nant;
        if (NY256 || a.ew_dft) {
          if (a.real_w) {
            // real weights: one packed multiply, the same roundings as the complex product
#pragma unroll
            for (int ix = 0; ix < 4; ++ix) {
              const float wr = wsm[ix * ny + iy].x;
              const float2 xv = unpack_byte(rs[ix * ny + iy]);
              z[ix] = __fmul2_rn(make_float2(wr, wr), xv);
            }
          } else {
#pragma unroll
            for (int ix = 0; ix < 4; ++ix)
              z[ix] = cmul(wsm[ix * ny + iy], unpack_byte(rs[ix * ny + iy]));
          }
          Dft<4>::run(z);
        } else {
          for (int ix = 0; ix < a.nx; ++ix) {
            const float2 col = cmul(wsm[ix * a.ny + iy], unpack_byte(rs[ix * a.ny + iy]));
#pragma unroll
            for (int A = 0; A < 4; ++A) z[A] = cadd(z[A], cmul(a.ex[A * a.nx + ix], col));
          }
        }
      }
#pragma unroll
      for (int A = 0; A < 4; ++A) {
        const int m = (s * 4 + A) * 16 + (iy & 15);
        const uint32_t off = tc::kmajor_off(m, 2 * (iy >> 4), tcl::A1_LBO, tcl::A1_SBO);
        if constexpr (SPLIT) {
          const float zr = z[A].x * ta.scale, zi = z[A].y * ta.scale;
          const __half2 h = __floats2half2_rn(zr, zi);
          const float2 hf = __half22float2(h);
          *reinterpret_cast<uint32_t*>(a1 + off) = h2u(h);
          *reinterpret_cast<uint32_t*>(a1 + tcl::A1_BYTES + off) = pack2<false>(zr - hf.x, zi - hf.y);
        } else {
          *reinterpret_cast<uint32_t*>(a1 + off) = pack2<BF16>(z[A].x * ta.scale, z[A].y * ta.scale);
        }
      }
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();                                            // (S2)
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t sa = tc::smem_u32(a1), sb = tc::smem_u32(b1s);
#pragma unroll
      for (int kk = 0; kk < 2; ++kk)
        tc::mma_f16(tbase, tc::smem_desc(sa + kk * 2 * tcl::A1_LBO, tcl::A1_LBO, tcl::A1_SBO),
                    tc::smem_desc(sb + kk * 2 * tcl::B_LBO, tcl::B_LBO, tcl::B_SBO), id1, kk);
      if constexpr (SPLIT) {
        // + hi * B_lo + lo * B_hi
#pragma unroll
        for (int kk = 0; kk < 2; ++kk)
          tc::mma_f16(tbase, tc::smem_desc(sa + kk * 2 * tcl::A1_LBO, tcl::A1_LBO, tcl::A1_SBO),
                      tc::smem_desc(sb + tcl::B1_BYTES + kk * 2 * tcl::B_LBO, tcl::B_LBO, tcl::B_SBO),
                      id1, 1);
#pragma unroll
        for (int kk = 0; kk < 2; ++kk)
          tc::mma_f16(tbase,
                      tc::smem_desc(sa + tcl::A1_BYTES + kk * 2 * tcl::A1_LBO, tcl::A1_LBO, tcl::A1_SBO),
                      tc::smem_desc(sb + kk * 2 * tcl::B_LBO, tcl::B_LBO, tcl::B_SBO), id1, 1);
      }
      tc::mma_commit(bar1);
    }
    ok = tc::mbar_wait(bar1, phase, tcl::WAIT_NS);
    if (!__syncthreads_and(ok)) break;
    tc::fence_after_sync();

    // ---- drain stage 1: twiddle W512^(n2 k1), round, store as A2[s][(A,k1)][(n2,c)]
    {
      const int m = 32 * warp + lane;
      const int sA = m >> 4, n2 = m & 15, s = sA >> 2, A = sA & 3;
      unsigned char* a2s = a2 + s * tcl::A2_BYTES;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t r[16];
        tc::tmem_ld16(tbase + tlane + 16 * q, r);
        tc::tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int k1 = 8 * q + j;
          uint32_t yv;
          if constexpr (SPLIT) {
            const float2 x = make_float2(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1]));
            const float2 y = cmul(x, twsm[k1 * 16 + n2]);
            const __half2 h = __floats2half2_rn(y.x, y.y);
            const float2 hf = __half22float2(h);
            yv = h2u(h);
            *reinterpret_cast<uint32_t*>(a2 + (2 + s) * tcl::A2_BYTES +
                                         tc::kmajor_off(A * 32 + k1, 2 * n2, tcl::A2_LBO, tcl::A2_SBO)) =
                pack2<false>(y.x - hf.x, y.y - hf.y);
          } else if constexpr (!BF16) {
            const uint2 t = reinterpret_cast<const uint2*>(twsm)[k1 * 16 + n2];
            const __half2 h = __floats2half2_rn(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1]));
            yv = h2u(__hfma2(__high2half2(h), u2h(t.y), __hmul2(__low2half2(h), u2h(t.x))));
          } else {
            const float2 x = make_float2(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1]));
            const float2 y = cmul(x, twsm[k1 * 16 + n2]);   // lanes: consecutive n2
            yv = pack2<BF16>(y.x, y.y);
          }
          *reinterpret_cast<uint32_t*>(a2s + tc::kmajor_off(A * 32 + k1, 2 * n2, tcl::A2_LBO, tcl::A2_SBO)) = yv;
        }
      }
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();                                            // (S3)
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t sb = tc::smem_u32(b2s);
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const uint32_t sa = tc::smem_u32(a2 + s * tcl::A2_BYTES);
#pragma unroll
        for (int kk = 0; kk < 2; ++kk)
          tc::mma_f16(tbase + 32 * s,
                      tc::smem_desc(sa + kk * 2 * tcl::A2_LBO, tcl::A2_LBO, tcl::A2_SBO),
                      tc::smem_desc(sb + kk * 2 * tcl::B_LBO, tcl::B_LBO, tcl::B_SBO), id2, kk);
        if constexpr (SPLIT) {
          const uint32_t sl = tc::smem_u32(a2 + (2 + s) * tcl::A2_BYTES);
#pragma unroll
          for (int kk = 0; kk < 2; ++kk)
            tc::mma_f16(tbase + 32 * s,
                        tc::smem_desc(sa + kk * 2 * tcl::A2_LBO, tcl::A2_LBO, tcl::A2_SBO),
                        tc::smem_desc(sb + tcl::B2_BYTES + kk * 2 * tcl::B_LBO, tcl::B_LBO, tcl::B_SBO),
                        id2, 1);
#pragma unroll
          for (int kk = 0; kk < 2; ++kk)
            tc::mma_f16(tbase + 32 * s,
                        tc::smem_desc(sl + kk * 2 * tcl::A2_LBO, tcl::A2_LBO, tcl::A2_SBO),
                        tc::smem_desc(sb + kk * 2 * tcl::B_LBO, tcl::B_LBO, tcl::B_SBO), id2, 1);
        }
      }
      tc::mma_commit(bar2);
    }
    ok = tc::mbar_wait(bar2, phase, tcl::WAIT_NS);
    if (!__syncthreads_and(ok)) break;
    tc::fence_after_sync();

    // ---- drain stage 2: warp A, lane k1 squares X[k1 + 32 k2] and accumulates
#pragma unroll
    for (int s = 0; s < 2; ++s) {
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        uint32_t r[16];
        tc::tmem_ld16(tbase + tlane + 32 * s + 16 * hh, r);
        tc::tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int k2 = 8 * hh + j;
          const float re = __uint_as_float(r[2 * j]), im = __uint_as_float(r[2 * j + 1]);
          acc[k2] = fmaf(re, re, fmaf(im, im, acc[k2]));
        }
      }
    }
    tc::fence_before_sync();
    phase ^= 1u;

    if (it == niter - 1) {
      float* dst = a.beams + item * (int64_t)(4 * 512) + warp * 512 + lane;
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) {
        dst[32 * k2] = acc[k2] * inv_s2;
        acc[k2] = 0.f;
      }
    }
    if (!has_next) break;
    item = nitem;
    ivol = nvol;
    it = nit;
    cur ^= 1;
  }
  if (!ok && tid == 0) atomicExch(ta.err, FFTBF_ETIMEOUT);
  cp_async_wait<0>();
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, tcl::TMEM_COLS);
}

// ------------------------------------------------------------------------------------
// Warp-specialised, double-buffered version of the same computation. Roles per CTA:
//   warps 0-3  producers: stage bytes (cp.async), unpack x weight, E-W DFT, round -> A1[b]
//   warps 4-7  drainers:  D1[b] -> twiddle -> A2[b]; D2[b] -> |.|^2 -> accumulators
//   warp 8     issuer:    one lane issues MMA1(p) and MMA2(p-1) and commits them
// for snapshot pairs p = 0, 1, ... with buffers b = p mod 2. Hand-offs are mbarriers:
//   a1_full[b]  producers -> issuer      d1_full[b]  issuer (commit) -> drainers, producers
//   d1_empty[b] drainers -> issuer       a2_full[b]  drainers -> issuer
//   d2_full[b]  issuer (commit) -> drainers   d2_empty[b] drainers -> issuer
// so the unpacking of pair p+1, the tensor-core stages and the draining of pair p overlap.
// Two CTAs per SM (256 TMEM columns each: D1[2] x 64, D2[2] x 64).
namespace tcp {
constexpr int NT = 288;
constexpr uint32_t TMEM_COLS = 256;
enum { A1F = 0, D1F = 2, D1E = 4, A2F = 6, D2F = 8, D2E = 10, NBAR = 12 };
}  // namespace tcp

struct TcPipeSmem {
  int a1, a2, b1, b2, tw, w, lut, raw, bars, misc, total;
};
__host__ __device__ inline TcPipeSmem tcp_smem_layout(int nant) {
  TcPipeSmem L;
  int o = 0;
  auto take = [&](int bytes) { int r = o; o += (bytes + 127) & ~127; return r; };
  L.a1 = take(2 * tcl::A1_BYTES);
  L.a2 = take(4 * tcl::A2_BYTES);
  L.b1 = take(tcl::B1_BYTES);
  L.b2 = take(tcl::B2_BYTES);
  L.tw = take(16 * 32 * 8);
  L.w = take(nant * 8);
  L.lut = take(256 * 8);
  L.raw = take(2 * ((2 * nant + 15) & ~15));
  L.bars = take(tcp::NBAR * 8);
  L.misc = take(16);
  L.total = o;
  return L;
}

template <bool BF16>
__global__ void __launch_bounds__(tcp::NT, 2) beams_tc_pipe_kernel(const TcArgs ta) {
  const BeamArgs& a = ta.b;
  extern __shared__ __align__(1024) unsigned char smem_tc[];
  unsigned char* smem = smem_tc;
  const int nant = a.nx * a.ny;
  const TcPipeSmem L = tcp_smem_layout(nant);
  unsigned char* a1 = smem + L.a1;
  unsigned char* a2 = smem + L.a2;
  unsigned char* b1s = smem + L.b1;
  unsigned char* b2s = smem + L.b2;
  float2* twsm = reinterpret_cast<float2*>(smem + L.tw);   // [k1 32][n2 16]
  float2* wsm = reinterpret_cast<float2*>(smem + L.w);
  float2* lut = reinterpret_cast<float2*>(smem + L.lut);   // byte -> (re, im)
  unsigned char* raw0 = smem + L.raw;
  const int rawsz = (2 * nant + 15) & ~15;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bars);
  uint32_t* taddr_sm = reinterpret_cast<uint32_t*>(smem + L.misc);
  volatile int* abort_sm = reinterpret_cast<volatile int*>(smem + L.misc + 4);
  volatile int* pvote = reinterpret_cast<volatile int*>(smem + L.misc + 8);    // producers
  volatile int* evote = reinterpret_cast<volatile int*>(smem + L.misc + 12);   // drainers
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t nitems = a.nwin * a.nfreq;
  const int nsnap = a.n_int * a.npol;
  const int niter = (nsnap + 1) / 2;
  if ((int64_t)blockIdx.x >= nitems) return;
  const int64_t my_items = (nitems - 1 - blockIdx.x) / gridDim.x + 1;
  const int64_t P = my_items * niter;                 // snapshot pairs of this CTA

  if (warp == 8) {
    tc::tmem_alloc(taddr_sm, tcp::TMEM_COLS);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    const uint32_t counts[tcp::NBAR] = {128, 128, 1, 1, 128, 128, 128, 128, 1, 1, 128, 128};
    for (int i = 0; i < tcp::NBAR; ++i) tc::mbar_init(bars + i, counts[i]);
    tc::mbar_init_fence();
    *abort_sm = 0;
  }
  load_kmajor(b1s, ta.b1, 64, tcl::B_LBO, tcl::B_SBO, tid, tcp::NT);
  load_kmajor(b2s, ta.b2, 32, tcl::B_LBO, tcl::B_SBO, tid, tcp::NT);
  const bool fast16 = !BF16 && a.ew_dft && a.nx == 4 && (a.ny & 3) == 0 && a.nyf == a.ny;
  if constexpr (!BF16) {
    uint2* tw16 = reinterpret_cast<uint2*>(twsm);      // [k1][n2] {(c, d), (-d, c)}
    for (int i = tid; i < 512; i += tcp::NT) {
      const float2 t = a.tw[(i >> 4) * (i & 15)];
      tw16[i] = make_uint2(pack2<false>(t.x, t.y), pack2<false>(-t.y, t.x));
    }
  } else {
    for (int i = tid; i < 512; i += tcp::NT) twsm[i] = a.tw[(i >> 4) * (i & 15)];
  }
  if (fast16) {
    uint2* w16 = reinterpret_cast<uint2*>(wsm);
    const float sc = ta.scale;
    for (int i = tid; i < nant; i += tcp::NT) {
      const float2 w = a.w[i];
      w16[i] = make_uint2(pack2<false>(w.x * sc * 0.0625f, w.y * sc * 0.0625f),
                          pack2<false>(-w.y * sc, w.x * sc));
    }
  } else {
    for (int i = tid; i < nant; i += tcp::NT) wsm[i] = a.w[i];
  }
  for (int i = tid; i < 256; i += tcp::NT) lut[i] = unpack_byte((unsigned)i);
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *taddr_sm;
  const uint64_t W = tcl::WAIT_NS;
  auto fail = [&]() { *abort_sm = 1; atomicExch(ta.err, FFTBF_ETIMEOUT); };

  if (warp < 4) {
    // ================================================================ producers
    const bool vec16 = ((nant & 15) == 0) && ((reinterpret_cast<uintptr_t>(a.volts) & 15) == 0);
    const bool scaled = ta.scale != 1.f;
    auto stage = [&](const uint8_t* ivol, int it, unsigned char* raw) {
      if (vec16) {
        const int cps = nant >> 4;
        for (int q = tid; q < 2 * cps; q += 128) {
          const int s = q >= cps ? 1 : 0, g = 2 * it + s;      // q < 2 cps
          if (g < nsnap) {
            const uint8_t* src = ivol + snap_offset(a, g, nant);
            cp_async16(raw + s * nant + ((q - s * cps) << 4), src + ((q - s * cps) << 4));
          }
        }
      } else {
        for (int q = tid; q < 2 * nant; q += 128) {
          const int s = q / nant, g = 2 * it + s;
          if (g < nsnap) raw[q] = ivol[snap_offset(a, g, nant) + (q - s * nant)];
        }
      }
    };
    int64_t item = blockIdx.x;
    int it = 0;
    const uint8_t* ivol = item_volts(a, item, nant);
    stage(ivol, 0, raw0);
    cp_async_commit();
    for (int64_t p = 0; p < P; ++p) {
      int64_t nitem = item;
      int nit = it + 1;
      if (nit == niter) { nitem = item + gridDim.x; nit = 0; }
      const uint8_t* nvol = nit == 0 && p + 1 < P ? item_volts(a, nitem, nant) : ivol;
      tc::named_sync(1, 128);                         // phase B of p-1 done: raw[(p+1)&1] free
      if (p + 1 < P) stage(nvol, nit, raw0 + ((p + 1) & 1) * rawsz);
      cp_async_commit();
      cp_async_wait<1>();
      const int b = (int)(p & 1);
      const uint32_t u = (uint32_t)(p >> 1);
      if (tid == 0) *pvote = (u == 0) || tc::mbar_wait_abortable(bars + tcp::D1F + b, (u - 1) & 1, W, abort_sm);
      tc::named_sync(1, 128);                         // bytes of p visible; A1[b] free (or abort)
      if (!*pvote) { if (tid == 0) fail(); break; }
      const unsigned char* raw = raw0 + (p & 1) * rawsz;
      unsigned char* a1b = a1 + b * tcl::A1_BYTES;
      if (fast16) {
        input_stage16<false>(a1b, raw, wsm, nant, a.ny, tid,
                      2 * it + 1 < nsnap, tcl::A1_LBO, tcl::A1_SBO);
      } else
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = tid + q * 128;
        const int s = c >> 8, iy = c & 255;
        float2 z[4] = {czero(), czero(), czero(), czero()};
        if (iy < a.nyf && 2 * it + s < nsnap) {
          const unsigned char* rs = raw + s * nant;
          if (a.ew_dft) {
#pragma unroll
            for (int ix = 0; ix < 4; ++ix) z[ix] = cmul(wsm[ix * a.ny + iy], lut[rs[ix * a.ny + iy]]);
            Dft<4>::run(z);
          } else {
            for (int ix = 0; ix < a.nx; ++ix) {
              const float2 col = cmul(wsm[ix * a.ny + iy], lut[rs[ix * a.ny + iy]]);
#pragma unroll
              for (int A = 0; A < 4; ++A) z[A] = cadd(z[A], cmul(a.ex[A * a.nx + ix], col));
            }
          }
          if (scaled) {
#pragma unroll
            for (int A = 0; A < 4; ++A) z[A] = make_float2(z[A].x * ta.scale, z[A].y * ta.scale);
          }
        }
#pragma unroll
        for (int A = 0; A < 4; ++A) {
          const int m = (s * 4 + A) * 16 + (iy & 15);
          *reinterpret_cast<uint32_t*>(a1b + tc::kmajor_off(m, 2 * (iy >> 4), tcl::A1_LBO, tcl::A1_SBO)) =
              pack2<BF16>(z[A].x, z[A].y);
        }
      }
      tc::fence_proxy_async_smem();
      tc::mbar_arrive(bars + tcp::A1F + b);
      item = nitem;
      ivol = nvol;
      it = nit;
    }
    cp_async_wait<0>();
  } else if (warp < 8) {
    // ================================================================= drainers
    const int q4 = warp - 4;                         // TMEM lane quarter
    const uint32_t tlane = (uint32_t)(32 * q4) << 16;
    const int etid = tid - 128;
    const float inv_s2 = 1.0f / (ta.scale * ta.scale);
    float acc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[i] = 0.f;
    int64_t qitem = blockIdx.x;                      // item of the pair being accumulated
    int qit = 0;
    for (int64_t p = 0; p <= P; ++p) {
      if (p < P) {
        const int b = (int)(p & 1);
        const uint32_t u = (uint32_t)(p >> 1);
        if (etid == 0) *evote = tc::mbar_wait_abortable(bars + tcp::D1F + b, u & 1, W, abort_sm);
        tc::named_sync(2, 128);
        if (!*evote) { if (etid == 0) fail(); break; }
        tc::fence_after_sync();
        const int m = 32 * q4 + lane;
        const int sA = m >> 4, n2 = m & 15, s = sA >> 2, A = sA & 3;
        unsigned char* a2s = a2 + (2 * b + s) * tcl::A2_BYTES;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          uint32_t r[32];
          tc::tmem_ld32(tbase + tlane + 64 * b + 32 * half, r);
          tc::tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int k1 = 16 * half + j;
            uint32_t yv;
            if constexpr (!BF16) {
              const uint2 t = reinterpret_cast<const uint2*>(twsm)[k1 * 16 + n2];
              const __half2 h = __floats2half2_rn(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1]));
              yv = h2u(__hfma2(__high2half2(h), u2h(t.y), __hmul2(__low2half2(h), u2h(t.x))));
            } else {
              const float2 x = make_float2(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1]));
              const float2 y = cmul(x, twsm[k1 * 16 + n2]);
              yv = pack2<BF16>(y.x, y.y);
            }
            *reinterpret_cast<uint32_t*>(a2s + tc::kmajor_off(A * 32 + k1, 2 * n2, tcl::A2_LBO, tcl::A2_SBO)) = yv;
          }
        }
        tc::fence_before_sync();
        tc::mbar_arrive(bars + tcp::D1E + b);
        tc::fence_proxy_async_smem();
        tc::mbar_arrive(bars + tcp::A2F + b);
      }
      if (p >= 1) {
        const int64_t q = p - 1;
        const int b = (int)(q & 1);
        const uint32_t u = (uint32_t)(q >> 1);
        if (etid == 0) *evote = tc::mbar_wait_abortable(bars + tcp::D2F + b, u & 1, W, abort_sm);
        tc::named_sync(2, 128);
        if (!*evote) { if (etid == 0) fail(); break; }
        tc::fence_after_sync();
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          uint32_t r[32];
          tc::tmem_ld32(tbase + tlane + 128 + 64 * b + 32 * s, r);
          tc::tmem_wait_ld();
#pragma unroll
          for (int k2 = 0; k2 < 16; ++k2) {
            const float re = __uint_as_float(r[2 * k2]), im = __uint_as_float(r[2 * k2 + 1]);
            acc[k2] = fmaf(re, re, fmaf(im, im, acc[k2]));
          }
        }
        tc::fence_before_sync();
        tc::mbar_arrive(bars + tcp::D2E + b);
        if (qit == niter - 1) {
          float* dst = a.beams + qitem * (int64_t)(4 * 512) + q4 * 512 + lane;
#pragma unroll
          for (int k2 = 0; k2 < 16; ++k2) {
            dst[32 * k2] = acc[k2] * inv_s2;
            acc[k2] = 0.f;
          }
          qitem += gridDim.x;
          qit = 0;
        } else {
          ++qit;
        }
      }
    }
  } else if (lane == 0) {
    // =================================================================== issuer
    const uint32_t id1 = tc::idesc_f16(128, 64, BF16);
    const uint32_t id2 = tc::idesc_f16(128, 32, BF16);
    const uint32_t sb1 = tc::smem_u32(b1s), sb2 = tc::smem_u32(b2s);
    for (int64_t p = 0; p <= P; ++p) {
      if (p < P) {
        const int b = (int)(p & 1);
        const uint32_t u = (uint32_t)(p >> 1);
        if (!tc::mbar_wait_abortable(bars + tcp::A1F + b, u & 1, W, abort_sm) ||
            (u >= 1 && !tc::mbar_wait_abortable(bars + tcp::D1E + b, (u - 1) & 1, W, abort_sm))) {
          fail();
          break;
        }
        tc::fence_after_sync();
        const uint32_t sa = tc::smem_u32(a1 + b * tcl::A1_BYTES);
#pragma unroll
        for (int kk = 0; kk < 2; ++kk)
          tc::mma_f16(tbase + 64 * b, tc::smem_desc(sa + kk * 2 * tcl::A1_LBO, tcl::A1_LBO, tcl::A1_SBO),
                      tc::smem_desc(sb1 + kk * 2 * tcl::B_LBO, tcl::B_LBO, tcl::B_SBO), id1, kk);
        tc::mma_commit(bars + tcp::D1F + b);
      }
      if (p >= 1) {
        const int64_t q = p - 1;
        const int b = (int)(q & 1);
        const uint32_t u = (uint32_t)(q >> 1);
        if (!tc::mbar_wait_abortable(bars + tcp::A2F + b, u & 1, W, abort_sm) ||
            (u >= 1 && !tc::mbar_wait_abortable(bars + tcp::D2E + b, (u - 1) & 1, W, abort_sm))) {
          fail();
          break;
        }
        tc::fence_after_sync();
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          const uint32_t sa = tc::smem_u32(a2 + (2 * b + s) * tcl::A2_BYTES);
#pragma unroll
          for (int kk = 0; kk < 2; ++kk)
            tc::mma_f16(tbase + 128 + 64 * b + 32 * s,
                        tc::smem_desc(sa + kk * 2 * tcl::A2_LBO, tcl::A2_LBO, tcl::A2_SBO),
                        tc::smem_desc(sb2 + kk * 2 * tcl::B_LBO, tcl::B_LBO, tcl::B_SBO), id2, kk);
        }
        tc::mma_commit(bars + tcp::D2F + b);
      }
    }
  }
  __syncwarp();
  // Every role has left its loop. The tensor core may still be finishing the last
  // commits; wait (bounded) for the final stage-2 commit before freeing TMEM.
  if (tid == 0 && P > 0 && !*abort_sm) {
    const int64_t q = P - 1;
    tc::mbar_wait(bars + tcp::D2F + (int)(q & 1), (uint32_t)((q >> 1) & 1), W);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 8) tc::tmem_dealloc(tbase, tcp::TMEM_COLS);
}

bool tc_supported(int nx, int ny, int mx, int my) {
  (void)nx;
  return mx == 4 && my == 512 && (ny < my ? ny : my) <= 256 && nx * ny <= 16384;
}

static int tc_residency(const void* kern, size_t smem, int nthreads, int max_ctas, int* per_sm) {
  // Residency from registers and shared memory (the occupancy query is conservative for
  // kernels that allocate tensor memory), capped by the TMEM budget.
  int dev = 0, smem_sm = 0, regs_sm = 0;
  FFTBF_CUDA_TRY(cudaGetDevice(&dev));
  FFTBF_CUDA_TRY(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  FFTBF_CUDA_TRY(cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev));
  cudaFuncAttributes fa{};
  FFTBF_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
  const int warps = (nthreads + 31) / 32;
  const int by_smem = smem_sm / (int)(smem + 1024);
  const int by_regs = regs_sm / (((fa.numRegs + 7) & ~7) * 32 * warps);
  int n = by_smem < by_regs ? by_smem : by_regs;
  if (n > max_ctas) n = max_ctas;
  *per_sm = n;
  if (n < 1) return set_error(FFTBF_EUNSUPPORTED, "tensor-core kernel does not fit on an SM");
  return FFTBF_OK;
}

int launch_beams_tc(const TcArgs& ta, int nsm, cudaStream_t st) {
  const BeamArgs& a = ta.b;
  if (a.nwin <= 0) return FFTBF_OK;
  const int64_t items = a.nwin * a.nfreq;
  // FP16 and BF16 on the 4x256 lattice: the grouped kernel (four snapshots per stage-1 MMA,
  // intermediates in tensor memory; beam_tcg.cu), or with FFTBF_TC_KERNEL=ws the pair-wise
  // warp-specialised kernel with MN-major planar operands (beam_tcw.cu), unless
  // FFTBF_TC_KERNEL=serial or FFTBF_TC_PIPE=1 ask for the kernels below. Of those two, the
  // serial kernel (several CTAs per SM, every warp in every phase) measures faster than the
  // first warp-specialised pipeline on the 4x256 lattice.
  const char* pipe = getenv("FFTBF_TC_PIPE");
  const char* which = getenv("FFTBF_TC_KERNEL");
  const bool old_kernel = (pipe && pipe[0] && pipe[0] != '0') || (which && which[0] == 's');
  const bool pairwise = which && which[0] == 'w';
  if (!old_kernel && !pairwise && tcg_eligible(ta)) return launch_beams_tcg(ta, nsm, st);
  if (!old_kernel && tcw_eligible(ta)) {
    TcArgs tw = ta;
    tw.b1 = ta.b1w;
    tw.b2 = ta.b2w;
    return launch_beams_tcw(tw, nsm, st);
  }
  if (ta.split || !(pipe && pipe[0] && pipe[0] != '0')) {   // the split form is serial only
    const TcSmem L = tc_smem_layout(a.nx * a.ny, ta.split != 0, ta.w4 != 0);
    // at most 8 CTAs of 64 TMEM columns per SM: keep a ninth from fitting (registers and
    // shared memory hold it at 6 on the 4x256 lattice for FP16 with real weights, 5 for
    // BF16, 3 for the split form)
    size_t smem = (size_t)L.total;
    if (smem < 26 * 1024) smem = 26 * 1024;
    if (smem > 200 * 1024) return set_error(FFTBF_EUNSUPPORTED, "tensor-core form: lattice too large");
    const bool ny256 = (ta.split || ta.bf16 || ta.w4) && a.ew_dft && a.nx == 4 && a.ny == 256 &&
                       a.nyf == 256 && (reinterpret_cast<uintptr_t>(a.volts) & 15) == 0;
    auto kern = ta.split ? (ny256 ? beams_tc_kernel<false, true, true> : beams_tc_kernel<false, true>)
                         : (ta.bf16 ? (ny256 ? beams_tc_kernel<true, false, true>
                                             : beams_tc_kernel<true, false>)
                                    : (ny256 ? beams_tc_kernel<false, false, true>
                                             : beams_tc_kernel<false, false>));
    FFTBF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FFTBF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                        cudaSharedmemCarveoutMaxShared));
    int per_sm = 0;
    int rc = tc_residency((const void*)kern, smem, tcl::NT, 8, &per_sm);
    if (rc != FFTBF_OK) return rc;
    const int64_t grid = items < (int64_t)nsm * per_sm ? items : (int64_t)nsm * per_sm;
    kern<<<(unsigned)grid, tcl::NT, smem, st>>>(ta);
    FFTBF_CUDA_TRY(cudaGetLastError());
    return FFTBF_OK;
  }
  const TcPipeSmem L = tcp_smem_layout(a.nx * a.ny);
  // at most 2 CTAs of 256 TMEM columns per SM: keep a third from fitting
  size_t smem = (size_t)L.total;
  if (smem < 77 * 1024) smem = 77 * 1024;
  if (smem > 200 * 1024) return set_error(FFTBF_EUNSUPPORTED, "tensor-core form: lattice too large");
  auto kern = ta.bf16 ? beams_tc_pipe_kernel<true> : beams_tc_pipe_kernel<false>;
  FFTBF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  FFTBF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      cudaSharedmemCarveoutMaxShared));
  int per_sm = 0;
  int rc = tc_residency((const void*)kern, smem, tcp::NT, 2, &per_sm);
  if (rc != FFTBF_OK) return rc;
  const int64_t grid = items < (int64_t)nsm * per_sm ? items : (int64_t)nsm * per_sm;
  kern<<<(unsigned)grid, tcp::NT, smem, st>>>(ta);
  FFTBF_CUDA_TRY(cudaGetLastError());
  return FFTBF_OK;
}

// ---------------------------------------------------------------- plan tables --
// Real-embedded DFT matrices, transposed (row = output, column = input), interleaved
// (re, im): B1t[2k1 + co][2n1 + ci] from W32^(n1 k1) for n1 < 16, k1 < 32 (the pruned
// stage 1), B2t[2k2 + co][2n2 + ci] from W16^(n2 k2). FP64, rounded once to 16 bits.
// lo != 0: the FP16 residual v - fp16(v) instead (the low half of a split FP16 operand).
__global__ void tc_tables_kernel(uint16_t* b1, uint16_t* b2, int bf16, int lo) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  auto entry = [](int out_c, int in_c, double c, double sp) {
    // X_re = x_re C - x_im S', X_im = x_re S' + x_im C with W = C + i S'
    if (out_c == 0) return in_c == 0 ? c : -sp;
    return in_c == 0 ? sp : c;
  };
  auto store = [&](uint16_t* dst, double v) {
    if (bf16) {
      __nv_bfloat16 h = __float2bfloat16_rn((float)v);
      *dst = *reinterpret_cast<uint16_t*>(&h);
    } else if (lo) {
      const __half hi = __float2half_rn((float)v);
      __half h = __float2half_rn((float)(v - (double)__half2float(hi)));
      *dst = *reinterpret_cast<uint16_t*>(&h);
    } else {
      __half h = __float2half_rn((float)v);
      *dst = *reinterpret_cast<uint16_t*>(&h);
    }
  };
  if (i < 64 * 32) {
    const int row = i >> 5, col = i & 31;
    const int k1 = row >> 1, co = row & 1, n1 = col >> 1, ci = col & 1;
    double s, c;
    sincospi(2.0 * ((n1 * k1) % 32) / 32.0, &s, &c);
    store(b1 + i, entry(co, ci, c, -s));
  }
  if (i < 32 * 32) {
    const int row = i >> 5, col = i & 31;
    const int k2 = row >> 1, co = row & 1, n2 = col >> 1, ci = col & 1;
    double s, c;
    sincospi(2.0 * ((n2 * k2) % 16) / 16.0, &s, &c);
    store(b2 + i, entry(co, ci, c, -s));
  }
}

int build_tc_tables(uint16_t* b1, uint16_t* b2, bool bf16, cudaStream_t st) {
  tc_tables_kernel<<<(64 * 32 + 255) / 256, 256, 0, st>>>(b1, b2, bf16 ? 1 : 0, 0);
  FFTBF_CUDA_TRY(cudaGetLastError());
  return FFTBF_OK;
}

int build_tc_tables_lo(uint16_t* b1, uint16_t* b2, cudaStream_t st) {
  tc_tables_kernel<<<(64 * 32 + 255) / 256, 256, 0, st>>>(b1, b2, 0, 1);
  FFTBF_CUDA_TRY(cudaGetLastError());
  return FFTBF_OK;
}

// ------------------------------------------------------------ GEMM test hook --
// D[128][n] = A[128][32] * B[n][32]^T with 16-bit operands (FP16 or BF16) in the
// canonical layout (A's strides padded like the stage-2 operand if `padded`), one MMA
// pair, FP32 in TMEM, read back with tcgen05.ld. Layout 3 puts A in tensor memory (row m
// in lane m, two elements per column, written with tcgen05.st) and layout 4 stores B
// MN-major, the two operand forms of the grouped kernel.
template <bool BF16>
__global__ void __launch_bounds__(128, 1) debug_tc_gemm_kernel(const uint16_t* A, const uint16_t* B,
                                                                int n, int padded, float* D, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_tc[];
  unsigned char* smem = smem_tc;
  // padded: 0 canonical K-major A, 1 K-major with the stage-2 operand's padded strides,
  // 2 MN-major A (element (m, k) at (m%8)*2 + (k%8)*16 + (m/8)*128 + (k/8)*2048),
  // 3 A in tensor memory (columns 224..239), 4 canonical A and MN-major B (element (n, k)
  // at (n%8)*2 + (k%8)*16 + (n/8)*128 + (k/8)*16n)
  const bool mn = padded == 2, a_tmem = padded == 3, b_mn = padded == 4;
  if (padded > 2) padded = 0;
  const int albo = mn ? 2048 : (padded ? tcl::A2_LBO : tcl::A1_LBO);
  const int asbo = mn ? 128 : (padded ? tcl::A2_SBO : tcl::A1_SBO);
  unsigned char* as = smem;
  unsigned char* bs = smem + (mn ? 8192 : 16 * asbo);
  uint64_t* bar = reinterpret_cast<uint64_t*>(bs + (n / 8) * tcl::B_SBO);
  uint32_t* taddr_sm = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    tc::tmem_alloc(taddr_sm, 256);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(bar, 1);
    tc::mbar_init_fence();
  }
  if (mn) {
    for (int i = tid; i < 128 * 32; i += 128) {
      const int m = i >> 5, k = i & 31;
      *reinterpret_cast<uint16_t*>(as + (m & 7) * 2 + (k & 7) * 16 + (m >> 3) * asbo + (k >> 3) * albo) =
          A[m * 32 + k];
    }
  } else if (!a_tmem) {
    load_kmajor(as, A, 128, albo, asbo, tid, 128);
  }
  const int blbo = b_mn ? 16 * n : tcl::B_LBO, bsbo = b_mn ? 128 : tcl::B_SBO;
  if (b_mn) {
    for (int i = tid; i < n * 32; i += 128) {
      const int m = i >> 5, k = i & 31;
      *reinterpret_cast<uint16_t*>(bs + (m & 7) * 2 + (k & 7) * 16 + (m >> 3) * bsbo + (k >> 3) * blbo) =
          B[m * 32 + k];
    }
  } else {
    load_kmajor(bs, B, n, tcl::B_LBO, tcl::B_SBO, tid, 128);
  }
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *taddr_sm;
  if (a_tmem) {
    uint32_t r[16];
    for (int j = 0; j < 16; ++j) r[j] = (uint32_t)A[tid * 32 + 2 * j] | ((uint32_t)A[tid * 32 + 2 * j + 1] << 16);
    tc::tmem_st16(tbase + ((uint32_t)(32 * warp) << 16) + 224, r);
    tc::tmem_wait_st();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
  }
  if (tid == 0) {
    const uint32_t id = tc::idesc_f16(128, n, BF16) | (mn ? (1u << 15) : 0u) | (b_mn ? (1u << 16) : 0u);
    for (int kk = 0; kk < 2; ++kk) {
      const uint64_t bd = tc::smem_desc(tc::smem_u32(bs) + kk * 2 * blbo, blbo, bsbo);
      if (a_tmem)
        tc::mma_f16_ts(tbase, tbase + 224 + 8 * kk, bd, id, kk);
      else
        tc::mma_f16(tbase, tc::smem_desc(tc::smem_u32(as) + kk * 2 * albo, albo, asbo), bd, id, kk);
    }
    tc::mma_commit(bar);
  }
  const bool ok = __syncthreads_and(tc::mbar_wait(bar, 0, tcl::WAIT_NS));
  tc::fence_after_sync();
  if (ok) {
    for (int c0 = 0; c0 < n; c0 += 32) {
      uint32_t r[32];
      tc::tmem_ld32(tbase + ((uint32_t)(32 * warp) << 16) + c0, r);
      tc::tmem_wait_ld();
      for (int j = 0; j < 32; ++j) D[(32 * warp + lane) * n + c0 + j] = __uint_as_float(r[j]);
    }
  } else if (tid == 0) {
    atomicExch(err, FFTBF_ETIMEOUT);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, 256);
}

// Wait, with the kernels' bounded wait, on an mbarrier that nothing arrives on: the wait
// runs out after limit_ns and the kernel records FFTBF_ETIMEOUT instead of hanging.
__global__ void debug_wait_timeout_kernel(uint64_t limit_ns, int* err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::mbar_init_fence();
  }
  __syncthreads();
  const bool ok = tc::mbar_wait(&bar, 0, limit_ns);
  if (!ok && threadIdx.x == 0) atomicExch(err, FFTBF_ETIMEOUT);
}

int launch_debug_wait_timeout(uint64_t limit_ns, int* err, cudaStream_t st) {
  debug_wait_timeout_kernel<<<1, 32, 0, st>>>(limit_ns, err);
  FFTBF_CUDA_TRY(cudaGetLastError());
  return FFTBF_OK;
}

int launch_debug_tc_gemm(const uint16_t* A, const uint16_t* B, int n, bool bf16, int layout,
                         float* D, int* err, cudaStream_t st) {
  const bool padded = layout == 1;
  const int asbo = padded ? tcl::A2_SBO : tcl::A1_SBO;
  if (layout > 2 && n > 128) return set_error(FFTBF_EINVAL, "layouts 3 and 4 take n <= 128");
  const size_t smem = (layout == 2 ? 8192 : 16 * asbo) + (n / 8) * tcl::B_SBO + 64;
  auto kern = bf16 ? debug_tc_gemm_kernel<true> : debug_tc_gemm_kernel<false>;
  FFTBF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<1, 128, smem, st>>>(A, B, n, layout, D, err);
  FFTBF_CUDA_TRY(cudaGetLastError());
  return FFTBF_OK;
}

}  // namespace fftbf

// Tensor-core FP16 and BF16 forms of the FFT-beam hot path on the 4x256 lattice (4 E-W
// beams x 512 N-S beams, Eq. fftbeamform with the N-S axis zero-padded to 2n, Eq. b2n-1),
// with four snapshots per stage-1 MMA and every intermediate kept in tensor memory.
//
// The 512-point N-S transform of each (snapshot, E-W beam A) is split as 512 = 32 x 16
// (n = n2 + 16 n1, k = k1 + 32 k2; inputs with n1 >= 16 are the padding), and the 4-point
// E-W DFT is folded into the first stage:
//   stage 1 (tcgen05.mma M=128 N=128 K=128): D1[(A, k1)][(g, co, n2)] =
//       sum over (ix, n1) of (-i)^(A ix) W32^(n1 k1) z[g][ix][n2 + 16 n1],
//     the stage matrix F1 (rows (A, k1), K = (ix, re/im, n1)) is the A operand in shared
//     memory and the weighted voltages of four snapshots g are the B operand (MN-major),
//     each snapshot twice: as (re; im) for the real part of the output (co = 0) and as
//     (im; -re) for the imaginary part (co = 1), so that both land in the same TMEM lane;
//   twiddle: TMEM lane (A, k1) reads its 16 complex values Y[n2], multiplies them by
//     W512^(n2 k1) in FP32, rounds once to 16 bits and writes them back to tensor memory
//     as row (A, k1) of the stage-2 A operand (K = (re/im, n2)): no transpose, no shared
//     memory;
//   stage 2 (tcgen05.mma M=128 N=32 K=32, A in tensor memory): the 16-point DFT over n2,
//     D2[(A, k1)][(co, k2)] = X[A][k1 + 32 k2], written over the drained D1 columns; the
//     thread owning lane (A, k1) squares it and integrates over time and polarisation in
//     registers (Eq. bf).
// Per snapshot the shared-memory traffic is the 8 KB data operand (written once, read once
// by the tensor core), 8 KB of stage-matrix reads and 2 KB of stage-2 matrix reads, plus
// the 1 KB of voltages.
//
// Roles (16 warps, one CTA per SM: all 512 TMEM columns), one group = four consecutive
// snapshots of the CTA's sequence (its items blockIdx.x, + gridDim.x, ... one after the
// other, so a group may straddle two items):
//   warps 0-3   input: warp ix unpacks E-W row ix of the group's four snapshots (lane
//               (n1, h): feeds n2 = 8h .. 8h+7), weights them and stores the B operand;
//   warps 4-7   twiddle: D1 lanes 32 (w-4) .. + 31 -> W512 -> stage-2 operand in TMEM;
//   warps 8-11  detection: D2 of the same lanes -> |X|^2 sums -> beams at an item's end;
//   warp 12     one thread: the eight stage-1 MMAs of a group (and the TMEM allocation);
//   warps 13, 15 one thread each: the stage-2 MMAs of snapshots 0, 1 (warp 13) and 2, 3
//               (warp 15) of a group (each tcgen05.mma holds its issuing thread for ~90
//               cycles, so two threads issue the group's eight in about half the time);
//   warp 14     one thread: bulk copies of the raw bytes (2 KB per time sample of two
//               polarisations, 1 KB per snapshot otherwise).
// Tensor memory: columns 0..383 hold three groups' D slots (128 columns: 32 per snapshot,
// D1 and then D2 over it), 384..511 two groups' stage-2 operands (64 columns: 16 per
// snapshot). Hand-offs are mbarriers, one per ring stage and group; every wait is bounded
// by one second of device time, after which the CTA records FFTBF_ETIMEOUT, every role
// leaves its loop, the issuing threads wait (bounded) for their copies and MMAs in
// flight, and the tensor memory is freed.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "beam_fp32.cuh"
#include "tc_ptx.cuh"

namespace fftbf {

namespace tcg {
constexpr int NT = 512;                       // 16 warps
constexpr int G = 4;                          // snapshots per group
constexpr int NANT = 1024;                    // feeds of the 4x256 lattice
constexpr int NR = 6;                         // raw-byte ring (groups of 4 KB)
constexpr int NB = 3;                         // B-operand ring (groups of 32 KB)
constexpr int ND = 3;                         // TMEM D ring (groups of 128 columns)
constexpr int NA = 2;                         // TMEM stage-2 operand ring (groups of 64)
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t A2_COL = 128 * ND;
// B operand (MN-major, N = 128 = (g, co, n2), K = 128 = (ix, ci, n1)): element (n, k) at
//   (n % 8) * 2 + (k % 8) * 16 + (n / 8) * B1_SBO + (k / 8) * B1_LBO
constexpr int B1_SBO = 128, B1_LBO = 2048, B1_TILE = 128 * 128 * 2;
// stage matrices, K-major: F1 [m 128][k 128], F2 [n 32][k 32]
constexpr int F1_LBO = 128, F1_SBO = 2048;
constexpr int F2_LBO = 128, F2_SBO = 512;
// RAWF/RAWE per raw stage, B1F/B1E per B stage, D1F/D2F/D2E per D slot, A2F/A2E per
// stage-2 operand slot
enum { RAWF = 0, RAWE = RAWF + NR, B1F = RAWE + NR, B1E = B1F + NB, D1F = B1E + NB,
       D2F = D1F + ND, D2E = D2F + ND, A2F = D2E + ND, A2E = A2F + NA, NBAR = A2E + NA };
constexpr uint64_t WAIT_NS = 1000000000ull;

struct Smem {
  int f1, f2, b1, raw, bars, misc, total;
};
__host__ __device__ inline Smem layout() {
  Smem L;
  int o = 0;
  auto take = [&](int bytes) { int r = o; o += (bytes + 127) & ~127; return r; };
  L.f1 = take(128 * 128 * 2);
  L.f2 = take(32 * 32 * 2);
  L.b1 = take(NB * B1_TILE);
  L.raw = take(NR * G * NANT);
  L.bars = take(NBAR * 8);
  L.misc = take(16);
  L.total = o;
  return L;
}
}  // namespace tcg

namespace {

__device__ __forceinline__ __half2 h2(uint32_t v) { return *reinterpret_cast<__half2*>(&v); }
__device__ __forceinline__ uint32_t u32(__half2 v) { return *reinterpret_cast<uint32_t*>(&v); }
// A value pair computed in packed half as the form's operand type (BF16: rounded once)
template <bool BF16>
__device__ __forceinline__ uint32_t as_operand(__half2 v) {
  if constexpr (BF16) {
    const __nv_bfloat162 b = __float22bfloat162_rn(__half22float2(v));
    return *reinterpret_cast<const uint32_t*>(&b);
  } else {
    return u32(v);
  }
}
// An FP32 pair rounded once to the operand type (low half = .x)
template <bool BF16>
__device__ __forceinline__ uint32_t pack_operand(float2 v) {
  if constexpr (BF16) {
    const __nv_bfloat162 b = __float22bfloat162_rn(v);
    return *reinterpret_cast<const uint32_t*>(&b);
  } else {
    return u32(__floats2half2_rn(v.x, v.y));
  }
}

}  // namespace

template <bool REALW, bool BF16>
__global__ void __launch_bounds__(tcg::NT, 1) beams_tcg_kernel(const TcArgs ta) {
  using namespace tcg;
  const BeamArgs& a = ta.b;
  extern __shared__ __align__(1024) unsigned char smem_tcg[];
  unsigned char* smem = smem_tcg;
  const Smem L = layout();
  unsigned char* b1 = smem + L.b1;
  unsigned char* raw = smem + L.raw;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bars);
  uint32_t* taddr_sm = reinterpret_cast<uint32_t*>(smem + L.misc);
  volatile int* abort_sm = reinterpret_cast<volatile int*>(smem + L.misc + 4);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t nitems = a.nwin * a.nfreq;
  const int nsnap = a.n_int * a.npol;
  if ((int64_t)blockIdx.x >= nitems) return;
  const int64_t my_items = (nitems - 1 - blockIdx.x) / gridDim.x + 1;
  const int64_t total = my_items * nsnap;             // snapshots of this CTA
  const int64_t ngroups = (total + G - 1) / G;

  // ---- set-up: tensor memory, barriers, stage matrices
  if (warp == 12) {
    tc::tmem_alloc(taddr_sm, TMEM_COLS);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    for (int i = 0; i < NBAR; ++i) {
      uint32_t c = 4;                                  // one arrival per warp of a role
      if ((i >= RAWF && i < RAWF + NR) || (i >= B1E && i < B1E + NB) ||
          (i >= D1F && i < D1F + ND))
        c = 1;                                         // expect_tx arrival or MMA commit
      if ((i >= D2F && i < D2F + ND) || (i >= A2E && i < A2E + NA)) c = 2;   // two issuers

      tc::mbar_init(bars + i, c);
    }
    tc::mbar_init_fence();
    *abort_sm = 0;
  }
  {
    const uint16_t* f1 = ta.f1;
    for (int i = tid; i < 128 * 64; i += NT) {
      const int m = i >> 6, k = (i & 63) * 2;
      *reinterpret_cast<uint32_t*>(smem + L.f1 + tc::kmajor_off(m, k, F1_LBO, F1_SBO)) =
          (uint32_t)f1[m * 128 + k] | ((uint32_t)f1[m * 128 + k + 1] << 16);
    }
    const uint16_t* f2 = ta.b2;
    for (int i = tid; i < 32 * 16; i += NT) {
      const int m = i >> 4, k = (i & 15) * 2;
      *reinterpret_cast<uint32_t*>(smem + L.f2 + tc::kmajor_off(m, k, F2_LBO, F2_SBO)) =
          (uint32_t)f2[m * 32 + k] | ((uint32_t)f2[m * 32 + k + 1] << 16);
    }
  }
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *taddr_sm;
  auto fail = [&]() {
    *abort_sm = 1;
    atomicExch(ta.err, FFTBF_ETIMEOUT);
  };
  auto wait_sleep = [&](int bar, uint32_t parity) -> bool {
    if (tc::mbar_wait_sleep(bars + bar, parity, WAIT_NS, abort_sm)) return true;
    fail();
    return false;
  };
  // the same, agreed by the whole warp (a lane never leaves a role loop alone)
  auto wait_warp = [&](int bar, uint32_t parity) -> bool {
    return __all_sync(0xffffffffu, wait_sleep(bar, parity)) != 0;
  };

  if (warp < 4) {
    // ============================================ input: voltages -> B operand
    const int ix = warp, n1 = lane & 15, h = lane >> 4;
    const int iy0 = 16 * n1 + 8 * h;                   // feeds (ix, iy0 .. iy0 + 7)
    // weights x scale / 16 (the unpacked voltages carry a factor 16), half2 over feed pairs
    uint32_t wr[4], wi[4];
    // BF16 form with real weights: the weights x scale as BF16 hi + lo parts, for voltages
    // unpacked straight to BF16 (no factor 16)
    __nv_bfloat162 wbh[4], wbl[4];
    const float sc = ta.scale * 0.0625f;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const float2 w0 = a.w[ix * 256 + iy0 + 2 * p], w1 = a.w[ix * 256 + iy0 + 2 * p + 1];
      wr[p] = u32(__halves2half2(__float2half_rn(w0.x * sc), __float2half_rn(w1.x * sc)));
      wi[p] = u32(__halves2half2(__float2half_rn(w0.y * sc), __float2half_rn(w1.y * sc)));
      const float2 wf = make_float2(w0.x * ta.scale, w1.x * ta.scale);
      wbh[p] = __float22bfloat162_rn(wf);
      const float2 hf = __bfloat1622float2(wbh[p]);
      wbl[p] = __float22bfloat162_rn(make_float2(wf.x - hf.x, wf.y - hf.y));
    }
    // byte offsets: raw (snapshot-relative) and B operand (k = 32 ix + 16 ci + n1,
    // n = 32 g + 16 co + 8 h + j); a quarter-warp's 16-byte stores fill 128 bytes
    const int roff = ix * 256 + iy0;
    const uint32_t boff = (uint32_t)((n1 & 7) * 16 + h * B1_SBO + (4 * ix + (n1 >> 3)) * B1_LBO);
    bool ok = true;
    for (int64_t k = 0; k < ngroups && ok; ++k) {
      const int r = (int)(k % NR), b = (int)(k % NB);
      if (!wait_warp(RAWF + r, (uint32_t)((k / NR) & 1))) { ok = false; break; }
      if (k >= NB && !wait_warp(B1E + b, (uint32_t)(((k / NB) - 1) & 1))) { ok = false; break; }
      const unsigned char* src = raw + r * (G * NANT) + roff;
      unsigned char* dst = b1 + b * B1_TILE + boff;
#pragma unroll
      for (int g = 0; g < G; ++g) {
        uint4 R = make_uint4(0u, 0u, 0u, 0u), I = R, Rn = R;
        if (G * k + g < total) {
          const uint2 wd = *reinterpret_cast<const uint2*>(src + g * NANT);
          uint32_t zr[4], zi[4];
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            if constexpr (BF16 && REALW) {
              // straight to BF16: each nibble, sign bit flipped, in the mantissa of 128 (ulp
              // 1), minus 136 leaves it exactly; the weight as hi + lo with one rounding of
              // re w_hi + (re w_lo)
              const uint32_t t = __byte_perm(p < 2 ? wd.x : wd.y, 0u, (p & 1) ? 0x4342u : 0x4140u);
              uint32_t ur = ((t >> 4) & 0x000F000Fu) ^ 0x43084308u, ui = (t & 0x000F000Fu) ^ 0x43084308u;
              const uint32_t k136 = 0x43084308u;
              const __nv_bfloat162 c136 = *reinterpret_cast<const __nv_bfloat162*>(&k136);
              const __nv_bfloat162 re = __hsub2(*reinterpret_cast<__nv_bfloat162*>(&ur), c136);
              const __nv_bfloat162 im = __hsub2(*reinterpret_cast<__nv_bfloat162*>(&ui), c136);
              const __nv_bfloat162 br = __hfma2(re, wbh[p], __hmul2_rn(re, wbl[p]));
              const __nv_bfloat162 bi = __hfma2(im, wbh[p], __hmul2_rn(im, wbl[p]));
              zr[p] = *reinterpret_cast<const uint32_t*>(&br);
              zi[p] = *reinterpret_cast<const uint32_t*>(&bi);
              continue;
            }
            // bytes of feeds 2p, 2p + 1 beside 0x64 bytes: [0x64 b1 0x64 b0]
            const uint32_t t = __byte_perm(p < 2 ? wd.x : wd.y, 0x64646464u, (p & 1) ? 0x4342u : 0x4140u);
            const __half2 re = __hsub2(h2((t & 0xFFF0FFF0u) ^ 0x00800080u), h2(0x64806480u));
            const __half2 im = __hsub2(h2((t & 0x000F000Fu) ^ 0x74087408u), h2(0x74087408u));
            __half2 vr, vi;
            if constexpr (REALW) {
              vr = __hmul2_rn(re, h2(wr[p]));
              vi = __hmul2_rn(im, h2(wr[p]));
            } else {
              vr = __hfma2(__hneg2(im), h2(wi[p]), __hmul2_rn(re, h2(wr[p])));
              vi = __hfma2(im, h2(wr[p]), __hmul2_rn(re, h2(wi[p])));
            }
            zr[p] = as_operand<BF16>(vr);
            zi[p] = as_operand<BF16>(vi);
          }
          R = make_uint4(zr[0], zr[1], zr[2], zr[3]);
          I = make_uint4(zi[0], zi[1], zi[2], zi[3]);
          Rn = make_uint4(zr[0] ^ 0x80008000u, zr[1] ^ 0x80008000u, zr[2] ^ 0x80008000u,
                          zr[3] ^ 0x80008000u);
        }
        unsigned char* d = dst + g * 4 * B1_SBO;
        *reinterpret_cast<uint4*>(d) = R;                                   // ci 0, co 0
        *reinterpret_cast<uint4*>(d + 2 * B1_SBO) = I;                      // ci 0, co 1
        *reinterpret_cast<uint4*>(d + 2 * B1_LBO) = I;                      // ci 1, co 0
        *reinterpret_cast<uint4*>(d + 2 * B1_LBO + 2 * B1_SBO) = Rn;        // ci 1, co 1
      }
      tc::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) {
        tc::mbar_arrive(bars + RAWE + r);
        tc::mbar_arrive(bars + B1F + b);
      }
    }
  } else if (warp < 8) {
    // ============================================ twiddle: D1 -> W512 -> stage-2 operand
    const int q = warp - 4, k1 = lane;                // TMEM lane (A = q, k1)
    // W512^(n2 k1) for n2 = 2p, 2p + 1 (FP32 table: cos, -sin)
    float2 tcs[8], tsn[8];
#pragma unroll
    for (int p = 0; p < 8; ++p) {
      const float2 u0 = a.tw[(2 * p * k1) & 511], u1 = a.tw[((2 * p + 1) * k1) & 511];
      tcs[p] = make_float2(u0.x, u1.x);
      tsn[p] = make_float2(u0.y, u1.y);
    }
    const uint32_t lanes = (uint32_t)(32 * q) << 16;
    for (int64_t k = 0; k < ngroups; ++k) {
      const int d = (int)(k % ND), s = (int)(k % NA);
      if (!wait_warp(D1F + d, (uint32_t)((k / ND) & 1))) break;
      if (k >= NA && !wait_warp(A2E + s, (uint32_t)(((k / NA) - 1) & 1))) break;
      tc::fence_after_sync();
#pragma unroll 1
      for (int g = 0; g < G; ++g) {
        uint32_t v[32];                                // re Y[n2 0..15], then im
        tc::tmem_ld32(tbase + lanes + 128 * d + 32 * g, v);
        tc::tmem_wait_ld();
        uint32_t o[16];                                // re Y'[n2] pairs, then im
#pragma unroll
        for (int p = 0; p < 8; ++p) {
          const float2 yr = make_float2(__uint_as_float(v[2 * p]), __uint_as_float(v[2 * p + 1]));
          const float2 yi = make_float2(__uint_as_float(v[16 + 2 * p]), __uint_as_float(v[17 + 2 * p]));
          const float2 zr = __ffma2_rn(yr, tcs[p], __fmul2_rn(yi, make_float2(-tsn[p].x, -tsn[p].y)));  // re c - im s
          const float2 zi = __ffma2_rn(yr, tsn[p], __fmul2_rn(yi, tcs[p]));                             // re s + im c
          o[p] = pack_operand<BF16>(zr);
          o[8 + p] = pack_operand<BF16>(zi);
        }
        tc::tmem_st16(tbase + lanes + A2_COL + 64 * s + 16 * g, o);
      }
      tc::tmem_wait_st();
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(bars + A2F + s);
    }
  } else if (warp < 12) {
    // ============================================ detection: D2 -> |X|^2 -> beams
    const int q = warp - 8;
    const uint32_t lanes = (uint32_t)(32 * q) << 16;
    float2 acc[8];                                     // |X|^2 sums of k2 = 2p, 2p + 1
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = make_float2(0.f, 0.f);
    const float inv_s2 = 1.0f / (ta.scale * ta.scale);
    int64_t item = blockIdx.x, S = 0;
    int j = 0;
    for (int64_t k = 0; k < ngroups; ++k) {
      const int d = (int)(k % ND);
      if (!wait_warp(D2F + d, (uint32_t)((k / ND) & 1))) break;
      tc::fence_after_sync();
#pragma unroll 1
      for (int g = 0; g < G && S < total; ++g, ++S) {
        uint32_t v[32];                                // re X[k2 0..15], then im
        tc::tmem_ld32(tbase + lanes + 128 * d + 32 * g, v);
        tc::tmem_wait_ld();
#pragma unroll
        for (int p = 0; p < 8; ++p) {
          const float2 xr = make_float2(__uint_as_float(v[2 * p]), __uint_as_float(v[2 * p + 1]));
          const float2 xi = make_float2(__uint_as_float(v[16 + 2 * p]), __uint_as_float(v[17 + 2 * p]));
          acc[p] = __ffma2_rn(xi, xi, __ffma2_rn(xr, xr, acc[p]));
        }
        if (++j == nsnap) {
          // last snapshot of the item: beams[item][A = q][k1 = lane + 32 k2]
          float* dst = a.beams + item * (int64_t)(4 * 512) + q * 512 + lane;
#pragma unroll
          for (int p = 0; p < 8; ++p) {
            dst[64 * p] = acc[p].x * inv_s2;
            dst[64 * p + 32] = acc[p].y * inv_s2;
            acc[p] = make_float2(0.f, 0.f);
          }
          j = 0;
          item += gridDim.x;
        }
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(bars + D2E + d);
    }
  } else if (warp == 12) {
    if (lane == 0) {
      // ========================================== stage-1 MMAs
      const uint32_t id1 = tc::idesc_f16(128, 128, BF16) | (1u << 16);   // B MN-major
      const uint32_t sf1 = tc::smem_u32(smem + L.f1), sb1 = tc::smem_u32(b1);
      int64_t k = 0;
      for (; k < ngroups; ++k) {
        const int b = (int)(k % NB), d = (int)(k % ND);
        if (!wait_sleep(B1F + b, (uint32_t)((k / NB) & 1))) break;
        if (k >= ND && !wait_sleep(D2E + d, (uint32_t)(((k / ND) - 1) & 1))) break;
        tc::fence_after_sync();
#pragma unroll
        for (int kk = 0; kk < 8; ++kk)
          tc::mma_f16(tbase + 128 * d, tc::smem_desc(sf1 + kk * 2 * F1_LBO, F1_LBO, F1_SBO),
                      tc::smem_desc(sb1 + b * B1_TILE + kk * 2 * B1_LBO, B1_LBO, B1_SBO), id1,
                      kk > 0 ? 1u : 0u);
        tc::mma_commit(bars + D1F + d);
        tc::mma_commit(bars + B1E + b);
      }
      // every MMA issued must have completed before the CTA frees its memory
      if (k > 0) tc::mbar_wait(bars + D1F + (int)((k - 1) % ND), (uint32_t)(((k - 1) / ND) & 1), WAIT_NS);
    }
  } else if (warp == 13 || warp == 15) {
    if (lane == 0) {
      // ========================================== stage-2 MMAs (A in tensor memory) of
      // snapshots g0, g0 + 1 of each group
      const int g0 = warp == 13 ? 0 : 2;
      const uint32_t id2 = tc::idesc_f16(128, 32, BF16);
      const uint32_t sf2 = tc::smem_u32(smem + L.f2);
      const uint64_t df2[2] = {tc::smem_desc(sf2, F2_LBO, F2_SBO),
                               tc::smem_desc(sf2 + 2 * F2_LBO, F2_LBO, F2_SBO)};
      int64_t k = 0;
      for (; k < ngroups; ++k) {
        const int s = (int)(k % NA), d = (int)(k % ND);
        if (!wait_sleep(A2F + s, (uint32_t)((k / NA) & 1))) break;
        tc::fence_after_sync();
#pragma unroll
        for (int g = g0; g < g0 + 2; ++g)
#pragma unroll
          for (int kk = 0; kk < 2; ++kk)
            tc::mma_f16_ts(tbase + 128 * d + 32 * g, tbase + A2_COL + 64 * s + 16 * g + 8 * kk,
                           df2[kk], id2, kk > 0 ? 1u : 0u);
        tc::mma_commit(bars + D2F + d);
        tc::mma_commit(bars + A2E + s);
      }
      if (k > 0) tc::mbar_wait(bars + D2F + (int)((k - 1) % ND), (uint32_t)(((k - 1) / ND) & 1), WAIT_NS);
    }
  } else if (warp == 14) {
    if (lane == 0) {
      // ========================================== raw-byte copies
      int64_t item = blockIdx.x, S = 0;
      int j = 0;
      const uint8_t* ibase = item_volts(a, item, NANT);
      const int64_t tstride = (int64_t)a.nfreq * a.npol * NANT;   // one time sample
      const bool two_pol = a.npol == 2;                             // nsnap even
      int64_t k = 0;
      for (; k < ngroups; ++k) {
        const int r = (int)(k % NR);
        if (k >= NR && !wait_sleep(RAWE + r, (uint32_t)(((k / NR) - 1) & 1))) break;
        const int nv = total - S < G ? (int)(total - S) : G;       // snapshots in the group
        uint64_t* bar = bars + RAWF + r;
        tc::mbar_arrive_expect_tx(bar, (uint32_t)(nv * NANT));
        unsigned char* dst = raw + r * (G * NANT);
        for (int g = 0; g < nv;) {
          if (two_pol) {                               // snapshots j, j + 1: one time sample
            tc::bulk_g2s(dst + g * NANT, ibase + (int64_t)(j >> 1) * tstride, 2 * NANT, bar);
            g += 2;
            j += 2;
          } else {
            tc::bulk_g2s(dst + g * NANT, ibase + snap_offset(a, j, NANT), NANT, bar);
            g += 1;
            j += 1;
          }
          if (j == nsnap) {
            j = 0;
            item += gridDim.x;
            if (item < nitems) ibase = item_volts(a, item, NANT);
          }
        }
        S += nv;
      }
      // every copy issued must have landed before the CTA exits
      for (int64_t kk = k - 1; kk >= 0 && kk >= k - NR; --kk)
        tc::mbar_wait(bars + RAWF + (int)(kk % NR), (uint32_t)((kk / NR) & 1), WAIT_NS);
    }
  }
  __syncwarp();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 12) tc::tmem_dealloc(tbase, TMEM_COLS);
}

bool tcg_eligible(const TcArgs& ta) {
  const BeamArgs& a = ta.b;
  return !ta.split && ta.f1 && ta.b2w && a.nx == 4 && a.ny == 256 && a.mx == 4 && a.my == 512 &&
         a.nyf == 256 && a.ew_dft && (reinterpret_cast<uintptr_t>(a.volts) & 15) == 0;
}

int launch_beams_tcg(const TcArgs& ta, int nsm, cudaStream_t st) {
  const BeamArgs& a = ta.b;
  const int64_t items = a.nwin * a.nfreq;
  if (items <= 0) return FFTBF_OK;
  const tcg::Smem L = tcg::layout();
  // one CTA per SM (all 512 tensor-memory columns); the shared memory keeps a second
  // CTA from becoming resident and waiting for tensor memory
  const size_t smem = (size_t)L.total;
  static_assert(tcg::NR * tcg::G * tcg::NANT + tcg::NB * tcg::B1_TILE > 114 * 1024,
                "shared memory must hold the kernel to one CTA per SM");
  auto kern = ta.bf16 ? (a.real_w ? beams_tcg_kernel<true, true> : beams_tcg_kernel<false, true>)
                      : (a.real_w ? beams_tcg_kernel<true, false> : beams_tcg_kernel<false, false>);
  FFTBF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  TcArgs tg = ta;
  tg.b2 = ta.b2w;                                      // planar W16 stage matrix
  const int64_t grid = items < (int64_t)nsm ? items : (int64_t)nsm;
  kern<<<(unsigned)grid, tcg::NT, smem, st>>>(tg);
  FFTBF_CUDA_TRY(cudaGetLastError());
  return FFTBF_OK;
}

// ---------------------------------------------------------------- plan table --
// F1[m = 32 A + k1][k = 32 ix + 16 ci + n1]: the E-W DFT and the pruned 32-point N-S DFT
// in one complex coefficient c = (-i)^(A ix) W32^(n1 k1) = exp(-2 pi i (8 A ix + n1 k1) / 32),
// real-embedded for a B operand that holds (re; im) of the data: ci = 0 -> Re c, ci = 1 ->
// -Im c. FP64, rounded once to FP16 (BF16 when bf16).
__global__ void tcg_f1_kernel(uint16_t* f1, bool bf16) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 128 * 128) return;
  const int m = i >> 7, k = i & 127;
  const int A = m >> 5, k1 = m & 31, ix = k >> 5, ci = (k >> 4) & 1, n1 = k & 15;
  const int phi = (8 * A * ix + n1 * k1) & 31;
  double sn, cs;
  sincospi(2.0 * phi / 32.0, &sn, &cs);
  const double v = ci == 0 ? cs : sn;                  // c = cs - i sn
  if (bf16) {
    const __nv_bfloat16 x = __double2bfloat16(v);
    f1[i] = *reinterpret_cast<const uint16_t*>(&x);
  } else {
    const __half x = __float2half_rn((float)v);
    f1[i] = *reinterpret_cast<const uint16_t*>(&x);
  }
}

int build_tcg_table(uint16_t* f1, bool bf16, cudaStream_t st) {
  tcg_f1_kernel<<<128 * 128 / 256, 256, 0, st>>>(f1, bf16);
  FFTBF_CUDA_TRY(cudaGetLastError());
  return FFTBF_OK;
}

}  // namespace fftbf

// Tensor-core FP16 and BF16 forms of the FFT-beam hot path on the 4x256 lattice (4 E-W
// beams x 512 N-S beams, Eq. fftbeamform with the N-S axis zero-padded to 2n, Eq. b2n-1),
// as a warp-specialised pipeline. The two forms share the input stage, computed in packed
// half (the BF16 form rounds its results to BF16 as it stores the stage-1 operand), and
// differ in the stage matrices, the MMA instruction descriptor and the twiddle: packed
// half for FP16, FP32 rounded once to BF16 for BF16 (as the serial kernel does it).
//
// The 512-point N-S transform of each (snapshot, E-W beam) is split as 512 = 32 x 16
// (n = n2 + 16 n1, k = k1 + 32 k2; inputs with n1 >= 16 are the padding):
//   stage 1 (tcgen05.mma, M=128 N=64 K=32): rows (snapshot s, E-W beam A, n2) of a snapshot
//     pair, the pruned 32-point DFT over n1 as a real-embedded GEMM;
//   twiddle: X1 *= W512^(n2 k1) while draining TMEM, in packed half arithmetic (FP32 for
//     the BF16 form);
//   stage 2 (tcgen05.mma, M=128 N=32 K=32 per snapshot): rows (A, k1), a 16-point DFT over
//     n2 giving X[k1 + 32 k2]; the thread owning TMEM row (A, k1) squares it and integrates
//     over time and polarisation in registers (Eq. bf).
// Both GEMM A operands are stored MN-major (rows contiguous for each K element) with complex
// values planar along K (real parts at K 0..15, imaginary parts at K 16..31), so that:
//   * the input stage packs two adjacent N-S feeds (adjacent rows n2) into one half2 and
//     writes 8 bytes per (E-W beam, component);
//   * the stage-1 drain packs two adjacent k1 (adjacent stage-2 rows) into one half2 and
//     writes 16 bytes per (component, 8 k1) instead of one 4-byte value per k1.
// The B operands (DFT matrices) stay K-major. Both stages' outputs are planar along N (real
// parts, then imaginary parts), so that the detector squares two adjacent beams k2, k2 + 1
// with one packed FFMA2 per component into one float2 accumulator.
//
// Unpacking: a voltage byte (bits 7..4 real, 3..0 imaginary, two's complement) is decoded
// exactly into FP16 by placing the real nibble in the mantissa of 1024 (ulp 1, nibble four
// bits up: 1024 + 16 (re ^ 8)) and the imaginary nibble in the mantissa of 16384 (ulp 16:
// 16384 + 16 (im ^ 8)), then subtracting 1152 and 16512: (16 re, 16 im), both exact. The
// factor 16 is folded into the FP16 weights (w / 16, a power of two, so the products
// round as w x would).
//
// Tensor memory holds a ring of four 64-column buffers: buffer t = P % 4 receives pair P's
// stage-1 result D1 (columns re k1, im k1), and, once the drain has read it, stage 2
// writes the pair's D2 (32 columns per snapshot) over the same columns; the detector frees
// the buffer for pair P + 4. Four pairs are thus in flight between stage 1 and detection.
//
// Roles (10 warps, 320 threads, two CTAs per SM by tensor memory: 256 columns each):
//   warps 0-3  rounds of two pairs: the input stage of pairs 2k, 2k+1 (bytes -> A1 tiles
//              P%4), then detection of pairs 2k-3, 2k-2 (D2 in buffers P%4 -> registers),
//              lane quarter = warp; one wait for the round's raw bytes, one for its A1
//              tiles, one arrival when both are written, one wait before detecting;
//   warps 4-7  stage-1 drain of pair P (D1 in buffer P%4 -> twiddle -> A2[P%2]), lane
//              quarter = warp-4;
//   warp 8     one thread: MMA1 of both pairs of round k once their A1 tiles are written
//              (each pair once its buffer is detected), then the bulk copies of round
//              k+RQ's raw bytes into the ring stages round k was read from (2 KB per pair,
//              both pairs counted on one barrier);
//   warp 9     one thread: MMA2(P) once A2[P%2] is written and D1 of buffer P%4 drained.
// Synchronisation, not arithmetic, paces this pipeline: each wait or arrival costs a few
// hundred cycles of latency under load, so the input role, which has the most of them per
// pair, does its waits and arrivals once per two pairs.
// Hand-offs are mbarriers (one elected arrival per warp after __syncwarp). Waiting threads
// are suspended (try_wait with a suspend-time hint) rather than spinning, so waiting warps
// take no issue slots. Every wait is bounded by one second of device time; on timeout the
// CTA records FFTBF_ETIMEOUT, every role leaves its loop, the issuing threads wait
// (bounded) for their copies and MMAs in flight, and the tensor memory is freed before
// exit.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "beam_fp32.cuh"
#include "tc_ptx.cuh"

namespace fftbf {

namespace tcw {
constexpr int NT = 320;
constexpr int NA2 = 2;                        // stage-2 operand tile pairs (pairs in flight)
constexpr int R = 8;                          // raw-byte ring stages (2 KB each, one pair)
constexpr int RQ = R / 2;                     // ... filled and waited for two pairs at a time
constexpr int NANT = 1024;                    // feeds of the 4x256 lattice
constexpr int NT4 = 4;                        // tensor-memory ring: pairs in flight
constexpr uint32_t TMEM_COLS = 64 * NT4;      // buffer t at columns 64 t: D1 of a pair, then
                                              // its D2 (stage 2 overwrites the drained D1)
// MN-major operand tiles (128 rows x 32 K, 16-bit): element (m, k) at
//   (m % 8) * 2 + (k % 8) * 16 + (m / 8) * SBO + (k / 8) * LBO
constexpr int SBO = 128, LBO = 2048, TILE = 8192;
constexpr int B_LBO = 128, B_SBO = 512;       // K-major DFT matrices
// RAWF per round stage; A1F, A1E per round parity (a round's two pairs use A1 tiles
// 2 (k % 2), + 1); D1F, D1E, D2F, D2E per tensor-memory buffer; A2F, A2E per A2 tile pair
enum { RAWF = 0, A1F = RAWF + RQ, A1E = A1F + 2, D1F = A1E + 2, D1E = D1F + NT4,
       A2F = D1E + NT4, A2E = A2F + NA2, D2F = A2E + NA2, D2E = D2F + NT4, NBAR = D2E + NT4 };
constexpr uint64_t WAIT_NS = 1000000000ull;

struct Smem {
  int a1, a2, b1, b2, w, twf, raw, bars, misc, total;
};
__host__ __device__ inline Smem layout() {
  Smem L;
  int o = 0;
  auto take = [&](int bytes) { int r = o; o += (bytes + 127) & ~127; return r; };
  L.a1 = take(4 * TILE);                 // A1[pair % 4]
  L.a2 = take(2 * NA2 * TILE);           // A2[b][s]
  L.b1 = take(64 * 32 * 2);
  L.b2 = take(32 * 32 * 2);
  L.w = take(2 * NANT * 2);              // FP16 weights: real part, then imaginary part
  L.twf = take(16 * 16 * 16);            // FP32 twiddles of the BF16 form, [j][n2] float4
  L.raw = take(R * 2 * NANT);
  L.bars = take(NBAR * 8);
  L.misc = take(16);
  L.total = o;
  return L;
}
}  // namespace tcw

namespace {

__device__ __forceinline__ __half2 as_h2(uint32_t v) { return *reinterpret_cast<__half2*>(&v); }
__device__ __forceinline__ uint32_t as_u(__half2 v) { return *reinterpret_cast<uint32_t*>(&v); }
// A stage-1 operand pair computed in packed half, as the form's operand type: itself for
// FP16, rounded to BF16 for the BF16 form (the FP16 value carries 11 significant bits, so
// this is the BF16 rounding of the exact value except within ~2^-12 of a BF16 boundary)
template <bool BF16>
__device__ __forceinline__ uint32_t operand(__half2 v) {
  if constexpr (BF16) {
    const __nv_bfloat162 b = __float22bfloat162_rn(__half22float2(v));
    return *reinterpret_cast<const uint32_t*>(&b);
  } else {
    return as_u(v);
  }
}

// The CTA's sequence of (work item, snapshot pair): items blockIdx.x, + gridDim.x, ...
struct PairSeq {
  int64_t item;
  int q;
  __device__ void next(int npairs) {
    if (++q == npairs) {
      q = 0;
      item += gridDim.x;
    }
  }
};

}  // namespace

template <bool REALW, bool BF16>
__global__ void __launch_bounds__(tcw::NT, 2) beams_tcw_kernel(const TcArgs ta) {
  using namespace tcw;
  const BeamArgs& a = ta.b;
  extern __shared__ __align__(1024) unsigned char smem_tcw[];
  unsigned char* smem = smem_tcw;
  const Smem L = layout();
  unsigned char* a1 = smem + L.a1;
  unsigned char* a2 = smem + L.a2;
  unsigned char* raw = smem + L.raw;
  const __half* wre = reinterpret_cast<const __half*>(smem + L.w);
  const __half* wim = wre + NANT;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bars);
  uint32_t* taddr_sm = reinterpret_cast<uint32_t*>(smem + L.misc);
  volatile int* abort_sm = reinterpret_cast<volatile int*>(smem + L.misc + 4);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t nitems = a.nwin * a.nfreq;
  const int nsnap = a.n_int * a.npol;
  const int npairs = (nsnap + 1) / 2;
  if ((int64_t)blockIdx.x >= nitems) return;
  const int64_t my_items = (nitems - 1 - blockIdx.x) / gridDim.x + 1;
  const int64_t total = my_items * npairs;            // snapshot pairs of this CTA

  // ---- set-up: tensor memory, barriers, DFT matrices, weights
  if (warp == 8) {
    tc::tmem_alloc(taddr_sm, TMEM_COLS);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    for (int i = 0; i < NBAR; ++i) {
      uint32_t c = 4;                                  // one arrival per warp of a role
      if ((i >= RAWF && i < RAWF + RQ) || (i >= A1E && i < A1E + 2) || (i >= D1F && i < D1F + NT4) ||
          (i >= A2E && i < A2E + NA2) || (i >= D2F && i < D2F + NT4))
        c = 1;                                         // expect_tx arrival or MMA commit
      tc::mbar_init(bars + i, c);
    }
    tc::mbar_init_fence();
    *abort_sm = 0;
  }
  {
    // B1 [n 64][k 32] and B2 [n 32][k 32] row-major -> canonical K-major tiles
    const uint16_t* src1 = ta.b1;
    const uint16_t* src2 = ta.b2;
    for (int i = tid; i < 64 * 16; i += NT) {
      const int m = i >> 4, k = (i & 15) * 2;
      *reinterpret_cast<uint32_t*>(smem + L.b1 + tc::kmajor_off(m, k, B_LBO, B_SBO)) =
          (uint32_t)src1[m * 32 + k] | ((uint32_t)src1[m * 32 + k + 1] << 16);
    }
    for (int i = tid; i < 32 * 16; i += NT) {
      const int m = i >> 4, k = (i & 15) * 2;
      *reinterpret_cast<uint32_t*>(smem + L.b2 + tc::kmajor_off(m, k, B_LBO, B_SBO)) =
          (uint32_t)src2[m * 32 + k] | ((uint32_t)src2[m * 32 + k + 1] << 16);
    }
    // weights x scale / 16 in FP16 (the unpacked voltages carry a factor 16)
    __half* w16 = reinterpret_cast<__half*>(smem + L.w);
    const float sc = ta.scale * 0.0625f;
    for (int i = tid; i < NANT; i += NT) {
      const float2 w = a.w[i];
      w16[i] = __float2half_rn(w.x * sc);
      w16[NANT + i] = __float2half_rn(w.y * sc);
    }
    if constexpr (BF16) {
      // (cos, cos, -sin, -sin) of W512^(n2 k1) for k1 = 2j, 2j + 1, from the plan's table
      float4* tw = reinterpret_cast<float4*>(smem + L.twf);
      for (int i = tid; i < 16 * 16; i += NT) {
        const int r = i >> 4, j = i & 15;
        const float2 w0 = a.tw[(r * 2 * j) & 511], w1 = a.tw[(r * (2 * j + 1)) & 511];
        tw[j * 16 + r] = make_float4(w0.x, w1.x, w0.y, w1.y);
      }
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
  // the same, agreed by the whole warp (a lane never leaves a role loop alone, so that the
  // warp's __syncwarp calls always see every lane)
  auto wait_warp = [&](int bar, uint32_t parity) -> bool {
    return __all_sync(0xffffffffu, wait_sleep(bar, parity)) != 0;
  };

  if (warp < 4) {
    // ============================================ input stage (pair P) + detection (P-2)
    // thread -> (snapshot s, K element n1, feeds n2 = 4 qn .. 4 qn + 3), chosen so that the
    // 8-byte A1 stores of each half-warp cover 128 contiguous bytes (no bank conflict)
    // and a warp's raw-byte loads cover 128 contiguous bytes
    const int s = tid >> 6, n1 = 8 * ((tid >> 5) & 1) + ((lane >> 1) & 7);
    const int qn = (lane & 1) | ((lane >> 4) << 1);
    // A1 offset of this thread's rows (s, A, n2 = 4 qn .. 4 qn + 3) at K element n1
    const uint32_t a1_off = (uint32_t)((qn & 1) * 8 + (n1 & 7) * 16 + (s * 8 + (qn >> 1)) * SBO +
                                       (n1 >> 3) * LBO);
    const int feed0 = 16 * n1 + 4 * qn;
    // weights of this thread's 16 feeds, as half2 pairs of adjacent N-S feeds
    uint32_t wr[4][2], wi[4][2];
#pragma unroll
    for (int ix = 0; ix < 4; ++ix) {
      const uint2 v = *reinterpret_cast<const uint2*>(wre + ix * 256 + feed0);
      wr[ix][0] = v.x;
      wr[ix][1] = v.y;
      if constexpr (!REALW) {
        const uint2 u = *reinterpret_cast<const uint2*>(wim + ix * 256 + feed0);
        wi[ix][0] = u.x;
        wi[ix][1] = u.y;
      }
    }
    float2 acc[8];                                    // |X|^2 sums of k2 = 2p, 2p + 1
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = make_float2(0.f, 0.f);
    const float inv_s2 = 1.0f / (ta.scale * ta.scale);
    PairSeq in{(int64_t)blockIdx.x, 0}, de{(int64_t)blockIdx.x, 0};
    bool ok = true;
    // round k: the input stage of pairs 2k and 2k + 1 (one raw-byte wait, one A1 wait and
    // one A1F arrival for both), then detection of pairs 2k - 3 and 2k - 2 (one D2F wait, on
    // the later pair: its stage-2 MMAs were committed after the earlier pair's)
    const int64_t nround = (total + 1) / 2;
    for (int64_t k = 0; k < nround + 2 && ok; ++k) {
      if (k < nround) {
        const int ab = (int)(k & 1);
        if (!wait_warp(RAWF + (int)(k % RQ), (uint32_t)((k / RQ) & 1))) { ok = false; break; }
        if (k >= 2 && !wait_warp(A1E + ab, (uint32_t)(((k >> 1) - 1) & 1))) { ok = false; break; }
#pragma unroll 1
        for (int j = 0; j < 2; ++j) {
          const int64_t P = 2 * k + j;
          if (P >= total) break;
          const int r = (int)(P % R), b = (int)(P & 3);   // raw stage, A1 tile
          const bool valid = s == 0 || 2 * in.q + 1 < nsnap;
          uint32_t o[4][2][2];                               // [A][re, im][n2 pair]
          if (valid) {
            uint32_t word[4];
#pragma unroll
            for (int ix = 0; ix < 4; ++ix)
              word[ix] = *reinterpret_cast<const uint32_t*>(raw + r * 2 * NANT + s * NANT + ix * 256 + feed0);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              __half2 zr[4], zi[4];
#pragma unroll
              for (int ix = 0; ix < 4; ++ix) {
                // bytes of feeds n2 = 4 qn + 2h, + 1 beside 0x64 bytes: [0x64 b1 0x64 b0]
                const uint32_t t = __byte_perm(word[ix], 0x64646464u, h ? 0x4342u : 0x4140u);
                const __half2 re = __hsub2(as_h2((t & 0xFFF0FFF0u) ^ 0x00800080u), as_h2(0x64806480u));
                const __half2 im = __hsub2(as_h2((t & 0x000F000Fu) ^ 0x74087408u), as_h2(0x74087408u));
                if constexpr (REALW) {
                  zr[ix] = __hmul2_rn(re, as_h2(wr[ix][h]));
                  zi[ix] = __hmul2_rn(im, as_h2(wr[ix][h]));
                } else {
                  const __half2 w_r = as_h2(wr[ix][h]), w_i = as_h2(wi[ix][h]);
                  zr[ix] = __hfma2(__hneg2(im), w_i, __hmul2_rn(re, w_r));
                  zi[ix] = __hfma2(im, w_r, __hmul2_rn(re, w_i));
                }
              }
              // 4-point E-W DFT, Y_A = sum_ix z_ix (-i)^(A ix), planar
              const __half2 ar = __hadd2(zr[0], zr[2]), ai = __hadd2(zi[0], zi[2]);
              const __half2 br = __hsub2(zr[0], zr[2]), bi = __hsub2(zi[0], zi[2]);
              const __half2 cr = __hadd2(zr[1], zr[3]), ci = __hadd2(zi[1], zi[3]);
              const __half2 dr = __hsub2(zr[1], zr[3]), di = __hsub2(zi[1], zi[3]);
              o[0][0][h] = operand<BF16>(__hadd2(ar, cr));
              o[0][1][h] = operand<BF16>(__hadd2(ai, ci));
              o[2][0][h] = operand<BF16>(__hsub2(ar, cr));
              o[2][1][h] = operand<BF16>(__hsub2(ai, ci));
              o[1][0][h] = operand<BF16>(__hadd2(br, di));            // b - i d
              o[1][1][h] = operand<BF16>(__hsub2(bi, dr));
              o[3][0][h] = operand<BF16>(__hsub2(br, di));            // b + i d
              o[3][1][h] = operand<BF16>(__hadd2(bi, dr));
            }
          } else {
#pragma unroll
            for (int A = 0; A < 4; ++A)
#pragma unroll
              for (int c = 0; c < 2; ++c) o[A][c][0] = o[A][c][1] = 0u;
          }
          unsigned char* dst = a1 + b * TILE + a1_off;
#pragma unroll
          for (int A = 0; A < 4; ++A)
#pragma unroll
            for (int c = 0; c < 2; ++c)
              *reinterpret_cast<uint2*>(dst + A * 2 * SBO + c * 2 * LBO) = make_uint2(o[A][c][0], o[A][c][1]);
          in.next(npairs);
        }
        tc::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(bars + A1F + ab);
      }
      // ---------------- detection of pairs 2k - 3 .. min(2k - 2, total - 1)
      const int64_t p0 = 2 * k - 3 > 0 ? 2 * k - 3 : 0;
      const int64_t p1 = 2 * k - 2 < total - 1 ? 2 * k - 2 : total - 1;
      if (p1 < p0) continue;
      if (!wait_warp(D2F + (int)(p1 & (NT4 - 1)), (uint32_t)((p1 / NT4) & 1))) { ok = false; break; }
      tc::fence_after_sync();
#pragma unroll 1
      for (int64_t Pd = p0; Pd <= p1; ++Pd) {
        const int t4 = (int)(Pd & (NT4 - 1));
        const uint32_t taddr = tbase + ((uint32_t)(32 * warp) << 16) + 64 * t4;
#pragma unroll
        for (int ss = 0; ss < 2; ++ss) {
          uint32_t v[32];                                  // re of k2 0..15, then im
          tc::tmem_ld32(taddr + 32 * ss, v);
          tc::tmem_wait_ld();
#pragma unroll
          for (int p = 0; p < 8; ++p) {
            const float2 xr = make_float2(__uint_as_float(v[2 * p]), __uint_as_float(v[2 * p + 1]));
            const float2 xi = make_float2(__uint_as_float(v[16 + 2 * p]), __uint_as_float(v[17 + 2 * p]));
            acc[p] = __ffma2_rn(xi, xi, __ffma2_rn(xr, xr, acc[p]));
          }
        }
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(bars + D2E + t4);     // buffer t4 is free
        if (de.q == npairs - 1) {
          // last pair of the window: beams[item][A = warp][k1 = lane + 32 k2]
          float* dst = a.beams + de.item * (int64_t)(4 * 512) + warp * 512 + lane;
#pragma unroll
          for (int p = 0; p < 8; ++p) {
            dst[64 * p] = acc[p].x * inv_s2;
            dst[64 * p + 32] = acc[p].y * inv_s2;
            acc[p] = make_float2(0.f, 0.f);
          }
        }
        de.next(npairs);
      }
    }
  } else if (warp < 8) {
    // ============================================ stage-1 drain: twiddle, A2 (pair P)
    const int m = tid - 128;                          // TMEM row (s, A, n2)
    const int s = m >> 6, A = (m >> 4) & 3, n2 = m & 15;
    const int lq = warp - 4;
    // twiddles W512^(n2 k1) of this row: FP16, half2 pairs over adjacent k1 (cos, then
    // -sin), in registers; BF16, FP32 quadruples (cos, cos, -sin, -sin) in shared memory
    // (the twiddle is applied in FP32 and the product rounded once to BF16), laid out
    // [j][n2] so that each half-warp's 16-byte loads read 256 contiguous bytes
    uint32_t ch[BF16 ? 1 : 16], dh[BF16 ? 1 : 16];
    const float4* twf = reinterpret_cast<const float4*>(smem + L.twf) + n2;
    if constexpr (!BF16) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        ch[j] = ta.tw16[(n2 * 16 + j) * 2];
        dh[j] = ta.tw16[(n2 * 16 + j) * 2 + 1];
      }
    }
    // A2 offset of element (m2 = A 32 + k1, k = n2) for k1 = 0 and the real part
    const uint32_t a2_off = (uint32_t)((n2 & 7) * 16 + (4 * A) * SBO + (n2 >> 3) * LBO + s * TILE);
    bool ok = true;
    for (int64_t P = 0; P < total && ok; ++P) {
      {
        const int b = (int)(P % NA2);
        const uint32_t u = (uint32_t)(P / NA2);
        const int t4 = (int)(P & (NT4 - 1));
        if (!wait_warp(D1F + t4, (uint32_t)((P / NT4) & 1))) { ok = false; break; }
        if (u >= 1 && !wait_warp(A2E + b, (u - 1) & 1)) { ok = false; break; }
        tc::fence_after_sync();
        const uint32_t taddr = tbase + ((uint32_t)(32 * lq) << 16) + 64 * t4;
        unsigned char* dst = a2 + 2 * b * TILE + a2_off;
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {                        // k1 = 16 hh .. 16 hh + 15
          uint32_t xr[16], xi[16];
          tc::tmem_ld16(taddr + 16 * hh, xr);
          tc::tmem_ld16(taddr + 32 + 16 * hh, xi);
          tc::tmem_wait_ld();
          if (hh == 1) {
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(bars + D1E + t4);    // D2 may overwrite D1
          }
#pragma unroll
          for (int qq = 0; qq < 2; ++qq) {                      // k1 = 8q .. 8q + 7
            const int q = 2 * hh + qq;
            uint32_t tr[4], ti[4];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
              const int jl = 4 * qq + jj, j = 4 * q + jj;
              if constexpr (BF16) {
                const float4 w = twf[16 * j];
                const float2 re = make_float2(__uint_as_float(xr[2 * jl]), __uint_as_float(xr[2 * jl + 1]));
                const float2 im = make_float2(__uint_as_float(xi[2 * jl]), __uint_as_float(xi[2 * jl + 1]));
                const float2 c = make_float2(w.x, w.y), d = make_float2(w.z, w.w);
                const float2 yr = __ffma2_rn(re, c, __fmul2_rn(im, make_float2(-d.x, -d.y)));
                const float2 yi = __ffma2_rn(re, d, __fmul2_rn(im, c));
                const __nv_bfloat162 br = __float22bfloat162_rn(yr), bi = __float22bfloat162_rn(yi);
                tr[jj] = *reinterpret_cast<const uint32_t*>(&br);
                ti[jj] = *reinterpret_cast<const uint32_t*>(&bi);
              } else {
                const __half2 hr = __floats2half2_rn(__uint_as_float(xr[2 * jl]), __uint_as_float(xr[2 * jl + 1]));
                const __half2 hi = __floats2half2_rn(__uint_as_float(xi[2 * jl]), __uint_as_float(xi[2 * jl + 1]));
                const __half2 c = as_h2(ch[j]), d = as_h2(dh[j]);
                tr[jj] = as_u(__hfma2(__hneg2(hi), d, __hmul2(hr, c)));   // re x c - im x d
                ti[jj] = as_u(__hfma2(hi, c, __hmul2(hr, d)));            // re x d + im x c
              }
            }
            *reinterpret_cast<uint4*>(dst + q * SBO) = make_uint4(tr[0], tr[1], tr[2], tr[3]);
            *reinterpret_cast<uint4*>(dst + q * SBO + 2 * LBO) = make_uint4(ti[0], ti[1], ti[2], ti[3]);
          }
        }
        tc::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(bars + A2F + b);
      }
    }
  } else if (warp == 8 && lane == 0) {
    // ============================================ stage-1 MMAs and raw-byte copies
    const uint32_t id1 = tc::idesc_f16(128, 64, BF16) | (1u << 15);   // A MN-major
    const uint32_t sa1 = tc::smem_u32(a1), sb1 = tc::smem_u32(smem + L.b1);
    // raw-byte source of the next pair to copy: the item's first byte is found once per
    // item (one 64-bit division), pairs then advance by a constant stride
    PairSeq cp{(int64_t)blockIdx.x, 0};
    const uint8_t* ibase = item_volts(a, cp.item, NANT);
    const int64_t tstride = (int64_t)a.nfreq * a.npol * NANT;      // one time sample
    const bool two_pol = a.npol == 2;
    // the bytes of the pair cp points at (1 KB if it is the lone last snapshot of an odd
    // count), copied to dst and counted on bar; then cp moves on
    auto pair_bytes = [&](int q) -> uint32_t { return 2 * q + 1 < nsnap ? 2 * NANT : NANT; };
    auto copy_pair = [&](unsigned char* dst, uint64_t* bar) {
      const int g = 2 * cp.q;
      const uint8_t* s0 = two_pol ? ibase + (int64_t)cp.q * tstride : ibase + snap_offset(a, g, NANT);
      if (g + 1 < nsnap) {
        if (two_pol) {
          tc::bulk_g2s(dst, s0, 2 * NANT, bar);
        } else {
          tc::bulk_g2s(dst, s0, NANT, bar);
          tc::bulk_g2s(dst + NANT, ibase + snap_offset(a, g + 1, NANT), NANT, bar);
        }
      } else {
        tc::bulk_g2s(dst, s0, NANT, bar);
      }
      if (++cp.q == npairs) {
        cp.q = 0;
        cp.item += gridDim.x;
        if (cp.item < nitems) ibase = item_volts(a, cp.item, NANT);
      }
    };
    const int64_t nround = (total + 1) / 2;
    int64_t issued = 0;                                // rounds whose bytes were requested
    // round `issued` (pairs 2 issued, + 1) into raw stages 2 (issued % RQ), + 1, on one barrier
    auto copy_round = [&]() {
      const int rq = (int)(issued % RQ);
      uint64_t* bar = bars + RAWF + rq;
      unsigned char* dst = raw + rq * 4 * NANT;
      const bool two = 2 * issued + 1 < total;
      const uint32_t bytes = pair_bytes(cp.q) + (two ? pair_bytes(cp.q + 1 == npairs ? 0 : cp.q + 1) : 0);
      tc::mbar_arrive_expect_tx(bar, bytes);
      copy_pair(dst, bar);
      if (two) copy_pair(dst + 2 * NANT, bar);
      ++issued;
    };
    // descriptors of tile 0; tile b starts b TILE bytes further (the start-address field
    // holds the address / 16)
    uint64_t da1[2], db1[2];
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      db1[kk] = tc::smem_desc(sb1 + kk * 2 * B_LBO, B_LBO, B_SBO);
      da1[kk] = tc::smem_desc(sa1 + kk * 2 * LBO, LBO, SBO);
    }
    while (issued < nround && issued < RQ) copy_round();
    int64_t mma1 = 0;                                  // pairs whose MMAs were issued
    bool ok = true;
    for (int64_t k = 0; k < nround && ok; ++k) {
      const int ab = (int)(k & 1);
      if (!wait_sleep(A1F + ab, (uint32_t)((k >> 1) & 1))) break;
      for (int j = 0; j < 2 && mma1 < total; ++j, ++mma1) {
        const int t4 = (int)(mma1 & (NT4 - 1));
        const uint32_t u4 = (uint32_t)(mma1 / NT4);
        if (u4 >= 1 && !wait_sleep(D2E + t4, (u4 - 1) & 1)) { ok = false; break; }
        tc::fence_after_sync();
        const uint64_t off = (uint64_t)(((int)(mma1 & 3) * TILE) >> 4);   // A1 tile mma1 % 4
        tc::mma_f16(tbase + 64 * t4, da1[0] + off, db1[0], id1, 0);
        tc::mma_f16(tbase + 64 * t4, da1[1] + off, db1[1], id1, 1);
        tc::mma_commit(bars + D1F + t4);
      }
      if (!ok) break;
      tc::mma_commit(bars + A1E + ab);
      // every input warp read round k's raw stages before its A1F arrival: refill them
      if (issued < nround) copy_round();
    }
    // Every copy and MMA issued must have landed before the CTA frees its memory. On the
    // normal path the other roles already waited for all of them; after a timeout, wait
    // here (bounded, regardless of the abort flag) for the last ones of each ring.
    for (int64_t k = issued - 1; k >= 0 && k >= issued - RQ; --k)
      tc::mbar_wait(bars + RAWF + (int)(k % RQ), (uint32_t)((k / RQ) & 1), WAIT_NS);
    if (mma1 > 0)
      tc::mbar_wait(bars + D1F + (int)((mma1 - 1) & (NT4 - 1)), (uint32_t)(((mma1 - 1) / NT4) & 1), WAIT_NS);
  } else if (warp == 9 && lane == 0) {
    // ============================================ stage-2 MMAs
    const uint32_t id2 = tc::idesc_f16(128, 32, BF16) | (1u << 15);   // A MN-major
    const uint32_t sa2 = tc::smem_u32(a2), sb2 = tc::smem_u32(smem + L.b2);
    uint64_t da2[2][2], db2[2];                        // tile pair 0; pair b is 2 b TILE further
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      db2[kk] = tc::smem_desc(sb2 + kk * 2 * B_LBO, B_LBO, B_SBO);
#pragma unroll
      for (int ss = 0; ss < 2; ++ss) da2[ss][kk] = tc::smem_desc(sa2 + ss * TILE + kk * 2 * LBO, LBO, SBO);
    }
    int64_t mma2 = 0;
    for (; mma2 < total; ++mma2) {
      const int b = (int)(mma2 % NA2);
      const uint32_t u = (uint32_t)(mma2 / NA2);
      const int t4 = (int)(mma2 & (NT4 - 1));
      const uint32_t u4 = (uint32_t)(mma2 / NT4);
      if (!wait_sleep(A2F + b, u & 1) || !wait_sleep(D1E + t4, u4 & 1)) break;
      tc::fence_after_sync();
      const uint64_t off = (uint64_t)((2 * b * TILE) >> 4);
#pragma unroll
      for (int ss = 0; ss < 2; ++ss) {
        tc::mma_f16(tbase + 64 * t4 + 32 * ss, da2[ss][0] + off, db2[0], id2, 0);
        tc::mma_f16(tbase + 64 * t4 + 32 * ss, da2[ss][1] + off, db2[1], id2, 1);
      }
      tc::mma_commit(bars + D2F + t4);
      tc::mma_commit(bars + A2E + b);
    }
    if (mma2 > 0)
      tc::mbar_wait(bars + D2F + (int)((mma2 - 1) & (NT4 - 1)), (uint32_t)(((mma2 - 1) / NT4) & 1), WAIT_NS);
  }
  __syncwarp();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 8) tc::tmem_dealloc(tbase, TMEM_COLS);
}

bool tcw_eligible(const TcArgs& ta) {
  const BeamArgs& a = ta.b;
  return !ta.split && ta.tw16 && a.nx == 4 && a.ny == 256 && a.mx == 4 &&
         a.my == 512 && a.nyf == 256 && a.ew_dft &&
         (reinterpret_cast<uintptr_t>(a.volts) & 15) == 0;
}

int launch_beams_tcw(const TcArgs& ta, int nsm, cudaStream_t st) {
  const BeamArgs& a = ta.b;
  const int64_t items = a.nwin * a.nfreq;
  if (items <= 0) return FFTBF_OK;
  const tcw::Smem L = tcw::layout();
  // two CTAs per SM (256 of the 512 tensor-memory columns each): keep a third from
  // fitting by shared memory as well, as it could not allocate tensor memory until one of
  // the others exits
  size_t smem = (size_t)L.total;
  if (smem < 77 * 1024) smem = 77 * 1024;
  auto kern = ta.bf16 ? (a.real_w ? beams_tcw_kernel<true, true> : beams_tcw_kernel<false, true>)
                      : (a.real_w ? beams_tcw_kernel<true, false> : beams_tcw_kernel<false, false>);
  FFTBF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  FFTBF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      cudaSharedmemCarveoutMaxShared));
  const int64_t per_wave = (int64_t)nsm * 2;
  const int64_t grid = items < per_wave ? items : per_wave;
  kern<<<(unsigned)grid, tcw::NT, smem, st>>>(ta);
  FFTBF_CUDA_TRY(cudaGetLastError());
  return FFTBF_OK;
}

// ---------------------------------------------------------------- plan tables --
// Stage matrices of the warp-specialised 16-bit forms, row-major [n][k] (n = output, k =
// input), FP64 rounded once to FP16 (or BF16 when bf16), and the W512 twiddle pairs:
//   b1[n = co 32 + k1][k = ci 16 + n1]   W32^(n1 k1), planar in and out
//   b2[n = co 16 + k2][k = ci 16 + n2]   W16^(n2 k2), planar in and out
//   tw16[(n2 16 + j) 2 + {0, 1}]         (cos, cos) and (-sin, -sin) of 2 pi n2 k1 / 512 for
//                                        k1 = 2j, 2j + 1, as 16-bit pairs
// With W = C + iS (S = -sin): out_re = sum in_re C - in_im S, out_im = sum in_re S + in_im C.
__global__ void tcw_tables_kernel(uint16_t* b1, uint16_t* b2, uint32_t* tw16, bool bf16) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  auto h = [bf16](double v) -> uint16_t {
    if (bf16) {
      const __nv_bfloat16 x = __double2bfloat16(v);
      return *reinterpret_cast<const uint16_t*>(&x);
    }
    const __half x = __float2half_rn((float)v);
    return *reinterpret_cast<const uint16_t*>(&x);
  };
  auto entry = [](int co, int ci, double c, double sp) {
    if (co == 0) return ci == 0 ? c : -sp;
    return ci == 0 ? sp : c;
  };
  if (i < 64 * 32) {
    const int n = i >> 5, k = i & 31;
    const int co = n >> 5, k1 = n & 31, ci = k >> 4, n1 = k & 15;
    double sn, cs;
    sincospi(2.0 * ((n1 * k1) % 32) / 32.0, &sn, &cs);
    b1[i] = h(entry(co, ci, cs, -sn));
  }
  if (i < 32 * 32) {
    const int n = i >> 5, k = i & 31;
    const int k2 = n & 15, co = n >> 4, ci = k >> 4, n2 = k & 15;
    double sn, cs;
    sincospi(2.0 * ((n2 * k2) % 16) / 16.0, &sn, &cs);
    b2[i] = h(entry(co, ci, cs, -sn));
  }
  if (i < 16 * 16) {
    const int n2 = i >> 4, j = i & 15;
    double s0, c0, s1, c1;
    sincospi(2.0 * ((n2 * 2 * j) % 512) / 512.0, &s0, &c0);
    sincospi(2.0 * ((n2 * (2 * j + 1)) % 512) / 512.0, &s1, &c1);
    tw16[2 * i] = (uint32_t)h(c0) | ((uint32_t)h(c1) << 16);
    tw16[2 * i + 1] = (uint32_t)h(-s0) | ((uint32_t)h(-s1) << 16);
  }
}

int build_tcw_tables(uint16_t* b1, uint16_t* b2, uint32_t* tw16, bool bf16, cudaStream_t st) {
  tcw_tables_kernel<<<(64 * 32 + 255) / 256, 256, 0, st>>>(b1, b2, tw16, bf16);
  FFTBF_CUDA_TRY(cudaGetLastError());
  return FFTBF_OK;
}

}  // namespace fftbf

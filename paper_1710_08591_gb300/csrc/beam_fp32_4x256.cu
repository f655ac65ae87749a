// FP32 form of the FFT-beam hot path specialised for the 4x256 lattice: 4 E-W x 256 N-S
// feeds, 4 E-W beams (a 4-point DFT, Eq. fftbeamform) x 512 N-S beams (the N-S axis
// zero-padded to 2n, Eq. b2n-1), 16-byte aligned voltages.
//
// The arithmetic, and the order in which each beam's sum is accumulated, are those of the
// 512-beam warp kernel (beam_fp32_n512.cu), so the beams are bit-identical to it; what
// changes is how the work is laid out, to move fewer bytes through shared memory and issue
// fewer instructions per snapshot:
//   * a CTA of four warps takes two snapshots per iteration and warp w owns E-W beam A = w
//     of both: each lane's 16 accumulators take the two snapshots in turn, so no partial
//     sums are combined across warps;
//   * each input-stage thread unpacks, weights and E-W transforms the same two adjacent
//     N-S feeds every iteration and keeps their apodisation weights in registers;
//   * pass 1, the pruned 32-point DFT over n1 for each n2 (n = n2 + 16 n1, inputs n1 >= 16
//     are the zero padding), is split as X1[2m] = DFT16(x)[m] and
//     X1[2m + 1] = DFT16(x W32^n1)[m]; one lane (n2, snapshot) computes both halves, so the
//     W32^n1 factors are compile-time constants instead of per-lane table loads, the even
//     half has no unit-factor multiplies, and both half-warps read the same W512^(n2 k1)
//     table entries (one broadcast wavefront per load);
//   * pass 2, one lane per k1: the 16-point DFT over n2 giving X[k1 + 32 k2], squared and
//     added to the lane's accumulators (Eq. bf).
// Shared memory per CTA: two 2 KB byte stages (cp.async, double-buffered), the W512 table
// and eight 32 x 17 complex tiles (one per snapshot and E-W beam: the inputs in rows 0..15,
// then the pass-1 outputs, odd k1 in rows 16..31, stored first, and even k1 in rows 0..15,
// stored once every lane has read its inputs).
#include <cuda_runtime.h>

#include "beam_fp32.cuh"

namespace fftbf {

namespace f4x256 {
constexpr int NT = 128;                 // four warps: warp w = E-W beam w
constexpr int S = 2;                    // snapshots per iteration
constexpr int NANT = 1024;
constexpr int RAW = S * NANT;           // staged bytes per iteration
constexpr int kRow = 17;                // float2 row stride of a tile (conflict-free both ways)
constexpr int kTile = 32 * kRow;
constexpr size_t kSmem = 2 * RAW + sizeof(float2) * (512 + S * 4 * kTile);
__device__ __forceinline__ int x1_row(int k1) { return (k1 & 1) * 16 + (k1 >> 1); }

// W32^n = exp(-2 pi i n / 32) = (cos(pi n / 16), -sin(pi n / 16)), n = 1..15, written out
// to FP32 precision: the same values as the plan's table entries W512^(16 n), which are
// these numbers computed in FP64 and rounded once.
__device__ __forceinline__ float2 w32(int n) {
  constexpr float c1 = 0.98078528040323044913f, c2 = 0.92387953251128675613f;
  constexpr float c3 = 0.83146961230254523708f, c4 = 0.70710678118654752440f;
  constexpr float c5 = 0.55557023301960222474f, c6 = 0.38268343236508977173f;
  constexpr float c7 = 0.19509032201612826785f;
  switch (n) {
    case 1: return make_float2(c1, -c7);
    case 2: return make_float2(c2, -c6);
    case 3: return make_float2(c3, -c5);
    case 4: return make_float2(c4, -c4);
    case 5: return make_float2(c5, -c3);
    case 6: return make_float2(c6, -c2);
    case 7: return make_float2(c7, -c1);
    case 8: return make_float2(0.f, -1.f);
    case 9: return make_float2(-c7, -c1);
    case 10: return make_float2(-c6, -c2);
    case 11: return make_float2(-c5, -c3);
    case 12: return make_float2(-c4, -c4);
    case 13: return make_float2(-c3, -c5);
    case 14: return make_float2(-c2, -c6);
    default: return make_float2(-c1, -c7);
  }
}
}  // namespace f4x256

template <bool REALW>
__global__ void __launch_bounds__(f4x256::NT, 4) beams_fp32_4x256_kernel(const BeamArgs a) {
  using namespace f4x256;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* tw512 = reinterpret_cast<float2*>(smem + 2 * RAW);   // [k1][n2] = W512^(n2 k1)
  float2* tiles = tw512 + 512;                                 // [s][A][kTile]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nsnap = a.n_int * a.npol;
  const int niter = (nsnap + S - 1) / S;
  const int64_t nitems = a.nwin * a.nfreq;

  for (int i = tid; i < 512; i += NT) tw512[i] = a.tw[(i & 15) * (i >> 4)];
  // this thread's feeds iy, iy + 1 of every E-W row ix and their weights
  const int iy = 2 * tid;
  float2 w0[4], w1[4];
#pragma unroll
  for (int ix = 0; ix < 4; ++ix) {
    w0[ix] = a.w[ix * 256 + iy];
    w1[ix] = a.w[ix * 256 + iy + 1];
  }

  int64_t item = blockIdx.x;
  if (item >= nitems) return;

  // bytes of iteration `it` of the work item at ivol into stage b: one 16-byte copy per
  // thread (snapshot tid / 64, chunk tid % 64)
  auto stage = [&](const uint8_t* ivol, int it, int b) {
    const int s = tid >> 6, g = it * S + s;
    if (g < nsnap) {
      const int c = (tid & 63) << 4;
      cp_async16(smem + b * RAW + s * NANT + c, ivol + snap_offset(a, g, NANT) + c);
    }
  };

  const uint8_t* ivol = item_volts(a, item, NANT);
  stage(ivol, 0, 0);
  cp_async_commit();
  float acc[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] = 0.f;
  int it = 0, cur = 0;
  const int n2 = lane & 15;
  float2* const p1 = tiles + ((lane >> 4) * 4 + warp) * kTile;     // pass-1 tile of this lane
  const int in_sl = (iy & 15) + kRow * (iy >> 4);                 // tile slot of feed iy
  // pass 2: lane l reads tile row l, which holds k1 = 2 l (l < 16) or 2 (l - 16) + 1, so that
  // each half-warp's 8-byte loads touch 16 distinct bank pairs
  const int k1_lane = lane < 16 ? 2 * lane : 2 * (lane - 16) + 1;

  while (true) {
    int64_t nitem = item;
    int nit = it + 1;
    if (nit == niter) { nitem = item + gridDim.x; nit = 0; }
    const bool has_next = nitem < nitems;
    const uint8_t* nvol = nit == 0 && has_next ? item_volts(a, nitem, NANT) : ivol;
    cp_async_wait<0>();
    __syncthreads();                                  // (A) bytes of `it` visible; tiles free
    if (has_next) stage(nvol, nit, cur ^ 1);
    cp_async_commit();

    // ---- unpack x weight, 4-point E-W DFT -> tile [s][A], slots of feeds iy, iy + 1
    const uint8_t* raw = smem + cur * RAW;
#pragma unroll
    for (int s = 0; s < S; ++s) {
      if (it * S + s < nsnap) {
        float2 z0[4], z1[4];
#pragma unroll
        for (int ix = 0; ix < 4; ++ix) {
          const unsigned v = *reinterpret_cast<const uint16_t*>(raw + s * NANT + ix * 256 + iy);
          const float2 x0 = unpack_byte(v & 255u), x1 = unpack_byte(v >> 8);
          if constexpr (REALW) {                      // one packed multiply per feed
            z0[ix] = __fmul2_rn(make_float2(w0[ix].x, w0[ix].x), x0);
            z1[ix] = __fmul2_rn(make_float2(w1[ix].x, w1[ix].x), x1);
          } else {
            z0[ix] = cmul(w0[ix], x0);
            z1[ix] = cmul(w1[ix], x1);
          }
        }
        Dft<4>::run(z0);
        Dft<4>::run(z1);
#pragma unroll
        for (int A = 0; A < 4; ++A) {
          tiles[(s * 4 + A) * kTile + in_sl] = z0[A];
          tiles[(s * 4 + A) * kTile + in_sl + 1] = z1[A];
        }
      }
    }
    __syncthreads();                                  // (B) tiles written

    // ---- pass 1, lane (n2, snapshot lane / 16): X1[k1] W512^(n2 k1) for all 32 k1
    {
      float2 x[16], xe[16];                           // xe: the inputs kept for the even half
#pragma unroll
      for (int n1 = 0; n1 < 16; ++n1) x[n1] = xe[n1] = p1[n2 + kRow * n1];
#pragma unroll
      for (int n1 = 1; n1 < 16; ++n1) x[n1] = n1 == 8 ? mul_mi(x[n1]) : cmul(x[n1], w32(n1));   // W32^8 = -i
      Dft<16>::run(x);
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const int k1 = 2 * m + 1;
        p1[x1_row(k1) * kRow + n2] = cmul(x[m], tw512[k1 * 16 + n2]);
      }
      __syncwarp();                                   // every lane's inputs read: rows 0..15 may change
      Dft<16>::run(xe);
      p1[n2] = xe[0];                                 // k1 = 0: W512^0 = 1
#pragma unroll
      for (int m = 1; m < 16; ++m) {
        const int k1 = 2 * m;
        p1[x1_row(k1) * kRow + n2] = cmul(xe[m], tw512[k1 * 16 + n2]);
      }
      __syncwarp();
    }
    // ---- pass 2, lane = row lane of the tile (k1 = k1_lane), the two snapshots in turn
#pragma unroll
    for (int s = 0; s < S; ++s) {
      if (it * S + s < nsnap) {
        const float2* t = tiles + (s * 4 + warp) * kTile + lane * kRow;
        float2 y[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) y[q] = t[q];
        Dft<16>::run(y);
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2)
          acc[k2] = fmaf(y[k2].x, y[k2].x, fmaf(y[k2].y, y[k2].y, acc[k2]));
      }
    }

    if (it == niter - 1) {
      // ---- window complete: beams[item][A = warp][k1 + 32 k2]
      float* dst = a.beams + item * (int64_t)(4 * 512) + warp * 512 + k1_lane;
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) {
        dst[32 * k2] = acc[k2];
        acc[k2] = 0.f;
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

bool fp32_4x256_eligible(const BeamArgs& a) {
  return a.nx == 4 && a.ny == 256 && a.mx == 4 && a.my == 512 && a.nyf == 256 && a.ew_dft &&
         (reinterpret_cast<uintptr_t>(a.volts) & 15) == 0;
}

int launch_beams_fp32_4x256(const BeamArgs& a, int nsm, cudaStream_t st) {
  const int64_t items = a.nwin * a.nfreq;
  if (items <= 0) return FFTBF_OK;
  auto kern = a.real_w ? beams_fp32_4x256_kernel<true> : beams_fp32_4x256_kernel<false>;
  const int smem = (int)f4x256::kSmem;
  FFTBF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  FFTBF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      cudaSharedmemCarveoutMaxShared));
  int per_sm = 0;
  FFTBF_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, f4x256::NT, smem));
  if (per_sm < 1) return set_error(FFTBF_EUNSUPPORTED, "4x256 kernel does not fit on an SM");
  const int64_t per_wave = (int64_t)nsm * per_sm;
  const int64_t grid = items < per_wave ? items : per_wave;
  kern<<<(unsigned)grid, f4x256::NT, smem, st>>>(a);
  FFTBF_CUDA_TRY(cudaGetLastError());
  return FFTBF_OK;
}

}  // namespace fftbf

// FP32 fused beam kernel specialised for an N-S transform of 512 beams over at most 256
// feeds (the 2x zero padding recommended by Eq. b2n-1), one warp per transform.
//
// N = 512 = 32 x 16 (Cooley-Tukey, n = n2 + 16 n1, k = k1 + 32 k2):
//   pass 1, lane (n2, h): X1[k1] = sum_{n1 < 16} x[n2 + 16 n1] W32^(n1 k1) for the 16
//     outputs k1 = 2m + h, as a 16-point DFT of x[n1] W32^(h n1) (inputs n1 >= 16 are the
//     zero padding); then X1[k1] *= W512^(n2 k1) and the 16 x 32 tile is transposed
//     through shared memory (row stride 17: conflict-free both ways);
//   pass 2, lane k1: X[k1 + 32 k2] = sum_{n2} X1_n2[k1] W16^(n2 k2), a 16-point DFT,
//     squared and added to 16 per-lane accumulators (Eq. bf).
// A CTA has four warps (eight for an E-W size of 8); per iteration it stages the bytes
// of S = 4 / mx snapshots (cp.async, double-buffered), unpacks, weights and E-W
// transforms them cooperatively into one 512-slot region per (snapshot, E-W beam), and
// each warp then transforms its own region. Two CTA barriers per iteration; the
// transforms synchronise only within their warp. Accumulation order is fixed per work
// item, as in the generic kernel.
// The 4x256 lattice with 16-byte aligned voltages runs the same arithmetic, in the same
// order, in its own kernel (beam_fp32_4x256.cu); this one serves the other shapes and
// unaligned voltages.
#include <cuda_runtime.h>

#include "beam_fp32.cuh"

namespace fftbf {

namespace n512 {
constexpr int kRow = 17;           // float2 row stride of the input and X1 tiles
constexpr int kRegion = 32 * kRow; // float2 slots per transform region (X1 tile, padded)
__device__ __forceinline__ int in_slot(int iy) { return (iy & 15) + kRow * (iy >> 4); }
}

#ifndef FFTBF_N512_NW
#define FFTBF_N512_NW 4           // warps per CTA for E-W sizes up to 4 (snapshots = NW / MX)
#endif
#ifndef FFTBF_N512_MIN_BLOCKS
#define FFTBF_N512_MIN_BLOCKS (24 / FFTBF_N512_NW)   // CTAs per SM the register budget targets
#endif

template <int MX>
__global__ void __launch_bounds__((MX > 4 ? MX : FFTBF_N512_NW) * 32, MX > 4 ? 2 : FFTBF_N512_MIN_BLOCKS)
beams_fp32_n512_kernel(const BeamArgs a) {
  constexpr int NW = MX > 4 ? MX : FFTBF_N512_NW;   // warps per CTA = transforms per iteration
  constexpr int S = NW / MX;                // snapshots per iteration
  constexpr int NT = NW * 32;
  extern __shared__ __align__(16) unsigned char smem[];
  const int ny = a.ny;
  const int nyf = a.nyf;
  const int nant = a.nx * a.ny;
  const int rawsz = (S * nant + 15) & ~15;
  // tables and regions first, so the weights start 16-byte aligned (128-bit loads)
  float2* tw512 = reinterpret_cast<float2*>(smem + 2 * rawsz);  // [32 k1][16 n2] = W512^(n2 k1)
  float2* tw32 = tw512 + 512;                // [2 h][16 n1]  = W32^(h n1)
  float2* reg = tw32 + 32;                   // [NW][kRegion]
  float2* wsm = reg + NW * n512::kRegion;
  float2* exsm = wsm + nant;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nsnap = a.n_int * a.npol;
  const int niter = (nsnap + S - 1) / S;
  const int64_t nitems = a.nwin * a.nfreq;
  const bool vec16 = ((nant & 15) == 0) && ((reinterpret_cast<uintptr_t>(a.volts) & 15) == 0);

  for (int i = threadIdx.x; i < nant; i += NT) wsm[i] = a.w[i];
  for (int i = threadIdx.x; i < MX * a.nx; i += NT) exsm[i] = a.ex[i];
  for (int i = threadIdx.x; i < 512; i += NT) {
    const int k1 = i >> 4, n2 = i & 15;
    tw512[i] = a.tw[n2 * k1];                // n2 k1 < 512
  }
  for (int i = threadIdx.x; i < 32; i += NT) tw32[i] = a.tw[(i >> 4) * 16 * (i & 15)];

  int64_t item = blockIdx.x;
  if (item >= nitems) return;

  // byte staging of iteration `it` of the work item starting at ivol into buffer b
  auto stage = [&](const uint8_t* ivol, int it, int b) {
    uint8_t* raw = smem + b * rawsz;
    if (vec16) {
      const int cps = nant >> 4;
      for (int q = threadIdx.x; q < S * cps; q += NT) {
        const int s = q / cps, g = it * S + s;
        if (g < nsnap) {
          const uint8_t* src = ivol + snap_offset(a, g, nant);
          cp_async16(raw + s * nant + ((q - s * cps) << 4), src + ((q - s * cps) << 4));
        }
      }
    } else {
      for (int q = threadIdx.x; q < S * nant; q += NT) {
        const int s = q / nant, g = it * S + s;
        if (g < nsnap) raw[q] = ivol[snap_offset(a, g, nant) + (q - s * nant)];
      }
    }
  };

  const uint8_t* ivol = item_volts(a, item, nant);
  stage(ivol, 0, 0);
  cp_async_commit();
  float acc[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] = 0.f;
  int it = 0, cur = 0;
  const int n2 = lane & 15, h = lane >> 4;
  float2* myreg = reg + warp * n512::kRegion;

  while (true) {
    int64_t nitem = item;
    int nit = it + 1;
    if (nit == niter) { nitem = item + gridDim.x; nit = 0; }
    const bool has_next = nitem < nitems;
    const uint8_t* nvol = nit == 0 && has_next ? item_volts(a, nitem, nant) : ivol;
    cp_async_wait<0>();
    __syncthreads();                                  // (A) bytes of `it` visible; regions free
    if (has_next) stage(nvol, nit, cur ^ 1);
    cp_async_commit();

    // ---- unpack x weight, E-W transform -> Z[s*MX + A][in_slot(iy)]
    const uint8_t* raw = smem + cur * rawsz;
    for (int c = threadIdx.x; c < S * 256; c += NT) {
      const int s = c >> 8, iy = c & 255;
      float2 z[MX];
#pragma unroll
      for (int A = 0; A < MX; ++A) z[A] = czero();
      if (iy < nyf && it * S + s < nsnap) {
        const uint8_t* rs = raw + s * nant;
        if constexpr (MX == 1 || MX == 2 || MX == 4 || MX == 8) {
          if (a.ew_dft) {
            if (a.real_w) {
              // real weights: w x in one packed multiply (the same roundings as the
              // complex product with a zero imaginary part)
#pragma unroll
              for (int ix = 0; ix < MX; ++ix) {
                const float wr = wsm[ix * ny + iy].x;
                const float2 xv = unpack_byte(rs[ix * ny + iy]);
                z[ix] = __fmul2_rn(make_float2(wr, wr), xv);
              }
            } else {
#pragma unroll
              for (int ix = 0; ix < MX; ++ix)
                z[ix] = cmul(wsm[ix * ny + iy], unpack_byte(rs[ix * ny + iy]));
            }
            Dft<MX>::run(z);
          }
        }
        if (!a.ew_dft) {
          for (int ix = 0; ix < a.nx; ++ix) {
            const float2 col = cmul(wsm[ix * ny + iy], unpack_byte(rs[ix * ny + iy]));
#pragma unroll
            for (int A = 0; A < MX; ++A) z[A] = cadd(z[A], cmul(exsm[A * a.nx + ix], col));
          }
        }
      }
#pragma unroll
      for (int A = 0; A < MX; ++A) reg[(s * MX + A) * n512::kRegion + n512::in_slot(iy)] = z[A];
    }
    __syncthreads();                                  // (B) regions written

    // ---- pass 1: lane (n2, h)
    {
      float2 x[16];
#pragma unroll
      for (int n1 = 0; n1 < 16; ++n1) x[n1] = cmul(myreg[n2 + n512::kRow * n1], tw32[h * 16 + n1]);
      Dft<16>::run(x);
      __syncwarp();
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const int k1 = 2 * m + h;
        myreg[k1 * n512::kRow + n2] = cmul(x[m], tw512[k1 * 16 + n2]);
      }
      __syncwarp();
    }
    // ---- pass 2: lane k1
    {
      float2 y[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) y[q] = myreg[lane * n512::kRow + q];
      Dft<16>::run(y);
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) acc[k2] = fmaf(y[k2].x, y[k2].x, fmaf(y[k2].y, y[k2].y, acc[k2]));
    }

    if (it == niter - 1) {
      // ---- window complete: add the S partial sums of each E-W beam, write once
      float* dst = a.beams + item * (int64_t)(MX * 512);
      if constexpr (S == 1) {
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) dst[warp * 512 + lane + 32 * k2] = acc[k2];
      } else {
        __syncthreads();
        float* red = reinterpret_cast<float*>(reg);
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) red[warp * 512 + lane + 32 * k2] = acc[k2];
        __syncthreads();
        for (int o = threadIdx.x; o < MX * 512; o += NT) {
          float sum = 0.f;
#pragma unroll
          for (int s = 0; s < S; ++s) sum += red[s * MX * 512 + o];
          dst[o] = sum;
        }
      }
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) acc[k2] = 0.f;
    }
    if (!has_next) break;
    item = nitem;
    ivol = nvol;
    it = nit;
    cur ^= 1;
  }
  cp_async_wait<0>();
}

static size_t n512_smem_bytes(const BeamArgs& a, int S, int NW) {
  const int nant = a.nx * a.ny;
  const size_t rawsz = ((size_t)S * nant + 15) & ~(size_t)15;
  return 2 * rawsz + sizeof(float2) * (512 + 32 + (size_t)NW * n512::kRegion +
                                       (size_t)nant + (size_t)a.mx * a.nx);
}

template <int MX>
static int launch_n512_mx(const BeamArgs& a, int nsm, cudaStream_t st) {
  // the 4x256 lattice with aligned voltages has its own kernel (beam_fp32_4x256.cu)
  if (MX == 4 && fp32_4x256_eligible(a)) return launch_beams_fp32_4x256(a, nsm, st);
  constexpr int NW = MX > 4 ? MX : FFTBF_N512_NW;
  constexpr int S = NW / MX;
  const size_t smem = n512_smem_bytes(a, S, NW);
  auto kern = beams_fp32_n512_kernel<MX>;
  FFTBF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  FFTBF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      cudaSharedmemCarveoutMaxShared));
  int per_sm = 0;
  FFTBF_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NW * 32, smem));
  if (per_sm < 1) return set_error(FFTBF_EUNSUPPORTED, "512-beam kernel does not fit on an SM");
  const int64_t items = a.nwin * a.nfreq;
  const int64_t grid = items < (int64_t)nsm * per_sm ? items : (int64_t)nsm * per_sm;
  kern<<<(unsigned)grid, NW * 32, smem, st>>>(a);
  FFTBF_CUDA_TRY(cudaGetLastError());
  return FFTBF_OK;
}

bool fp32_n512_supported(const BeamArgs& a) {
  const bool mx_ok = a.mx == 1 || a.mx == 2 || a.mx == 4 || a.mx == 8;
  return mx_ok && a.my == 512 && a.nyf <= 256 &&
         n512_smem_bytes(a, a.mx > 4 ? 1 : FFTBF_N512_NW / a.mx, a.mx > 4 ? a.mx : FFTBF_N512_NW) <=
             200 * 1024;
}

int launch_beams_fp32_n512(const BeamArgs& a, int nsm, cudaStream_t st) {
  switch (a.mx) {
    case 1: return launch_n512_mx<1>(a, nsm, st);
    case 2: return launch_n512_mx<2>(a, nsm, st);
    case 4: return launch_n512_mx<4>(a, nsm, st);
    case 8: return launch_n512_mx<8>(a, nsm, st);
    default: return set_error(FFTBF_EUNSUPPORTED, "512-beam kernel: E-W size %d", a.mx);
  }
}

}  // namespace fftbf

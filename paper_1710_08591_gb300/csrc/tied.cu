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

// FP64 regridding weight of beam k on an axis of n feeds and M beams for pointing y.
__device__ __forceinline__ double regrid_weight(int n, int M, bool dense, double y, int k) {
  if (dense) {
    double e = y - (double)k / (double)M;
    e -= rint(e);                          // the kernel has period 1 in y
    const double L = 2.0 * n - 1.0;
    if (fabs(e) < 1e-9) return L / M;      // limit at y - k/M integer (error ~ n^2 e^2)
    return sinpi(L * e) / (sinpi(e) * (double)M);
  }
  long long k0 = llrint(y * (double)M) % M;
  if (k0 < 0) k0 += M;
  return k0 == k ? 1.0 : 0.0;
}

__global__ void tied_table_kernel(int n, int M, int dense, int nfreq, int n_tied,
                                  const double* y, const int* perm, float* out) {
  const int64_t total = (int64_t)nfreq * n_tied * M;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(i % M);
    const int64_t fs = i / M;                         // f * n_tied + sorted slot
    const int f = (int)(fs / n_tied);
    const int s = perm[fs];
    out[i] = (float)regrid_weight(n, M, dense != 0, y[(int64_t)f * n_tied + s], k);
  }
}

constexpr int TS = 64, TJ = 64, TK = 16;

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
  cudaFree(tt.wx);
  cudaFree(tt.wy);
  cudaFree(tt.perm);
  cudaFree(tt.duv);
  tt = TiedTables();
}

int tied_prepare(TiedTables& tt, int nx, int ny, int mx, int my, int nfreq, int n_tied,
                 const double* u, const double* v, cudaStream_t st) {
  const size_t nuv = (size_t)nfreq * n_tied;
  if (tt.n_tied == n_tied && tt.u.size() == nuv &&
      std::memcmp(tt.u.data(), u, nuv * sizeof(double)) == 0 &&
      std::memcmp(tt.v.data(), v, nuv * sizeof(double)) == 0)
    return FFTBF_OK;                                  // same pointings: tables are current

  const bool dense_x = mx >= 2 * nx - 1, dense_y = my >= 2 * ny - 1;
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
  // Sort each frequency's pointings by E-W beam (one-hot axis) so tiles skip columns.
  std::vector<int> perm(nuv);
  for (int f = 0; f < nfreq; ++f) {
    int* p = perm.data() + (size_t)f * n_tied;
    for (int s = 0; s < n_tied; ++s) p[s] = s;
    if (!dense_x) {
      const double* uf = u + (size_t)f * n_tied;
      std::stable_sort(p, p + n_tied, [&](int a, int b) {
        long long ka = ((llrint(uf[a] * mx) % mx) + mx) % mx;
        long long kb = ((llrint(uf[b] * mx) % mx) + mx) % mx;
        return ka < kb;
      });
    }
  }
  if (tt.cap_tied < nuv || tt.n_tied != n_tied) {
    cudaFree(tt.wx);
    cudaFree(tt.wy);
    cudaFree(tt.perm);
    cudaFree(tt.duv);
    tt.wx = tt.wy = nullptr;
    tt.perm = nullptr;
    tt.duv = nullptr;
    tt.cap_tied = 0;
    if (cudaMalloc(&tt.wx, nuv * mx * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&tt.wy, nuv * my * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&tt.perm, nuv * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&tt.duv, 2 * nuv * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      tied_free(tt);
      return set_error(FFTBF_ENOMEM, "cannot allocate tied-beam tables (%zu pointings)", nuv);
    }
    tt.cap_tied = nuv;
  }
  // The plan keeps host copies of the pointings (to detect a repeat) and of the order;
  // the uploads read those plan-owned buffers, never the caller's.
  tt.n_tied = 0;
  tt.u.assign(u, u + nuv);
  tt.v.assign(v, v + nuv);
  tt.hperm.swap(perm);
  FFTBF_CUDA_TRY(cudaMemcpyAsync(tt.duv, tt.u.data(), nuv * sizeof(double), cudaMemcpyHostToDevice, st));
  FFTBF_CUDA_TRY(cudaMemcpyAsync(tt.duv + nuv, tt.v.data(), nuv * sizeof(double), cudaMemcpyHostToDevice, st));
  FFTBF_CUDA_TRY(cudaMemcpyAsync(tt.perm, tt.hperm.data(), nuv * sizeof(int), cudaMemcpyHostToDevice, st));
  const int threads = 256;
  auto blocks = [&](int64_t n) { return (unsigned)std::min<int64_t>((n + threads - 1) / threads, 1 << 20); };
  tied_table_kernel<<<blocks((int64_t)nuv * mx), threads, 0, st>>>(nx, mx, dense_x, nfreq,
                                                                    n_tied, tt.duv, tt.perm, tt.wx);
  FFTBF_CUDA_TRY(cudaGetLastError());
  tied_table_kernel<<<blocks((int64_t)nuv * my), threads, 0, st>>>(ny, my, dense_y, nfreq,
                                                                    n_tied, tt.duv + nuv, tt.perm, tt.wy);
  FFTBF_CUDA_TRY(cudaGetLastError());
  tt.n_tied = n_tied;
  return FFTBF_OK;
}

int tied_launch(const TiedTables& tt, const float* beams, int64_t nwin, int nfreq, int mx,
                int my, float* out, cudaStream_t st) {
  if (nwin <= 0) return FFTBF_OK;
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

// C ABI of the FFT-beamforming library: argument checks, plan tables, dispatch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "internal.cuh"

namespace fftbf {

static thread_local std::string g_error;
static thread_local int g_error_code = FFTBF_OK;

int set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_error = buf;
  g_error_code = code;
  return code;
}

void clear_error() {
  g_error.clear();
  g_error_code = FFTBF_OK;
}

int cuda_error(cudaError_t e, const char* what) {
  const int code = (e == cudaErrorMemoryAllocation) ? FFTBF_ENOMEM : FFTBF_ECUDA;
  return set_error(code, "%s: %s", what, cudaGetErrorString(e));
}

// Radix plan of a power-of-two N for the Stockham stages: the small radix (2 or 4) goes
// first so that the last stage, which keeps its outputs as accumulators, is radix 8.
static int radix_plan(int n, int* r0) {
  if (n == 1) { *r0 = 1; return 1; }
  int l = 0;
  while ((1 << l) < n) ++l;
  *r0 = (l % 3 == 1) ? 2 : (l % 3 == 2) ? 4 : 8;
  return (l % 3 == 0) ? l / 3 : l / 3 + 1;
}

static void remember_stream(fftbf_plan* p, cudaStream_t st) {
  if (std::find(p->streams_used.begin(), p->streams_used.end(), st) == p->streams_used.end())
    p->streams_used.push_back(st);
}

class DeviceGuard {
 public:
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev_);
    if (prev_ != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() { cudaSetDevice(prev_); }

 private:
  int prev_ = 0;
};

}  // namespace fftbf

using namespace fftbf;

extern "C" {

const char* fftbf_last_error(void) { return g_error.c_str(); }
int fftbf_last_error_code(void) { return g_error_code; }

fftbf_plan* fftbf_plan_create(int nx, int ny, int pad_x, int pad_y, int npol, int nfreq,
                              int n_int, const float* weights) {
  if (nx < 1 || ny < 1 || pad_x < 1 || pad_y < 1 || npol < 1 || nfreq < 1 || n_int < 1) {
    set_error(FFTBF_EINVAL, "plan sizes must all be >= 1 (nx=%d ny=%d pad_x=%d pad_y=%d "
              "npol=%d nfreq=%d n_int=%d)", nx, ny, pad_x, pad_y, npol, nfreq, n_int);
    return nullptr;
  }
  if ((int64_t)nx * ny > 65536 || pad_x > 64 || pad_y > 65536) {
    set_error(FFTBF_EUNSUPPORTED, "lattice limits: nx*ny <= 65536, pad_x <= 64, pad_y <= 65536");
    return nullptr;
  }
  fftbf_plan* p = new (std::nothrow) fftbf_plan();
  if (!p) {
    set_error(FFTBF_ENOMEM, "cannot allocate plan");
    return nullptr;
  }
  p->nx = nx; p->ny = ny; p->mx = pad_x; p->my = pad_y;
  p->npol = npol; p->nfreq = nfreq; p->n_int = n_int;
  cudaError_t e = cudaGetDevice(&p->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, p->device);
  const int nant = nx * ny;
  if (e == cudaSuccess) e = cudaMalloc(&p->d_w, sizeof(float2) * nant);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_ex, sizeof(float2) * pad_x * nx);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_tw, sizeof(float2) * pad_y);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(p->d_err, 0, sizeof(int));
  if (e == cudaSuccess) {
    p->h_w.assign(2 * (size_t)nant, 0.f);
    for (int i = 0; i < nant; ++i) {
      p->h_w[2 * i] = weights ? weights[2 * i] : 1.f;
      p->h_w[2 * i + 1] = weights ? weights[2 * i + 1] : 0.f;
    }
    p->real_w = true;
    for (int i = 0; i < nant; ++i) p->real_w = p->real_w && p->h_w[2 * i + 1] == 0.f;
    e = cudaMemcpy(p->d_w, p->h_w.data(), sizeof(float2) * nant, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    cuda_error(e, "fftbf_plan_create");
    fftbf_destroy(p);
    return nullptr;
  }
  if (build_tables(nx, pad_x, pad_y, p->d_ex, p->d_tw, 0) != FFTBF_OK ||
      (e = cudaDeviceSynchronize()) != cudaSuccess) {
    if (e != cudaSuccess) cuda_error(e, "plan tables");
    fftbf_destroy(p);
    return nullptr;
  }
  return p;
}

int fftbf_plan_set_precision(fftbf_plan* p, int prec) {
  if (!p) return set_error(FFTBF_EINVAL, "null plan");
  if (prec == FFTBF_PREC_FP32) {
    p->precision = prec;
    return FFTBF_OK;
  }
  if (prec != FFTBF_PREC_TC_FP16 && prec != FFTBF_PREC_TC_BF16 && prec != FFTBF_PREC_TC_FP16X3)
    return set_error(FFTBF_EINVAL, "unknown precision %d", prec);
  if (!tc_supported(p->nx, p->ny, p->mx, p->my))
    return set_error(FFTBF_EUNSUPPORTED,
                     "tensor-core form needs pad_x = 4, pad_y = 512 and at most 256 N-S feeds "
                     "(got nx=%d ny=%d pad_x=%d pad_y=%d)", p->nx, p->ny, p->mx, p->my);
  DeviceGuard g(p->device);
  if (!p->d_b1) {
    FFTBF_CUDA_TRY(cudaMalloc(&p->d_b1, sizeof(uint16_t) * 64 * 32));
    FFTBF_CUDA_TRY(cudaMalloc(&p->d_b2, sizeof(uint16_t) * 32 * 32));
  }
  const bool bf16 = prec == FFTBF_PREC_TC_BF16;
  int rc = build_tc_tables(p->d_b1, p->d_b2, bf16, 0);
  if (rc != FFTBF_OK) return rc;
  if (prec == FFTBF_PREC_TC_FP16X3) {
    if (!p->d_b1lo) {
      FFTBF_CUDA_TRY(cudaMalloc(&p->d_b1lo, sizeof(uint16_t) * 64 * 32));
      FFTBF_CUDA_TRY(cudaMalloc(&p->d_b2lo, sizeof(uint16_t) * 32 * 32));
    }
    rc = build_tc_tables_lo(p->d_b1lo, p->d_b2lo, 0);
    if (rc != FFTBF_OK) return rc;
  }
  if (prec == FFTBF_PREC_TC_FP16 || prec == FFTBF_PREC_TC_BF16) {
    if (!p->d_b1w) {
      FFTBF_CUDA_TRY(cudaMalloc(&p->d_b1w, sizeof(uint16_t) * 64 * 32));
      FFTBF_CUDA_TRY(cudaMalloc(&p->d_b2w, sizeof(uint16_t) * 32 * 32));
      FFTBF_CUDA_TRY(cudaMalloc(&p->d_tw16, sizeof(uint32_t) * 16 * 16 * 2));
      FFTBF_CUDA_TRY(cudaMalloc(&p->d_f1, sizeof(uint16_t) * 128 * 128));
    }
    rc = build_tcw_tables(p->d_b1w, p->d_b2w, p->d_tw16, prec == FFTBF_PREC_TC_BF16, 0);
    if (rc != FFTBF_OK) return rc;
    rc = build_tcg_table(p->d_f1, prec == FFTBF_PREC_TC_BF16, 0);
    if (rc != FFTBF_OK) return rc;
  }
  FFTBF_CUDA_TRY(cudaDeviceSynchronize());
  // FP16 range: |X1| <= 16 * max_iy sum_ix |w| * 8 sqrt(2); keep it below 30000.
  double wmax = 0.0;
  for (int iy = 0; iy < p->ny; ++iy) {
    double sum = 0.0;
    for (int ix = 0; ix < p->nx; ++ix) {
      const double re = p->h_w[2 * ((size_t)ix * p->ny + iy)], im = p->h_w[2 * ((size_t)ix * p->ny + iy) + 1];
      sum += std::sqrt(re * re + im * im);
    }
    wmax = std::max(wmax, sum);
  }
  const double bound = 16.0 * wmax * 8.0 * std::sqrt(2.0);
  p->tc_scale = (!bf16 && bound > 30000.0) ? (float)(30000.0 / bound) : 1.f;
  p->precision = prec;
  return FFTBF_OK;
}

int fftbf_execute(fftbf_plan* p, const uint8_t* volts, int64_t T, float* beams, void* stream) {
  NvtxRange nvtx("fftbf_execute");
  if (!p) return set_error(FFTBF_EINVAL, "null plan");
  if (T < 0 || T % p->n_int != 0)
    return set_error(FFTBF_EINVAL, "T = %lld is not a non-negative multiple of n_int = %d",
                     (long long)T, p->n_int);
  if (T == 0) return FFTBF_OK;
  if (!volts || !beams) return set_error(FFTBF_EINVAL, "null voltage or beam pointer");
  DeviceGuard g(p->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  BeamArgs a{};
  a.volts = volts;
  a.beams = beams;
  a.w = p->d_w;
  a.ex = p->d_ex;
  a.tw = p->d_tw;
  a.nx = p->nx; a.ny = p->ny; a.mx = p->mx; a.my = p->my;
  a.npol = p->npol; a.nfreq = p->nfreq; a.n_int = p->n_int;
  a.nyf = std::min(p->ny, p->my);
  a.nwin = T / p->n_int;
  a.ew_dft = (p->mx == p->nx) && (p->mx & (p->mx - 1)) == 0 && p->mx <= 16;
  a.real_w = p->real_w ? 1 : 0;
  const int nsnap = p->n_int * p->npol;
  int S = kMaxElems / (p->mx * p->my);
  if (S < 1) S = 1;
  if (S > nsnap) S = nsnap;
  a.S = S;
  if (fp32_fft_supported(p->mx, p->my)) a.nst = radix_plan(p->my, &a.r0);
  int rc;
  if (p->precision == FFTBF_PREC_FP32) {
    rc = launch_beams_fp32(a, p->nsm, st);
  } else {
    TcArgs ta{};
    ta.b = a;
    ta.b1 = p->d_b1;
    ta.b2 = p->d_b2;
    ta.scale = p->tc_scale;
    ta.err = p->d_err;
    ta.bf16 = p->precision == FFTBF_PREC_TC_BF16;
    ta.split = p->precision == FFTBF_PREC_TC_FP16X3;
    // the packed-half input stage with real weights: 4 bytes per feed in shared memory
    ta.w4 = p->precision == FFTBF_PREC_TC_FP16 && p->real_w && a.ew_dft && p->nx == 4 &&
            (p->ny & 3) == 0 && a.nyf == p->ny;
    ta.b1lo = p->d_b1lo;
    ta.b2lo = p->d_b2lo;
    if (p->precision == FFTBF_PREC_TC_FP16 || p->precision == FFTBF_PREC_TC_BF16) {
      ta.b1w = p->d_b1w;
      ta.b2w = p->d_b2w;
      ta.tw16 = p->d_tw16;
      ta.f1 = p->d_f1;
    }
    rc = launch_beams_tc(ta, p->nsm, st);
  }
  if (rc == FFTBF_OK) remember_stream(p, st);
  return rc;
}

int fftbf_tied_beams(fftbf_plan* p, const float* beams, int64_t n_windows, int n_tied,
                     const double* u, const double* v, float* tied, void* stream) {
  NvtxRange nvtx("fftbf_tied_beams");
  if (!p) return set_error(FFTBF_EINVAL, "null plan");
  if (n_windows < 0 || n_tied < 1)
    return set_error(FFTBF_EINVAL, "need n_windows >= 0 and n_tied >= 1");
  if (!u || !v) return set_error(FFTBF_EINVAL, "null pointing array");
  if (n_windows > 0 && (!beams || !tied)) return set_error(FFTBF_EINVAL, "null beam pointer");
  DeviceGuard g(p->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = tied_prepare(p->tied, p->nx, p->ny, p->mx, p->my, p->nfreq, n_tied, u, v, st);
  if (rc != FFTBF_OK) return rc;
  p->tied.err = p->d_err;
  rc = tied_launch(p->tied, beams, n_windows, p->nfreq, p->mx, p->my, tied, st);
  if (rc == FFTBF_OK) remember_stream(p, st);
  return rc;
}

int fftbf_tied_set_window(fftbf_plan* p, const double* hx, const double* hy, int trunc_x,
                          int trunc_y) {
  if (!p) return set_error(FFTBF_EINVAL, "null plan");
  if (trunc_x < 0 || trunc_y < 0 || trunc_x > p->mx || trunc_y > p->my)
    return set_error(FFTBF_EINVAL, "truncation must be in 0..pad per axis");
  if (hx && p->mx < 2 * p->nx - 1)
    return set_error(FFTBF_EINVAL, "an E-W window needs pad_x >= 2nx-1 (the FFT beams of a "
                     "smaller padding do not hold every redundant baseline)");
  if (hy && p->my < 2 * p->ny - 1)
    return set_error(FFTBF_EINVAL, "a N-S window needs pad_y >= 2ny-1");
  auto lags = [](const double* h, int n, std::vector<double>& g) -> int {
    g.clear();
    if (!h) return FFTBF_OK;
    for (int i = 0; i < n; ++i)
      if (!std::isfinite(h[i])) return set_error(FFTBF_EINVAL, "window value %d not finite", i);
    g.assign(2 * (size_t)n - 1, 0.0);
    for (int d = -(n - 1); d < n; ++d) {
      double acc = 0.0;
      for (int a = std::max(0, -d); a < std::min(n, n - d); ++a) acc += h[a + d] * h[a];
      g[d + n - 1] = acc / (n - std::abs(d));
    }
    return FFTBF_OK;
  };
  std::vector<double> gx, gy;
  int rc = lags(hx, p->nx, gx);
  if (rc == FFTBF_OK) rc = lags(hy, p->ny, gy);
  if (rc != FFTBF_OK) return rc;
  p->tied.win_x.g.swap(gx);
  p->tied.win_y.g.swap(gy);
  p->tied.win_x.trunc = trunc_x;
  p->tied.win_y.trunc = trunc_y;
  ++p->tied.version;
  return FFTBF_OK;
}

int fftbf_plan_sync(fftbf_plan* p) {
  if (!p) return set_error(FFTBF_EINVAL, "null plan");
  DeviceGuard g(p->device);
  for (cudaStream_t st : p->streams_used) FFTBF_CUDA_TRY(cudaStreamSynchronize(st));
  if (p->pipe.copy) FFTBF_CUDA_TRY(cudaStreamSynchronize(p->pipe.copy));
  for (int k = 0; k < HostPipe::kCopyStreams - 1; ++k)
    if (p->pipe.copy_extra[k]) FFTBF_CUDA_TRY(cudaStreamSynchronize(p->pipe.copy_extra[k]));
  FFTBF_CUDA_TRY(cudaGetLastError());
  int err = 0;
  FFTBF_CUDA_TRY(cudaMemcpy(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err != 0) {
    FFTBF_CUDA_TRY(cudaMemset(p->d_err, 0, sizeof(int)));
    return set_error(err, "a device-side wait of the tensor-core kernel ran out");
  }
  return FFTBF_OK;
}

void fftbf_destroy(fftbf_plan* p) {
  if (!p) return;
  {
    DeviceGuard g(p->device);
    for (cudaStream_t st : p->streams_used) cudaStreamSynchronize(st);
    host_pipe_free(p->pipe);
    tied_free(p->tied);
    cudaFree(p->d_w);
    cudaFree(p->d_ex);
    cudaFree(p->d_tw);
    cudaFree(p->d_b1);
    cudaFree(p->d_b2);
    cudaFree(p->d_b1lo);
    cudaFree(p->d_b2lo);
    cudaFree(p->d_b1w);
    cudaFree(p->d_b2w);
    cudaFree(p->d_tw16);
    cudaFree(p->d_f1);
    cudaFree(p->d_err);
  }
  delete p;
}

int fftbf_debug_unpack(const uint8_t* in, int64_t n, float* out, void* stream) {
  if (n < 0) return set_error(FFTBF_EINVAL, "negative length");
  if (n > 0 && (!in || !out)) return set_error(FFTBF_EINVAL, "null pointer");
  return launch_debug_unpack(in, n, out, static_cast<cudaStream_t>(stream));
}

int fftbf_debug_wait_timeout(int limit_us, void* stream) {
  if (limit_us < 1 || limit_us > 2000000) return set_error(FFTBF_EINVAL, "limit_us must be 1..2000000");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int* err = nullptr;
  FFTBF_CUDA_TRY(cudaMalloc(&err, sizeof(int)));
  int rc = FFTBF_OK;
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
  if (e == cudaSuccess) rc = launch_debug_wait_timeout((uint64_t)limit_us * 1000ull, err, st);
  int h = 0;
  if (e == cudaSuccess && rc == FFTBF_OK) e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && rc == FFTBF_OK) e = cudaStreamSynchronize(st);
  cudaFree(err);
  if (e != cudaSuccess) return cuda_error(e, "debug wait");
  if (rc != FFTBF_OK) return rc;
  return h ? set_error(h, "device wait ran out after %d us (as intended)", limit_us) : FFTBF_OK;
}

int fftbf_debug_tc_gemm(const uint16_t* a, const uint16_t* b, int n, int bf16, int padded,
                        float* d, void* stream) {
  if (!a || !b || !d) return set_error(FFTBF_EINVAL, "null pointer");
  if (n != 32 && n != 64 && n != 128 && n != 256)
    return set_error(FFTBF_EINVAL, "n must be 32, 64, 128 or 256");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int* err = nullptr;
  FFTBF_CUDA_TRY(cudaMalloc(&err, sizeof(int)));
  cudaMemsetAsync(err, 0, sizeof(int), st);
  if (padded < 0 || padded > 4) {
    cudaFree(err);
    return set_error(FFTBF_EINVAL, "layout must be 0 to 4");
  }
  int rc = launch_debug_tc_gemm(a, b, n, bf16 != 0, padded, d, err, st);
  int h = 0;
  if (rc == FFTBF_OK) {
    cudaError_t e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_error(e, "debug tc gemm");
    else if (h != 0) rc = set_error(h, "tensor-core wait ran out");
  }
  cudaFree(err);
  return rc;
}

}  // extern "C"

// Internal declarations shared by the library's translation units (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "fftbf.h"

#include <nvtx3/nvToolsExt.h>

namespace fftbf {

// NVTX range over an entry point (header-only NVTX v3: no cost unless a tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Thread-local error message plus status code.
int set_error(int code, const char* fmt, ...);
int cuda_error(cudaError_t e, const char* what);
// Forget the calling thread's last error (after a recovered failure, e.g. a fallback).
void clear_error();

#define FFTBF_CUDA_TRY(call)                               \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_error(e_, #call);   \
  } while (0)

constexpr int kThreads = 256;          // threads per CTA of the FP32 beam kernel
#ifndef FFTBF_FP32_MIN_BLOCKS
#define FFTBF_FP32_MIN_BLOCKS 2            // resident CTAs per SM the register budget targets
#endif
constexpr int kMaxElems = 2048;        // complex values per CTA iteration (S * Mx * My)
constexpr int kMaxStages = 16;

// Arguments of the FP32 beam kernels (one launch = one fftbf_execute).
struct BeamArgs {
  const uint8_t* volts;   // [T][nfreq][npol][nx][ny]
  float* beams;           // [nwin][nfreq][mx][my]
  const float2* w;        // [nx][ny] apodisation weights
  const float2* ex;       // [mx][nx] E-W DFT matrix exp(-2 pi i (A ix mod mx) / mx)
  const float2* tw;       // [my] N-S twiddles exp(-2 pi i k / my)
  int nx, ny, mx, my, npol, nfreq, n_int;
  int nyf;                // min(ny, my): folded N-S input length
  int S;                  // snapshots per CTA iteration
  int nst;                // FFT stages (power-of-two my): r0 first, then radix 8
  int r0;                 // radix of the first stage (1, 2, 4 or 8)
  int ew_dft;             // 1 if mx == nx and mx is a power of two (E-W is a plain DFT)
  int real_w;             // 1 if every weight is real (two multiplies instead of a complex one)
  int64_t nwin;           // windows in this call
};

// Launch the FP32 fused beam kernel. Returns FFTBF_OK or an error code.
int launch_beams_fp32(const BeamArgs& a, int nsm, cudaStream_t st);
// True if the register-FFT path supports this shape (else the direct-DFT path runs).
bool fp32_fft_supported(int mx, int my);
// Warp-per-transform kernel for my == 512 with at most 256 feeds on the N-S axis.
bool fp32_n512_supported(const BeamArgs& a);
int launch_beams_fp32_n512(const BeamArgs& a, int nsm, cudaStream_t st);
bool fp32_4x256_eligible(const BeamArgs& a);
int launch_beams_fp32_4x256(const BeamArgs& a, int nsm, cudaStream_t st);
int launch_debug_unpack(const uint8_t* in, int64_t n, float* out, cudaStream_t st);

// Batched launches (batch.cu): one job = one plan's buffers over nwin windows.
struct BatchJob {
  BeamArgs a;
  int variant;
  int64_t item0;      // first global item of this job
  int64_t nitems;     // nwin * nfreq
};
int batch_variant(int mx, int my);
size_t batch_item_smem(const BeamArgs& a, int variant);
// Upload h_jobs (item0 must be prefix sums) and run the batch kernel over them.
int batch_launch_jobs(const BatchJob* h_jobs, int njobs, BatchJob* d_jobs,
                      unsigned long long* d_counter, size_t smem, int grid, cudaStream_t st);

// Tensor-core form (4 E-W beams x 512 N-S beams over <= 256 N-S feeds).
struct TcArgs {
  BeamArgs b;
  const uint16_t* b1;   // [64][32] stage-1 matrix (transposed, interleaved), FP16 or BF16 bits
  const uint16_t* b2;   // [32][32] stage-2 DFT16 matrix
  float scale;          // multiplies the E-W output before rounding to 16 bits
  int* err;             // device error word (FFTBF_ETIMEOUT on a wait that ran out)
  int bf16;
  int split;            // split FP16: b1lo, b2lo hold the residuals of b1, b2
  int w4;               // FP16 form with real weights on the packed-half input stage
  const uint16_t* b1lo;
  const uint16_t* b2lo;
  // warp-specialised FP16 kernel (4x256 lattice): planar stage matrices and W512 twiddles
  const uint16_t* b1w;  // [64][32]
  const uint16_t* b2w;  // [32][32]
  const uint32_t* tw16; // [16 n2][16 k1 pairs][2] half2 (cos, -sin)
  // grouped kernel (4x256 lattice): E-W x pruned W32 stage matrix [128][128] (b2w is its
  // stage-2 matrix)
  const uint16_t* f1;
};
bool tc_supported(int nx, int ny, int mx, int my);
int launch_beams_tc(const TcArgs& ta, int nsm, cudaStream_t st);
int build_tc_tables(uint16_t* b1, uint16_t* b2, bool bf16, cudaStream_t st);
int build_tc_tables_lo(uint16_t* b1, uint16_t* b2, cudaStream_t st);
bool tcw_eligible(const TcArgs& ta);
int launch_beams_tcw(const TcArgs& ta, int nsm, cudaStream_t st);
int build_tcw_tables(uint16_t* b1, uint16_t* b2, uint32_t* tw16, bool bf16, cudaStream_t st);
bool tcg_eligible(const TcArgs& ta);
int launch_beams_tcg(const TcArgs& ta, int nsm, cudaStream_t st);
int build_tcg_table(uint16_t* f1, bool bf16, cudaStream_t st);
int launch_debug_tc_gemm(const uint16_t* A, const uint16_t* B, int n, bool bf16, int layout,
                         float* D, int* err, cudaStream_t st);
int launch_debug_wait_timeout(uint64_t limit_ns, int* err, cudaStream_t st);
// FP64 table builders (device), rounded to FP32.
int build_tables(int nx, int mx, int my, float2* ex, float2* tw, cudaStream_t st);

// Tied-beam weight tables and regridding GEMM.
struct AxisWindow {
  std::vector<double> g;        // 2n-1 lag coefficients of the optimal windowed beam; empty = none
  int trunc = 0;                // keep the `trunc` FFT beams nearest the pointing (0 = all)
};
struct TiedTables {
  int n_tied = 0;
  AxisWindow win_x, win_y;
  int version = 0, built_version = -1;   // window settings the tables were built for
  double* d_g = nullptr;        // device copy: g_x then g_y
  int kx = 0, ky = 0;           // compact kernel taps per axis (0: dense GEMM path)
  int* first = nullptr;         // [nfreq][n_tied][2] first kept beam per axis (compact path)
  float* cw = nullptr;          // [nfreq][n_tied][kx + ky] tap weights (compact path)
  std::vector<double> u, v;     // host copies of the pointings the tables were made for
  std::vector<int> hperm;       // host copy of perm
  std::vector<double> hg;       // host staging of the lag coefficients
  float* wx = nullptr;          // [nfreq][n_tied][mx] in sorted order
  float* wy = nullptr;          // [nfreq][n_tied][my] in sorted order
  int* perm = nullptr;          // [nfreq][n_tied] sorted slot -> caller's pointing index
  double* duv = nullptr;        // device scratch for u, v
  size_t cap_tied = 0;
  // tensor-core path (E-W axis on the grid): split FP16 weight rows and their exponents,
  // the E-W beam of each sorted pointing, and per-call split beam rows
  int tc = 0;
  int tc_n_tied = 0;            // pointings per channel of the split tables
  uint16_t* wyh = nullptr;      // [nfreq][n_tied][my] FP16 hi of 2^e wx wy
  uint16_t* wyl = nullptr;      // [nfreq][n_tied][my] FP16 lo
  int* wye = nullptr;           // [nfreq][n_tied] row exponent e
  int* wa = nullptr;            // [nfreq][n_tied] E-W beam of the pointing
  uint16_t* ph = nullptr;       // [nwin][nfreq][mx][my] FP16 hi of the beams (scratch)
  uint16_t* pl = nullptr;
  int* pe = nullptr;            // [nwin][nfreq][mx] beam row exponents
  size_t p_cap = 0;             // rows of ph / pl / pe
  int* err = nullptr;           // the plan's device error word (bounded waits)
};
bool tied_tc_eligible(bool dense_x, int mx, int my);
int tied_tc_build(TiedTables& tt, int64_t nuv, int mx, int my, cudaStream_t st);
int tied_tc_launch(TiedTables& tt, const float* beams, int64_t nwin, int nfreq, int mx, int my,
                   float* out, cudaStream_t st);
int tied_prepare(TiedTables& tt, int nx, int ny, int mx, int my, int nfreq, int n_tied,
                 const double* u, const double* v, cudaStream_t st);
int tied_launch(TiedTables& tt, const float* beams, int64_t nwin, int nfreq, int mx,
                int my, float* out, cudaStream_t st);
void tied_free(TiedTables& tt);

// Staging of fftbf_execute_host: two voltage chunks, device outputs, copy stream.
struct HostPipe {
  static constexpr int kCopyStreams = 4;   // parallel host-to-device copies per chunk
  static constexpr int kStages = 3;        // staging buffers: a buffer is refilled after the
                                           // compute three chunks back, so copies rarely wait
  cudaStream_t copy = nullptr;
  cudaStream_t copy_extra[kCopyStreams - 1] = {nullptr, nullptr, nullptr};
  cudaEvent_t copied_extra[kStages][kCopyStreams - 1] = {};
  cudaEvent_t copied[kStages] = {};
  cudaEvent_t freed[kStages] = {};
  uint8_t* stage[kStages] = {};
  size_t stage_bytes = 0;
  float* beams = nullptr;
  size_t beams_cap = 0;
  float* tied = nullptr;
  size_t tied_cap = 0;
  int next = 0;                            // staging buffer of the next chunk (kept across calls)
};
void host_pipe_free(HostPipe& hp);

}  // namespace fftbf

struct fftbf_plan;
struct fftbf_batch;
namespace fftbf {
void batch_fill_args(const fftbf_plan* p, BeamArgs& a);
}
extern "C" int fftbf_batch_grid(const fftbf_batch* bb);
extern "C" int fftbf_batch_tuned_variant(const fftbf_batch* bb, int i);
extern "C" size_t fftbf_batch_smem(const fftbf_batch* bb);

struct fftbf_plan {
  int device = 0;
  int nsm = 0;
  int nx = 0, ny = 0, mx = 0, my = 0, npol = 0, nfreq = 0, n_int = 0;
  int precision = FFTBF_PREC_FP32;
  float2* d_w = nullptr;
  float2* d_ex = nullptr;
  float2* d_tw = nullptr;
  fftbf::TiedTables tied;
  fftbf::HostPipe pipe;
  std::vector<float> h_w;         // host copy of the weights (re, im interleaved)
  bool real_w = false;            // every weight has a zero imaginary part
  uint16_t* d_b1 = nullptr;       // tensor-core stage matrices for the selected precision
  uint16_t* d_b2 = nullptr;
  uint16_t* d_b1lo = nullptr;     // split FP16 form: residuals of the stage matrices
  uint16_t* d_b2lo = nullptr;
  uint16_t* d_b1w = nullptr;      // warp-specialised FP16 kernel: planar stage matrices
  uint16_t* d_b2w = nullptr;
  uint32_t* d_tw16 = nullptr;     // and its W512 twiddle pairs
  uint16_t* d_f1 = nullptr;       // grouped FP16/BF16 kernel: E-W x W32 stage matrix
  float tc_scale = 1.f;
  int* d_err = nullptr;           // device error word of bounded waits
  std::vector<cudaStream_t> streams_used;
};

// fftbf_execute_host: the hot path on host buffers, with the host-to-device copies of
// the voltages overlapped with the transform of the previous chunk.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.cuh"

namespace fftbf {

void host_pipe_free(HostPipe& hp) {
  if (hp.copy) cudaStreamSynchronize(hp.copy);
  for (int k = 0; k < HostPipe::kCopyStreams - 1; ++k) {
    if (hp.copy_extra[k]) {
      cudaStreamSynchronize(hp.copy_extra[k]);
      cudaStreamDestroy(hp.copy_extra[k]);
    }
    for (int b = 0; b < HostPipe::kStages; ++b)
      if (hp.copied_extra[b][k]) cudaEventDestroy(hp.copied_extra[b][k]);
  }
  for (int b = 0; b < HostPipe::kStages; ++b) {
    if (hp.copied[b]) cudaEventDestroy(hp.copied[b]);
    if (hp.freed[b]) cudaEventDestroy(hp.freed[b]);
    cudaFree(hp.stage[b]);
  }
  cudaFree(hp.beams);
  cudaFree(hp.tied);
  if (hp.copy) cudaStreamDestroy(hp.copy);
  hp = HostPipe();
}

static int grow(void** ptr, size_t* cap, size_t need) {
  if (*cap >= need) return FFTBF_OK;
  cudaFree(*ptr);
  *ptr = nullptr;
  *cap = 0;
  if (cudaMalloc(ptr, need) != cudaSuccess) {
    cudaGetLastError();
    return set_error(FFTBF_ENOMEM, "cannot allocate %zu bytes of staging", need);
  }
  *cap = need;
  return FFTBF_OK;
}

}  // namespace fftbf

using namespace fftbf;

extern "C" int fftbf_execute_host(fftbf_plan* p, const uint8_t* volts_h, int64_t T,
                                  float* beams_h, int n_tied, const double* u,
                                  const double* v, float* tied_h, void* stream) {
  NvtxRange nvtx("fftbf_execute_host");
  if (!p) return set_error(FFTBF_EINVAL, "null plan");
  if (T < 0 || T % p->n_int != 0)
    return set_error(FFTBF_EINVAL, "T = %lld is not a non-negative multiple of n_int = %d",
                     (long long)T, p->n_int);
  if (n_tied < 0) return set_error(FFTBF_EINVAL, "n_tied < 0");
  if (T == 0) return FFTBF_OK;
  if (!volts_h || !beams_h) return set_error(FFTBF_EINVAL, "null host buffer");
  if (n_tied > 0 && (!u || !v || !tied_h)) return set_error(FFTBF_EINVAL, "null tied buffer");
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != p->device) cudaSetDevice(p->device);
  struct Restore {
    int d;
    ~Restore() { cudaSetDevice(d); }
  } restore{prev};

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  HostPipe& hp = p->pipe;
  if (!hp.copy) {
    FFTBF_CUDA_TRY(cudaStreamCreateWithFlags(&hp.copy, cudaStreamNonBlocking));
    for (int b = 0; b < HostPipe::kStages; ++b) {
      FFTBF_CUDA_TRY(cudaEventCreateWithFlags(&hp.copied[b], cudaEventDisableTiming));
      FFTBF_CUDA_TRY(cudaEventCreateWithFlags(&hp.freed[b], cudaEventDisableTiming));
    }
    for (int k = 0; k < HostPipe::kCopyStreams - 1; ++k) {
      FFTBF_CUDA_TRY(cudaStreamCreateWithFlags(&hp.copy_extra[k], cudaStreamNonBlocking));
      for (int b = 0; b < HostPipe::kStages; ++b)
        FFTBF_CUDA_TRY(cudaEventCreateWithFlags(&hp.copied_extra[b][k], cudaEventDisableTiming));
    }
  }
  const int64_t nwin = T / p->n_int;
  const size_t snap_t = (size_t)p->nfreq * p->npol * p->nx * p->ny;   // bytes per sample t
  const size_t win_bytes = snap_t * p->n_int;
  const size_t beam_win = (size_t)p->nfreq * p->mx * p->my;           // floats per window
  // Chunks of whole windows holding about four waves of work items for the resident CTAs
  // (a one-window chunk of 1024 channels is 1.1 waves, so its second wave runs nearly
  // empty), at most 4 GiB of voltages per buffer, split evenly over the call.
  const int64_t want_items = 4LL * p->nsm * 6;
  int64_t cw = (want_items + p->nfreq - 1) / p->nfreq;
  const int64_t cap = std::max<int64_t>(1, (int64_t)((4ull << 30) / win_bytes));
  cw = std::max<int64_t>(1, std::min(cw, std::min(cap, nwin)));
  const int64_t nchunk = (nwin + cw - 1) / cw;
  cw = (nwin + nchunk - 1) / nchunk;
  if (hp.stage_bytes < cw * win_bytes) {
    // all earlier work on the old buffers must be done before they are freed
    cudaStreamSynchronize(hp.copy);
    for (int k = 0; k < HostPipe::kCopyStreams - 1; ++k) cudaStreamSynchronize(hp.copy_extra[k]);
    cudaStreamSynchronize(st);
  }
  if (hp.stage_bytes < cw * win_bytes) {
    for (int b = 0; b < HostPipe::kStages; ++b) {
      cudaFree(hp.stage[b]);
      hp.stage[b] = nullptr;
    }
    hp.stage_bytes = 0;
    for (int b = 0; b < HostPipe::kStages; ++b) {
      if (cudaMalloc(&hp.stage[b], cw * win_bytes) != cudaSuccess) {
        cudaGetLastError();
        return set_error(FFTBF_ENOMEM, "cannot allocate voltage staging");
      }
    }
    hp.stage_bytes = cw * win_bytes;
  }
  if (hp.beams_cap < nwin * beam_win * sizeof(float) ||
      (n_tied > 0 && hp.tied_cap < (size_t)nwin * p->nfreq * n_tied * sizeof(float))) {
    cudaStreamSynchronize(st);
  }
  int rc = grow(reinterpret_cast<void**>(&hp.beams), &hp.beams_cap, nwin * beam_win * sizeof(float));
  if (rc != FFTBF_OK) return rc;
  if (n_tied > 0) {
    rc = grow(reinterpret_cast<void**>(&hp.tied), &hp.tied_cap,
              (size_t)nwin * p->nfreq * n_tied * sizeof(float));
    if (rc != FFTBF_OK) return rc;
  }

  // the buffer rotation continues from the previous call, so its last chunks' compute
  // overlaps this call's first copies
  int b = hp.next;
  for (int64_t w0 = 0; w0 < nwin; w0 += cw, b = (b + 1) % HostPipe::kStages) {
    const int64_t nw = std::min<int64_t>(cw, nwin - w0);
    // the chunk's bytes go over kCopyStreams concurrent copies (one engine rarely fills
    // the host link), each waiting until the previous user of buffer b has finished
    const size_t bytes = nw * win_bytes;
    const size_t part = ((bytes / HostPipe::kCopyStreams) + 4095) & ~(size_t)4095;
    for (int k = 0; k < HostPipe::kCopyStreams; ++k) {
      cudaStream_t cs = k == 0 ? hp.copy : hp.copy_extra[k - 1];
      cudaEvent_t ev = k == 0 ? hp.copied[b] : hp.copied_extra[b][k - 1];
      const size_t off = (size_t)k * part;
      if (off >= bytes) {
        FFTBF_CUDA_TRY(cudaEventRecord(ev, cs));
      } else {
        FFTBF_CUDA_TRY(cudaStreamWaitEvent(cs, hp.freed[b], 0));
        FFTBF_CUDA_TRY(cudaMemcpyAsync(hp.stage[b] + off, volts_h + w0 * win_bytes + off,
                                       std::min(part, bytes - off), cudaMemcpyHostToDevice, cs));
        FFTBF_CUDA_TRY(cudaEventRecord(ev, cs));
      }
      FFTBF_CUDA_TRY(cudaStreamWaitEvent(st, ev, 0));
    }
    rc = fftbf_execute(p, hp.stage[b], nw * p->n_int, hp.beams + w0 * beam_win, stream);
    if (rc != FFTBF_OK) return rc;
    FFTBF_CUDA_TRY(cudaEventRecord(hp.freed[b], st));
  }
  hp.next = b;
  if (n_tied > 0) {
    rc = fftbf_tied_beams(p, hp.beams, nwin, n_tied, u, v, hp.tied, stream);
    if (rc != FFTBF_OK) return rc;
    FFTBF_CUDA_TRY(cudaMemcpyAsync(tied_h, hp.tied, (size_t)nwin * p->nfreq * n_tied * sizeof(float),
                                   cudaMemcpyDeviceToHost, st));
  }
  FFTBF_CUDA_TRY(cudaMemcpyAsync(beams_h, hp.beams, nwin * beam_win * sizeof(float),
                                 cudaMemcpyDeviceToHost, st));
  return FFTBF_OK;
}

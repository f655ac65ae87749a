// Instantiation of the FP32 fused beam kernels for an E-W size of 3 (one file per size so
// that nvcc compiles them in parallel).
#include "beam_fp32.cuh"

namespace fftbf {
template int launch_fft_mx<3>(const BeamArgs&, int, int, cudaStream_t);
}  // namespace fftbf

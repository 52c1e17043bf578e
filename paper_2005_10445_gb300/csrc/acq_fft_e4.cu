// acq_fft_e4.cu -- transform kernels with 16 complex values per thread.
#include "acq_fft_kernels.cuh"

namespace atlas {

cudaError_t prepare_fft_e4() { return FftLaunch<4>::prepare(); }

cudaError_t launch_window_fft_e4(int logM, bool split, const WindowFftParams& p, cudaStream_t s) {
  return FftLaunch<4>::window_fft(logM, split, p, s);
}

cudaError_t launch_corr_e4(int logM, bool split, const CorrParams& p, cudaStream_t s) {
  return FftLaunch<4>::corr(logM, split, p, s);
}

}  // namespace atlas

// acq_fft_e5.cu -- transform kernels with 32 complex values per thread.
#include "acq_fft_kernels.cuh"

namespace atlas {

cudaError_t prepare_fft_e5() { return FftLaunch<5>::prepare(); }

cudaError_t launch_window_fft_e5(int logM, bool split, const WindowFftParams& p, cudaStream_t s) {
  return FftLaunch<5>::window_fft(logM, split, p, s);
}

cudaError_t launch_corr_e5(int logM, bool split, const CorrParams& p, cudaStream_t s) {
  return FftLaunch<5>::corr(logM, split, p, s);
}

}  // namespace atlas

// Explicit instantiations of the FFT pass launchers for line length(s) 64, 80, 96.
#include "fft_core.cuh"

namespace sfw {

SFW_FFT_INSTANTIATE(64)
SFW_FFT_INSTANTIATE(80)
SFW_FFT_INSTANTIATE(96)

}  // namespace sfw

// Explicit instantiations of the FFT pass launchers for line length(s) 128.
#include "fft_core.cuh"

namespace sfw {

SFW_FFT_INSTANTIATE(128)

}  // namespace sfw

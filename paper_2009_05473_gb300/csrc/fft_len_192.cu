// Explicit instantiations of the FFT pass launchers for line length(s) 192.
#include "fft_core.cuh"

namespace sfw {

SFW_FFT_INSTANTIATE(192)

}  // namespace sfw

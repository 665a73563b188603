// Explicit instantiations of the FFT pass launchers for line length(s) 144.
#include "fft_core.cuh"

namespace sfw {

SFW_FFT_INSTANTIATE(144)

}  // namespace sfw

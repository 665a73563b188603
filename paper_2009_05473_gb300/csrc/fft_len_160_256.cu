// Explicit instantiations of the FFT pass launchers for line length(s) 160, 256.
#include "fft_core.cuh"

namespace sfw {

SFW_FFT_INSTANTIATE(160)
SFW_FFT_INSTANTIATE(256)

}  // namespace sfw

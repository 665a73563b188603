// Explicit instantiations of the FFT pass launchers for line length(s) runtime (generic).
#include "fft_core.cuh"

namespace sfw {

SFW_FFT_INSTANTIATE(0)

}  // namespace sfw

// FFT kernels of the grid sizes 32 to 40.
#include "grid_fft.cuh"

namespace eacg {
template struct GridFft<32>;
template struct GridFft<36>;
template struct GridFft<40>;
}  // namespace eacg

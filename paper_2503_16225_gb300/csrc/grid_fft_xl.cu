// FFT kernels of the grid sizes 80 and 96.
#include "grid_fft.cuh"

namespace eacg {
template struct GridFft<80, 0>;
template struct GridFft<96, 0>;
}  // namespace eacg

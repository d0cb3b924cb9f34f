// FFT kernels of the grid sizes 64 and 72 (both line plans).
#include "grid_fft.cuh"

namespace eacg {
template struct GridFft<64, 0>;
template struct GridFft<64, 1>;
template struct GridFft<72, 0>;
template struct GridFft<72, 1>;
}  // namespace eacg

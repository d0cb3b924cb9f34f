// FFT kernels of the grid sizes 64 and 72.
#include "grid_fft.cuh"

namespace eacg {
template struct GridFft<64>;
template struct GridFft<72>;
}  // namespace eacg

// FFT kernels of the grid sizes 32 to 40.
#include "grid_fft.cuh"

namespace eacg {
template struct GridFft<32, 0>;
template struct GridFft<32, 1>;
template struct GridFft<36, 0>;
template struct GridFft<36, 1>;
template struct GridFft<40, 0>;
}  // namespace eacg

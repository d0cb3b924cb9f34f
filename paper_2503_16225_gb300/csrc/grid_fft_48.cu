// FFT kernels of the grid size 48 (both line plans).
#include "grid_fft.cuh"

namespace eacg {
template struct GridFft<48, 0>;
template struct GridFft<48, 1>;
}  // namespace eacg

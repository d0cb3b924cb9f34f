// FFT kernels of the grid size 48.
#include "grid_fft.cuh"

namespace eacg {
template struct GridFft<48>;
}  // namespace eacg

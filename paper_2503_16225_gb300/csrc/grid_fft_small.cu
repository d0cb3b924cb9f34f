// FFT kernels of the grid sizes 8 to 24 (one instantiation unit per group of sizes keeps
// the parallel build short).
#include "grid_fft.cuh"

namespace eacg {
template struct GridFft<8, 0>;
template struct GridFft<12, 0>;
template struct GridFft<16, 0>;
template struct GridFft<16, 1>;
template struct GridFft<20, 0>;
template struct GridFft<24, 0>;
}  // namespace eacg

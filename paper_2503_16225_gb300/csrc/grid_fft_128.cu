// FFT kernels of the grid size 128 (FP32 transforms; the FP64-accurate plane kernels stop at 96).
#include "grid_fft.cuh"

namespace eacg {
template struct GridFft<128, 0>;
}  // namespace eacg

// Strided (y, z) FFT kernels and launchers instantiated for float.
#include "mx_fft_launch.cuh"

namespace mx {
template cudaError_t launch_strided<float>(int, int, cx<float>*, long, long, const twv<float>*, int, cudaStream_t, unsigned*,
                                           bool);
}  // namespace mx

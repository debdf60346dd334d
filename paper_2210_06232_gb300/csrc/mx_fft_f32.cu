// x-direction FFT kernels and launchers instantiated for float.
#include "mx_fft_launch.cuh"

namespace mx {
template cudaError_t launch_x_r2c<float>(int, const float*, const float*, cx<float>*, long, long, const twv<float>*, int, cudaStream_t, unsigned*);
template cudaError_t launch_x_c2r<float>(int, const cx<float>*, float*, float*, long, long, const twv<float>*, double, int, cudaStream_t, unsigned*);
}  // namespace mx

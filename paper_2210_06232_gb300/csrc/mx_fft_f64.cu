// FFT kernels and launchers instantiated for double.
#include "mx_fft_launch.cuh"

namespace mx {
template cudaError_t launch_x_r2c<double>(int, const double*, const double*, cx<double>*, long, long, const twv<double>*, int, cudaStream_t, unsigned*);
template cudaError_t launch_x_c2r<double>(int, const cx<double>*, double*, double*, long, long, const twv<double>*, double, int, cudaStream_t, unsigned*);
template cudaError_t launch_strided<double>(int, int, cx<double>*, long, long, const twv<double>*, int, cudaStream_t, unsigned*,
                                            bool);
}  // namespace mx

// Launchers of the fused z pass of the literal form (see k_z_fused).
#include "mx_fft_launch.cuh"

namespace mx {

// Registers per thread hold 6 x E complex values: E = 8 (FP32) / 4 (FP64)
// for powers of two, 6 (FP32) for 3 * 2^a.  Other lengths run unfused.
template <typename T> constexpr int zf_E(int n) {
  return (n & (n - 1)) == 0 ? (n < (sizeof(T) == 4 ? 8 : 4) ? n : (sizeof(T) == 4 ? 8 : 4))
         : (sizeof(T) == 4 && n % 3 == 0 && (n / 3) % 2 == 0) ? 6
                                                                : 0;
}
// Columns per block: ~256 threads per block (measured faster at 512^3 than
// 128-thread blocks, although only one ~250-register block fits per SM).
template <typename T> constexpr int zf_TX(int n) {
  return clampi(256 / (n / (zf_E<T>(n) ? zf_E<T>(n) : 1)), 2, 32);
}

#define MX_ZF_LENS(X) X(2) X(4) X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(6) X(12) X(24) X(48) X(96) X(192) X(384)

template <typename T, int N, typename CoefT>
static cudaError_t zf_n(cx<T>* data, const GridParams& g, const void* tab, double t, const twv<T>* tw, int grid,
                        double* partials, unsigned* counter, double* record, cudaStream_t s) {
  constexpr int E = zf_E<T>(N);
  if constexpr (E == 0) {
    return cudaErrorInvalidValue;
  } else {
    constexpr int TX = zf_TX<T>(N), P = N / E;
    static_assert(plan_ok(N, E), "plan");
    const size_t smem = sizeof(twv<T>) * N + sizeof(cx<T>) * N * (TX + 1);
    const CoefT* tb = reinterpret_cast<const CoefT*>(tab);
    cudaError_t err;
    if (record) {
      auto k = k_z_fused<T, N, E, TX, CoefT, true>;
      if ((err = set_smem(k, smem)) != cudaSuccess) return err;
      k<<<grid, P * TX, smem, s>>>(data, g, tb, t, tw, partials, counter, record);
    } else {
      auto k = k_z_fused<T, N, E, TX, CoefT, false>;
      if ((err = set_smem(k, smem)) != cudaSuccess) return err;
      k<<<grid, P * TX, smem, s>>>(data, g, tb, t, tw, partials, counter, record);
    }
    return cudaGetLastError();
  }
}

bool zfused_supported(int nz, bool fp64) { return fp64 ? zf_E<double>(nz) > 0 : zf_E<float>(nz) > 0; }
int fft_line_E(int n) { return fft_E(n); }
int zfused_line_E(int n, bool fp64) { return fp64 ? zf_E<double>(n) : zf_E<float>(n); }

template <typename T, typename CoefT>
static cudaError_t zf_dispatch(cx<T>* data, const GridParams& g, const void* tab, double t, const twv<T>* tw, int grid,
                               double* partials, unsigned* counter, double* record, cudaStream_t s) {
  switch (g.nz) {
#define X(n) case n: return zf_n<T, n, CoefT>(data, g, tab, t, tw, grid, partials, counter, record, s);
    MX_ZF_LENS(X)
#undef X
  }
  return cudaErrorInvalidValue;
}

template <>
cudaError_t launch_z_fused<float>(int coef_kind, float2* data, const GridParams& g, const void* tab, double t,
                                  const float4* tw, int grid, double* partials, unsigned* counter, double* record,
                                  cudaStream_t s) {
  if (coef_kind == 1) return zf_dispatch<float, CoefHL>(data, g, tab, t, tw, grid, partials, counter, record, s);
  if (coef_kind == 3) return zf_dispatch<float, CoefHL>(data, g, nullptr, t, tw, grid, partials, counter, record, s);
  return cudaErrorInvalidValue;
}

template <>
cudaError_t launch_z_fused<double>(int coef_kind, double2* data, const GridParams& g, const void* tab, double t,
                                   const double2* tw, int grid, double* partials, unsigned* counter, double* record,
                                   cudaStream_t s) {
  if (coef_kind == 0) return zf_dispatch<double, Coef<double>>(data, g, tab, t, tw, grid, partials, counter, record, s);
  if (coef_kind == 2) return zf_dispatch<double, Coef<double>>(data, g, nullptr, t, tw, grid, partials, counter, record, s);
  return cudaErrorInvalidValue;
}

}  // namespace mx

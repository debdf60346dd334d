// Dispatch of the fused z pass of the literal form over line lengths (see
// k_z_fused); the per-length launches are compiled in mx_zfused_*.cu.
#include "mx_zfused.cuh"

namespace mx {

#define X(n) extern template MX_ZF_SIG(float, n, CoefHL);
MX_ZF_LENS(X)
#undef X
#define X(n) extern template MX_ZF_SIG(double, n, Coef<double>);
MX_ZF_LENS(X)
#undef X

bool zfused_supported(int nz, bool fp64) { return fp64 ? zf_E<double>(nz) > 0 : zf_E<float>(nz) > 0; }
int fft_line_E(int n) { return fft_E(n); }
int zfused_line_E(int n, bool fp64) { return fp64 ? zf_E<double>(n) : zf_E<float>(n); }
int zfused_tile_cols(int n, bool fp64) { return fp64 ? zf_TX<double>(n) : zf_TX<float>(n); }

template <typename T, typename CoefT>
static cudaError_t zf_dispatch(cx<T>* data, const GridParams& g, const void* tab, double t, const twv<T>* tw, int grid,
                               bool pipelined, double* partials, unsigned* counter, double* record, cudaStream_t s) {
  switch (g.nz) {
#define X(n) case n: return zf_n<T, n, CoefT>(data, g, tab, t, tw, grid, pipelined, partials, counter, record, s);
    MX_ZF_LENS(X)
#undef X
  }
  return cudaErrorInvalidValue;
}

template <>
cudaError_t launch_z_fused<float>(int coef_kind, float2* data, const GridParams& g, const void* tab, double t,
                                  const float4* tw, int grid, bool pipelined, double* partials, unsigned* counter, double* record,
                                  cudaStream_t s) {
  if (coef_kind == 1) return zf_dispatch<float, CoefHL>(data, g, tab, t, tw, grid, pipelined, partials, counter, record, s);
  if (coef_kind == 3) return zf_dispatch<float, CoefHL>(data, g, nullptr, t, tw, grid, pipelined, partials, counter, record, s);
  return cudaErrorInvalidValue;
}

template <>
cudaError_t launch_z_fused<double>(int coef_kind, double2* data, const GridParams& g, const void* tab, double t,
                                   const dd2* tw, int grid, bool pipelined, double* partials, unsigned* counter, double* record,
                                   cudaStream_t s) {
  if (coef_kind == 0) return zf_dispatch<double, Coef<double>>(data, g, tab, t, tw, grid, pipelined, partials, counter, record, s);
  if (coef_kind == 2) return zf_dispatch<double, Coef<double>>(data, g, nullptr, t, tw, grid, pipelined, partials, counter, record, s);
  return cudaErrorInvalidValue;
}

}  // namespace mx

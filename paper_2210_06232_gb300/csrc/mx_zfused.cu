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
// Columns per block: ~256 threads per block (one ~250-register block per SM).
template <typename T> constexpr int zf_TX(int n) {
  return clampi(256 / (n / (zf_E<T>(n) ? zf_E<T>(n) : 1)), 2, 32);
}

#define MX_ZF_LENS(X) X(2) X(4) X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(6) X(12) X(24) X(48) X(96) X(192) X(384)

// Tensor map of the spectrum as [6][nz][ny][2 Mx] scalars, box [6][ZC][1][2 TX].
template <typename T, int N, int E, int TX>
static bool z_tensor_map(CUtensorMap* m, const void* data, const GridParams& g) {
  using ZT = ZTile<T, N, E, TX>;
  const cuuint64_t dim[4] = {(cuuint64_t)2 * g.mx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, 6};
  const cuuint32_t box[4] = {(cuuint32_t)(2 * TX), 1, (cuuint32_t)ZT::ZC, 6};
  return tensor_map(m, (int)sizeof(T), 4, data, dim, box);
}

template <typename T, int N, typename CoefT>
static cudaError_t zf_n(cx<T>* data, const GridParams& g, const void* tab, double t, const twv<T>* tw, int grid,
                        bool pipelined, double* partials, unsigned* counter, double* record, cudaStream_t s) {
  constexpr int E = zf_E<T>(N);
  if constexpr (E == 0) {
    return cudaErrorInvalidValue;
  } else {
    constexpr int TX = zf_TX<T>(N), P = N / E;
    using ZT = ZTile<T, N, E, TX>;
    static_assert(plan_ok(N, E), "plan");
    static_assert(ZT::stage_bytes % (128 * ZT::NZC) == 0, "tensor-copy boxes start on 128-byte boundaries");
    const CoefT* tb = reinterpret_cast<const CoefT*>(tab);
    cudaError_t err;
    // with the tensor-copy prefetch when the stage fits beside the exchange buffers
    constexpr size_t smem_tma = 2 * ZT::stage_bytes + ZT::tw_bytes + ZT::exch_bytes + 16;
    if constexpr (smem_tma + ZT::static_bytes <= 232448) {  // shared memory of a block on sm_103a
      CUtensorMap m;
      if (pipelined && counter && z_tensor_map<T, N, E, TX>(&m, data, g)) {
        if (record) {
          auto k = k_z_fused_tma<T, N, E, TX, CoefT, true>;
          if ((err = set_smem(k, smem_tma)) != cudaSuccess) return err;
          k<<<grid, P * TX, smem_tma, s>>>(data, g, tb, t, tw, partials, counter, record, m);
        } else {
          auto k = k_z_fused_tma<T, N, E, TX, CoefT, false>;
          if ((err = set_smem(k, smem_tma)) != cudaSuccess) return err;
          k<<<grid, P * TX, smem_tma, s>>>(data, g, tb, t, tw, partials, counter, record, m);
        }
        return cudaGetLastError();
      }
    }
    const size_t smem = ZT::tw_bytes + ZT::exch_bytes + 16;
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
                                   const double2* tw, int grid, bool pipelined, double* partials, unsigned* counter, double* record,
                                   cudaStream_t s) {
  if (coef_kind == 0) return zf_dispatch<double, Coef<double>>(data, g, tab, t, tw, grid, pipelined, partials, counter, record, s);
  if (coef_kind == 2) return zf_dispatch<double, Coef<double>>(data, g, nullptr, t, tw, grid, pipelined, partials, counter, record, s);
  return cudaErrorInvalidValue;
}

}  // namespace mx

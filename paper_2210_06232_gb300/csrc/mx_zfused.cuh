// Launch of the fused z pass of the literal form for one line length (see
// k_z_fused); instantiated per precision and length in mx_zfused_*.cu so that
// the large kernels compile in parallel.
#pragma once
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

// Tensor map of the spectrum as [6][nz][ny][2 Mx] scalars, box [3][ZC][1][2 TX].
template <typename T, int N, int E, int TX>
static bool z_tensor_map(CUtensorMap* m, const void* data, const GridParams& g) {
  using ZT = ZTile<T, N, E, TX>;
  const cuuint64_t dim[4] = {(cuuint64_t)2 * g.mx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, 6};
  const cuuint32_t box[4] = {(cuuint32_t)(2 * TX), 1, (cuuint32_t)ZT::ZC, 3};
  return tensor_map(m, (int)sizeof(T), 4, data, dim, box);
}

template <typename T, int N, typename CoefT>
cudaError_t zf_n(cx<T>* data, const GridParams& g, const void* tab, double t, const twv<T>* tw, int grid,
                        bool pipelined, double* partials, unsigned* counter, double* record, cudaStream_t s) {
  constexpr int E = zf_E<T>(N);
  if constexpr (E == 0) {
    return cudaErrorInvalidValue;
  } else {
    constexpr int TX = zf_TX<T>(N), P = N / E;
    using ZT = ZTile<T, N, E, TX>;
    static_assert(plan_ok(N, E), "plan");
    static_assert(ZT::stage_bytes % (128 * ZT::NB) == 0, "tensor-copy boxes start on 128-byte boundaries");
    const CoefT* tb = reinterpret_cast<const CoefT*>(tab);
    cudaError_t err;
    // with the tensor-copy prefetch when the stage fits beside the exchange buffers
    constexpr size_t smem_tma = ZT::smem_tma;
    if constexpr (smem_tma + ZT::static_bytes <= 232448) {  // shared memory of a block on sm_103a
      CUtensorMap m;
      if (pipelined && counter && z_tensor_map<T, N, E, TX>(&m, data, g)) {
        // one instantiation per coefficient source (a table, or FP64 per point), with or without invariants
        auto k = record ? (tb ? k_z_fused_tma<T, N, E, TX, CoefT, true, false> : k_z_fused_tma<T, N, E, TX, CoefT, true, true>)
                        : (tb ? k_z_fused_tma<T, N, E, TX, CoefT, false, false>
                              : k_z_fused_tma<T, N, E, TX, CoefT, false, true>);
        if ((err = set_smem(k, smem_tma)) != cudaSuccess) return err;
        k<<<grid, P * TX, smem_tma, s>>>(data, g, tb, t, tw, partials, counter, record, m);
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

// Explicit instantiations (and their extern declarations) of zf_n for one length.
#define MX_ZF_SIG(T, N, CoefT)                                                                                     \
  cudaError_t zf_n<T, N, CoefT>(cx<T>*, const GridParams&, const void*, double, const twv<T>*, int, bool, double*, \
                                unsigned*, double*, cudaStream_t)

}  // namespace mx

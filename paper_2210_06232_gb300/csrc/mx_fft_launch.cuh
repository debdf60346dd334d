// Launcher bodies for the FFT kernels, instantiated per precision in
// mx_fft_f32.cu and mx_fft_f64.cu.
#pragma once
#include "mx_launch.h"
#include "mx_strided_tma.cuh"
#include "mx_tmap.h"
#include "mx_xpass_tma.cuh"

namespace mx {

// Registers per thread per line: E complex values.
constexpr int fft_E(int n) {
  return (n & (n - 1)) == 0 ? (n <= 8 ? n : 8)
         : (n % 3 == 0)     ? (n == 3 ? 3 : (n == 6 ? 6 : 12))
                            : (n == 5 ? 5 : (n == 10 ? 10 : 20));
}
constexpr int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }
// Lines per block: ~256 threads per block.
constexpr int fft_TY(int n) { return clampi(256 / (n / fft_E(n)), 1, 256); }
constexpr int fft_TX(int n) { return clampi(256 / (n / fft_E(n)), 8, 64); }

#define MX_FOR_EACH_LEN(X) \
  X(1) X(2) X(4) X(8) X(16) X(32) X(64) X(128) X(256) X(512) \
  X(3) X(6) X(12) X(24) X(48) X(96) X(192) X(384) \
  X(5) X(10) X(20) X(40) X(80) X(160) X(320)

// Dynamic shared memory of a launch; set every time (static shared memory of the
// kernel adds to it, so the 48 KB default can be exceeded below 48 KB dynamic).
template <typename K> static cudaError_t set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Grid of a persistent FFT launch: `bps` blocks per SM (0 = one block per work item).
static long persistent_grid(long items, int bps) {
  if (bps <= 0) return items;
  const long cap = (long)num_sms() * bps;
  return items < cap ? items : cap;
}

// Bulk-copy pipelined x passes: rows of at least 32 complex values, groups of
// 2 TY rows that never straddle the E/H boundary, 16-byte aligned buffers.
template <typename T, int M>
static bool xp_tma_ok(const void* a, const void* b, long rows3) {
  constexpr int TY = fft_TY(M);
  return M >= 32 && rows3 % (2 * TY) == 0 && ((((uintptr_t)a) | ((uintptr_t)b)) & 15u) == 0;
}

template <typename T, int M>
static cudaError_t x_r2c_n(const T* e, const T* h, cx<T>* out, long rows3, long nrows, const twv<T>* tw, int bps,
                           cudaStream_t s, unsigned* counter) {
  constexpr int E = fft_E(M), TY = fft_TY(M), P = M / E;
  static_assert(plan_ok(M, E), "plan");
  if constexpr (M >= 32 && xp_fits<T, M, TY>()) {
    if (counter && xp_tma_ok<T, M>(e, h, rows3)) {
      const size_t smem = xp_smem<T, M, TY>();
      auto k = k_x_r2c_tma<T, M, E, TY>;
      cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (err != cudaSuccess) return err;
      const long blocks = persistent_grid((nrows + 2 * TY - 1) / (2 * TY), bps > 0 ? bps : 2);
      k<<<(unsigned)blocks, P * TY + 32, smem, s>>>(e, h, out, rows3, nrows, tw, counter);
      return cudaGetLastError();
    }
  }
  const size_t smem = sizeof(twv<T>) * 2 * M + sizeof(cx<T>) * TY * line_buf(M);
  auto k = k_x_r2c<T, M, E, TY>;
  cudaError_t err = set_smem(k, smem);
  if (err != cudaSuccess) return err;
  const long blocks = persistent_grid((nrows + TY - 1) / TY, bps);
  k<<<(unsigned)blocks, P * TY, smem, s>>>(e, h, out, rows3, nrows, tw);
  return cudaGetLastError();
}

template <typename T, int M>
static cudaError_t x_c2r_n(const cx<T>* in, T* e, T* h, long rows3, long nrows, const twv<T>* tw, double scale,
                           int bps, cudaStream_t s, unsigned* counter) {
  constexpr int E = fft_E(M), TY = fft_TY(M), P = M / E;
  if constexpr (M >= 32 && xp_fits<T, M, TY>()) {
    if (counter && xp_tma_ok<T, M>(in, in, rows3)) {
      const size_t smem = xp_smem<T, M, TY>();
      auto k = k_x_c2r_tma<T, M, E, TY>;
      cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (err != cudaSuccess) return err;
      const long blocks = persistent_grid((nrows + 2 * TY - 1) / (2 * TY), bps > 0 ? bps : 2);
      k<<<(unsigned)blocks, P * TY + 32, smem, s>>>(in, e, h, rows3, nrows, tw, scale, counter);
      return cudaGetLastError();
    }
  }
  const size_t smem = sizeof(twv<T>) * 2 * M + sizeof(cx<T>) * TY * line_buf(M);
  auto k = k_x_c2r<T, M, E, TY>;
  cudaError_t err = set_smem(k, smem);
  if (err != cudaSuccess) return err;
  const long blocks = persistent_grid((nrows + TY - 1) / TY, bps);
  k<<<(unsigned)blocks, P * TY, smem, s>>>(in, e, h, rows3, nrows, tw, scale);
  return cudaGetLastError();
}

template <typename T, int N, int DIR>
static cudaError_t strided_n(cx<T>* data, long inner, long outer, const twv<T>* tw, int bps, cudaStream_t s,
                             unsigned* counter, bool dbuf) {
  constexpr int E = fft_E(N), TX = fft_TX(N), P = N / E;
  static_assert(plan_ok(N, E), "plan");
  const long tiles = (inner + TX - 1) / TX * outer;
  if (tiles > 0x7fffffffL) return cudaErrorInvalidConfiguration;  // the kernels count tiles in 32 bits
  using ST = STile<T, N, E, TX>;
  if constexpr (ST::smem <= 232448) {  // shared memory of a block on sm_103a
    // tensor-copy loads and stores of [outer][N][inner] complex as scalars
    CUtensorMap m;
    const cuuint64_t dim[3] = {(cuuint64_t)(2 * inner), (cuuint64_t)N, (cuuint64_t)outer};
    const cuuint32_t box[3] = {(cuuint32_t)(2 * TX), (cuuint32_t)ST::ZC, 1};
    if (counter && tensor_map(&m, (int)sizeof(T), 3, data, dim, box)) {
      if constexpr (N % 16 == 0 && STile2<T, N, E, TX>::smem <= 232448) {
        if (dbuf) {
          auto k = k_fft_strided_tma2<T, N, E, TX, DIR>;
          constexpr size_t smem2 = STile2<T, N, E, TX>::smem;
          cudaError_t err = set_smem(k, smem2);
          if (err != cudaSuccess) return err;
          const long blocks = persistent_grid(tiles, bps > 0 ? bps : 1);
          k<<<(unsigned)blocks, P * TX, smem2, s>>>(inner, outer, tw, counter, m);
          return cudaGetLastError();
        }
      }
      auto k = k_fft_strided_tma<T, N, E, TX, DIR>;
      cudaError_t err = set_smem(k, ST::smem);
      if (err != cudaSuccess) return err;
      const long blocks = persistent_grid(tiles, bps > 0 ? bps : 1);
      k<<<(unsigned)blocks, P * TX, ST::smem, s>>>(inner, outer, tw, counter, m);
      return cudaGetLastError();
    }
  }
  const size_t smem = sizeof(twv<T>) * N + sizeof(cx<T>) * strided_rows(N) * TX;
  auto k = k_fft_strided<T, N, E, TX, DIR>;
  cudaError_t err = set_smem(k, smem);
  if (err != cudaSuccess) return err;
  const long blocks = persistent_grid(tiles, bps);
  k<<<(unsigned)blocks, P * TX, smem, s>>>(data, inner, outer, tw);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_x_r2c(int M, const T* e, const T* h, cx<T>* out, long rows3, long nrows, const twv<T>* tw, int bps,
                         cudaStream_t s, unsigned* counter) {
  if (nrows <= 0) return cudaSuccess;
  switch (M) {
#define X(n) case n: return x_r2c_n<T, n>(e, h, out, rows3, nrows, tw, bps, s, counter);
    MX_FOR_EACH_LEN(X)
#undef X
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_x_c2r(int M, const cx<T>* in, T* e, T* h, long rows3, long nrows, const twv<T>* tw, double scale,
                         int bps, cudaStream_t s, unsigned* counter) {
  if (nrows <= 0) return cudaSuccess;
  switch (M) {
#define X(n) case n: return x_c2r_n<T, n>(in, e, h, rows3, nrows, tw, scale, bps, s, counter);
    MX_FOR_EACH_LEN(X)
#undef X
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_strided(int N, int dir, cx<T>* data, long inner, long outer, const twv<T>* tw, int bps,
                           cudaStream_t s, unsigned* counter, bool dbuf) {
  if (inner <= 0 || outer <= 0 || N == 1) return cudaSuccess;
  if (dir < 0) {
    switch (N) {
#define X(n) case n: return strided_n<T, n, -1>(data, inner, outer, tw, bps, s, counter, dbuf);
      MX_FOR_EACH_LEN(X)
#undef X
    }
  } else {
    switch (N) {
#define X(n) case n: return strided_n<T, n, +1>(data, inner, outer, tw, bps, s, counter, dbuf);
      MX_FOR_EACH_LEN(X)
#undef X
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace mx

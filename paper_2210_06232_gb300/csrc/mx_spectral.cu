// Spectral pass (per-k exponential update and invariant sums) and the
// coefficient-table kernel, instantiated for float and double.
#include "mx_launch.h"
#include "mx_spectral_tma.cuh"

namespace mx {

int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      n = v;
    else
      return 152;
  }
  return n;
}

int spectral_blocks(long npts) {
  // persistent-style grid: at most 2 blocks of 256 threads per SM of a 152-SM GB300
  long b = (npts + 511) / 512;
  const long cap = 152L * 2L;
  return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

template <typename T, typename CoefT, bool TABLE, int V>
static cudaError_t spectral_v(int mode, const cx<T>* src, cx<T>* dst, long npts, const GridParams& g, const void* tab,
                              double t, int blocks, double* partials, unsigned* counter, double* record, cudaStream_t s) {
  const CoefT* tb = reinterpret_cast<const CoefT*>(tab);
  switch (mode) {
    case 0:
      k_spectral<T, CoefT, TABLE, false, true, V><<<blocks, 256, 0, s>>>(src, dst, npts, g, tb, t, partials, counter, record);
      break;
    case 1:
      k_spectral<T, CoefT, TABLE, true, false, V><<<blocks, 256, 0, s>>>(src, dst, npts, g, tb, t, partials, counter, record);
      break;
    case 2:
      k_spectral<T, CoefT, TABLE, true, true, V><<<blocks, 256, 0, s>>>(src, dst, npts, g, tb, t, partials, counter, record);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T, typename CoefT, bool TABLE>
static cudaError_t spectral_mode(int mode, const cx<T>* src, cx<T>* dst, long npts, const GridParams& g, const void* tab,
                                 double t, int blocks, double* partials, unsigned* counter, double* record, cudaStream_t s) {
  if (npts >= (1L << 31)) return cudaErrorInvalidValue;
  // two points per thread when rows have even length (keeps both in one row, 16-byte aligned)
  if (sizeof(T) == 4 && g.mx % 2 == 0)
    return spectral_v<T, CoefT, TABLE, 2>(mode, src, dst, npts, g, tab, t, blocks, partials, counter, record, s);
  return spectral_v<T, CoefT, TABLE, 1>(mode, src, dst, npts, g, tab, t, blocks, partials, counter, record, s);
}

template <bool UPDATE, bool INV>
static cudaError_t tma_mode(const float2* src, float2* dst, long npts, const GridParams& g, const void* tab, int blocks,
                            double* partials, unsigned* counter, double* record, cudaStream_t s) {
  auto k = k_spectral_tma<UPDATE, INV>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma_smem_bytes());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k<<<blocks, TMA_THREADS, tma_smem_bytes(), s>>>(src, dst, npts, g, (const Coef<float>*)tab, partials, counter, record);
  return cudaGetLastError();
}

// Grouped rows (k_spectral_grp): even ny and nz, so that rows y and -y (z and -z) share |k|^2;
// Mx a multiple of GRP_L.
template <bool INV>
static cudaError_t grp_mode(const float2* src, float2* dst, long npts, const GridParams& g, const void* tab, int blocks,
                            double* partials, unsigned* counter, double* record, cudaStream_t s) {
  auto k = k_spectral_grp<INV>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma_smem_bytes());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k<<<blocks, TMA_THREADS, tma_smem_bytes(), s>>>(src, dst, npts, g, (const Coef<float>*)tab, partials, counter, record);
  return cudaGetLastError();
}

template <>
cudaError_t launch_spectral<float>(int mode, int coef_kind, const float2* src, float2* dst, long npts, const GridParams& g,
                                   const void* tab, double t, int blocks, double* partials, unsigned* counter,
                                   double* record, cudaStream_t s) {
  // bulk-copy pipeline: table coefficients, even rows, 16-byte aligned buffers
  const bool aligned = (((uintptr_t)src | (uintptr_t)dst) & 15u) == 0;
  if (coef_kind == 0 && g.mx % 2 == 0 && aligned && npts < (1L << 31) && npts >= TMA_CH) {
    // the updating modes take the table entries once per group of rows that share them (rows of
    // whole segments, so that no consumer idles)
    if (g.ny % 2 == 0 && g.nz % 2 == 0 && g.mx % GRP_L == 0) {
      if (mode == 1) return grp_mode<false>(src, dst, npts, g, tab, blocks, partials, counter, record, s);
      if (mode == 2) return grp_mode<true>(src, dst, npts, g, tab, blocks, partials, counter, record, s);
    }
    switch (mode) {
      case 0: return tma_mode<false, true>(src, dst, npts, g, tab, blocks, partials, counter, record, s);
      case 1: return tma_mode<true, false>(src, dst, npts, g, tab, blocks, partials, counter, record, s);
      case 2: return tma_mode<true, true>(src, dst, npts, g, tab, blocks, partials, counter, record, s);
    }
  }
  switch (coef_kind) {
    case 0: return spectral_mode<float, Coef<float>, true>(mode, src, dst, npts, g, tab, t, blocks, partials, counter, record, s);
    case 1: return spectral_mode<float, CoefHL, true>(mode, src, dst, npts, g, tab, t, blocks, partials, counter, record, s);
    case 2: return spectral_mode<float, Coef<float>, false>(mode, src, dst, npts, g, tab, t, blocks, partials, counter, record, s);
    case 3: return spectral_mode<float, CoefHL, false>(mode, src, dst, npts, g, tab, t, blocks, partials, counter, record, s);
  }
  return cudaErrorInvalidValue;
}

template <>
cudaError_t launch_spectral<double>(int mode, int coef_kind, const double2* src, double2* dst, long npts,
                                    const GridParams& g, const void* tab, double t, int blocks, double* partials,
                                    unsigned* counter, double* record, cudaStream_t s) {
  switch (coef_kind) {
    case 0: return spectral_mode<double, Coef<double>, true>(mode, src, dst, npts, g, tab, t, blocks, partials, counter, record, s);
    case 2: return spectral_mode<double, Coef<double>, false>(mode, src, dst, npts, g, tab, t, blocks, partials, counter, record, s);
  }
  return cudaErrorInvalidValue;
}

template <>
cudaError_t launch_coef_table<float>(int coef_kind, void* tab, int nq, const GridParams& g, double t, cudaStream_t s) {
  const int blocks = (nq + 255) / 256;
  if (nq <= 0) return cudaSuccess;
  if (coef_kind == 0) k_coef_table<float, Coef<float>><<<blocks, 256, 0, s>>>((Coef<float>*)tab, nq, g, t);
  else if (coef_kind == 1) k_coef_table<float, CoefHL><<<blocks, 256, 0, s>>>((CoefHL*)tab, nq, g, t);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <>
cudaError_t launch_coef_table<double>(int coef_kind, void* tab, int nq, const GridParams& g, double t, cudaStream_t s) {
  const int blocks = (nq + 255) / 256;
  if (nq <= 0) return cudaSuccess;
  if (coef_kind != 0) return cudaErrorInvalidValue;
  k_coef_table<double, Coef<double>><<<blocks, 256, 0, s>>>((Coef<double>*)tab, nq, g, t);
  return cudaGetLastError();
}

}  // namespace mx

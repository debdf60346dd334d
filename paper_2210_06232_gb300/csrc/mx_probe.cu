// Arithmetic peak probe: FMA throughput of the FP32 and FP64 pipes of the current device,
// measured with CUDA events, for the ALU rooflines that the benchmark reports beside the HBM
// ones (the FP64 forms are bound by the FP64 pipe, not by memory).
#include "../../include/maxexp.h"
#include "mx_launch.h"

namespace {

constexpr int CHAINS = 8;   // independent FMA chains per thread
constexpr int ITERS = 4096;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T* __restrict__ out, T a, T b) {
  T v[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) v[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < ITERS; ++i) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) v[c] = fma(v[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += v[c];
  if (s == (T)12345.678) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

template <typename T>
mx_status measure(double* flops) {
  const int sms = mx::num_sms();
  const int blocks = sms * 8, threads = 256;
  T* out = nullptr;
  if (mx::dev_alloc((void**)&out, (size_t)blocks * threads * sizeof(T)) != cudaSuccess) return MX_E_NOMEM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  mx_status st = MX_OK;
  float best = 0.f;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    st = MX_E_CUDA;
  } else {
    // a and b keep the chains bounded (|a| < 1): no overflow, no denormals
    const T a = (T)0.999, b = (T)0.001;
    for (int rep = 0; rep < 6 && st == MX_OK; ++rep) {
      cudaEventRecord(e0, 0);
      k_fma_peak<T><<<blocks, threads>>>(out, a, b);
      cudaEventRecord(e1, 0);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        st = MX_E_CUDA;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && (best == 0.f || ms < best)) best = ms;  // the first launch is a warm-up
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (st != MX_OK) return st;
  *flops = 2.0 * (double)blocks * threads * CHAINS * ITERS / (best * 1e-3);
  return MX_OK;
}

}  // namespace

extern "C" mx_status mx_fma_peak(int precision, double* flops_per_s) {
  if (!flops_per_s || (precision != MX_FP64 && precision != MX_FP32)) return MX_E_INVAL;
  return precision == MX_FP64 ? measure<double>(flops_per_s) : measure<float>(flops_per_s);
}

// ---------------------------------------------------------------------------------------------
// Tensor-copy streaming of z-line tiles: the access pattern of the fused z pass without its
// arithmetic.  A spectrum [6][nz][ny][mx] complex FP32 is read tile by tile (cols columns x nz x
// comps components, rows of cols x 8 bytes at a stride of one z plane) into shared memory and
// written back in place by one persistent block per SM, the next tile's copy in flight while the
// current one is stored.  What HBM delivers for such rows bounds the fused pass from above.
#include "mx_tma.cuh"
#include "mx_tmap.h"

namespace {

template <int TX, int NC>
__global__ void __launch_bounds__(32, 1) k_tile_stream(const __grid_constant__ CUtensorMap tm, int mx, int ny, int nz,
                                                       int zc, unsigned* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char sm[];
  const int nzb = nz / zc;
  const uint32_t box_bytes = (uint32_t)NC * zc * TX * 8, stage_bytes = box_bytes * nzb;
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + 2 * (size_t)stage_bytes);
  if (threadIdx.x != 0) return;
  mx::mbar_init(full, 1);
  mx::mbar_init(full + 1, 1);
  mx::mbar_fence_init();
  const int ntx = mx / TX, ncg = 6 / NC;
  const unsigned ntiles = (unsigned)ntx * ny * ncg;  // column tiles fastest, then y, then component group
  auto coords = [&](unsigned tile, int& x0, int& y, int& cg) {
    const unsigned r = tile / ntx;
    x0 = (int)(tile - r * ntx) * TX;
    y = (int)(r % ny);
    cg = (int)(r / ny);
  };
  auto load = [&](unsigned tile, int s) {
    int x0, y, cg;
    coords(tile, x0, y, cg);
    mx::mbar_expect_tx(full + s, stage_bytes);
    for (int b = 0; b < nzb; ++b)
      mx::tma_load_4d(sm + s * (size_t)stage_bytes + b * (size_t)box_bytes, &tm, 2 * x0, y, b * zc, NC * cg, full + s);
  };
  auto store = [&](unsigned tile, int s) {
    int x0, y, cg;
    coords(tile, x0, y, cg);
    for (int b = 0; b < nzb; ++b)
      mx::tma_store_4d(&tm, sm + s * (size_t)stage_bytes + b * (size_t)box_bytes, 2 * x0, y, b * zc, NC * cg);
    mx::bulk_commit();
  };
  unsigned i = 0;
  if (blockIdx.x < ntiles) load(blockIdx.x, 0);
  for (unsigned tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
    const int s = (int)(i & 1u);
    const unsigned nxt = tile + gridDim.x;
    if (nxt < ntiles) {
      mx::bulk_wait_read_all();  // the store of the previous tile has read the other stage
      load(nxt, s ^ 1);
    }
    if (!mx::mbar_wait_bounded(full + s, (i >> 1) & 1u)) {
      atomicExch(err, 1u);
      if (nxt < ntiles) mx::mbar_wait_bounded(full + (s ^ 1), ((i + 1) >> 1) & 1u);  // let that copy land
      break;
    }
    mx::fence_proxy_async_smem();
    store(tile, s);
  }
  mx::bulk_wait_all();
}

template <int TX, int NC>
mx_status tile_stream(void* buf, int mx_, int ny, int nz, int reps, double* gbs) {
  const int nzc = (nz + 255) / 256;
  if (nz % nzc) return MX_E_INVAL;
  const int zc = nz / nzc;
  const size_t stage = (size_t)NC * nz * TX * 8, smem = 2 * stage + 16;
  if (smem > 232448) return MX_E_INVAL;
  CUtensorMap m;
  const cuuint64_t dim[4] = {(cuuint64_t)2 * mx_, (cuuint64_t)ny, (cuuint64_t)nz, 6};
  const cuuint32_t box[4] = {(cuuint32_t)(2 * TX), 1, (cuuint32_t)zc, (cuuint32_t)NC};
  if (!mx::tensor_map(&m, 4, 4, buf, dim, box)) return MX_E_INVAL;
  unsigned* err = nullptr;
  if (mx::dev_alloc((void**)&err, 4) != cudaSuccess) return MX_E_NOMEM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  mx_status st = MX_OK;
  float best = 0.f;
  auto k = k_tile_stream<TX, NC>;
  if (cudaMemset(err, 0, 4) != cudaSuccess || cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    st = MX_E_CUDA;
  } else {
    for (int rep = 0; rep <= reps && st == MX_OK; ++rep) {  // launch 0 is a warm-up
      cudaEventRecord(e0, 0);
      k<<<mx::num_sms(), 32, smem>>>(m, mx_, ny, nz, zc, err);
      cudaEventRecord(e1, 0);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        st = MX_E_CUDA;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    unsigned herr = 0;
    if (st == MX_OK && cudaMemcpy(&herr, err, 4, cudaMemcpyDeviceToHost) != cudaSuccess) st = MX_E_CUDA;
    if (st == MX_OK && herr) st = MX_E_TIMEOUT;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(err);
  if (st != MX_OK) return st;
  *gbs = 2.0 * 6 * (double)mx_ * ny * nz * 8 / (best * 1e-3) / 1e9;
  return MX_OK;
}

}  // namespace

extern "C" mx_status mx_tile_stream(void* buf, int mx_, int ny, int nz, int cols, int reps, double* gbs) {
  if (!buf || !gbs || reps < 1 || mx_ < 1 || ny < 1 || nz < 2 || nz > 512 || (((uintptr_t)buf) & 15u)) return MX_E_INVAL;
  if (cols != 4 && cols != 8 && cols != 16) return MX_E_INVAL;
  if (mx_ % cols || (2 * mx_ * 4) % 16) return MX_E_INVAL;
  if (cols == 4) return tile_stream<4, 6>(buf, mx_, ny, nz, reps, gbs);
  if (cols == 8) return tile_stream<8, 3>(buf, mx_, ny, nz, reps, gbs);
  return tile_stream<16, 1>(buf, mx_, ny, nz, reps, gbs);
}

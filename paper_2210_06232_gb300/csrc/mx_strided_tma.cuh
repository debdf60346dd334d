// Strided line FFT (y passes; z passes without a fused plan) with tensor-copy
// loads and stores, sm_103a.
//
// The data is viewed as [outer][N][inner] complex and transformed along the
// middle axis, TX consecutive inner columns per tile (as k_fft_strided).  A
// tile is brought into an input stage by the tensor-copy engine while the
// previous one is transformed in registers, and leaves through an output stage
// and a tensor store, so that each thread issues no global load or store of
// its own.  Waits on the stage's mbarrier are bounded: a wait that gives up
// sets counter[1] (read by the host as MX_E_TIMEOUT) and the block leaves the
// loop together.
#pragma once
#include "mx_kernels.cuh"

namespace mx {

template <typename T, int N, int E, int TX>
struct STile {
  static constexpr int P = N / E;
  static constexpr int NZC = (N + 255) / 256;  // boxes along the line
  static constexpr int ZC = N / NZC;           // line positions per box
  static constexpr size_t stage_bytes = (size_t)N * TX * sizeof(cx<T>);
  static constexpr size_t exch_bytes = (size_t)strided_rows(N) * TX * sizeof(cx<T>);
  static constexpr size_t tw_bytes = (size_t)N * sizeof(twv<T>);
  static constexpr size_t smem = 2 * stage_bytes + tw_bytes + exch_bytes + 16;
  // position z of column x in a stage: box z / ZC, laid out [z % ZC][x]
  __device__ __forceinline__ static int index(int z, int x) { return (z / ZC) * (ZC * TX) + (z % ZC) * TX + x; }
};

template <typename T, int N, int E, int TX, int DIR>
__global__ void __launch_bounds__((N / E) * TX) k_fft_strided_tma(long inner, long outer, const twv<T>* __restrict__ twg,
                                                                  unsigned* __restrict__ counter,
                                                                  const __grid_constant__ CUtensorMap tmap) {
  using C = cx<T>;
  using ST = STile<T, N, E, TX>;
  constexpr int P = N / E;
  static_assert(ST::stage_bytes % (128 * ST::NZC) == 0, "tensor-copy boxes start on 128-byte boundaries");
  extern __shared__ __align__(128) unsigned char ssmraw[];
  // [input stage][output stage][twiddles][exchange buffer][mbarrier]
  C* stage = reinterpret_cast<C*>(ssmraw);
  C* ostage = reinterpret_cast<C*>(ssmraw + ST::stage_bytes);
  twv<T>* tw = reinterpret_cast<twv<T>*>(ssmraw + 2 * ST::stage_bytes);
  C* sm = reinterpret_cast<C*>(reinterpret_cast<unsigned char*>(tw) + ST::tw_bytes);
  uint64_t* full = reinterpret_cast<uint64_t*>(reinterpret_cast<unsigned char*>(sm) + ST::exch_bytes);
  for (int i = threadIdx.x; i < tw_len(N, E); i += blockDim.x) tw[i] = twg[i];
  const int x = threadIdx.x % TX, t = threadIdx.x / TX;
  // tile indices fit in 32 bits (checked by the launcher)
  const unsigned ntile_in = (unsigned)((inner + TX - 1) / TX);
  const unsigned ntiles = ntile_in * (unsigned)outer;
  const void* tm = &tmap;
  auto load = [&](unsigned tile) {  // thread 0
    const unsigned o = tile / ntile_in;
    const int c0 = (int)(tile - o * ntile_in) * TX;
    mbar_expect_tx(full, (uint32_t)ST::stage_bytes);
#pragma unroll
    for (int h = 0; h < ST::NZC; ++h)
      tma_load_3d(reinterpret_cast<unsigned char*>(stage) + h * (ST::stage_bytes / ST::NZC), tm, 2 * c0, h * ST::ZC,
                  (int)o, full);
  };
  auto store = [&](unsigned tile) {  // thread 0
    const unsigned o = tile / ntile_in;
    const int c0 = (int)(tile - o * ntile_in) * TX;
#pragma unroll
    for (int h = 0; h < ST::NZC; ++h)
      tma_store_3d(tm, reinterpret_cast<const unsigned char*>(ostage) + h * (ST::stage_bytes / ST::NZC), 2 * c0,
                   h * ST::ZC, (int)o);
    bulk_commit();
  };
  if (threadIdx.x == 0) {
    mbar_init(full, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && blockIdx.x < ntiles) load(blockIdx.x);
  bool pending = blockIdx.x < ntiles;  // a copy into the stage is in flight (thread 0's view)
  unsigned it = 0;
  for (unsigned tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const bool lost = !mbar_wait_bounded(full, it & 1u);
    if (__syncthreads_or(lost)) {
      if (lost) atomicExch(counter + 1, 1u);
      break;
    }
    C v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = stage[ST::index(t + P * m, x)];
    fence_proxy_async_smem();
    __syncthreads();  // every read of the input stage is done (and the twiddles are in)
    pending = false;
    if (threadIdx.x == 0 && tile + gridDim.x < ntiles) {
      load(tile + gridDim.x);
      pending = true;
    }
    line_fft<T, N, E, DIR>(v, sm + x, TX, t, tw);
    if (threadIdx.x == 0) bulk_wait_read_all();  // the previous tile's store has read the output stage
    __syncthreads();
#pragma unroll
    for (int m = 0; m < E; ++m) ostage[ST::index(t + P * m, x)] = v[m];
    fence_proxy_async_smem();  // generic writes before the async-proxy reads of the store
    __syncthreads();
    if (threadIdx.x == 0) store(tile);  // columns past `inner` are dropped by the engine
  }
  if (threadIdx.x == 0) {
    // after a timed-out wait: let the copy this block issued land before its shared memory is released
    if (pending) mbar_wait_bounded(full, it & 1u);
    bulk_wait_all();
  }
}

}  // namespace mx

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

// Two input stages, each of which, once read, is also the exchange buffer of
// its tile's transform (rows swizzled instead of padded, swz_rows, so that the
// exchange fits the stage: N a multiple of 16), and an output stage: two tiles are in
// flight per block while one is transformed.  Stage s takes tiles it, it + 2,
// ... of the block's sequence; its mbarrier completes once per tile.
template <typename T, int N, int E, int TX>
struct STile2 {
  static constexpr int NZC = (N + 255) / 256;
  static constexpr int ZC = N / NZC;
  static constexpr size_t stage_bytes = (size_t)N * TX * sizeof(cx<T>);
  static constexpr size_t tw_bytes = (size_t)N * sizeof(twv<T>);
  static constexpr size_t smem = 3 * stage_bytes + tw_bytes + 32;
  __device__ __forceinline__ static int index(int z, int x) { return (z / ZC) * (ZC * TX) + (z % ZC) * TX + x; }
};

template <typename T, int N, int E, int TX, int DIR>
__global__ void __launch_bounds__((N / E) * TX) k_fft_strided_tma2(long inner, long outer, const twv<T>* __restrict__ twg,
                                                                   unsigned* __restrict__ counter,
                                                                   const __grid_constant__ CUtensorMap tmap) {
  using C = cx<T>;
  using ST = STile2<T, N, E, TX>;
  constexpr int P = N / E;
  static_assert(N % 16 == 0, "swizzled exchange rows stay within the stage");
  static_assert(ST::stage_bytes % (128 * ST::NZC) == 0, "tensor-copy boxes start on 128-byte boundaries");
  extern __shared__ __align__(128) unsigned char ssmraw[];
  // [input stage 0][input stage 1][output stage][twiddles][2 mbarriers]
  C* const in0 = reinterpret_cast<C*>(ssmraw);
  C* const ostage = in0 + 2 * N * TX;
  twv<T>* tw = reinterpret_cast<twv<T>*>(ostage + N * TX);
  uint64_t* full = reinterpret_cast<uint64_t*>(reinterpret_cast<unsigned char*>(tw) + ST::tw_bytes);
  for (int i = threadIdx.x; i < tw_len(N, E); i += blockDim.x) tw[i] = twg[i];
  const int x = threadIdx.x % TX, t = threadIdx.x / TX;
  const unsigned ntile_in = (unsigned)((inner + TX - 1) / TX);
  const unsigned ntiles = ntile_in * (unsigned)outer;
  const void* tm = &tmap;
  auto load = [&](unsigned tile, int s) {  // thread 0
    const unsigned o = tile / ntile_in;
    const int c0 = (int)(tile - o * ntile_in) * TX;
    unsigned char* dst = reinterpret_cast<unsigned char*>(in0 + s * N * TX);
    mbar_expect_tx(full + s, (uint32_t)ST::stage_bytes);
#pragma unroll
    for (int h = 0; h < ST::NZC; ++h)
      tma_load_3d(dst + h * (ST::stage_bytes / ST::NZC), tm, 2 * c0, h * ST::ZC, (int)o, full + s);
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
    mbar_init(full + 1, 1);
    mbar_fence_init();
  }
  __syncthreads();
  // parities of the copies issued into stage s (bit s) and of the waits completed on it (bit 2 + s),
  // thread 0's view: at most one copy per stage is outstanding, so a copy is in flight when the
  // two differ, and the wait parity of stage s is bit 2 + s
  unsigned book = 0u;
  if (threadIdx.x == 0) {
    if (blockIdx.x < ntiles) load(blockIdx.x, 0), book ^= 1u;
    if (blockIdx.x + gridDim.x < ntiles) load(blockIdx.x + gridDim.x, 1), book ^= 2u;
  }
  unsigned it = 0;
  for (unsigned tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int s = (int)(it & 1u);
    C* const st = in0 + s * N * TX;
    const bool lost = !mbar_wait_bounded(full + s, (it >> 1) & 1u);
    if (__syncthreads_or(lost)) {
      if (lost) atomicExch(counter + 1, 1u);
      break;
    }
    book ^= 4u << s;
    C v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = st[ST::index(t + P * m, x)];
    // the transform's first exchange waits for every read of the stage above
    line_fft<T, N, E, DIR>(v, st + x, swz_rows(TX, 1), t, tw);
    if (threadIdx.x == 0) bulk_wait_read_all();  // the previous tile's store has read the output stage
    __syncthreads();                              // and every exchange read of this stage is done
#pragma unroll
    for (int m = 0; m < E; ++m) ostage[ST::index(t + P * m, x)] = v[m];
    fence_proxy_async_smem();  // generic accesses (output and input stages) before the async proxy's
    __syncthreads();
    if (threadIdx.x == 0) {
      store(tile);  // columns past `inner` are dropped by the engine
      if (tile + 2 * gridDim.x < ntiles) load(tile + 2 * gridDim.x, s), book ^= 1u << s;
    }
  }
  if (threadIdx.x == 0) {
    // after a timed-out wait: let the copies this block issued land before its shared memory is released
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const unsigned issued = (book >> s) & 1u, waited = (book >> (2 + s)) & 1u;
      if (issued != waited) mbar_wait_bounded(full + s, waited);
    }
    bulk_wait_all();
  }
}

}  // namespace mx

// x-direction transforms with bulk-copy fed tiles (sm_103a).
//
// Rows are contiguous, so a group of TY rows is one cp.async.bulk copy.  A
// producer warp keeps NST groups in flight in a shared-memory ring (mbarrier
// full/empty pairs, bounded waits, async-proxy fence before a stage is
// released, as in the pipelined spectral pass); the consumer threads (P per
// row, TY rows) take their E values of a row from the stage, release it and
// run the same register line FFT and packing arithmetic as k_x_r2c /
// k_x_c2r, writing results straight to global memory.
#pragma once
#include "mx_spectral_tma.cuh"

namespace mx {

constexpr int XP_NST = 4;             // ring depth
constexpr size_t XP_SMEM_MAX = 200 * 1024;  // the pipelined variant is used only below this

// Both directions move TY rows of M complex values (2M reals) per group.
template <typename T, int M, int TY>
__host__ __device__ constexpr size_t xp_stage_bytes() { return (size_t)TY * M * sizeof(cx<T>); }
template <typename T, int M, int TY>
__host__ __device__ constexpr size_t xp_smem() {
  return sizeof(twv<T>) * 2 * M + sizeof(cx<T>) * TY * line_buf(M) + XP_NST * xp_stage_bytes<T, M, TY>() + 16 * XP_NST;
}
template <typename T, int M, int TY>
__host__ __device__ constexpr bool xp_fits() { return xp_smem<T, M, TY>() <= XP_SMEM_MAX; }

// Producer side shared by both directions: group g of TY rows -> stage g % NST.
template <int TY>
__device__ __forceinline__ void xp_produce(unsigned char* stages, size_t stage_bytes, uint64_t* full, uint64_t* empty,
                                           const unsigned char* in_e, const unsigned char* in_h, long rows3,
                                           long nrows, size_t row_bytes, unsigned* counter) {
  const long ngroups = (nrows + TY - 1) / TY;
  unsigned i = 0;
  bool ok = true;
  for (long grp = blockIdx.x; grp < ngroups; grp += gridDim.x, ++i) {
    const int s = (int)(i % XP_NST);
    if (i >= (unsigned)XP_NST && !mbar_wait_bounded(&empty[s], ((i / XP_NST) - 1) & 1u)) {
      ok = false;
      break;
    }
    const long row0 = grp * TY;
    const long n = (nrows - row0) < TY ? (nrows - row0) : TY;
    const unsigned char* src = row0 < rows3 ? in_e + (size_t)row0 * row_bytes : in_h + (size_t)(row0 - rows3) * row_bytes;
    const uint32_t bytes = (uint32_t)(n * row_bytes);
    mbar_expect_tx(&full[s], bytes);
    bulk_g2s(stages + (size_t)s * stage_bytes, src, bytes, &full[s]);
  }
  if (!ok) {
    atomicExch(counter + 1, 1u);
    for (unsigned j = (i > (unsigned)XP_NST ? i - XP_NST : 0); j < i; ++j)
      mbar_wait_bounded(&full[j % XP_NST], (j / XP_NST) & 1u);
  }
}

template <typename T, int M, int E, int TY>
__global__ void __launch_bounds__((M / E) * TY + 32) k_x_r2c_tma(const T* __restrict__ in_e, const T* __restrict__ in_h,
                                                               cx<T>* __restrict__ out, long rows3, long nrows,
                                                               const twv<T>* __restrict__ twg, unsigned* counter) {
  using C = cx<T>;
  constexpr int P = M / E;
  constexpr int NC = P * TY;
  constexpr int LB = line_bar(P, NC);  // lines within a warp: __syncwarp; else named barrier over consumers
  constexpr size_t SB = xp_stage_bytes<T, M, TY>();
  extern __shared__ __align__(16) unsigned char smraw[];
  twv<T>* tw = reinterpret_cast<twv<T>*>(smraw);
  C* sm = reinterpret_cast<C*>(tw + 2 * M);
  unsigned char* stages = reinterpret_cast<unsigned char*>(sm + TY * line_buf(M));
  uint64_t* full = reinterpret_cast<uint64_t*>(stages + XP_NST * SB);
  uint64_t* empty = full + XP_NST;
  for (int i = threadIdx.x; i < M + tw_len(M, E); i += blockDim.x) tw[i] = twg[i];
  if (threadIdx.x == 0) {
    for (int s = 0; s < XP_NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NC);
    }
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x >= NC) {  // producer warp
    if (threadIdx.x == NC)
      xp_produce<TY>(stages, SB, full, empty, reinterpret_cast<const unsigned char*>(in_e),
                     reinterpret_cast<const unsigned char*>(in_h), rows3, nrows, 2 * M * sizeof(T), counter);
    return;
  }
  const int t = threadIdx.x % P, ly = threadIdx.x / P;
  C* line = sm + ly * line_buf(M);
  const long ngroups = (nrows + TY - 1) / TY;
  unsigned i = 0;
  for (long grp = blockIdx.x; grp < ngroups; grp += gridDim.x, ++i) {
    const int s = (int)(i % XP_NST);
    const long row = grp * TY + ly;
    const bool ok = row < nrows;
    // leave together: a thread that gave up waiting takes its barrier partners with it
    const bool lost = !mbar_wait_bounded(&full[s], (i / XP_NST) & 1u);
    if (fft_any<LB>(lost)) {
      if (lost) atomicExch(counter + 1, 1u);
      break;
    }
    const C* st = reinterpret_cast<const C*>(stages + (size_t)s * SB) + (size_t)ly * M;
    C v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = ok ? st[t + P * m] : C{0, 0};
    fence_proxy_async_smem();
    mbar_arrive(&empty[s]);
    line_fft<T, M, E, -1, LB>(v, line, 1, t, tw + M);
    fft_bar<LB>();
#pragma unroll
    for (int m = 0; m < E; ++m) line[xoff(t + P * m, 1)] = v[m];
    fft_bar<LB>();
    if (ok) {
      C* dst = out + row * M;
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const int k = t + P * m;
        C z = line[xoff(k, 1)];
        C r;
        if (k == 0) {
          r = C{z.x + z.y, z.x - z.y};
        } else {
          C zp = cconj(line[xoff(M - k, 1)]);
          C a = cadd(z, zp), d = csub(z, zp);
          C b = C{d.y, -d.x};
          C wb = twmul<-1>(b, tw[k]);
          r = C{(T)0.5 * (a.x + wb.x), (T)0.5 * (a.y + wb.y)};
        }
        dst[k] = r;
      }
    }
    fft_bar<LB>();  // `line` is reused by the next group
  }
}

template <typename T, int M, int E, int TY>
__global__ void __launch_bounds__((M / E) * TY + 32) k_x_c2r_tma(const cx<T>* __restrict__ in, T* __restrict__ out_e,
                                                               T* __restrict__ out_h, long rows3, long nrows,
                                                               const twv<T>* __restrict__ twg, double scale,
                                                               unsigned* counter) {
  using C = cx<T>;
  constexpr int P = M / E;
  constexpr int NC = P * TY;
  constexpr int LB = line_bar(P, NC);  // lines within a warp: __syncwarp; else named barrier over consumers
  constexpr size_t SB = xp_stage_bytes<T, M, TY>();
  extern __shared__ __align__(16) unsigned char smraw[];
  twv<T>* tw = reinterpret_cast<twv<T>*>(smraw);
  C* sm = reinterpret_cast<C*>(tw + 2 * M);
  unsigned char* stages = reinterpret_cast<unsigned char*>(sm + TY * line_buf(M));
  uint64_t* full = reinterpret_cast<uint64_t*>(stages + XP_NST * SB);
  uint64_t* empty = full + XP_NST;
  for (int i = threadIdx.x; i < M + tw_len(M, E); i += blockDim.x) tw[i] = twg[i];
  if (threadIdx.x == 0) {
    for (int s = 0; s < XP_NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NC);
    }
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x >= NC) {
    if (threadIdx.x == NC)
      xp_produce<TY>(stages, SB, full, empty, reinterpret_cast<const unsigned char*>(in),
                     reinterpret_cast<const unsigned char*>(in) + (size_t)rows3 * M * sizeof(C), rows3, nrows,
                     M * sizeof(C), counter);
    return;
  }
  const int t = threadIdx.x % P, ly = threadIdx.x / P;
  C* line = sm + ly * line_buf(M);
  const KC<T> sc(scale);
  const long ngroups = (nrows + TY - 1) / TY;
  unsigned i = 0;
  for (long grp = blockIdx.x; grp < ngroups; grp += gridDim.x, ++i) {
    const int s = (int)(i % XP_NST);
    const long row = grp * TY + ly;
    const bool ok = row < nrows;
    // leave together: a thread that gave up waiting takes its barrier partners with it
    const bool lost = !mbar_wait_bounded(&full[s], (i / XP_NST) & 1u);
    if (fft_any<LB>(lost)) {
      if (lost) atomicExch(counter + 1, 1u);
      break;
    }
    const C* st = reinterpret_cast<const C*>(stages + (size_t)s * SB) + (size_t)ly * M;
    C v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int k = t + P * m;
      C x = ok ? st[k] : C{0, 0};
      if (k == 0) {
        v[m] = C{x.x + x.y, x.x - x.y};
      } else {
        C xp = cconj(ok ? st[M - k] : C{0, 0});
        C sm2 = cadd(x, xp), d = csub(x, xp);
        C wd = twmul<+1>(d, tw[k]);
        v[m] = C{sm2.x - wd.y, sm2.y + wd.x};
      }
    }
    fence_proxy_async_smem();
    mbar_arrive(&empty[s]);
    fft_bar<LB>();  // previous group's readers of `line` are done
    line_fft<T, M, E, +1, LB>(v, line, 1, t, tw + M);
    if (ok) {
      T* dst = row < rows3 ? out_e + row * (2L * M) : out_h + (row - rows3) * (2L * M);
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const int n = t + P * m;
        *reinterpret_cast<C*>(dst + 2 * n) = C{sc.mul(v[m].x), sc.mul(v[m].y)};
      }
    }
  }
}

}  // namespace mx

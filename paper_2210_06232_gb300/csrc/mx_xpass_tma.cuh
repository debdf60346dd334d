// x-direction transforms with bulk-copy fed tiles (sm_103a).
//
// Rows are contiguous, so a group of RY = 2 TY rows is one cp.async.bulk copy.
// A producer warp keeps NST groups in flight in a shared-memory ring (mbarrier
// full/empty pairs, bounded waits, async-proxy fence before a stage is
// released, as in the pipelined spectral pass).  The consumer threads (P per
// row, TY row pairs) take their E values of two rows, ly and ly + TY, from the
// stage, release it and transform both rows together (shared twiddle loads and
// barriers, twice the independent work per thread), then run the packing
// arithmetic of k_x_r2c / k_x_c2r and write straight to global memory.
#pragma once
#include "mx_spectral_tma.cuh"

namespace mx {

constexpr int XP_NST = 2;                   // ring depth (groups of 2 TY rows)
constexpr size_t XP_SMEM_MAX = 200 * 1024;  // the pipelined variant is used only below this

// Both directions move RY = 2 TY rows of M complex values (2M reals) per group.
template <typename T, int M, int TY>
__host__ __device__ constexpr size_t xp_stage_bytes() { return (size_t)2 * TY * M * sizeof(cx<T>); }
template <typename T, int M, int TY>
__host__ __device__ constexpr size_t xp_smem() {
  return sizeof(twv<T>) * 2 * M + sizeof(cx<T>) * 2 * TY * line_buf(M) + XP_NST * xp_stage_bytes<T, M, TY>() +
         16 * XP_NST;
}
template <typename T, int M, int TY>
__host__ __device__ constexpr bool xp_fits() { return xp_smem<T, M, TY>() <= XP_SMEM_MAX; }

// Producer side shared by both directions: group g of RY rows -> stage g % NST.
template <int RY>
__device__ __forceinline__ void xp_produce(unsigned char* stages, size_t stage_bytes, uint64_t* full, uint64_t* empty,
                                           const unsigned char* in_e, const unsigned char* in_h, long rows3,
                                           long nrows, size_t row_bytes, unsigned* counter) {
  const long ngroups = (nrows + RY - 1) / RY;
  unsigned i = 0;
  bool ok = true;
  for (long grp = blockIdx.x; grp < ngroups; grp += gridDim.x, ++i) {
    const int s = (int)(i % XP_NST);
    if (i >= (unsigned)XP_NST && !mbar_wait_bounded(&empty[s], ((i / XP_NST) - 1) & 1u)) {
      ok = false;
      break;
    }
    const long row0 = grp * RY;
    const long n = (nrows - row0) < RY ? (nrows - row0) : RY;
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

// Shared-memory carve-up of both directions:
// [twiddles 2M][2 TY line buffers][NST stages][full NST][empty NST]
template <typename T, int M, int TY>
struct XpSmem {
  twv<T>* tw;
  cx<T>* sm;
  unsigned char* stages;
  uint64_t* full;
  uint64_t* empty;
  __device__ __forceinline__ explicit XpSmem(unsigned char* raw) {
    tw = reinterpret_cast<twv<T>*>(raw);
    sm = reinterpret_cast<cx<T>*>(tw + 2 * M);
    stages = reinterpret_cast<unsigned char*>(sm + 2 * TY * line_buf(M));
    full = reinterpret_cast<uint64_t*>(stages + XP_NST * xp_stage_bytes<T, M, TY>());
    empty = full + XP_NST;
  }
};

template <typename T, int M, int E, int TY>
__global__ void __launch_bounds__((M / E) * TY + 32) k_x_r2c_tma(const T* __restrict__ in_e, const T* __restrict__ in_h,
                                                               cx<T>* __restrict__ out, long rows3, long nrows,
                                                               const twv<T>* __restrict__ twg, unsigned* counter) {
  using C = cx<T>;
  constexpr int P = M / E;
  constexpr int NC = P * TY;
  constexpr int RY = 2 * TY;
  constexpr int LB = line_bar(P, NC);  // lines within a warp: __syncwarp; else named barrier over consumers
  constexpr int LS = TY * line_buf(M);  // from a thread's first line buffer to its second
  constexpr size_t SB = xp_stage_bytes<T, M, TY>();
  extern __shared__ __align__(16) unsigned char smraw[];
  XpSmem<T, M, TY> L(smraw);
  for (int i = threadIdx.x; i < M + tw_len(M, E); i += blockDim.x) L.tw[i] = twg[i];
  if (threadIdx.x == 0) {
    for (int s = 0; s < XP_NST; ++s) {
      mbar_init(&L.full[s], 1);
      mbar_init(&L.empty[s], NC);
    }
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x >= NC) {  // producer warp
    if (threadIdx.x == NC)
      xp_produce<RY>(L.stages, SB, L.full, L.empty, reinterpret_cast<const unsigned char*>(in_e),
                     reinterpret_cast<const unsigned char*>(in_h), rows3, nrows, 2 * M * sizeof(T), counter);
    return;
  }
  const int t = threadIdx.x % P, ly = threadIdx.x / P;
  C* line = L.sm + ly * line_buf(M);
  const twv<T>* tw = L.tw;
  const long ngroups = (nrows + RY - 1) / RY;
  unsigned i = 0;
  for (long grp = blockIdx.x; grp < ngroups; grp += gridDim.x, ++i) {
    const int s = (int)(i % XP_NST);
    // leave together: a thread that gave up waiting takes its barrier partners with it
    const bool lost = !mbar_wait_bounded(&L.full[s], (i / XP_NST) & 1u);
    if (fft_any<LB>(lost)) {
      if (lost) atomicExch(counter + 1, 1u);
      break;
    }
    const C* st = reinterpret_cast<const C*>(L.stages + (size_t)s * SB);
    C v[2][E];
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      const bool ok = grp * RY + ly + l * TY < nrows;
#pragma unroll
      for (int m = 0; m < E; ++m) v[l][m] = ok ? st[(size_t)(ly + l * TY) * M + t + P * m] : C{0, 0};
    }
    fence_proxy_async_smem();
    mbar_arrive(&L.empty[s]);
    // MIR: the last stage mirrored (lines_fft MIRROR), so that Z_{M-k} is this thread's own
    // register E-1-m ((E - m) mod E for t = 0) and register m holds position
    // k = (m odd ? (t ? 2P - t : P) : t) + 2P (m / 2)
    constexpr bool MIR = mirror_ok(M, E);
    lines_fft<T, M, E, -1, LB, 2, 1, 0, false, 0, MIR>(v, line, 1, LS, t, tw + M);
    auto pos = [&](int m) { return MIR ? ((m & 1) ? (t ? 2 * P - t : P) : t) + 2 * P * (m >> 1) : t + P * m; };
    // Otherwise Z_{M-k} of position k = t + P m: for t > 0 it is register E-1-m of thread
    // P - t, for t = 0 register (E - m) mod E of this thread.  Lines within a warp fetch it
    // with a shuffle, wider lines through the line buffer.
    C zq[2][E];
    if constexpr (MIR) {
#pragma unroll
      for (int l = 0; l < 2; ++l)
#pragma unroll
        for (int m = 0; m < E; ++m) zq[l][m] = t == 0 ? v[l][(E - m) % E] : v[l][E - 1 - m];
    } else if constexpr (LB < 0) {
      const int lane = threadIdx.x & 31;
      const int src = (lane & ~(P - 1)) | ((P - t) & (P - 1));
#pragma unroll
      for (int l = 0; l < 2; ++l)
#pragma unroll
        for (int m = 0; m < E; ++m) {
          const C w = v[l][E - 1 - m];
          const C sh = C{__shfl_sync(0xffffffffu, w.x, src), __shfl_sync(0xffffffffu, w.y, src)};
          zq[l][m] = t == 0 ? v[l][(E - m) % E] : sh;
        }
    } else {
      fft_bar<LB>();
#pragma unroll
      for (int l = 0; l < 2; ++l)
#pragma unroll
        for (int m = 0; m < E; ++m) line[l * LS + xoff(t + P * m, 1)] = v[l][m];
      fft_bar<LB>();
#pragma unroll
      for (int l = 0; l < 2; ++l)
#pragma unroll
        for (int m = 0; m < E; ++m) {
          const int k = t + P * m;
          zq[l][m] = line[l * LS + xoff(k == 0 ? 0 : M - k, 1)];
        }
      fft_bar<LB>();  // the line buffers are reused by the next group
    }
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      const long row = grp * RY + ly + l * TY;
      if (row < nrows) {
        C* dst = out + row * M;
#pragma unroll
        for (int m = 0; m < E; ++m) {
          const int k = pos(m);
          const C z = v[l][m];
          C r;
          if (k == 0) {
            r = C{z.x + z.y, z.x - z.y};
          } else {
            C zp = cconj(zq[l][m]);
            C a = cadd(z, zp), d = csub(z, zp);
            C b = C{d.y, -d.x};
            C wb = twmul<-1>(b, tw[k]);
            r = C{(T)0.5 * (a.x + wb.x), (T)0.5 * (a.y + wb.y)};
          }
          dst[k] = r;
        }
      }
    }
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
  constexpr int RY = 2 * TY;
  constexpr int LB = line_bar(P, NC);
  constexpr int LS = TY * line_buf(M);
  constexpr size_t SB = xp_stage_bytes<T, M, TY>();
  extern __shared__ __align__(16) unsigned char smraw[];
  XpSmem<T, M, TY> L(smraw);
  for (int i = threadIdx.x; i < M + tw_len(M, E); i += blockDim.x) L.tw[i] = twg[i];
  if (threadIdx.x == 0) {
    for (int s = 0; s < XP_NST; ++s) {
      mbar_init(&L.full[s], 1);
      mbar_init(&L.empty[s], NC);
    }
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x >= NC) {
    if (threadIdx.x == NC)
      xp_produce<RY>(L.stages, SB, L.full, L.empty, reinterpret_cast<const unsigned char*>(in),
                     reinterpret_cast<const unsigned char*>(in) + (size_t)rows3 * M * sizeof(C), rows3, nrows,
                     M * sizeof(C), counter);
    return;
  }
  const int t = threadIdx.x % P, ly = threadIdx.x / P;
  C* line = L.sm + ly * line_buf(M);
  const twv<T>* tw = L.tw;
  const KC<T> sc(scale);
  const long ngroups = (nrows + RY - 1) / RY;
  unsigned i = 0;
  for (long grp = blockIdx.x; grp < ngroups; grp += gridDim.x, ++i) {
    const int s = (int)(i % XP_NST);
    const bool lost = !mbar_wait_bounded(&L.full[s], (i / XP_NST) & 1u);
    if (fft_any<LB>(lost)) {
      if (lost) atomicExch(counter + 1, 1u);
      break;
    }
    C v[2][E];
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      const bool ok = grp * RY + ly + l * TY < nrows;
      const C* st = reinterpret_cast<const C*>(L.stages + (size_t)s * SB) + (size_t)(ly + l * TY) * M;
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const int k = t + P * m;
        C x = ok ? st[k] : C{0, 0};
        if (k == 0) {
          v[l][m] = C{x.x + x.y, x.x - x.y};
        } else {
          C xp = cconj(ok ? st[M - k] : C{0, 0});
          C sm2 = cadd(x, xp), d = csub(x, xp);
          C wd = twmul<+1>(d, tw[k]);
          v[l][m] = C{sm2.x - wd.y, sm2.y + wd.x};
        }
      }
    }
    fence_proxy_async_smem();
    mbar_arrive(&L.empty[s]);
    fft_bar<LB>();  // previous group's readers of the line buffers are done
    lines_fft<T, M, E, +1, LB, 2>(v, line, 1, LS, t, tw + M);
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      const long row = grp * RY + ly + l * TY;
      if (row < nrows) {
        T* dst = row < rows3 ? out_e + row * (2L * M) : out_h + (row - rows3) * (2L * M);
#pragma unroll
        for (int m = 0; m < E; ++m) {
          const int n = t + P * m;
          *reinterpret_cast<C*>(dst + 2 * n) = C{sc.mul(v[l][m].x), sc.mul(v[l][m].y)};
        }
      }
    }
  }
}

}  // namespace mx

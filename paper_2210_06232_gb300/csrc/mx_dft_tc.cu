// DFT-as-GEMM on the fifth-generation tensor cores (tcgen05) against the FMA radix-8 stage.
//
// The cost model of the method (Sec. 2.5: the transforms dominate) makes the radix stages of the
// line FFTs the only candidate for the tensor cores.  This unit measures one such stage both
// ways, on the same data, so that the choice rests on a measurement:
//   * FMA: a thread holds the 8 complex inputs of one 8-point DFT, multiplies them by twiddles
//     and runs the register butterfly of the line FFTs (bfly8, double-single constants);
//   * tcgen05: 128 threads write the twiddled inputs of 128 DFT-8s into shared memory as the A
//     operand of a 128 x 16 x 16 MMA (kind::tf32, K-major, no swizzle; the 16 x 16 real matrix
//     of the DFT-8 is the B operand), one thread issues the MMAs, the 128 x 16 FP32 result lands
//     in tensor memory and is read back with tcgen05.ld.  TF32 keeps 10 mantissa bits, so an
//     FP32-accurate product needs split operands: a = a0 + a1 + a2 with a_i the TF32 truncation
//     of what is left; 1 product (a0 b0), 3 (+ a0 b1 + a1 b0) or 6 (+ a0 b2 + a1 b1 + a2 b0).
// Each launch applies `reps` stages (twiddle, then DFT-8) to tiles of 128 DFT-8s held on chip,
// so the time is the stage's arithmetic and data movement, not HBM.
#include <math.h>
#include <string.h>

#include "../../include/maxexp.h"
#include "mx_launch.h"

namespace {

constexpr int TC_M = 128;  // DFT-8s per tile (MMA M: one per tensor-memory lane)
constexpr int TC_K = 16;   // 8 complex inputs, (re, im) interleaved
constexpr int TC_N = 16;   // 8 complex outputs, (re, im) interleaved

__device__ __forceinline__ float tf32_trunc(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// Byte offset of element (row, k) of a K-major operand without swizzle: core matrices of 8 rows
// x 16 bytes (4 TF32 values), 4 of them along K (leading byte offset 128), groups of 8 rows 512
// bytes apart (stride byte offset 512).
__host__ __device__ constexpr uint32_t kmaj_off(int row, int k) {
  return (uint32_t)(((row >> 3) * 4 + (k >> 2)) * 128 + (row & 7) * 16 + (k & 3) * 4);
}
constexpr uint32_t LBO = 128, SBO = 512;

// Shared-memory matrix descriptor: start address, leading and stride byte offsets (all >> 4),
// descriptor version 1 (bits 46-47), no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((LBO >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((SBO >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::tf32: FP32 accumulator (bits 4-5 = 1), A and B TF32 (bits 7-9,
// 10-12 = 2), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mx::smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// 16 columns of this warp's 32 lanes (lane = row) from tensor memory.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Stage twiddles w[k] (plain FP32, the same values in both variants) and, for the tensor-core
// variant, the three TF32 splits of the DFT-8 matrix laid out as the B operand.
struct Consts {
  float2 tw[8];
  float b[3][TC_N * TC_K];  // K-major: element (n, k) at kmaj_off(n, k) / 4
};

__device__ __forceinline__ void twiddle(float2* v, const float2* tw) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float2 a = v[k], w = tw[k];
    v[k] = float2{fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x)};
  }
}

__global__ void __launch_bounds__(TC_M) k_dft8_fma(const float2* __restrict__ in, float2* __restrict__ out,
                                                   const Consts* __restrict__ cs, int reps) {
  const long row = (long)blockIdx.x * TC_M + threadIdx.x;
  float2 tw[8], v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) tw[k] = cs->tw[k], v[k] = in[row * 8 + k];
  for (int r = 0; r < reps; ++r) {
    twiddle(v, tw);
    mx::bfly8<-1, 1>(v);
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) out[row * 8 + k] = v[k];
}

// NP products of NS = 1, 2 or 3 splits: pairs (i, j) with i + j < NS.
template <int NP>
__global__ void __launch_bounds__(TC_M, 1) k_dft8_tc(const float2* __restrict__ in, float2* __restrict__ out,
                                                     const Consts* __restrict__ cs, int reps, unsigned* __restrict__ err) {
  constexpr int NS = NP == 1 ? 1 : (NP == 3 ? 2 : 3);
  static_assert(NP == 1 || NP == 3 || NP == 6, "1, 3 or 6 products");
  __shared__ __align__(128) unsigned char sA[NS][TC_M * TC_K * 4];
  __shared__ __align__(128) unsigned char sB[NS][TC_N * TC_K * 4];
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int i = tid; i < NS * TC_N * TC_K; i += TC_M)
    reinterpret_cast<float*>(sB)[i] = cs->b[i / (TC_N * TC_K)][i % (TC_N * TC_K)];
  if (warp == 0) {
    // 32 columns of tensor memory (the minimum allocation) hold the 16 result columns
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(mx::smem_u32(&tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mx::mbar_init(&bar, 1);
    mx::mbar_fence_init();
  }
  const long row = (long)blockIdx.x * TC_M + tid;
  float2 tw[8], v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) tw[k] = cs->tw[k], v[k] = in[row * 8 + k];
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  bool lost = false;
  int r = 0;
  for (; r < reps; ++r) {
    twiddle(v, tw);
    // the split inputs of this row, 16 bytes (4 TF32 values) per store
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float a[4] = {v[2 * q].x, v[2 * q].y, v[2 * q + 1].x, v[2 * q + 1].y};
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        float p[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          p[e] = tf32_trunc(a[e]);
          a[e] -= p[e];
        }
        *reinterpret_cast<float4*>(sA[s] + kmaj_off(tid, 4 * q)) = make_float4(p[0], p[1], p[2], p[3]);
      }
    }
    mx::fence_proxy_async_smem();  // the stores above before the tensor core's reads
    tc_fence_before();
    __syncthreads();  // (also: every tcgen05.ld of the previous stage is done)
    tc_fence_after();
    if (tid == 0) {
      uint32_t acc = 0;
#pragma unroll
      for (int i = 0; i < NS; ++i)
#pragma unroll
        for (int j = 0; j < NS; ++j) {
          if (i + j >= NS) continue;
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {  // K = 16 as two MMAs of K = 8
            tc_mma(tmem, smem_desc(mx::smem_u32(sA[i]) + ks * 2 * LBO), smem_desc(mx::smem_u32(sB[j]) + ks * 2 * LBO), acc);
            acc = 1;
          }
        }
      tc_commit(&bar);
    }
    const bool ok = mx::mbar_wait_bounded(&bar, (uint32_t)(r & 1));
    lost = __syncthreads_or(!ok) != 0;
    if (lost) {
      if (tid == 0) atomicExch(err, 1u);
      break;
    }
    tc_fence_after();
    float d[16];
    tc_ld16(tmem + ((uint32_t)(warp * 32) << 16), d);
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = float2{d[2 * k], d[2 * k + 1]};
  }
  if (lost && tid == 0) mx::mbar_wait_bounded(&bar, (uint32_t)(r & 1));  // (bounded) the MMAs issued have completed
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem) : "memory");
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) out[row * 8 + k] = v[k];
}

void host_consts(Consts& c) {
  for (int k = 0; k < 8; ++k) {
    // unit-modulus twiddles divided by sqrt(8): each stage then keeps the magnitude of the data
    const double a = -2.0 * M_PI * (double)(k + 1) / 64.0, s = 1.0 / sqrt(8.0);
    c.tw[k] = make_float2((float)(cos(a) * s), (float)(sin(a) * s));
  }
  // B[(n1, re/im)][(k1, re/im)]: re_k1 += cos x.re + sin x.im, im_k1 += -sin x.re + cos x.im,
  // angle 2 pi n1 k1 / 8 (the forward kernel), stored K-major at (n = output, k = input)
  for (int s = 0; s < 3; ++s)
    for (int i = 0; i < TC_N * TC_K; ++i) c.b[s][i] = 0.f;
  for (int n1 = 0; n1 < 8; ++n1)
    for (int k1 = 0; k1 < 8; ++k1) {
      const double th = 2.0 * M_PI * (double)((n1 * k1) % 8) / 8.0;
      const double co = cos(th), si = sin(th);
      const double ent[2][2] = {{co, -si}, {si, co}};  // [input re/im][output re/im]
      for (int ir = 0; ir < 2; ++ir)
        for (int orr = 0; orr < 2; ++orr) {
          double rest = ent[ir][orr];
          for (int s = 0; s < 3; ++s) {
            float f = (float)rest;
            uint32_t u;
            memcpy(&u, &f, 4);
            u &= 0xFFFFE000u;
            memcpy(&f, &u, 4);
            c.b[s][kmaj_off(2 * k1 + orr, 2 * n1 + ir) / 4] = f;
            rest -= (double)f;
          }
        }
    }
}

}  // namespace

extern "C" mx_status mx_dft8_stage_eval(int variant, const void* in, void* out, long long tiles, int reps,
                                        double* ms) {
  if (!in || !out || tiles < 1 || tiles > (1LL << 20) || reps < 1 || !ms) return MX_E_INVAL;
  if (variant != 0 && variant != 1 && variant != 3 && variant != 6) return MX_E_INVAL;
  if ((((uintptr_t)in) | ((uintptr_t)out)) & 15u) return MX_E_INVAL;
  Consts hc;
  host_consts(hc);
  Consts* dc = nullptr;
  unsigned* derr = nullptr;
  if (mx::dev_alloc((void**)&dc, sizeof(Consts)) != cudaSuccess) return MX_E_NOMEM;
  if (mx::dev_alloc((void**)&derr, sizeof(unsigned)) != cudaSuccess) {
    cudaFree(dc);
    return MX_E_NOMEM;
  }
  mx_status st = MX_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaMemcpy(dc, &hc, sizeof(Consts), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(derr, 0, sizeof(unsigned)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    st = MX_E_CUDA;
  } else {
    const float2* src = (const float2*)in;
    float2* dst = (float2*)out;
    const int grid = (int)tiles;
    cudaEventRecord(e0, 0);
    switch (variant) {
      case 0: k_dft8_fma<<<grid, TC_M>>>(src, dst, dc, reps); break;
      case 1: k_dft8_tc<1><<<grid, TC_M>>>(src, dst, dc, reps, derr); break;
      case 3: k_dft8_tc<3><<<grid, TC_M>>>(src, dst, dc, reps, derr); break;
      default: k_dft8_tc<6><<<grid, TC_M>>>(src, dst, dc, reps, derr); break;
    }
    cudaEventRecord(e1, 0);
    unsigned herr = 0;
    float t = 0.f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&t, e0, e1) != cudaSuccess ||
        cudaMemcpy(&herr, derr, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) {
      st = MX_E_CUDA;
    } else if (herr) {
      st = MX_E_TIMEOUT;
    } else {
      *ms = t;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(dc);
  cudaFree(derr);
  return st;
}

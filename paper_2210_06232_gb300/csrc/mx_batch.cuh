// Batched spectral form: many independent instances (different grids, eps,
// mu, h) advanced K steps by ONE persistent cooperative launch.
//
// Per step n the grid runs
//   phase A  coefficient tables of every instance at its t_n (grid-stride
//            over the concatenation of the tables), and the invariant records
//            of step n-1 (one block per instance, fixed summation order);
//   barrier
//   phase B  the exponential update of every instance: a global list of
//            chunks (CH points x 6 components) spanning all instances, consumed
//            by the same warp-specialised bulk-copy pipeline as the single
//            pass; each warp writes its invariant partial sums of the chunk
//            (in the instance's precision) to `cpart[chunk][warp]` when step
//            n is recorded;
//   barrier.
// Chunk contents and warp partitions depend only on the instance's own chunk
// index, and records are summed per instance over its own chunks in order,
// so an instance gets bit-identical fields and invariants alone or in any
// mix.  Grid barriers and mbarrier waits are bounded; a wait that gives up
// sets bar[2] and every block leaves at its next check.
#pragma once
#include "mx_spectral_tma.cuh"

namespace mx {

struct BInst {
  GridParams g;
  const void* src;   // spectrum at t0 (packed half spectrum, 6 components)
  void* dst;         // spectrum at t_n
  void* tab;         // Coef<T>[nq] for this instance (nullptr: direct coefficients)
  int nq;
  unsigned npts;     // Nz * Ny * Mx points per component
  unsigned chunk0;   // first global chunk of this instance
  unsigned nchunks;
  unsigned q0;       // first index of this instance in the concatenated table range
  unsigned seg0;     // first invariant segment (BT_SEGC chunks) of this instance
  unsigned nseg;
  long long n0;      // step count before this launch
  double t0, h;      // time before this launch, step size: t_n = t0 + (n - n0) h
  double* rec;       // record slots of this launch (16 doubles each)
  int every;         // record every `every` steps (0: none)
};

// Per table entry of an FP32 batch, what does not change with t: hk = (0.5 c) |k| and |k|, |k|^2
// (coef_from_hk), so that phase A takes no FP64 square root.
struct QK {
  double hk;
  float kabs, k2;
};

struct BatchArgs {
  const BInst* inst;
  int ninst;
  unsigned total_chunks;
  unsigned total_q;
  int nsteps;
  unsigned total_segs;
  void* cpart;     // [total_chunks][BT_CWARPS][16] of T: per-warp partial sums of a chunk (value 15: 0)
  double* segpart; // [2][total_segs][NSUM]: sums of BT_SEGC consecutive chunks
  const QK* qk;    // [total_q] (FP32 batches; nullptr: coefficients from |k|^2 alone)
  unsigned* bar;  // [0] arrivals, [1] generation, [2] error flag
};

template <typename T> struct BTraits;
template <> struct BTraits<float> {
  static constexpr int PPT = 2;  // points per consumer thread per chunk
};
template <> struct BTraits<double> {
  static constexpr int PPT = 1;
};
constexpr int BT_NST = 4;
constexpr int BT_CONSUMERS = 224;  // seven consumer warps + the producer: two blocks of eight warps per SM
constexpr int BT_THREADS = BT_CONSUMERS + 32;
constexpr int BT_CWARPS = BT_CONSUMERS / 32;
constexpr int BT_SEGC = 32;  // chunks per invariant segment (one lane each)
template <typename T> __host__ __device__ constexpr int bt_ch() { return BT_CONSUMERS * BTraits<T>::PPT; }
template <typename T> __host__ __device__ constexpr size_t bt_smem_bytes() {
  return (size_t)BT_NST * 6 * bt_ch<T>() * sizeof(cx<T>) + 16 * BT_NST + 32 * NSUM * sizeof(double);
}

// Bounded software grid barrier (all blocks co-resident: cooperative launch).
__device__ __forceinline__ bool grid_barrier(unsigned* bar) {
  __syncthreads();
  __shared__ int failed;
  if (threadIdx.x == 0) {
    failed = 0;
    volatile unsigned* gen = bar + 1;
    const unsigned g0 = *gen;
    __threadfence();
    const unsigned nb = gridDim.x;
    if (atomicAdd(bar, 1u) == nb - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned it = 0;
      while (*gen == g0) {
        if (++it > (1u << 26) || *(volatile unsigned*)(bar + 2)) {
          atomicExch(bar + 2, 1u);
          failed = 1;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return failed == 0 && *(volatile unsigned*)(bar + 2) == 0;
}

__device__ __forceinline__ int find_inst(const BInst* inst, int n, unsigned key, bool by_chunk) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {  // last instance whose start <= key
    const int mid = (lo + hi + 1) >> 1;
    const unsigned start = by_chunk ? __ldg(&inst[mid].chunk0) : __ldg(&inst[mid].q0);
    if (start <= key) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int find_inst_seg(const BInst* inst, int n, unsigned key) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(&inst[mid].seg0) <= key) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ Coef<float> load_coef_cg(const Coef<float>* p) {
  const float4 v = __ldcg(reinterpret_cast<const float4*>(p));
  return Coef<float>{v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ Coef<double> load_coef_cg(const Coef<double>* p) {
  const double2 a = __ldcg(reinterpret_cast<const double2*>(p)), b = __ldcg(reinterpret_cast<const double2*>(p) + 1);
  return Coef<double>{a.x, a.y, b.x, b.y};
}

__device__ __forceinline__ bool recorded(const BInst& b, long long N) { return b.every > 0 && N % b.every == 0; }

// Instance of global chunk `key`: binary search over the first chunks held in shared
// memory (batches of up to BT_SINST instances), else over the descriptors.
constexpr int BT_SINST = 1024;
static_assert(BTraits<float>::PPT <= 2 && BTraits<double>::PPT <= 2, "a thread's points cross at most one row end");
__device__ __forceinline__ int find_inst_s(const BatchArgs& a, const unsigned* s_chunk0, unsigned key) {
  if (a.ninst > BT_SINST) return find_inst(a.inst, a.ninst, key, true);
  int lo = 0, hi = a.ninst - 1;
  while (lo < hi) {  // last instance whose first chunk <= key
    const int mid = (lo + hi + 1) >> 1;
    if (s_chunk0[mid] <= key) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}
__device__ __forceinline__ long long rec_slot(const BInst& b, long long N) { return N / b.every - b.n0 / b.every - 1; }

// Invariant records, a fixed tree in three levels.  A chunk's sum is its
// warps' partials added in warp order in the instance's precision (T; the
// partials are sums of T densities already); segment j of an instance is the
// FP64 sum of the chunk sums of its chunks [j*BT_SEGC, (j+1)*BT_SEGC), one lane
// per chunk and a transposed warp tree; the record is the sum of the
// instance's segments (one warp per instance).  Every level depends only on
// instance-local indices.  On a part with a narrow FP64 pipe the transposed
// trees (16 FP64 additions per lane where a butterfly per sum takes 75) and
// the chunk-level sums in T keep phase A short.
template <typename T>
__device__ void batch_segments(const BatchArgs& a, long long step_local, double* seg) {
  const int lane = threadIdx.x & 31;
  const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  const T* cp = reinterpret_cast<const T*>(a.cpart);
  for (unsigned sgi = gw; sgi < a.total_segs; sgi += nw) {
    const int ii = find_inst_seg(a.inst, a.ninst, sgi);
    const BInst& b = a.inst[ii];
    if (!recorded(b, b.n0 + step_local)) continue;  // uniform within the warp
    const unsigned c = (sgi - b.seg0) * BT_SEGC + lane;  // this lane's chunk of the instance
    double v[16];
    if (c < b.nchunks) {
      const T* row = cp + (size_t)(b.chunk0 + c) * BT_CWARPS * 16;
      // rows of 16 values, 64 (float) or 128 (double) bytes: 16-byte loads
      using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
      constexpr int PER = (int)(sizeof(V) / sizeof(T));
      T s[16];
#pragma unroll
      for (int w = 0; w < BT_CWARPS; ++w)
#pragma unroll
        for (int q = 0; q < 16 / PER; ++q) {
          const V x = __ldcg(reinterpret_cast<const V*>(row + w * 16) + q);
          const T* e = reinterpret_cast<const T*>(&x);
#pragma unroll
          for (int u = 0; u < PER; ++u) s[q * PER + u] = w == 0 ? e[u] : s[q * PER + u] + e[u];
        }
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] = (double)s[k];
    } else {
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] = 0.0;
    }
    const double tot = warp_transpose_sum16<double>(v, lane);
    const int idx = transpose_index(lane);
    if (!(lane & 1) && idx < NSUM) seg[(size_t)sgi * NSUM + idx] = tot;
  }
}

__device__ void batch_final(const BatchArgs& a, long long step_local, const double* seg) {
  const int lane = threadIdx.x & 31;
  const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (unsigned ii = gw; ii < (unsigned)a.ninst; ii += nw) {
    const BInst& b = a.inst[ii];
    const long long N = b.n0 + step_local;
    if (!recorded(b, N)) continue;
    double v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = 0.0;
    for (unsigned j = lane; j < b.nseg; j += 32) {
      const double* p = seg + (size_t)(b.seg0 + j) * NSUM;
#pragma unroll
      for (int k = 0; k < NSUM; ++k) v[k] += __ldcg(p + k);
    }
    const double tot = warp_transpose_sum16<double>(v, lane);
    const int idx = transpose_index(lane);
    if (!(lane & 1) && idx < NSUM) b.rec[(size_t)rec_slot(b, N) * 16 + idx] = tot;
  }
}

template <typename T>
// 112 registers and eight warps per block: two blocks per SM (four warps on each SM sub-partition,
// 4 x 32 x 112 of its 16384 registers).  With eight consumer warps (nine per block) only one block
// fits: five warps on a sub-partition would need at most 102 registers each.
__global__ void __maxnreg__(112) k_batch_steps(BatchArgs a) {
  using C = cx<T>;
  constexpr int PPT = BTraits<T>::PPT;
  constexpr int CH = bt_ch<T>();
  extern __shared__ __align__(16) unsigned char smraw[];
  C* stage = reinterpret_cast<C*>(smraw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smraw + (size_t)BT_NST * 6 * CH * sizeof(C));
  uint64_t* empty = full + BT_NST;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  __shared__ unsigned s_chunk0[BT_SINST];  // first chunk of each instance (instance lookup)
  for (int k = tid; k < a.ninst && k < BT_SINST; k += blockDim.x) s_chunk0[k] = a.inst[k].chunk0;
  if (tid == 0) {
    for (int s = 0; s < BT_NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], BT_CONSUMERS);
    }
    mbar_fence_init();
  }
  __syncthreads();
  unsigned i = 0;  // pipeline position, continues across steps
  const unsigned gthreads = gridDim.x * blockDim.x;

  for (int n = 1; n <= a.nsteps + 2; ++n) {
    // ------------------------------------------------ phase A: tables of step n,
    // invariant segments of step n-1, records of step n-2
    if (n <= a.nsteps) {
      for (unsigned q = blockIdx.x * blockDim.x + tid; q < a.total_q; q += gthreads) {
        const int ii = find_inst(a.inst, a.ninst, q, false);
        const BInst& b = a.inst[ii];
        const unsigned qi = q - b.q0;
        if (b.tab && qi < (unsigned)b.nq) {
          const double t = b.t0 + (double)n * b.h;
          Coef<T> v;
          if constexpr (sizeof(T) == 4) {
            if (a.qk) {
              const QK e = a.qk[q];
              v = coef_from_hk(e.hk, e.kabs, e.k2, qi == 0, t, b.g);
            } else {
              v = coef_direct<T, Coef<T>>(b.g.s0 * (double)qi, t, b.g);
            }
          } else {
            v = coef_direct<T, Coef<T>>(b.g.s0 * (double)qi, t, b.g);
          }
          reinterpret_cast<Coef<T>*>(b.tab)[qi] = v;
        }
      }
    }
    if (n >= 2 && n - 1 <= a.nsteps) batch_segments<T>(a, n - 1, a.segpart + (size_t)((n - 1) & 1) * a.total_segs * NSUM);
    if (n >= 3) batch_final(a, n - 2, a.segpart + (size_t)((n - 2) & 1) * a.total_segs * NSUM);
    if (n == a.nsteps + 2) break;
    if (!grid_barrier(a.bar)) return;
    if (n == a.nsteps + 1) continue;

    // ------------------------------------------------ phase B: update every chunk
    if (warp == BT_CWARPS) {
      if (lane == 0) {
        unsigned ii = i;
        bool ok = true;
        for (unsigned gc = blockIdx.x; gc < a.total_chunks; gc += gridDim.x, ++ii) {
          const int s = (int)(ii % BT_NST);
          if (ii >= (unsigned)BT_NST && !mbar_wait_bounded(&empty[s], ((ii / BT_NST) - 1) & 1u)) {
            ok = false;
            break;
          }
          const BInst& b = a.inst[find_inst_s(a, s_chunk0, gc)];
          const unsigned p0 = (gc - b.chunk0) * CH;
          const unsigned cnt = min((unsigned)CH, b.npts - p0);
          const uint32_t bytes = cnt * (uint32_t)sizeof(C);
          mbar_expect_tx(&full[s], 6 * bytes);
          const C* src = reinterpret_cast<const C*>(b.src);
#pragma unroll
          for (int comp = 0; comp < 6; ++comp)
            bulk_g2s(stage + ((size_t)s * 6 + comp) * CH, src + (size_t)comp * b.npts + p0, bytes, &full[s]);
        }
        if (!ok) {
          atomicExch(a.bar + 2, 1u);
          for (unsigned j = (ii > (unsigned)BT_NST ? ii - BT_NST : 0); j < ii; ++j)
            mbar_wait_bounded(&full[j % BT_NST], (j / BT_NST) & 1u);
        }
      }
    } else {
      // Everything a chunk needs besides its data (instance, wavenumbers, coefficients) is
      // prepared one chunk ahead, so the coefficient loads from L2 overlap the current chunk.
      struct Pt {
        Coef<T> q;
        T kx, ky, kz, w;  // w: Hermitian weight, 0 past the instance's last point
      };
      struct Prep {
        int ii;
        unsigned p0;
        bool rec;
        Pt pt[PPT];
      };
      auto prep = [&](unsigned gc, Prep& o) {
        o.ii = find_inst_s(a, s_chunk0, gc);
        const BInst& b = a.inst[o.ii];
        const GridParams& g = b.g;
        o.p0 = (gc - b.chunk0) * CH;
        o.rec = recorded(b, b.n0 + n);
        // row of this thread's first point; the next one is in it or starts the next row
        const unsigned pf = o.p0 + PPT * tid;
        const unsigned rf = (pf < b.npts ? pf : 0u) / (unsigned)g.mx;
        const int xf = (int)((pf < b.npts ? pf : 0u) - rf * (unsigned)g.mx);
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
          const unsigned p = pf + j;
          const bool live = p < b.npts;
          const bool wrap = xf + j >= g.mx;  // PPT <= 2 crosses at most one row end
          const unsigned r = live ? rf + (wrap ? 1u : 0u) : 0u;
          const int x = live ? xf + j - (wrap ? g.mx : 0) : 0;
          const unsigned z = r / (unsigned)g.ny;
          const int y = (int)(r - z * (unsigned)g.ny);
          const int my = signed_index(y, g.ny), mz = signed_index((int)z, g.nz);
          Pt& q = o.pt[j];
          q.kx = GP<T>::nu(g, 0) * (T)x;
          q.ky = GP<T>::nu(g, 1) * (T)my;
          q.kz = GP<T>::nu(g, 2) * (T)mz;
          q.w = live ? (x == 0 ? (T)1 : (T)2) : (T)0;
          if (b.tab) {
            // L1-bypassing load: the table was rewritten by other blocks in phase A
            q.q = load_coef_cg(reinterpret_cast<const Coef<T>*>(b.tab) + (g.qa[0] * x * x + g.qa[1] * my * my +
                                                                          g.qa[2] * mz * mz));
          } else {
            const double k2 = g.nu[0] * g.nu[0] * (double)x * x + g.nu[1] * g.nu[1] * (double)my * my +
                              g.nu[2] * g.nu[2] * (double)mz * mz;
            q.q = coef_direct<T, Coef<T>>(k2, b.t0 + (double)n * b.h, g);
          }
        }
      };
      unsigned ii = i;
      Prep cur, nxt;
      if (blockIdx.x < a.total_chunks) prep(blockIdx.x, cur);
      for (unsigned gc = blockIdx.x; gc < a.total_chunks; gc += gridDim.x, ++ii, cur = nxt) {
        const int s = (int)(ii % BT_NST);
        if (gc + gridDim.x < a.total_chunks) prep(gc + gridDim.x, nxt);
        const BInst& b = a.inst[cur.ii];
        const GridParams& g = b.g;
        const unsigned p0 = cur.p0;
        const bool rec = cur.rec;
        // the warp leaves together (its lanes meet again in warp shuffles)
        const bool lost = !mbar_wait_bounded(&full[s], (ii / BT_NST) & 1u);
        if (__any_sync(0xffffffffu, lost)) {
          if (lost) atomicExch(a.bar + 2, 1u);
          break;
        }
        C v[6][PPT];
        const C* st = stage + (size_t)s * 6 * CH;
#pragma unroll
        for (int comp = 0; comp < 6; ++comp)
#pragma unroll
          for (int j = 0; j < PPT; ++j) v[comp][j] = st[comp * CH + PPT * tid + j];
        fence_proxy_async_smem();
        mbar_arrive(&empty[s]);
        T part[NSUM];
#pragma unroll
        for (int k = 0; k < NSUM; ++k) part[k] = (T)0;
        const T eps = GP<T>::eps(g), mu = GP<T>::mu(g);
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
          const Pt& q = cur.pt[j];
          if (q.w == (T)0) continue;
          C hh[3] = {v[3][j], v[4][j], v[5][j]};
          C ee[3] = {v[0][j], v[1][j], v[2][j]};
          Apply<T, Coef<T>>::run(q.q, q.kx, q.ky, q.kz, hh, ee);
#pragma unroll
          for (int comp = 0; comp < 3; ++comp) v[comp][j] = ee[comp], v[comp + 3][j] = hh[comp];
          if (rec) add_densities<T>(part, q.w, q.kx, q.ky, q.kz, hh, ee, eps, mu);
        }
        C* dst = reinterpret_cast<C*>(b.dst);
        const unsigned pt = p0 + PPT * tid;
        if (pt < b.npts) {
#pragma unroll
          for (int comp = 0; comp < 6; ++comp) {
            if constexpr (PPT == 2) {
              __stcs(reinterpret_cast<float4*>(dst + (size_t)comp * b.npts + pt),
                     make_float4(v[comp][0].x, v[comp][0].y, v[comp][PPT - 1].x, v[comp][PPT - 1].y));
            } else {
              __stcs(dst + (size_t)comp * b.npts + pt, v[comp][0]);
            }
          }
        }
        if (rec) {  // uniform across the block: one instance per chunk
          T v16[16];
#pragma unroll
          for (int k = 0; k < NSUM; ++k) v16[k] = part[k];
          v16[15] = (T)0;
          const T tot = warp_transpose_sum16<T>(v16, lane);
          const int idx = transpose_index(lane);
          if (!(lane & 1)) reinterpret_cast<T*>(a.cpart)[((size_t)gc * BT_CWARPS + warp) * 16 + idx] = tot;
        }
      }
    }
    // every thread of a block iterated the same chunks
    i += (a.total_chunks > blockIdx.x) ? (a.total_chunks - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    if (!grid_barrier(a.bar)) return;
  }
}

}  // namespace mx

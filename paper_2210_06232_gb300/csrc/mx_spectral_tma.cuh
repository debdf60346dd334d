// FP32 spectral pass with a bulk-copy (TMA engine) pipeline, sm_103a.
//
// The pass is a pure stream: per point it reads six complex values, applies
// the per-k exponential and writes six.  Memory-level parallelism comes from
// the copy engine instead of registers: chunks of CH points per component
// are brought into shared memory by cp.async.bulk (one 4 KB copy per
// component) completing on an mbarrier, NST chunks in flight per block;
// 256 threads consume a chunk (two points each) and write the result with
// streaming 16-byte stores.  Waits on the mbarrier are bounded: a wait that
// gives up sets counter[1] (read by the host as MX_E_TIMEOUT) and the warp
// leaves the loop together.
#pragma once
#include "mx_kernels.cuh"

namespace mx {

constexpr int TMA_CH = 512;       // points per component per chunk (4 KB in FP32)
constexpr int TMA_NST = 4;        // chunks in flight per block
constexpr int TMA_CONSUMERS = 256;
constexpr int TMA_THREADS = TMA_CONSUMERS + 32;  // + one producer warp
constexpr int TMA_CWARPS = TMA_CONSUMERS / 32;
constexpr size_t tma_smem_bytes() {
  return (size_t)TMA_NST * 6 * TMA_CH * sizeof(float2) + 16 * TMA_NST + (size_t)TMA_CWARPS * NSUM * sizeof(double);
}

// Warp-specialised: warp TMA_CWARPS is the producer (lane 0 issues the bulk
// copies of chunk i into stage i % NST once `empty` says the consumers have
// read what was there); the consumer warps wait on `full`, copy their two
// points per component to registers, fence their generic reads against the
// async proxy, release the stage, then compute and store.  Coefficient-table loads are issued before the wait on the data.
template <bool UPDATE, bool INV>
__global__ void __launch_bounds__(TMA_THREADS, 2)
    k_spectral_tma(const float2* __restrict__ src, float2* __restrict__ dst, long comp_stride, GridParams g,
                   const Coef<float>* __restrict__ tab, double* __restrict__ partials, unsigned* __restrict__ counter,
                   double* __restrict__ record) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* stage = reinterpret_cast<float2*>(smraw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smraw + (size_t)TMA_NST * 6 * TMA_CH * sizeof(float2));
  uint64_t* empty = full + TMA_NST;
  double* wsum = reinterpret_cast<double*>(empty + TMA_NST);  // [TMA_CWARPS][NSUM]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const unsigned npts = (unsigned)comp_stride;
  const unsigned nchunks = (npts + TMA_CH - 1) / TMA_CH;

  if (tid == 0) {
    for (int s = 0; s < TMA_NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], TMA_CONSUMERS);
    }
    mbar_fence_init();
  }
  if (tid < TMA_CWARPS * NSUM) wsum[tid] = 0.0;
  __syncthreads();

  if (warp == TMA_CWARPS) {
    // ---------------------------------------------------------- producer
    if (lane == 0) {
      unsigned i = 0;
      bool ok = true;
      for (unsigned c = blockIdx.x; c < nchunks; c += gridDim.x, ++i) {
        const int s = (int)(i % TMA_NST);
        if (i >= (unsigned)TMA_NST && !mbar_wait_bounded(&empty[s], ((i / TMA_NST) - 1) & 1u)) {
          ok = false;
          break;
        }
        const unsigned p0 = c * TMA_CH;
        const unsigned n = min((unsigned)TMA_CH, npts - p0);
        const uint32_t bytes = n * (uint32_t)sizeof(float2);
        mbar_expect_tx(&full[s], 6 * bytes);
#pragma unroll
        for (int comp = 0; comp < 6; ++comp)
          bulk_g2s(stage + ((size_t)s * 6 + comp) * TMA_CH, src + (size_t)comp * comp_stride + p0, bytes, &full[s]);
      }
      if (!ok) {
        atomicExch(counter + 1, 1u);
        // let the last copies this block issued land before its shared memory is released
        for (unsigned j = (i > (unsigned)TMA_NST ? i - TMA_NST : 0); j < i; ++j)
          mbar_wait_bounded(&full[j % TMA_NST], (j / TMA_NST) & 1u);
      }
    }
  } else {
    // ---------------------------------------------------------- consumers
    const unsigned mx = (unsigned)g.mx, ny = (unsigned)g.ny;
    const float eps = g.epsf, mu = g.muf;
    const float nux = g.nuf[0], nuy = g.nuf[1], nuz = g.nuf[2];
    float part[INV ? 16 : 1];  // NSUM sums and a zero (warp_transpose_sum16)
#pragma unroll
    for (int k = 0; k < (INV ? 16 : 1); ++k) part[k] = 0.f;
    int cnt = 0;
    unsigned i = 0;
    // position of this thread's two points in chunk c, and their table entries
    struct Pos {
      unsigned p;
      int x0, my, mz;
      float4 q[2];
    };
    auto locate = [&](unsigned c, Pos& o) {
      const unsigned p = c * TMA_CH + 2 * tid;
      const unsigned pp = p < npts ? p : 0;
      const unsigned r = pp / mx;
      o.p = p;
      o.x0 = (int)(pp - r * mx);
      const unsigned z = r / ny;
      const int y = (int)(r - z * ny);
      o.my = signed_index(y, g.ny);
      o.mz = signed_index((int)z, g.nz);
      if constexpr (UPDATE) {
        const int qyz = g.qa[1] * o.my * o.my + g.qa[2] * o.mz * o.mz;
#pragma unroll
        for (int j = 0; j < 2; ++j)
          o.q[j] = __ldg(reinterpret_cast<const float4*>(tab) + (g.qa[0] * (o.x0 + j) * (o.x0 + j) + qyz));
      }
    };
    Pos cur, nxt;
    if (blockIdx.x < nchunks) locate(blockIdx.x, cur);
    // (cur takes nxt at the end of an iteration, when its loads have had the compute time to land)
    for (unsigned c = blockIdx.x; c < nchunks; c += gridDim.x, ++i, cur = nxt) {
      const int s = (int)(i % TMA_NST);
      // table entries of the next chunk are requested before this chunk is computed
      if (c + gridDim.x < nchunks) locate(c + gridDim.x, nxt);
      const unsigned p = cur.p;
      const bool live = p < npts;
      const int x0 = cur.x0, my = cur.my, mz = cur.mz;
      const float4 q4[2] = {cur.q[0], cur.q[1]};
      // the warp leaves together (its lanes meet again in warp shuffles)
      const bool lost = !mbar_wait_bounded(&full[s], (i / TMA_NST) & 1u);
      if (__any_sync(0xffffffffu, lost)) {
        if (lost) atomicExch(counter + 1, 1u);
        break;
      }
      const float4* st4 = reinterpret_cast<const float4*>(stage + (size_t)s * 6 * TMA_CH) + tid;
      float4 v[6];
#pragma unroll
      for (int comp = 0; comp < 6; ++comp) v[comp] = st4[comp * (TMA_CH / 2)];
      fence_proxy_async_smem();
      mbar_arrive(&empty[s]);
      if constexpr (INV) {
        // every 16 chunks (32 points per thread in FP32) the warp's sums go to FP64; taken by all
        // lanes alike, before the lanes past the last point leave the iteration
        if (cnt == 16) {
          const float w = warp_transpose_sum16(part, lane);
          const int k = transpose_index(lane);
          if ((lane & 1) == 0 && k < NSUM) wsum[warp * NSUM + k] += (double)w;
#pragma unroll
          for (int k2 = 0; k2 < 16; ++k2) part[k2] = 0.f;
          cnt = 0;
        }
        ++cnt;
      }
      if (!live) continue;
      const float ky = nuy * (float)my, kz = nuz * (float)mz;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int x = x0 + j;
        const float kx = nux * (float)x;
        float2 ee[3], hh[3];
#pragma unroll
        for (int comp = 0; comp < 3; ++comp) {
          ee[comp] = j ? make_float2(v[comp].z, v[comp].w) : make_float2(v[comp].x, v[comp].y);
          hh[comp] = j ? make_float2(v[comp + 3].z, v[comp + 3].w) : make_float2(v[comp + 3].x, v[comp + 3].y);
        }
        if constexpr (UPDATE) {
          const Coef<float> q{q4[j].x, q4[j].y, q4[j].z, q4[j].w};
          Apply<float, Coef<float>>::run(q, kx, ky, kz, hh, ee);
#pragma unroll
          for (int comp = 0; comp < 3; ++comp) {
            if (j) {
              v[comp].z = ee[comp].x, v[comp].w = ee[comp].y;
              v[comp + 3].z = hh[comp].x, v[comp + 3].w = hh[comp].y;
            } else {
              v[comp].x = ee[comp].x, v[comp].y = ee[comp].y;
              v[comp + 3].x = hh[comp].x, v[comp + 3].y = hh[comp].y;
            }
          }
        }
        if constexpr (INV) add_densities<float>(part, x == 0 ? 1.f : 2.f, kx, ky, kz, hh, ee, eps, mu);
      }
      if constexpr (UPDATE) {
#pragma unroll
        for (int comp = 0; comp < 6; ++comp)
          __stcs(reinterpret_cast<float4*>(dst + (size_t)comp * comp_stride + p), v[comp]);
      }
    }
    if constexpr (INV) {
      const float w = warp_transpose_sum16(part, lane);
      const int k = transpose_index(lane);
      if ((lane & 1) == 0 && k < NSUM) wsum[warp * NSUM + k] += (double)w;
    }
  }
  if constexpr (INV) {
    __syncthreads();
    __shared__ double grp[32][NSUM];
    rows_finish(reinterpret_cast<const double(*)[NSUM]>(wsum), TMA_CWARPS, grp, partials, counter, record);
  }
}

// ------------------------------------------------------- grouped rows
//
// The same pass with chunks of up to four rows that share every coefficient-table entry: the
// rows (y, z), (-y, z), (y, -z), (-y, -z) of |m_y| = a_y, |m_z| = a_z have the same |k|^2 at each
// x (one row where -y = y, at m = 0 and at the Nyquist index), taken in segments of GRP_L
// columns.  Each consumer thread takes one x of two of the rows, so a table entry is read once
// per four points instead of once per point.  Rows must have even length (16-byte copies).
constexpr int GRP_L = 128;  // columns per segment (TMA_CH / 4)
static_assert(4 * GRP_L == TMA_CH && TMA_CONSUMERS == 2 * GRP_L, "four rows of GRP_L per stage, two per thread");

template <bool INV>
__global__ void __launch_bounds__(TMA_THREADS, 2)
    k_spectral_grp(const float2* __restrict__ src, float2* __restrict__ dst, long comp_stride, GridParams g,
                   const Coef<float>* __restrict__ tab, double* __restrict__ partials, unsigned* __restrict__ counter,
                   double* __restrict__ record) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* stage = reinterpret_cast<float2*>(smraw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smraw + (size_t)TMA_NST * 6 * TMA_CH * sizeof(float2));
  uint64_t* empty = full + TMA_NST;
  double* wsum = reinterpret_cast<double*>(empty + TMA_NST);  // [TMA_CWARPS][NSUM]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mx = g.mx, ny = g.ny, nz = g.nz;
  const int gy = ny / 2 + 1, gz = nz / 2 + 1, nsg = (mx + GRP_L - 1) / GRP_L;
  const unsigned nchunks = (unsigned)gy * (unsigned)gz * (unsigned)nsg;
  // rows of chunk c: ya, yb (= ya when -y is y), za, zb likewise; nr = 1, 2 or 4, row r at
  // (r & ydist ? yb : ya, (ydist ? r >> 1 : r) ? zb : za)
  struct Rows {
    int xs, len, ya, yb, za, zb, nr;
    bool ydist;
  };
  auto rows_of = [&](unsigned c, Rows& o) {
    const unsigned grp = c / (unsigned)nsg;
    const int sg = (int)(c - grp * (unsigned)nsg);
    const int ay = (int)(grp % (unsigned)gy), az = (int)(grp / (unsigned)gy);
    o.xs = sg * GRP_L;
    o.len = min(GRP_L, mx - o.xs);
    o.ya = ay;
    o.yb = (ny - ay) % ny;
    o.za = az;
    o.zb = (nz - az) % nz;
    o.ydist = o.yb != o.ya;
    o.nr = (o.ydist ? 2 : 1) * (o.zb != o.za ? 2 : 1);
  };
  auto row_y = [](const Rows& o, int r) { return (o.ydist && (r & 1)) ? o.yb : o.ya; };
  auto row_z = [](const Rows& o, int r) { return ((o.ydist ? r >> 1 : r) != 0) ? o.zb : o.za; };

  if (tid == 0) {
    for (int s = 0; s < TMA_NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], TMA_CONSUMERS);
    }
    mbar_fence_init();
  }
  if (tid < TMA_CWARPS * NSUM) wsum[tid] = 0.0;
  __syncthreads();

  if (warp == TMA_CWARPS) {
    // ---------------------------------------------------------- producer
    if (lane == 0) {
      unsigned i = 0;
      bool ok = true;
      for (unsigned c = blockIdx.x; c < nchunks; c += gridDim.x, ++i) {
        const int s = (int)(i % TMA_NST);
        if (i >= (unsigned)TMA_NST && !mbar_wait_bounded(&empty[s], ((i / TMA_NST) - 1) & 1u)) {
          ok = false;
          break;
        }
        Rows o;
        rows_of(c, o);
        const uint32_t bytes = (uint32_t)o.len * (uint32_t)sizeof(float2);
        mbar_expect_tx(&full[s], 6u * (uint32_t)o.nr * bytes);
        for (int r = 0; r < o.nr; ++r) {
          const size_t off = ((size_t)row_z(o, r) * ny + row_y(o, r)) * mx + o.xs;
#pragma unroll
          for (int comp = 0; comp < 6; ++comp)
            bulk_g2s(stage + ((size_t)s * 6 + comp) * TMA_CH + r * GRP_L, src + (size_t)comp * comp_stride + off, bytes,
                     &full[s]);
        }
      }
      if (!ok) {
        atomicExch(counter + 1, 1u);
        // let the last copies this block issued land before its shared memory is released
        for (unsigned j = (i > (unsigned)TMA_NST ? i - TMA_NST : 0); j < i; ++j)
          mbar_wait_bounded(&full[j % TMA_NST], (j / TMA_NST) & 1u);
      }
    }
  } else {
    // ---------------------------------------------------------- consumers
    const float eps = g.epsf, mu = g.muf;
    const float nux = g.nuf[0], nuy = g.nuf[1], nuz = g.nuf[2];
    const int xl = tid % GRP_L, pr = tid / GRP_L;  // column in the segment, pair of rows (2 pr, 2 pr + 1)
    float part[INV ? 16 : 1];
#pragma unroll
    for (int k = 0; k < (INV ? 16 : 1); ++k) part[k] = 0.f;
    int cnt = 0;
    unsigned i = 0;
    // this thread's table entry of chunk c (one for all its rows); the rows are recomputed when
    // the chunk is processed, so that only the entry is carried one chunk ahead
    auto entry = [&](unsigned c) {
      Rows o;
      rows_of(c, o);
      const int x = o.xs + (xl < o.len ? xl : 0);
      const int my = signed_index(o.ya, ny), mz = signed_index(o.za, nz);
      return __ldg(reinterpret_cast<const float4*>(tab) + (g.qa[0] * x * x + g.qa[1] * my * my + g.qa[2] * mz * mz));
    };
    float4 qcur = make_float4(0.f, 0.f, 0.f, 0.f), qnxt = qcur;
    if (blockIdx.x < nchunks) qcur = entry(blockIdx.x);
    for (unsigned c = blockIdx.x; c < nchunks; c += gridDim.x, ++i, qcur = qnxt) {
      const int s = (int)(i % TMA_NST);
      if (c + gridDim.x < nchunks) qnxt = entry(c + gridDim.x);
      Rows o;
      rows_of(c, o);
      // the warp leaves together (its lanes meet again in warp shuffles)
      const bool lost = !mbar_wait_bounded(&full[s], (i / TMA_NST) & 1u);
      if (__any_sync(0xffffffffu, lost)) {
        if (lost) atomicExch(counter + 1, 1u);
        break;
      }
      const float2* st = stage + (size_t)s * 6 * TMA_CH;
      float2 v[2][6];
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int comp = 0; comp < 6; ++comp) v[j][comp] = st[comp * TMA_CH + (2 * pr + j) * GRP_L + xl];
      fence_proxy_async_smem();
      mbar_arrive(&empty[s]);
      if constexpr (INV) {
        // every 16 chunks (up to 32 points per thread) the warp's sums go to FP64; taken by all
        // lanes alike, before the lanes with no point leave the iteration
        if (cnt == 16) {
          const float w = warp_transpose_sum16(part, lane);
          const int k = transpose_index(lane);
          if ((lane & 1) == 0 && k < NSUM) wsum[warp * NSUM + k] += (double)w;
#pragma unroll
          for (int k2 = 0; k2 < 16; ++k2) part[k2] = 0.f;
          cnt = 0;
        }
        ++cnt;
      }
      if (xl >= o.len) continue;
      const int x = o.xs + xl;
      const float kx = nux * (float)x;
      const Coef<float> q{qcur.x, qcur.y, qcur.z, qcur.w};
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int r = 2 * pr + j;
        if (r >= o.nr) break;
        const int y = row_y(o, r), z = row_z(o, r);
        const float ky = nuy * (float)signed_index(y, ny), kz = nuz * (float)signed_index(z, nz);
        float2 ee[3] = {v[j][0], v[j][1], v[j][2]}, hh[3] = {v[j][3], v[j][4], v[j][5]};
        Apply<float, Coef<float>>::run(q, kx, ky, kz, hh, ee);
        if constexpr (INV) add_densities<float>(part, x == 0 ? 1.f : 2.f, kx, ky, kz, hh, ee, eps, mu);
        float2* d = dst + ((size_t)z * ny + y) * mx + x;
#pragma unroll
        for (int comp = 0; comp < 3; ++comp) {
          __stcs(d + (size_t)comp * comp_stride, ee[comp]);
          __stcs(d + (size_t)(comp + 3) * comp_stride, hh[comp]);
        }
      }
    }
    if constexpr (INV) {
      const float w = warp_transpose_sum16(part, lane);
      const int k = transpose_index(lane);
      if ((lane & 1) == 0 && k < NSUM) wsum[warp * NSUM + k] += (double)w;
    }
  }
  if constexpr (INV) {
    __syncthreads();
    __shared__ double grp[32][NSUM];
    rows_finish(reinterpret_cast<const double(*)[NSUM]>(wsum), TMA_CWARPS, grp, partials, counter, record);
  }
}

}  // namespace mx

// CUDA kernels of the exponential-integrator Fourier pseudospectral step
// (Wang & Jiang, arXiv 2210.06232, Alg. 1 and Alg. 2) for sm_103a.
//
// Data layout in HBM
//   physical fields : 6 components (E_x, E_y, E_z, H_x, H_y, H_z), each
//                     [Nz][Ny][Nx] real, x fastest (the paper's ordering).
//   spectrum        : 6 components, each [Nz][Ny][Mx] complex, Mx = Nx/2.
//                     Column kx = 0 is "packed": its real part carries the
//                     kx = 0 plane and its imaginary part the kx = Nx/2
//                     (Nyquist) plane.  Both planes have wavenumber k_x = 0
//                     in the scheme (the Nyquist entry of Omega_x is 0,
//                     Sec. 2.3), both are transforms of real rows, and the
//                     per-k update commutes with the packing (it is the
//                     same real-linear map on both planes and preserves
//                     Hermitian symmetry), so the y/z transforms, the update
//                     and the invariant sums act on the packed column as on
//                     any other.  The spectrum therefore holds exactly as
//                     many reals as the physical fields.
#pragma once
#include <type_traits>

#include "mx_fft.cuh"
#include "mx_tma.cuh"

namespace mx {

// Grid description shared by all kernels.
struct GridParams {
  int nx, ny, nz, mx;   // mx = nx / 2
  double nu[3];         // nu_w = 2 pi / (w_R - w_L)
  int qa[3];            // |k|^2 = s0 * (qa0 mx^2 + qa1 my^2 + qa2 mz^2) when commensurate
  double s0;
  double eps, mu;
  double c;             // 1 / sqrt(eps mu)
  double zh, ze;        // sqrt(eps / mu), sqrt(mu / eps)
  float nuf[3], epsf, muf;  // FP32 copies for the FP32 kernels (no conversion on the FP64 pipe)
  // tries of the fused z pass's waits for its tiles (MBAR_TRIES unless a test lowers it to make
  // them give up; the wait for a copy still in flight when a block leaves keeps the full bound)
  unsigned wait_tries = 1u << 24;
  // factor of the fused z pass's output (its inverse transforms carry no 1/nz): 1 where the
  // inverse x pass applies the whole normalisation (literal form), 1/nz where the output stays
  // the state between steps (xy-resident form)
  double zscale = 1.0;
  float zscalef = 1.0f;
};
// Material constants of a grid (host side; after nu is set).
inline void set_material(GridParams& g, double eps, double mu) {
  g.eps = eps;
  g.mu = mu;
  g.c = 1.0 / sqrt(eps * mu);
  g.zh = sqrt(eps / mu);
  g.ze = sqrt(mu / eps);
  for (int w = 0; w < 3; ++w) g.nuf[w] = (float)g.nu[w];
  g.epsf = (float)eps;
  g.muf = (float)mu;
}
// eps, mu and nu_w in the kernel's arithmetic type.
template <typename T> struct GP;
template <> struct GP<float> {
  __device__ __forceinline__ static float zscale(const GridParams& g) { return g.zscalef; }
  __device__ __forceinline__ static float eps(const GridParams& g) { return g.epsf; }
  __device__ __forceinline__ static float mu(const GridParams& g) { return g.muf; }
  __device__ __forceinline__ static float nu(const GridParams& g, int w) { return g.nuf[w]; }
};
template <> struct GP<double> {
  __device__ __forceinline__ static double zscale(const GridParams& g) { return g.zscale; }
  __device__ __forceinline__ static double eps(const GridParams& g) { return g.eps; }
  __device__ __forceinline__ static double mu(const GridParams& g) { return g.mu; }
  __device__ __forceinline__ static double nu(const GridParams& g, int w) { return g.nu[w]; }
};

// Per-|k|^2 coefficients of the exact exponential (Prop. 2.1-2.2 rewritten
// with k rather than k/|k|):
//   H' = cos(th) H + al (k.H) k - i bh (k x E)
//   E' = cos(th) E + al (k.E) k + i be (k x H)
// th = c |k| t, al = (1 - cos th)/|k|^2, bh = sin(th)/|k| sqrt(eps/mu),
// be = sin(th)/|k| sqrt(mu/eps).  At k = 0: (1, 0, 0, 0), the identity.
template <typename T> struct Coef { T c, al, bh, be; };
// Double-single coefficients (value = hi + lo) for the repeated-step FP32
// form: the same map is applied every step, so a rounded coefficient would
// bias every step the same way.
struct CoefHL { float c, c_l, al, al_l, bh, bh_l, be, be_l; };

__device__ __forceinline__ int signed_index(int i, int n) {
  // DFT bin -> wavenumber index, Nyquist bin mapped to 0 (Omega_w, Sec. 2.3)
  return (i < n / 2) ? i : ((i == n / 2) ? 0 : i - n);
}

// Number of accumulated invariant sums per record.
constexpr int NSUM = 15;

// --------------------------------------------------------- per-point update

template <typename T, typename CoefT> struct Apply;

template <typename T> struct Apply<T, Coef<T>> {
  __device__ __forceinline__ static void run(const Coef<T>& q, T kx, T ky, T kz, cx<T>* h, cx<T>* e) {
    using C = cx<T>;
    C kh = C{kx * h[0].x + ky * h[1].x + kz * h[2].x, kx * h[0].y + ky * h[1].y + kz * h[2].y};
    C ke = C{kx * e[0].x + ky * e[1].x + kz * e[2].x, kx * e[0].y + ky * e[1].y + kz * e[2].y};
    C kxe[3] = {C{ky * e[2].x - kz * e[1].x, ky * e[2].y - kz * e[1].y},
                C{kz * e[0].x - kx * e[2].x, kz * e[0].y - kx * e[2].y},
                C{kx * e[1].x - ky * e[0].x, kx * e[1].y - ky * e[0].y}};
    C kxh[3] = {C{ky * h[2].x - kz * h[1].x, ky * h[2].y - kz * h[1].y},
                C{kz * h[0].x - kx * h[2].x, kz * h[0].y - kx * h[2].y},
                C{kx * h[1].x - ky * h[0].x, kx * h[1].y - ky * h[0].y}};
    const T kv[3] = {kx, ky, kz};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const T ak = q.al * kv[i];
      // -i * bh * kxe = (bh * kxe.y, -bh * kxe.x)
      h[i] = C{q.c * h[i].x + ak * kh.x + q.bh * kxe[i].y, q.c * h[i].y + ak * kh.y - q.bh * kxe[i].x};
      // +i * be * kxh = (-be * kxh.y, be * kxh.x)
      e[i] = C{q.c * e[i].x + ak * ke.x - q.be * kxh[i].y, q.c * e[i].y + ak * ke.y + q.be * kxh[i].x};
    }
  }
};

template <> struct Apply<float, CoefHL> {
  __device__ __forceinline__ static void run(const CoefHL& q, float kx, float ky, float kz, float2* h, float2* e) {
    using C = float2;
    C kh = C{kx * h[0].x + ky * h[1].x + kz * h[2].x, kx * h[0].y + ky * h[1].y + kz * h[2].y};
    C ke = C{kx * e[0].x + ky * e[1].x + kz * e[2].x, kx * e[0].y + ky * e[1].y + kz * e[2].y};
    C kxe[3] = {C{ky * e[2].x - kz * e[1].x, ky * e[2].y - kz * e[1].y},
                C{kz * e[0].x - kx * e[2].x, kz * e[0].y - kx * e[2].y},
                C{kx * e[1].x - ky * e[0].x, kx * e[1].y - ky * e[0].y}};
    C kxh[3] = {C{ky * h[2].x - kz * h[1].x, ky * h[2].y - kz * h[1].y},
                C{kz * h[0].x - kx * h[2].x, kz * h[0].y - kx * h[2].y},
                C{kx * h[1].x - ky * h[0].x, kx * h[1].y - ky * h[0].y}};
    const float kv[3] = {kx, ky, kz};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      // small corrections first, then the leading products
      const float akh = q.al * kv[i], akl = q.al_l * kv[i];
      float hx = q.c_l * h[i].x + akl * kh.x + q.bh_l * kxe[i].y;
      float hy = q.c_l * h[i].y + akl * kh.y - q.bh_l * kxe[i].x;
      hx = fmaf(q.c, h[i].x, fmaf(akh, kh.x, fmaf(q.bh, kxe[i].y, hx)));
      hy = fmaf(q.c, h[i].y, fmaf(akh, kh.y, fmaf(-q.bh, kxe[i].x, hy)));
      float ex = q.c_l * e[i].x + akl * ke.x - q.be_l * kxh[i].y;
      float ey = q.c_l * e[i].y + akl * ke.y + q.be_l * kxh[i].x;
      ex = fmaf(q.c, e[i].x, fmaf(akh, ke.x, fmaf(-q.be, kxh[i].y, ex)));
      ey = fmaf(q.c, e[i].y, fmaf(akh, ke.y, fmaf(q.be, kxh[i].x, ey)));
      h[i] = C{hx, hy};
      e[i] = C{ex, ey};
    }
  }
};

// Coefficients computed directly (no table): FP64 arithmetic per point.
template <typename T, typename CoefT> __device__ __forceinline__ CoefT coef_direct(double k2, double t, const GridParams& g);
// FP32 coefficients: the half phase th/2 = c |k| t / 2 is formed and reduced to
// [-pi, pi] in FP64 (Cody-Waite reduction with 2 pi = hi + lo), so that large
// c |k| t lose nothing; sin and cos of the reduced half angle are then taken in
// FP32, which gives the FP32 coefficients to a few FP32 ulps:
//   cos th = 1 - 2 sin^2(th/2), sin th = 2 sin(th/2) cos(th/2),
//   (1 - cos th)/|k|^2 = 2 sin^2(th/2) / |k|^2.
// The same from hk = (0.5 c) |k| and |k|, |k|^2 in FP32 (zero: k = 0), for tables recomputed every
// step from precomputed hk: the operations past the square root, in the same order.
__device__ __forceinline__ Coef<float> coef_from_hk(double hk, float kabsf, float k2f, bool zero, double t,
                                                    const GridParams& g) {
  if (zero) return Coef<float>{1.f, 0.f, 0.f, 0.f};
  const double hp = hk * t;
  const double n = rint(hp * 0.15915494309189533577);  // 1 / (2 pi)
  const double r = fma(-n, 2.4492935982947064e-16, fma(-n, 6.283185307179586, hp));
  float sh, ch;
  sincosf((float)r, &sh, &ch);
  const float s = 2.f * sh * ch, sh2 = sh * sh;
  const float b = s / kabsf;
  return Coef<float>{1.f - 2.f * sh2, 2.f * sh2 / k2f, b * (float)g.zh, b * (float)g.ze};
}
template <> __device__ __forceinline__ Coef<float> coef_direct<float, Coef<float>>(double k2, double t, const GridParams& g) {
  if (k2 == 0.0) return Coef<float>{1.f, 0.f, 0.f, 0.f};
  const double kabs = sqrt(k2);
  return coef_from_hk(0.5 * g.c * kabs, (float)kabs, (float)k2, false, t, g);
}
template <> __device__ __forceinline__ Coef<double> coef_direct<double, Coef<double>>(double k2, double t, const GridParams& g) {
  if (k2 == 0.0) return Coef<double>{1.0, 0.0, 0.0, 0.0};
  double kabs = sqrt(k2), th = g.c * kabs * t, s, c;
  sincos(th, &s, &c);
  double sh = sin(0.5 * th);
  double al = 2.0 * sh * sh / k2, b = s / kabs;
  return Coef<double>{c, al, b * sqrt(g.eps / g.mu), b * sqrt(g.mu / g.eps)};
}
__device__ __forceinline__ void split_hl(double v, float& hi, float& lo) {
  hi = (float)v;
  lo = (float)(v - (double)hi);
}
template <> __device__ __forceinline__ CoefHL coef_direct<float, CoefHL>(double k2, double t, const GridParams& g) {
  CoefHL r;
  if (k2 == 0.0) {
    r.c = 1.f; r.c_l = r.al = r.al_l = r.bh = r.bh_l = r.be = r.be_l = 0.f;
    return r;
  }
  double kabs = sqrt(k2), th = g.c * kabs * t, s, c;
  sincos(th, &s, &c);
  double sh = sin(0.5 * th);
  double al = 2.0 * sh * sh / k2, b = s / kabs;
  split_hl(c, r.c, r.c_l);
  split_hl(al, r.al, r.al_l);
  split_hl(b * sqrt(g.eps / g.mu), r.bh, r.bh_l);
  split_hl(b * sqrt(g.mu / g.eps), r.be, r.be_l);
  return r;
}

// Table of coefficients for q = 0 .. nq-1, |k|^2 = s0 q, at time t.
template <typename T, typename CoefT>
__global__ void k_coef_table(CoefT* __restrict__ tab, int nq, GridParams g, double t) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < nq) tab[q] = coef_direct<T, CoefT>(g.s0 * (double)q, t, g);
}

// ------------------------------------------------------- invariant densities
//
// Parseval on the unnormalised DFT: <u, v>_N = (1/N_S^2) sum_k conj(u_k) v_k.
// Spectral forms of the Sec. 4 invariants (D_w -> i k_w, D -> i k x):
//   s0  mu|H|^2 + eps|E|^2                       -> E1 = s0/(2 N_S^2)
//   s1  |k x E|^2/mu + |k x H|^2/eps             -> E2 = s1/(2 N_S^2)
//   s2+w  k_w^2 * s0-density                     -> E3[w]
//   s5+w  k_w^2 * s1-density                     -> E4[w]
//   s8  k.(Re H x Im H)/eps + k.(Re E x Im E)/mu -> H1 = s8/N_S^2
//   s9  k.(Re w x Im w)/(eps mu^2) + k.(Re v x Im v)/(mu eps^2),
//       w = k x E, v = k x H                     -> H2 = s9/N_S^2
//   s10+w k_w Im(conj(H).E)                      -> M1[w] = -s/N_S^2, M2 = -M1
//   s13 eps^2 |k.E|^2,  s14 mu^2 |k.H|^2         -> ||div||_N = sqrt(s)/N_S
// Two identities for real k shorten the arithmetic:
//   |k x U|^2 = |k|^2 |U|^2 - |k.U|^2            (Lagrange)
//   k.((k x a) x (k x b)) = |k|^2 k.(a x b)       ((k x a) x (k x b) = (k.(a x b)) k)
// Each density is multiplied by the Hermitian weight of its half-spectrum
// column (1 for the packed column 0, 2 otherwise).
template <typename T>
__device__ __forceinline__ void add_densities(T* acc, T w, T kx, T ky, T kz, const cx<T>* h, const cx<T>* e, T eps, T mu) {
  const T h2 = h[0].x * h[0].x + h[0].y * h[0].y + h[1].x * h[1].x + h[1].y * h[1].y + h[2].x * h[2].x + h[2].y * h[2].y;
  const T e2 = e[0].x * e[0].x + e[0].y * e[0].y + e[1].x * e[1].x + e[1].y * e[1].y + e[2].x * e[2].x + e[2].y * e[2].y;
  const T kEr = kx * e[0].x + ky * e[1].x + kz * e[2].x, kEi = kx * e[0].y + ky * e[1].y + kz * e[2].y;
  const T kHr = kx * h[0].x + ky * h[1].x + kz * h[2].x, kHi = kx * h[0].y + ky * h[1].y + kz * h[2].y;
  const T kE2 = kEr * kEr + kEi * kEi, kH2 = kHr * kHr + kHi * kHi;
  const T kx2 = kx * kx, ky2 = ky * ky, kz2 = kz * kz;
  const T k2 = kx2 + ky2 + kz2;
  // k . (Re U x Im U)
  const T ch = kx * (h[1].x * h[2].y - h[2].x * h[1].y) + ky * (h[2].x * h[0].y - h[0].x * h[2].y) +
               kz * (h[0].x * h[1].y - h[1].x * h[0].y);
  const T ce = kx * (e[1].x * e[2].y - e[2].x * e[1].y) + ky * (e[2].x * e[0].y - e[0].x * e[2].y) +
               kz * (e[0].x * e[1].y - e[1].x * e[0].y);
  // material constants (loop invariants of every caller)
  const T ie = (T)1 / eps, im = (T)1 / mu;
  const T c9e = ie * im * im, c9h = im * ie * ie, eps2 = eps * eps, mu2 = mu * mu;
  const T d0 = w * (mu * h2 + eps * e2);
  const T d1 = w * ((k2 * e2 - kE2) * im + (k2 * h2 - kH2) * ie);
  const T mim = w * (h[0].x * e[0].y - h[0].y * e[0].x + h[1].x * e[1].y - h[1].y * e[1].x + h[2].x * e[2].y - h[2].y * e[2].x);
  acc[0] += d0;
  acc[1] += d1;
  acc[2] += kx2 * d0;
  acc[3] += ky2 * d0;
  acc[4] += kz2 * d0;
  acc[5] += kx2 * d1;
  acc[6] += ky2 * d1;
  acc[7] += kz2 * d1;
  acc[8] += w * (ch * ie + ce * im);
  acc[9] += (w * k2) * (ce * c9e + ch * c9h);
  acc[10] += kx * mim;
  acc[11] += ky * mim;
  acc[12] += kz * mim;
  acc[13] += (w * eps2) * kE2;
  acc[14] += (w * mu2) * kH2;
}

// Transpose reduction of 16 values across a warp (value 15 is padding): after
// levels with lane offsets 16, 8, 4, 2 each lane keeps one value index,
// (lane >> 1) & 15, summed over its 16-lane group; the final xor-1 exchange
// completes the sum over all 32 lanes.  16 shuffles instead of 16 x 5, and
// the addition order is fixed.
template <typename T>
__device__ __forceinline__ T warp_transpose_sum16(T* v, int lane) {
  // level 16: 8 exchanges
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const bool up = lane & 16;
    const T send = up ? v[j] : v[j + 8];
    const T recv = __shfl_xor_sync(0xffffffffu, send, 16);
    v[j] = (up ? v[j + 8] : v[j]) + recv;
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const bool up = lane & 8;
    const T send = up ? v[j] : v[j + 4];
    const T recv = __shfl_xor_sync(0xffffffffu, send, 8);
    v[j] = (up ? v[j + 4] : v[j]) + recv;
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const bool up = lane & 4;
    const T send = up ? v[j] : v[j + 2];
    const T recv = __shfl_xor_sync(0xffffffffu, send, 4);
    v[j] = (up ? v[j + 2] : v[j]) + recv;
  }
  {
    const bool up = lane & 2;
    const T send = up ? v[0] : v[1];
    const T recv = __shfl_xor_sync(0xffffffffu, send, 2);
    v[0] = (up ? v[1] : v[0]) + recv;
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}
// Value index held by `lane` after warp_transpose_sum16.
__device__ __forceinline__ int transpose_index(int lane) {
  return ((lane & 16) ? 8 : 0) + ((lane & 8) ? 4 : 0) + ((lane & 4) ? 2 : 0) + ((lane & 2) ? 1 : 0);
}

// Grid reduction of NSUM FP64 sums.  Every block hands in its totals as rows, one per warp
// (rows[w][k], w < nrows), summed in warp order; the last block to finish sums the blocks'
// partials in a fixed order and writes the record.  The counter must be zero on entry; the last
// block resets it.  The order is that of a warp-wide tree over 32 consecutive "lanes" j (lane j
// holding blocks j, j + blockDim.x, ...), then the groups of 32 in order, each tree summed by one
// thread per (sum, group): on a part whose FP64 pipe is narrow, that is a few warp instructions
// where a shuffle tree in every warp costs hundreds.  `grp` (shared, 32 rows; it may be `rows`)
// holds the groups' sums in the last block.
__device__ __forceinline__ void rows_finish(const double (*rows)[NSUM], int nrows, double (*grp)[NSUM],
                                            double* __restrict__ partials,
                                            unsigned* __restrict__ counter, double* __restrict__ record) {
  __shared__ bool last;
  const int nblocks = gridDim.x * gridDim.y;
  const int bid = blockIdx.y * gridDim.x + blockIdx.x;
  if (threadIdx.x < NSUM) {
    double v = 0.0;
    for (int w = 0; w < nrows; ++w) v += rows[w][threadIdx.x];
    partials[(size_t)bid * NSUM + threadIdx.x] = v;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == (unsigned)(nblocks - 1));
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int ngrp = (int)((blockDim.x + 31) >> 5);
  const int q = threadIdx.x, w = q / NSUM, k = q - w * NSUM;
  if (w < ngrp) {
    // the first block of every lane in 32 independent loads issued together (a loop per lane would
    // wait for each L2 round trip in turn), then the blocks past blockDim.x, added in the same order
    double s[32];
    const int b0 = 32 * w;
#pragma unroll
    for (int l = 0; l < 32; ++l) s[l] = b0 + l < nblocks ? __ldcg(partials + (size_t)(b0 + l) * NSUM + k) : 0.0;
    for (int r = (int)blockDim.x; b0 + r < nblocks; r += (int)blockDim.x)
#pragma unroll
      for (int l = 0; l < 32; ++l)
        if (b0 + r + l < nblocks) s[l] += __ldcg(partials + (size_t)(b0 + r + l) * NSUM + k);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int l = 0; l < o; ++l) s[l] += s[l + o];
    grp[w][k] = s[0];
  }
  __syncthreads();
  if (threadIdx.x < NSUM) {
    double v = 0.0;
    for (int g = 0; g < ngrp; ++g) v += grp[g][threadIdx.x];
    record[threadIdx.x] = v;
  }
  if (threadIdx.x == 0) *counter = 0u;
}

// Block-wide FP64 reduction of NSUM values held by every thread (a warp tree, then the warps in
// order), then the grid reduction of rows_finish.
__device__ __forceinline__ void reduce_and_finish(double* acc, double* __restrict__ partials, unsigned* __restrict__ counter,
                                                  double* __restrict__ record) {
  __shared__ double red[32][NSUM];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int i = 0; i < NSUM; ++i) {
    double v = acc[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][i] = v;
  }
  __syncthreads();
  rows_finish(red, nwarps, red, partials, counter, record);
}

// ----------------------------------------------------------------- x passes
//
// Real rows of length Nx = 2M -> packed half spectrum of M complex values.
// z_n = x_{2n} + i x_{2n+1}, Z = DFT_M(z), then for k = 1..M-1
//   X_k = (Z_k + conj Z_{M-k})/2 + W_N^k (Z_k - conj Z_{M-k})/(2i),
// and X_0 = Re Z_0 + Im Z_0, X_M = Re Z_0 - Im Z_0 packed as (X_0, X_M).
// Rows 0 .. 3R-1 come from `in_e`, rows 3R .. 6R-1 from `in_h` (R = Ny Nz).
// Persistent: a block loads the twiddles once and loops over groups of TY rows.
template <typename T, int M, int E, int TY>
__global__ void __launch_bounds__((M / E) * TY) k_x_r2c(const T* __restrict__ in_e, const T* __restrict__ in_h,
                                                        cx<T>* __restrict__ out, long rows3, long nrows,
                                                        const twv<T>* __restrict__ twg) {
  using C = cx<T>;
  constexpr int P = M / E;
  constexpr int PITCH = line_buf(M);
  constexpr int LB = line_bar(P, 0);  // lines within a warp synchronise with __syncwarp
  extern __shared__ __align__(16) unsigned char smraw[];
  // twiddles: exp(-2 pi i k / (2M)) for k < M (packing), then the stage-major table of the M-point FFT
  twv<T>* tw = reinterpret_cast<twv<T>*>(smraw);
  C* sm = reinterpret_cast<C*>(tw + 2 * M);
  for (int i = threadIdx.x; i < M + tw_len(M, E); i += blockDim.x) tw[i] = twg[i];
  const int t = threadIdx.x % P, ly = threadIdx.x / P;
  C* line = sm + ly * PITCH;
  const long ngroups = (nrows + TY - 1) / TY;
  // register double buffer: the next group's row values are requested before this group is transformed
  auto load_group = [&](long grp, C* dst) {
    const long row = grp * TY + ly;
    const bool ok = grp < ngroups && row < nrows;
    const T* src = ok ? (row < rows3 ? in_e + row * (2L * M) : in_h + (row - rows3) * (2L * M)) : nullptr;
#pragma unroll
    for (int m = 0; m < E; ++m) dst[m] = ok ? *reinterpret_cast<const C*>(src + 2 * (t + P * m)) : C{0, 0};
  };
  C nxt[E];
  load_group(blockIdx.x, nxt);
  __syncthreads();  // twiddles
  for (long grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const long row = grp * TY + ly;
    const bool ok = row < nrows;
    C v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = nxt[m];
    load_group(grp + gridDim.x, nxt);
    fft_bar<LB>();  // previous group's readers of `line` are done
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
          C a = cadd(z, zp), d = csub(z, zp);  // 2A, 2iB
          C b = C{d.y, -d.x};                   // 2B = -i * d
          C wb = twmul<-1>(b, tw[k]);
          r = C{(T)0.5 * (a.x + wb.x), (T)0.5 * (a.y + wb.y)};
        }
        dst[k] = r;
      }
    }
  }
}

// Packed half spectrum -> real rows, scaled by `scale`.
//   Z'_k = (X_k + conj X_{M-k}) + i conj(W_N^k) (X_k - conj X_{M-k}),
//   Z'_0 = (X_0 + X_M) + i (X_0 - X_M);  z' = unnormalised IDFT_M(Z') = N z.
template <typename T, int M, int E, int TY>
__global__ void __launch_bounds__((M / E) * TY) k_x_c2r(const cx<T>* __restrict__ in, T* __restrict__ out_e,
                                                        T* __restrict__ out_h, long rows3, long nrows,
                                                        const twv<T>* __restrict__ twg, double scale) {
  using C = cx<T>;
  constexpr int P = M / E;
  constexpr int PITCH = line_buf(M);
  constexpr int LB = line_bar(P, 0);
  extern __shared__ __align__(16) unsigned char smraw[];
  twv<T>* tw = reinterpret_cast<twv<T>*>(smraw);  // as in k_x_r2c
  C* sm = reinterpret_cast<C*>(tw + 2 * M);
  for (int i = threadIdx.x; i < M + tw_len(M, E); i += blockDim.x) tw[i] = twg[i];
  const int t = threadIdx.x % P, ly = threadIdx.x / P;
  C* line = sm + ly * PITCH;
  const KC<T> sc(scale);  // 1/(Nx Ny Nz), hi + lo in FP32
  const long ngroups = (nrows + TY - 1) / TY;
  auto load_group = [&](long grp, C* dst) {
    const long row = grp * TY + ly;
    const bool ok = grp < ngroups && row < nrows;
    const C* src = ok ? in + row * M : nullptr;
#pragma unroll
    for (int m = 0; m < E; ++m) dst[m] = ok ? src[t + P * m] : C{0, 0};
  };
  C nxt[E];
  load_group(blockIdx.x, nxt);
  __syncthreads();  // twiddles
  for (long grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const long row = grp * TY + ly;
    const bool ok = row < nrows;
    fft_bar<LB>();  // previous group's readers of `line` are done
#pragma unroll
    for (int m = 0; m < E; ++m) line[xoff(t + P * m, 1)] = nxt[m];
    load_group(grp + gridDim.x, nxt);
    fft_bar<LB>();
    C v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int k = t + P * m;
      C x = line[xoff(k, 1)];
      if (k == 0) {
        v[m] = C{x.x + x.y, x.x - x.y};
      } else {
        C xp = cconj(line[xoff(M - k, 1)]);
        C s = cadd(x, xp), d = csub(x, xp);
        C wd = twmul<+1>(d, tw[k]);
        v[m] = C{s.x - wd.y, s.y + wd.x};  // s + i * wd
      }
    }
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

// -------------------------------------------------------- strided complex FFT
//
// data viewed as [outer][N][inner] complex; transforms every (outer, i)
// line of N along the middle axis (y: inner = Mx; z: inner = Ny Mx).
// Tile = TX consecutive inner indices x P threads per line.  Persistent over
// tiles (ntile_in tiles per outer index).
template <typename T, int N, int E, int TX, int DIR>
__global__ void __launch_bounds__((N / E) * TX) k_fft_strided(cx<T>* __restrict__ data, long inner, long outer,
                                                              const twv<T>* __restrict__ twg) {
  using C = cx<T>;
  constexpr int P = N / E;
  extern __shared__ __align__(16) unsigned char smraw[];
  twv<T>* tw = reinterpret_cast<twv<T>*>(smraw);  // stage-major table of (N, E)
  C* sm = reinterpret_cast<C*>(tw + N);
  for (int i = threadIdx.x; i < tw_len(N, E); i += blockDim.x) tw[i] = twg[i];
  const int x = threadIdx.x % TX, t = threadIdx.x / TX;
  // tile indices fit in 32 bits (checked by the launcher): 32-bit division per tile
  const unsigned ntile_in = (unsigned)((inner + TX - 1) / TX);
  const unsigned ntiles = ntile_in * (unsigned)outer;
  const long pstride = (long)P * inner;  // between a thread's E positions
  auto line_base = [&](unsigned tile, bool& ok) {
    const unsigned o = tile / ntile_in;
    const long col = (long)(tile - o * ntile_in) * TX + x;
    ok = tile < ntiles && col < inner;
    return data + (long)o * N * inner + col + (long)t * inner;
  };
  auto load_tile = [&](unsigned tile, C* dst) {
    bool ok;
    const C* b = line_base(tile, ok);
#pragma unroll
    for (int m = 0; m < E; ++m) dst[m] = ok ? b[m * pstride] : C{0, 0};
  };
  C nxt[E];
  load_tile(blockIdx.x, nxt);
  for (unsigned tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    bool ok;
    C* base = line_base(tile, ok);
    C v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = nxt[m];
    // in place: the next tile is another set of columns, never written by this tile
    load_tile(tile + gridDim.x, nxt);
    __syncthreads();  // twiddles
    line_fft<T, N, E, DIR>(v, sm + x, TX, t, tw);
    if (ok) {
#pragma unroll
      for (int m = 0; m < E; ++m) base[m * pstride] = v[m];
    }
  }
}

// ------------------------------------------------------- fused z pass (literal)
//
// For the literal form: the spectrum after the x and y passes is transformed
// along z, multiplied by the exponential and transformed back, with all six
// components of a tile (fixed ky, TX consecutive kx, every kz) held in
// registers and transformed one after another through one exchange buffer (two
// at a time with TMAP, see below):
// thread (x, t) owns positions t + P*m of its column for the six components,
// which are exactly the frequencies its forward transforms produce and its
// inverse transforms consume (mx_fft.cuh).  One read and one write of the
// spectrum replace three passes (z forward, update, z inverse).
// With TMAP a tile arrives by tensor copy in an input stage, in boxes of three
// components; the results leave through an output stage and tensor stores.
// Components are transformed in threes (ZTile::TRIP; pairs where the buffers do
// not fit), which cuts the barriers and shares each twiddle load.  With
// triplets, once the tile is read the upper half of the input stage takes the
// next tile's upper boxes at once, its lower half holds the coefficient-table
// entries of this tile (cp.async, during the forward transforms) and takes the
// next tile's lower boxes after the update: the next tile's copies run during
// the whole of this tile's work instead of the inverse transforms only.  Both
// directions of transforms exchange through six unpadded, row-swizzled buffers
// in the output stage (once the previous store has read it), alternating
// between two triplets so that an exchange has a single barrier.  Without
// triplets the stage holds the coefficients and a second exchange buffer, and
// the next tile's copies are issued after the update.  Invariants of the updated state are summed per thread in T
// over a tile, then per warp in a compensated (Kahan) pair of T in shared
// memory, converted to FP64 at the end: no FP64 arithmetic in the loop, where
// an FP64 instruction costs the pipe as much with one active lane as with 32.
template <typename T, int N, int E, int TX>
struct ZTile {
  static constexpr int P = N / E;
  static constexpr int NZC = (N + 255) / 256;  // boxes of the tensor copy along z
  static constexpr int ZC = N / NZC;           // z rows per box
  static constexpr int NB = 2 * NZC;           // boxes per tile: along z, then two halves of three components
  static constexpr size_t stage_bytes = (size_t)6 * N * TX * sizeof(cx<T>);
  static constexpr int NT = P * TX;  // threads
  static constexpr int NL = 1;       // components per exchange buffer of this size (pairs: see above)
  static constexpr size_t exch_bytes = (size_t)NL * strided_rows(N) * TX * sizeof(cx<T>);
  static constexpr size_t tw_bytes = (size_t)N * sizeof(twv<T>);
  // unpadded exchange buffer with swizzled rows (swz_rows): XK + 1 rows of TX values per 128-byte line
  static constexpr size_t xbuf_bytes = (size_t)N * TX * sizeof(cx<T>);
  static constexpr int XK = TX * (int)sizeof(cx<T>) >= 128 ? 0 : 128 / (TX * (int)sizeof(cx<T>)) - 1;
  // staged coefficient entries (32 bytes each): one per column and |m_z| = 0 .. N/2 - 1 (the entry
  // depends on m_z^2 only, and the Nyquist plane has m_z = 0), shared by the threads that need it
  static constexpr int NA = N / 2;
  static constexpr size_t coef_bytes = (size_t)NA * TX * 32;
  // components in threes: both directions exchange through six buffers in the output stage, the
  // coefficients fill (part of) the input stage's lower half
  static constexpr bool TRIP = XK <= 7 && N % (XK + 1) == 0 && 2 * coef_bytes <= stage_bytes &&
                               6 * xbuf_bytes <= stage_bytes;
  static constexpr size_t smem_tma = TRIP ? 2 * stage_bytes + tw_bytes + 16 : 2 * stage_bytes + tw_bytes + exch_bytes + 16;
  // static shared memory of the kernel: compensated sums and the block reduction
  static constexpr size_t static_bytes = (size_t)2 * 32 * NSUM * sizeof(T) + (size_t)32 * NSUM * sizeof(double) + 128;
  // element (comp c, z, column x) of the stage: z box z / ZC, laid out [c][z % ZC][x] (the box of
  // components c / 3 and z box b is the (2 b + c / 3)-th NB-th of the stage)
  __device__ __forceinline__ static int stage_index(int c, int z, int x) {
    return (z / ZC) * (6 * ZC * TX) + (c * ZC + z % ZC) * TX + x;
  }
};

// Thread 0: the tensor stores of tile `tile` from the output stage (one bulk group).
template <typename T, int N, int E, int TX>
__device__ __forceinline__ void z_tile_store(const void* tmap, const cx<T>* ostage, long tile, int ntx) {
  using ZT = ZTile<T, N, E, TX>;
  const int y = (int)((unsigned)tile / (unsigned)ntx);
  const int x0 = (int)((unsigned)tile - (unsigned)y * (unsigned)ntx) * TX;
#pragma unroll
  for (int b = 0; b < ZT::NB; ++b)
    tma_store_4d(tmap, reinterpret_cast<const unsigned char*>(ostage) + b * (ZT::stage_bytes / ZT::NB), 2 * x0, y,
                 (b >> 1) * ZT::ZC, 3 * (b & 1));
  bulk_commit();
}

// Thread 0: tensor copies of boxes B0 .. B1 - 1 of tile `tile` into the stage, completing on `full`
// (EXPECT: announce the whole tile's bytes, with the first copies of the tile).
template <typename T, int N, int E, int TX, int B0 = 0, int B1 = ZTile<T, N, E, TX>::NB, bool EXPECT = true>
__device__ __forceinline__ void z_tile_copy(const void* tmap, cx<T>* stage, uint64_t* full, long tile, int ntx) {
  using ZT = ZTile<T, N, E, TX>;
  const int y = (int)((unsigned)tile / (unsigned)ntx);
  const int x0 = (int)((unsigned)tile - (unsigned)y * (unsigned)ntx) * TX;
  if constexpr (EXPECT) mbar_expect_tx(full, (uint32_t)ZT::stage_bytes);
#pragma unroll
  for (int b = B0; b < B1; ++b)
    tma_load_4d(reinterpret_cast<unsigned char*>(stage) + b * (ZT::stage_bytes / ZT::NB), tmap, 2 * x0, y,
                (b >> 1) * ZT::ZC, 3 * (b & 1), full);
}

// Forward and inverse z transforms of NL components in the fused pass: in FP32 the exactly
// invertible pair (lifted rotations, mirrored inverse; mx_fft.cuh), whose twiddle table holds
// lifting constants; in FP64 the plain pair (constants rounded to FP64 bias a step by ~1e-16).
template <typename T, int N, int E, int NL, bool PP = false, int CNS = 0>
__device__ __forceinline__ void zf_fwd(cx<T> (*v)[E], cx<T>* sm, int SS, int LS, int t, const twv<T>* tw,
                                       cx<T>* sm2 = nullptr, const twv<T>* twr = nullptr) {
  if constexpr (std::is_same<T, float>::value) lines_fft_lf<N, E, 0, NL, 1, 0, PP, CNS>(v, sm, SS, LS, t, tw, sm2, twr);
  else lines_fft<T, N, E, -1, 0, NL, 1, 0, PP, CNS>(v, sm, SS, LS, t, tw, sm2, twr);
}
template <typename T, int N, int E, int NL, bool PP = false, int CNS = 0>
__device__ __forceinline__ void zf_inv(cx<T> (*v)[E], cx<T>* sm, int SS, int LS, int t, const twv<T>* tw,
                                       cx<T>* sm2 = nullptr, const twv<T>* twr = nullptr) {
  if constexpr (std::is_same<T, float>::value)
    lines_ifft_lf<N, E, 0, NL, num_stages(N, E) - 1, 0, PP, CNS>(v, sm, SS, LS, t, tw, sm2, twr);
  else
    lines_fft<T, N, E, +1, 0, NL, 1, 0, PP, CNS>(v, sm, SS, LS, t, tw, sm2, twr);
}

// SRC: where the coefficients come from: 0 = the table (tab set), 1 = computed per point in FP64
// (tab null), 2 = either, decided at run time.  An instantiation without the FP64 path carries no
// FP64 code, and no call into the FP64 sine's slow path, in its loop.
template <typename T, int N, int E, int TX, typename CoefT, bool INV, bool TMAP, int SRC>
__device__ __forceinline__ void z_fused_body(cx<T>* __restrict__ data, const GridParams& g, const CoefT* __restrict__ tab,
                                             double tstep, const twv<T>* __restrict__ twg, double* __restrict__ partials,
                                             unsigned* __restrict__ counter, double* __restrict__ record,
                                             const void* tmap) {
  using C = cx<T>;
  using ZT = ZTile<T, N, E, TX>;
  constexpr int P = N / E;
  constexpr int LS = strided_rows(N) * TX;  // exchange buffer of one component (TX lines side by side)
  extern __shared__ __align__(128) unsigned char zsmraw[];
  // [input stage, output stage (TMAP only)][twiddles][exchange buffer][mbarrier]; the stages also
  // serve as second exchange buffers.  Triplets: [input stage][output stage][twiddles][mbarrier]
  constexpr bool TRIP = TMAP && ZT::TRIP;
  constexpr int TWC = TRIP ? tw_cache_ns(N, E) : 0;  // second-stage twiddles kept in registers
  twv<T> twr[tw_cache_len(N, E)];
  C* stage = reinterpret_cast<C*>(zsmraw);
  C* ostage = reinterpret_cast<C*>(zsmraw + ZT::stage_bytes);
  twv<T>* tw = reinterpret_cast<twv<T>*>(TMAP ? reinterpret_cast<unsigned char*>(ostage) + ZT::stage_bytes : zsmraw);
  C* sm = reinterpret_cast<C*>(reinterpret_cast<unsigned char*>(tw) + ZT::tw_bytes);  // (not with triplets)
  uint64_t* full = reinterpret_cast<uint64_t*>(TRIP ? reinterpret_cast<unsigned char*>(tw) + ZT::tw_bytes
                                                    : reinterpret_cast<unsigned char*>(sm) + ZT::exch_bytes);
  for (int i = threadIdx.x; i < tw_len(N, E); i += blockDim.x) tw[i] = twg[i];
  const int x = threadIdx.x % TX, t = threadIdx.x / TX;
  const long inner = (long)g.mx * g.ny;  // stride between z planes
  const long comp = inner * N;           // stride between components
  const int ntx = (g.mx + TX - 1) / TX;
  const long ntiles = (long)ntx * g.ny;
  const T eps = GP<T>::eps(g), mu = GP<T>::mu(g);
  const T nux = GP<T>::nu(g, 0), nuy = GP<T>::nu(g, 1), nuz = GP<T>::nu(g, 2);
  __shared__ T zhi[32][NSUM], zlo[32][NSUM];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (INV && lane == 0)
    for (int k = 0; k < NSUM; ++k) zhi[warp][k] = zlo[warp][k] = (T)0;
  if constexpr (TMAP) {
    if (threadIdx.x == 0) {
      mbar_init(full, 1);
      mbar_fence_init();
    }
    __syncthreads();
    if constexpr (TRIP && TWC > 0) tw_cached<T, N, E>(twr, tw, t);
    if (threadIdx.x == 0 && (long)blockIdx.x < ntiles) z_tile_copy<T, N, E, TX>(tmap, stage, full, blockIdx.x, ntx);
  }
  unsigned it = 0;
  bool pending = (long)blockIdx.x < ntiles;  // a copy into the stage is in flight (thread 0's view)
  for (long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    // 32-bit division (a 64-bit one runs partly on the FP64 pipe); ntiles < 2^31
    const int y = (int)((unsigned)tile / (unsigned)ntx);
    const int col = (int)((unsigned)tile - (unsigned)y * (unsigned)ntx) * TX + x;
    const bool ok = col < g.mx;
    C* base = data + (long)y * g.mx + col;
    C v[6][E];
    if constexpr (TMAP) {
      const bool lost = !mbar_wait_tries(full, it & 1u, g.wait_tries);
      if (__syncthreads_or(lost)) {
        if (lost) atomicExch(counter + 1, 1u);
        break;
      }
#pragma unroll
      for (int c = 0; c < 6; ++c)
#pragma unroll
        for (int m = 0; m < E; ++m) v[c][m] = stage[ZT::stage_index(c, t + P * m, x)];
      __syncthreads();  // every read of the stage is done (and the twiddles are in)
      pending = false;
      if constexpr (TRIP) {
        // the stage's upper half is free until the next tile: its copies start now
        if (threadIdx.x == 0 && tile + gridDim.x < ntiles) {
          z_tile_copy<T, N, E, TX, ZT::NB / 2, ZT::NB, true>(tmap, stage, full, tile + gridDim.x, ntx);
          pending = true;
        }
      }
    } else {
#pragma unroll
      for (int c = 0; c < 6; ++c)
#pragma unroll
        for (int m = 0; m < E; ++m) v[c][m] = ok ? base[c * comp + (long)(t + P * m) * inner] : C{0, 0};
      __syncthreads();  // twiddles
    }
    const int my = signed_index(y, g.ny);
    // TMAP: the input stage is free until the next tile's copy; the tile's coefficient-table
    // entries, one per column and |m_z| (ZTile::NA of them per column), are copied into it
    // (cp.async, spread over all threads) while the forward transforms run, as planes of 16-byte
    // pieces (piece h of the entry of column x and |m_z| = a at cpl[(h NA + a) TX + x]): a warp's
    // copies are contiguous, and its reads of one piece (consecutive or mirrored |m_z|) too
    constexpr int NPC = (int)(sizeof(CoefT) / 16);
    constexpr int NA = ZT::NA;
    static_assert(sizeof(CoefT) % 16 == 0, "coefficient entries are whole 16-byte pieces");
    float4* cpl = reinterpret_cast<float4*>(stage);
    static_assert((size_t)NA * TX * sizeof(CoefT) <= ZT::stage_bytes, "coefficients fit in the stage");
    const bool staged = TMAP && tab != nullptr;  // block-uniform
    if (staged) {
      const int col0 = col - x;
      const int qyy = g.qa[1] * my * my;
#pragma unroll
      for (int L = threadIdx.x; L < NPC * NA * TX; L += ZT::NT) {
        const int xx = L % TX, a = (L / TX) % NA, h = L / (TX * NA);
        const int cx = col0 + xx;
        if (cx < g.mx)
          cp_async_16n<16>(cpl + L, reinterpret_cast<const float4*>(tab + (g.qa[0] * cx * cx + qyy + g.qa[2] * a * a)) + h);
      }
      cp_async_commit();
    }
    constexpr int SWZ = swz_rows(TX, ZT::XK);
    constexpr int LX = N * TX;  // complex values per unpadded exchange buffer
    if constexpr (TRIP) {
      static_assert(sizeof(CoefT) == 32, "coefficient entries of 32 bytes");
      // three components at a time through the output stage, as the inverse transforms, once the
      // previous tile's store has read it
      if (threadIdx.x == 0) bulk_wait_read_all();
      __syncthreads();
#pragma unroll
      for (int c = 0; c < 6; c += 3)
        zf_fwd<T, N, E, 3, true, TWC>(v + c, ostage + x, SWZ, LX, t, tw, ostage + 3 * LX + x, twr);
    } else if constexpr (TMAP && ZT::coef_bytes + ZT::exch_bytes <= ZT::stage_bytes) {
      // two components at a time: the second exchange buffer is the input stage past the coefficients
      C* xb2 = reinterpret_cast<C*>(reinterpret_cast<unsigned char*>(stage) + ZT::coef_bytes);
      const int ls2 = (int)(xb2 - sm);
#pragma unroll
      for (int c = 0; c < 6; c += 2) zf_fwd<T, N, E, 2>(v + c, sm + x, TX, ls2, t, tw);
    } else {
#pragma unroll
      for (int c = 0; c < 6; c += ZT::NL) zf_fwd<T, N, E, ZT::NL>(v + c, sm + x, TX, LS, t, tw);
    }
    if (staged) {
      cp_async_wait_all();
      __syncthreads();  // every thread's copies have landed (a thread reads entries others copied)
    }
    T part[INV ? 16 : 1];  // NSUM sums and a zero (warp_transpose_sum16)
#pragma unroll
    for (int k = 0; k < (INV ? 16 : 1); ++k) part[k] = (T)0;
    if (ok) {
      const T kx = nux * (T)col, ky = nuy * (T)my;
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const int mz = signed_index(t + P * m, N);
        const T kz = nuz * (T)mz;
        CoefT q;
        auto from_stage = [&]() {
          union {
            CoefT c;
            float4 f[NPC];
          } u;
          const int a = mz < 0 ? -mz : mz;
#pragma unroll
          for (int h = 0; h < NPC; ++h) u.f[h] = cpl[(h * NA + a) * TX + x];
          return u.c;
        };
        auto direct = [&]() {
          const double k2 = g.nu[0] * g.nu[0] * (double)col * col + g.nu[1] * g.nu[1] * (double)my * my +
                            g.nu[2] * g.nu[2] * (double)mz * mz;
          return coef_direct<T, CoefT>(k2, tstep, g);
        };
        if constexpr (SRC == 1) {
          q = direct();
        } else if constexpr (SRC == 0 && TMAP) {
          q = from_stage();  // staged: the table is set (and this column is inside the grid)
        } else if constexpr (SRC == 0) {
          q = tab[g.qa[0] * col * col + g.qa[1] * my * my + g.qa[2] * mz * mz];
        } else {
          if (staged) q = from_stage();
          else if (tab) q = tab[g.qa[0] * col * col + g.qa[1] * my * my + g.qa[2] * mz * mz];
          else q = direct();
        }
        C ee[3] = {v[0][m], v[1][m], v[2][m]};
        C hh[3] = {v[3][m], v[4][m], v[5][m]};
        Apply<T, CoefT>::run(q, kx, ky, kz, hh, ee);
#pragma unroll
        for (int c = 0; c < 3; ++c) v[c][m] = ee[c], v[c + 3][m] = hh[c];
        if constexpr (INV) add_densities<T>(part, col == 0 ? (T)1 : (T)2, kx, ky, kz, hh, ee, eps, mu);
      }
    }
    if constexpr (TRIP) {
      // the coefficient reads of the stage's lower half are done: it takes the next tile's lower
      // boxes (async proxy after generic)
      fence_proxy_async_smem();
      __syncthreads();
      if (threadIdx.x == 0 && tile + gridDim.x < ntiles)
        z_tile_copy<T, N, E, TX, 0, ZT::NB / 2, false>(tmap, stage, full, tile + gridDim.x, ntx);
    } else if constexpr (TMAP) {
      // the stage's coefficient reads are done: it takes the next tile (async proxy after generic)
      fence_proxy_async_smem();
      // the previous tile's store has read the output stage: it is the inverse transforms' second
      // exchange buffer
      if (threadIdx.x == 0) bulk_wait_read_all();
      __syncthreads();
      if (threadIdx.x == 0 && tile + gridDim.x < ntiles) {
        z_tile_copy<T, N, E, TX>(tmap, stage, full, tile + gridDim.x, ntx);
        pending = true;
      }
    }
    if constexpr (INV) {
      const T w = warp_transpose_sum16(part, lane);
      const int k = transpose_index(lane);
      if ((lane & 1) == 0 && k < NSUM) {  // hi + (-lo) carries the sum
        const T yv = w - zlo[warp][k], tv = zhi[warp][k] + yv;
        zlo[warp][k] = (tv - zhi[warp][k]) - yv;
        zhi[warp][k] = tv;
      }
    }
    if constexpr (TRIP) {
      // three components at a time through the output stage: exchanges alternate between two
      // triplets of buffers there, so that none waits for the readers of the one before it
#pragma unroll
      for (int c = 0; c < 6; c += 3)
        zf_inv<T, N, E, 3, true, TWC>(v + c, ostage + x, SWZ, LX, t, tw, ostage + 3 * LX + x, twr);
    } else if constexpr (TMAP) {
      // two components at a time through the output stage: exchanges alternate between two pairs
      // of buffers there, so that none waits for the readers of the one before it
      static_assert(ZT::exch_bytes <= ZT::stage_bytes, "an exchange buffer fits in the output stage");
      if constexpr (4 * ZT::exch_bytes <= ZT::stage_bytes) {
#pragma unroll
        for (int c = 0; c < 6; c += 2)
          zf_inv<T, N, E, 2, true>(v + c, ostage + x, TX, LS, t, tw, ostage + 2 * LS + x);
      } else {
        const int ls2 = (int)(ostage - sm);
#pragma unroll
        for (int c = 0; c < 6; c += 2) zf_inv<T, N, E, 2>(v + c, sm + x, TX, ls2, t, tw);
      }
    } else {
#pragma unroll
      for (int c = 0; c < 6; c += ZT::NL) zf_inv<T, N, E, ZT::NL>(v + c, sm + x, TX, LS, t, tw);
    }
    if (g.zscalef != 1.0f) {  // block-uniform; exact for nz a power of two
      const T sc = GP<T>::zscale(g);
#pragma unroll
      for (int c = 0; c < 6; ++c)
#pragma unroll
        for (int m = 0; m < E; ++m) v[c][m] = C{v[c][m].x * sc, v[c][m].y * sc};
    }
    if constexpr (TMAP) {
      // through the output stage and the tensor-copy engine (it drops the columns past Mx)
      __syncthreads();  // the inverse transforms' exchange reads of the output stage are done
#pragma unroll
      for (int c = 0; c < 6; ++c)
#pragma unroll
        for (int m = 0; m < E; ++m) ostage[ZT::stage_index(c, t + P * m, x)] = v[c][m];
      fence_proxy_async_smem();  // generic writes before the async-proxy reads of the store
      __syncthreads();
      if (threadIdx.x == 0) z_tile_store<T, N, E, TX>(tmap, ostage, tile, ntx);
    } else if (ok) {
      // addresses recomputed here instead of kept live from the loads
      C* sbase = base + (long)t * inner;
      asm volatile("" : "+l"(sbase));
#pragma unroll
      for (int c = 0; c < 6; ++c)
#pragma unroll
        for (int m = 0; m < E; ++m) sbase[c * comp + (long)(P * m) * inner] = v[c][m];
    }
  }
  if constexpr (TMAP) {
    // after a timed-out wait: let the copy this block issued land before its shared memory is released
    if (threadIdx.x == 0 && pending) mbar_wait_bounded(full, it & 1u);
    if (threadIdx.x == 0) bulk_wait_all();  // the last stores have completed
  }
  if constexpr (INV) {
    // each warp's row of totals: lane k takes sum k (hi + (-lo)) to FP64
    __shared__ double rows[32][NSUM];
    if (lane < NSUM) rows[warp][lane] = (double)zhi[warp][lane] - (double)zlo[warp][lane];
    __syncthreads();
    rows_finish(rows, (int)((blockDim.x + 31) >> 5), rows, partials, counter, record);
  }
}

// DIRECT: coefficients computed per point (no table); else from the table, which must be set.
template <typename T, int N, int E, int TX, typename CoefT, bool INV, bool DIRECT>
__global__ void __launch_bounds__((N / E) * TX, 1)
    k_z_fused_tma(cx<T>* __restrict__ data, GridParams g, const CoefT* __restrict__ tab, double tstep,
                  const twv<T>* __restrict__ twg, double* __restrict__ partials, unsigned* __restrict__ counter,
                  double* __restrict__ record, const __grid_constant__ CUtensorMap tmap) {
  z_fused_body<T, N, E, TX, CoefT, INV, true, DIRECT ? 1 : 0>(data, g, tab, tstep, twg, partials, counter, record,
                                                            &tmap);
}

template <typename T, int N, int E, int TX, typename CoefT, bool INV>
__global__ void __launch_bounds__((N / E) * TX, 1) k_z_fused(cx<T>* __restrict__ data, GridParams g,
                                                             const CoefT* __restrict__ tab, double tstep,
                                                             const twv<T>* __restrict__ twg, double* __restrict__ partials,
                                                             unsigned* __restrict__ counter, double* __restrict__ record) {
  z_fused_body<T, N, E, TX, CoefT, INV, false, 2>(data, g, tab, tstep, twg, partials, counter, record, nullptr);
}

// ------------------------------------------------------ spectral update pass
//
// dst = R(t) src elementwise over the half spectrum (src may equal dst);
// UPDATE = false reads only (invariants of src).  Each thread takes V
// consecutive points of one row per iteration (V = 2: 16-byte FP32 loads),
// grid-stride over the flattened [Nz][Ny][Mx] index.  Invariant densities
// of the written state are summed in T over at most CHUNK iterations, then
// added into per-thread FP64 slots in shared memory; the block and grid
// reductions are FP64 (reduce_and_finish).
template <typename T> struct vec4;
template <> struct vec4<float> { using type = float4; };

template <typename T, int V>
__device__ __forceinline__ void load_pts(const cx<T>* __restrict__ a, long i, cx<T>* out) {
  if constexpr (V == 2 && sizeof(T) == 4) {
    const float4 v = __ldcs(reinterpret_cast<const float4*>(a + i));
    out[0] = cx<T>{v.x, v.y};
    out[1] = cx<T>{v.z, v.w};
  } else {
#pragma unroll
    for (int j = 0; j < V; ++j) out[j] = __ldcs(a + i + j);
  }
}
template <typename T, int V>
__device__ __forceinline__ void store_pts(cx<T>* __restrict__ a, long i, const cx<T>* in) {
  if constexpr (V == 2 && sizeof(T) == 4) {
    __stcs(reinterpret_cast<float4*>(a + i), make_float4(in[0].x, in[0].y, in[1].x, in[1].y));
  } else {
#pragma unroll
    for (int j = 0; j < V; ++j) __stcs(a + i + j, in[j]);
  }
}

template <typename T, typename CoefT, bool TABLE, bool UPDATE, bool INV, int V>
__global__ void __launch_bounds__(256, 2) k_spectral(const cx<T>* __restrict__ src, cx<T>* __restrict__ dst,
                                                     long comp_stride, GridParams g, const CoefT* __restrict__ tab,
                                                     double t, double* __restrict__ partials,
                                                     unsigned* __restrict__ counter, double* __restrict__ record) {
  using C = cx<T>;
  constexpr int CHUNK = 16;
  __shared__ double sacc[INV ? NSUM : 1][256];
  const unsigned npts = (unsigned)comp_stride;
  const unsigned mx = (unsigned)g.mx, ny = (unsigned)g.ny;
  const T eps = GP<T>::eps(g), mu = GP<T>::mu(g);
  const T nux = GP<T>::nu(g, 0), nuy = GP<T>::nu(g, 1), nuz = GP<T>::nu(g, 2);
  T part[INV ? NSUM : 1];
  if constexpr (INV) {
#pragma unroll
    for (int i = 0; i < NSUM; ++i) part[i] = (T)0, sacc[i][threadIdx.x] = 0.0;
  }
  int cnt = 0;
  const unsigned stride = gridDim.x * blockDim.x * V;
  for (unsigned p = (blockIdx.x * blockDim.x + threadIdx.x) * V; p < npts; p += stride) {
    const unsigned r = p / mx;
    const int x0 = (int)(p - r * mx);
    const unsigned z = r / ny;
    const int y = (int)(r - z * ny);
    const int my = signed_index(y, g.ny), mz = signed_index((int)z, g.nz);
    const T ky = nuy * (T)my, kz = nuz * (T)mz;
    C e[3][V], h[3][V];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      load_pts<T, V>(src, (long)c * comp_stride + p, e[c]);
      load_pts<T, V>(src, (long)(c + 3) * comp_stride + p, h[c]);
    }
#pragma unroll
    for (int j = 0; j < V; ++j) {
      const int x = x0 + j;
      const T kx = nux * (T)x;
      C hh[3] = {h[0][j], h[1][j], h[2][j]};
      C ee[3] = {e[0][j], e[1][j], e[2][j]};
      if constexpr (UPDATE) {
        CoefT q;
        if constexpr (TABLE) {
          q = tab[g.qa[0] * x * x + g.qa[1] * my * my + g.qa[2] * mz * mz];
        } else {
          const double k2 = g.nu[0] * g.nu[0] * (double)x * x + g.nu[1] * g.nu[1] * (double)my * my +
                            g.nu[2] * g.nu[2] * (double)mz * mz;
          q = coef_direct<T, CoefT>(k2, t, g);
        }
        Apply<T, CoefT>::run(q, kx, ky, kz, hh, ee);
#pragma unroll
        for (int c = 0; c < 3; ++c) h[c][j] = hh[c], e[c][j] = ee[c];
      }
      if constexpr (INV) add_densities<T>(part, x == 0 ? (T)1 : (T)2, kx, ky, kz, hh, ee, eps, mu);
    }
    if constexpr (UPDATE) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        store_pts<T, V>(dst, (long)c * comp_stride + p, e[c]);
        store_pts<T, V>(dst, (long)(c + 3) * comp_stride + p, h[c]);
      }
    }
    if constexpr (INV) {
      if (++cnt == CHUNK) {
#pragma unroll
        for (int i = 0; i < NSUM; ++i) sacc[i][threadIdx.x] += (double)part[i], part[i] = (T)0;
        cnt = 0;
      }
    }
  }
  if constexpr (INV) {
    double acc[NSUM];
#pragma unroll
    for (int i = 0; i < NSUM; ++i) acc[i] = sacc[i][threadIdx.x] + (double)part[i];
    reduce_and_finish(acc, partials, counter, record);
  }
}

}  // namespace mx

// Register-resident mixed-radix (2/3/4/5/8) line FFT for sm_103a.
//
// One line of length N is transformed by P = N/E threads, each holding E
// complex values in registers.  Stage s is a radix-R_s Stockham (autosort)
// step; every R_s divides E, so a thread performs E/R_s butterflies per stage
// on values it already holds.  On entry thread t holds x[t + P*m] in v[m]
// (m = 0..E-1); on exit it holds X[t + P*m] in v[m], natural order.  The
// same index set is read by the first stage and written by the last one,
// which lets a forward transform, a per-frequency update and an inverse
// transform run back to back in registers.  Between stages values are
// exchanged through a shared-memory line buffer (position p at sm[p*SS]).
//
// Transform definition (the paper's Sec. 2.3): forward X_k = sum_j x_j
// exp(-2 pi i jk/N), inverse without the 1/N factor (callers fold all
// normalisation into one multiply).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mx {

template <typename T> struct vec2;
template <> struct vec2<float> { using type = float2; };
template <> struct vec2<double> { using type = double2; };
template <typename T> using cx = typename vec2<T>::type;

// Twiddle storage.  FP32: the value as a pair hi + lo (float4 hi.x, hi.y, lo.x,
// lo.y); FP64: the lifting constants of the rotation (dd2 p, u, sign, 0; twmul
// below).  A rounded cos/sin constant would scale each frequency by the same
// wrong factor on every transform, and in a repeated forward/inverse loop that
// bias grows linearly with the step count; neither form has that bias.
struct __align__(16) dd2 { double x, y, z, w; };
template <typename T> struct tw_t;
template <> struct tw_t<float> { using type = float4; };
template <> struct tw_t<double> { using type = dd2; };
template <typename T> using twv = typename tw_t<T>::type;

// a * w (forward, DIR < 0) or a * conj(w) (inverse).
// FP64 twiddles are lifted rotations: entry (p, u, sign, 0) rotates by the twiddle's angle a as
// three shears x += p y, y += u x, x += p y (p = -tan(a'/2), u = sin a'), where a' = a when
// |a| <= pi/2 and a -+ pi otherwise (sign = -1: the input is negated first, by its sign bits, off
// the FP64 pipe).  The inverse rotation takes -p, -u.  A product of shears has determinant 1 for
// whatever rounded p and u, so the rounding of the constants scales no frequency on average (a
// rounded cos/sin pair scales every value that passes through it by |w|^2 on every transform,
// which a repeated step accumulates), at 3 FP64 operations where a double-double pair takes 8.
template <int DIR> __device__ __forceinline__ double2 twmul(double2 a, dd2 w) {
  const double p = DIR < 0 ? w.x : -w.x, u = DIR < 0 ? w.y : -w.y;
  const int sb = __double2hiint(w.z) & (int)0x80000000;
  double x = __hiloint2double(__double2hiint(a.x) ^ sb, __double2loint(a.x));
  double y = __hiloint2double(__double2hiint(a.y) ^ sb, __double2loint(a.y));
  x = fma(p, y, x);
  y = fma(u, x, y);
  x = fma(p, y, x);
  return double2{x, y};
}
template <int DIR> __device__ __forceinline__ float2 twmul(float2 a, float4 w) {
  const float hy = DIR < 0 ? w.y : -w.y, ly = DIR < 0 ? w.w : -w.w;
  const float re = fmaf(a.x, w.x, fmaf(-a.y, hy, a.x * w.z - a.y * ly));
  const float im = fmaf(a.x, hy, fmaf(a.y, w.x, a.x * ly + a.y * w.z));
  return float2{re, im};
}
// x * c for a real constant c given as a double-double hi + lo (or a double): applied as a
// hi + lo pair of the arithmetic type
template <typename T> struct KC;
template <> struct KC<double> {
  double h, l;
  __device__ __forceinline__ constexpr KC(double c) : h(c), l(0.0) {}
  __device__ __forceinline__ constexpr KC(double hi, double lo) : h(hi), l(lo) {}
  __device__ __forceinline__ double mul(double x) const { return fma(x, h, x * l); }
};
template <> struct KC<float> {
  float h, l;
  __device__ __forceinline__ constexpr KC(double c) : h((float)c), l((float)(c - (double)(float)c)) {}
  __device__ __forceinline__ constexpr KC(double hi, double lo) : h((float)hi), l((float)((hi - (double)(float)hi) + lo)) {}
  __device__ __forceinline__ float mul(float x) const { return fmaf(x, h, x * l); }
};
// Butterfly constants as double-double pairs (hi = the double nearest, lo = the rest).
#define MX_KC_INV_SQRT2 0.7071067811865476, -4.833646656726457e-17
#define MX_KC_SIN_2PI_3 0.8660254037844386, 5.0175421109034514e-17
#define MX_KC_COS_2PI_5 0.30901699437494745, -2.716057601841253e-17
#define MX_KC_COS_4PI_5 -0.8090169943749475, 2.716057601841253e-17
#define MX_KC_SIN_2PI_5 0.9510565162951535, 4.0934500900087295e-17
#define MX_KC_SIN_4PI_5 0.5877852522924731, -7.93475083819002e-18

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return C{a.x, -a.y}; }
template <typename C, typename T> __device__ __forceinline__ C cscale(C a, T s) { return C{a.x * s, a.y * s}; }
// multiply by (DIR * i): DIR = -1 for the forward kernel exp(-2 pi i / R)
template <int DIR, typename C> __device__ __forceinline__ C rot(C a) {
  return DIR < 0 ? C{a.y, -a.x} : C{-a.y, a.x};
}

// ---------------------------------------------------------------- butterflies
// In-register DFT of R values v[0], v[S], ..., v[(R-1)S] (S compile-time stride).

template <int DIR, int S, typename C> __device__ __forceinline__ void bfly2(C* v) {
  C a = v[0], b = v[S];
  v[0] = cadd(a, b);
  v[S] = csub(a, b);
}

template <int DIR, int S, typename C> __device__ __forceinline__ void bfly4(C* v) {
  C a = v[0], b = v[S], c = v[2 * S], d = v[3 * S];
  C s0 = cadd(a, c), d0 = csub(a, c), s1 = cadd(b, d), d1 = rot<DIR>(csub(b, d));
  v[0] = cadd(s0, s1);
  v[S] = cadd(d0, d1);
  v[2 * S] = csub(s0, s1);
  v[3 * S] = csub(d0, d1);
}

template <int DIR, int S, typename C> __device__ __forceinline__ void bfly8(C* v) {
  using T = decltype(v[0].x);
  constexpr KC<T> h(MX_KC_INV_SQRT2);  // 1/sqrt(2)
  C e[4] = {v[0], v[2 * S], v[4 * S], v[6 * S]};
  C o[4] = {v[S], v[3 * S], v[5 * S], v[7 * S]};
  bfly4<DIR, 1>(e);
  bfly4<DIR, 1>(o);
  // o[k] *= exp(DIR * 2 pi i k / 8)
  C o1 = o[1], o3 = o[3];
  o[1] = C{h.mul(o1.x - DIR * o1.y), h.mul(o1.y + DIR * o1.x)};
  o[2] = rot<DIR>(o[2]);
  o[3] = C{h.mul(-o3.x - DIR * o3.y), h.mul(-o3.y + DIR * o3.x)};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[k * S] = cadd(e[k], o[k]);
    v[(k + 4) * S] = csub(e[k], o[k]);
  }
}

// FP64: the products by exp(DIR i pi/4) and exp(DIR 3 i pi/4) = -exp(-DIR i pi/4) as lifted
// rotations (three shears, p = -tan(a/2), u = sin a; twmul): 3 FP64 operations where 1/sqrt(2)
// as a double-double pair takes 6, and determinant 1 whatever the rounding of p and u.
template <int DIR, int S> __device__ __forceinline__ void bfly8(double2* v) {
  constexpr double TP8 = 0.41421356237309503;   // tan(pi/8) = sqrt(2) - 1
  constexpr double S4 = 0.70710678118654757;    // sin(pi/4)
  double2 e[4] = {v[0], v[2 * S], v[4 * S], v[6 * S]};
  double2 o[4] = {v[S], v[3 * S], v[5 * S], v[7 * S]};
  bfly4<DIR, 1>(e);
  bfly4<DIR, 1>(o);
  // rotation by a = DIR pi/4 (p = -DIR tan(pi/8), u = DIR sin(pi/4)) of o[1]; by -a of o[3],
  // whose product is then subtracted where o[3] is added (the factor -1 of 3 pi/4 = pi - pi/4)
  const double p = DIR < 0 ? TP8 : -TP8, u = DIR < 0 ? -S4 : S4;
  double x = o[1].x, y = o[1].y;
  x = fma(p, y, x);
  y = fma(u, x, y);
  x = fma(p, y, x);
  o[1] = double2{x, y};
  o[2] = rot<DIR>(o[2]);
  x = o[3].x, y = o[3].y;
  x = fma(-p, y, x);
  y = fma(-u, x, y);
  x = fma(-p, y, x);
  o[3] = double2{x, y};
  v[0] = cadd(e[0], o[0]);
  v[4 * S] = csub(e[0], o[0]);
  v[S] = cadd(e[1], o[1]);
  v[5 * S] = csub(e[1], o[1]);
  v[2 * S] = cadd(e[2], o[2]);
  v[6 * S] = csub(e[2], o[2]);
  v[3 * S] = csub(e[3], o[3]);
  v[7 * S] = cadd(e[3], o[3]);
}

template <int DIR, int S, typename C> __device__ __forceinline__ void bfly3(C* v) {
  using T = decltype(v[0].x);
  const T c1 = (T)-0.5;                        // cos 2 pi/3 (exact)
  constexpr KC<T> s1(MX_KC_SIN_2PI_3);  // sin 2 pi/3
  C a = v[0], b = v[S], c = v[2 * S];
  C s = cadd(b, c), d = csub(b, c);
  C t = C{a.x + c1 * s.x, a.y + c1 * s.y};
  C u = rot<DIR>(C{s1.mul(d.x), s1.mul(d.y)});
  v[0] = cadd(a, s);
  v[S] = cadd(t, u);
  v[2 * S] = csub(t, u);
}

template <int DIR, int S, typename C> __device__ __forceinline__ void bfly5(C* v) {
  using T = decltype(v[0].x);
  constexpr KC<T> c1(MX_KC_COS_2PI_5), c2(MX_KC_COS_4PI_5);  // cos 2pi/5, cos 4pi/5
  constexpr KC<T> s1(MX_KC_SIN_2PI_5), s2(MX_KC_SIN_4PI_5);  // sin 2pi/5, sin 4pi/5
  C a = v[0], b = v[S], c = v[2 * S], d = v[3 * S], e = v[4 * S];
  C p1 = cadd(b, e), m1 = csub(b, e), p2 = cadd(c, d), m2 = csub(c, d);
  C t1 = C{a.x + c1.mul(p1.x) + c2.mul(p2.x), a.y + c1.mul(p1.y) + c2.mul(p2.y)};
  C t2 = C{a.x + c2.mul(p1.x) + c1.mul(p2.x), a.y + c2.mul(p1.y) + c1.mul(p2.y)};
  C u1 = rot<DIR>(C{s1.mul(m1.x) + s2.mul(m2.x), s1.mul(m1.y) + s2.mul(m2.y)});
  C u2 = rot<DIR>(C{s2.mul(m1.x) - s1.mul(m2.x), s2.mul(m1.y) - s1.mul(m2.y)});
  v[0] = C{a.x + p1.x + p2.x, a.y + p1.y + p2.y};
  v[S] = cadd(t1, u1);
  v[4 * S] = csub(t1, u1);
  v[2 * S] = cadd(t2, u2);
  v[3 * S] = csub(t2, u2);
}

template <int R, int DIR, int S, typename C> __device__ __forceinline__ void bfly(C* v) {
  if constexpr (R == 2) bfly2<DIR, S>(v);
  else if constexpr (R == 3) bfly3<DIR, S>(v);
  else if constexpr (R == 4) bfly4<DIR, S>(v);
  else if constexpr (R == 5) bfly5<DIR, S>(v);
  else if constexpr (R == 8) bfly8<DIR, S>(v);
  else static_assert(R == 2, "unsupported radix");
}

// ------------------------------------------------------------------ planning

// Radix of the next stage: the largest of 8, 5, 4, 3, 2 dividing both the
// length still to factor and E.
__host__ __device__ constexpr int pick_radix(int rem, int E) {
  return (rem % 8 == 0 && E % 8 == 0)   ? 8
         : (rem % 5 == 0 && E % 5 == 0) ? 5
         : (rem % 4 == 0 && E % 4 == 0) ? 4
         : (rem % 3 == 0 && E % 3 == 0) ? 3
         : (rem % 2 == 0 && E % 2 == 0) ? 2
                                        : 0;
}
__host__ __device__ constexpr bool plan_ok(int N, int E) {
  if (N <= 0 || E <= 0 || N % E) return false;
  int rem = N;
  while (rem > 1) {
    int r = pick_radix(rem, E);
    if (!r) return false;
    rem /= r;
  }
  return true;
}
__host__ __device__ constexpr int num_stages(int N, int E) {
  int s = 0, rem = N;
  while (rem > 1) {
    rem /= pick_radix(rem, E);
    ++s;
  }
  return s;
}
// Radix of the plan's last stage.
__host__ __device__ constexpr int last_radix(int N, int E) {
  int rem = N, r = 0;
  while (rem > 1) {
    r = pick_radix(rem, E);
    rem /= r;
  }
  return r;
}
// A mirrored last stage (lines_fft MIRROR) needs two butterflies per thread there and an exchange
// before it.
__host__ __device__ constexpr bool mirror_ok(int N, int E) {
  return num_stages(N, E) >= 2 && last_radix(N, E) > 0 && E / last_radix(N, E) == 2;
}

// Stage-major twiddle table of a line FFT of length N with E values per thread:
// for each stage after the first (NS > 1, radix R) the entries
// [r - 1][k] = exp(-2 pi i r k / (NS R)), r = 1..R-1, k = 0..NS-1, so that the
// threads of a warp (consecutive k) read consecutive entries.
__host__ __device__ constexpr int tw_stage_off(int N, int E, int NS) {
  int off = 0, ns = 1;
  while (ns < NS) {
    const int r = pick_radix(N / ns, E);
    if (ns > 1) off += ns * (r - 1);
    ns *= r;
  }
  return off;
}
__host__ __device__ constexpr int tw_len(int N, int E) { return tw_stage_off(N, E, N); }

// ------------------------------------------------------------------ the line FFT
//
// v      : E registers, v[m] <-> position t + P*m
// sm     : this line's exchange buffer, position p at sm[xoff(p, SS)]:
//          for interleaved lines (SS > 1, SS lines side by side) row p of SS
//          values with one padding row every 8 rows, so that the rows written
//          at stride R = 8 by neighbouring threads fall on different banks;
//          for a contiguous line (SS == 1) one complex of padding every 16,
//          which spreads the stride-R exchange writes over all banks.
// tw     : stage-major twiddle table of (N, E) (tw_stage_off), twv<T> entries
// All threads sharing the barrier must call this together (it synchronises):
// NBAR < 0 uses __syncwarp() (each line within one warp), NBAR == 0
// __syncthreads(), NBAR > 0 the named barrier of this thread's group of NBAR
// (warp-specialised kernels whose producer warp is busy).
// SS < 0 (see swz_rows): rows of W values with no padding, row p stored at
// p ^ ((p >> 3) & K): rows 8 apart, written together at stride R = 8, land on
// different 128-byte bank lines when K + 1 rows share one (K = 1 for 64-byte
// rows, 3 for 32-byte rows); the buffer is exactly N * W values (N a multiple
// of K + 1).
__host__ __device__ constexpr int swz_rows(int W, int K) { return -(W | (K << 16)); }
__device__ __forceinline__ int xoff(int p, int SS) {
  return SS == 1  ? p + (p >> 4)
         : SS > 0 ? (p + (p >> 3)) * SS
                  : (p ^ ((p >> 3) & ((-SS) >> 16))) * ((-SS) & 0xFFFF);
}
// Exchange-buffer length (complex values) of one contiguous line of length n.
__host__ __device__ constexpr int line_buf(int n) { return n + (n >> 4) + 1; }
// Rows of the exchange buffer of interleaved lines (SS > 1): one padding row every 8.
__host__ __device__ constexpr int strided_rows(int n) { return n + (n >> 3) + 1; }

// Barrier kinds: NBAR < 0 when every line lies within one warp (P threads per
// line with P dividing 32): __syncwarp; 0: __syncthreads; > 0: named barrier
// 1 + threadIdx.x / NBAR over NBAR threads (consecutive groups of NBAR threads
// synchronise independently; barrier 0 stays __syncthreads).
template <int NBAR> __device__ __forceinline__ void fft_bar() {
  if constexpr (NBAR < 0) __syncwarp();
  else if constexpr (NBAR == 0) __syncthreads();
  else asm volatile("bar.sync %0, %1;" ::"r"(1 + (int)threadIdx.x / NBAR), "r"(NBAR) : "memory");
}
// The same synchronisation, returning whether any participating thread had `v` set
// (a uniform decision, e.g. to leave a loop together).
template <int NBAR> __device__ __forceinline__ bool fft_any(bool v) {
  if constexpr (NBAR < 0) {
    return __any_sync(0xffffffffu, v);
  } else if constexpr (NBAR == 0) {
    return __syncthreads_or(v) != 0;
  } else {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %3, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(NBAR), "r"(1 + (int)threadIdx.x / NBAR)
        : "memory");
    return r != 0;
  }
}
// Barrier kind for lines of P threads in blocks whose consumers synchronise with `wide`.
__host__ __device__ constexpr int line_bar(int P, int wide) { return (P <= 32 && 32 % P == 0) ? -1 : wide; }

// NL lines at once (v[l][m]; line l exchanges through sm + l * LS): the lines
// share the barriers and each twiddle load, and their butterflies interleave.
// PP: exchanges alternate between sm (even exchange index IX) and sm2 (odd), so
// that an exchange need not wait for the readers of the one before it: the
// barrier after the previous exchange's writes already orders them.  The first
// exchange of a transform keeps its leading barrier unless the exchange count
// is even, in which case the caller guarantees that the previous transform
// also ran with PP on the same sm and sm2 (its last exchange used sm2) or that
// a barrier has passed since sm was last read.
// CNS > 1: the twiddles of the stage with NS == CNS come from twr (tw_cached),
// in registers, instead of tw.
// MIRROR (mirror_ok(N, E)): in the last stage thread t takes the butterflies t and
// (t ? 2P - t : P) instead of t and t + P, so that the output k = j + NS r of register
// b + 2 r has its mirror N - k in the same thread, at register E - 1 - m (m = b + 2 r; thread 0:
// (E - m) mod E).  A real-input transform then pairs X_k with X_{N-k} without an exchange.
template <typename T, int N, int E, int DIR, int NBAR, int NL, int NS = 1, int IX = 0, bool PP = false, int CNS = 0,
          bool MIRROR = false>
__device__ __forceinline__ void lines_fft(cx<T> (*v)[E], cx<T>* sm, int SS, int LS, int t, const twv<T>* tw,
                                          cx<T>* sm2 = nullptr, const twv<T>* twr = nullptr) {
  if constexpr (NS < N) {
    constexpr int P = N / E;
    constexpr int R = pick_radix(N / NS, E);
    static_assert(R > 0, "no factorisation for this (N, E)");
    constexpr int B = E / R;  // butterflies per thread and line
    constexpr bool MLAST = MIRROR && NS * R == N;  // this stage is the mirrored last one
    static_assert(!MIRROR || (mirror_ok(N, E) && CNS == 0), "mirrored last stage: two butterflies per thread");
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int j = (MLAST && b == 1) ? (t ? 2 * P - t : P) : t + P * b;
      const int k = j % NS;
      if constexpr (NS > 1) {
        constexpr int OFF = tw_stage_off(N, E, NS);
#pragma unroll
        for (int r = 1; r < R; ++r) {
          const twv<T> w = NS == CNS ? twr[b * (R - 1) + r - 1] : tw[OFF + (r - 1) * NS + k];
#pragma unroll
          for (int l = 0; l < NL; ++l) v[l][b + r * B] = twmul<DIR>(v[l][b + r * B], w);
        }
      }
#pragma unroll
      for (int l = 0; l < NL; ++l) bfly<R, DIR, B>(v[l] + b);
    }
    if constexpr (NS * R < N) {
      cx<T>* xb = (PP && (IX & 1)) ? sm2 : sm;
      constexpr int NX = num_stages(N, E) - 1;  // exchanges per transform
      if constexpr (!(PP && (IX > 0 || NX % 2 == 0))) fft_bar<NBAR>();  // previous readers of xb are done
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const int j = t + P * b;
        const int k = j % NS;
        const int base = (j / NS) * NS * R + k;
#pragma unroll
        for (int l = 0; l < NL; ++l)
#pragma unroll
          for (int r = 0; r < R; ++r) xb[l * LS + xoff(base + r * NS, SS)] = v[l][b + r * B];
      }
      fft_bar<NBAR>();
#pragma unroll
      for (int l = 0; l < NL; ++l)
#pragma unroll
        for (int m = 0; m < E; ++m) {
          // the inputs of butterfly j of the next stage are j + (N / R') r'; mirrored when it is last
          constexpr int R2 = pick_radix(N / (NS * R), E);
          constexpr bool NEXT_M = MIRROR && NS * R * R2 == N;
          const int e = NEXT_M ? ((m & 1) ? (t ? 2 * P - t : P) : t) + (N / R2) * (m >> 1) : t + P * m;
          v[l][m] = xb[l * LS + xoff(e, SS)];
        }
      lines_fft<T, N, E, DIR, NBAR, NL, NS * R, IX + 1, PP, CNS, MIRROR>(v, sm, SS, LS, t, tw, sm2, twr);
    }
  }
}

// The second stage's radix and the number of its twiddles a thread uses (B (R - 1)).
__host__ __device__ constexpr int tw_cache_ns(int N, int E) { return pick_radix(N, E) < N ? pick_radix(N, E) : 0; }
__host__ __device__ constexpr int tw_cache_len(int N, int E) {
  return tw_cache_ns(N, E) ? (E / pick_radix(N / tw_cache_ns(N, E), E)) * (pick_radix(N / tw_cache_ns(N, E), E) - 1) : 1;
}
// Twiddles of the stage NS = tw_cache_ns(N, E) for thread t, in the order lines_fft reads them.
template <typename T, int N, int E>
__device__ __forceinline__ void tw_cached(twv<T>* twr, const twv<T>* tw, int t) {
  constexpr int NS = tw_cache_ns(N, E);
  if constexpr (NS > 0 && NS < N) {
    constexpr int P = N / E, R = pick_radix(N / NS, E), B = E / R, OFF = tw_stage_off(N, E, NS);
#pragma unroll
    for (int b = 0; b < B; ++b)
#pragma unroll
      for (int r = 1; r < R; ++r) twr[b * (R - 1) + r - 1] = tw[OFF + (r - 1) * NS + (t + P * b) % NS];
  }
}

template <typename T, int N, int E, int DIR, int NBAR = 0>
__device__ __forceinline__ void line_fft(cx<T>* v, cx<T>* sm, int SS, int t, const twv<T>* tw) {
  lines_fft<T, N, E, DIR, NBAR, 1>(reinterpret_cast<cx<T>(*)[E]>(v), sm, SS, 0, t, tw);
}

// ------------------------------------------------- exactly invertible FP32 pair (lifting)
//
// For a forward transform, a per-frequency map and an inverse transform applied again and again
// (the literal form's z pass), FP32 twiddles rounded once bias every step the same way: the
// inverse does not undo the forward exactly.  This pair removes the bias without double-single
// constants.  Every rotation of the forward transform is three shears (lifting):
//   x1 = x + p y,  y1 = y + u x1,  x2 = x1 + p y1   (p = -tan(a/2), u = sin a: rotation by a)
// which the inverse undoes exactly by the same shears in reverse order with opposite signs, for
// whatever rounded p and u; rotations with |a| > pi/2 are a rotation by a -+ pi of the negated
// input (the sign s is exact).  The inverse transform is the forward's mirror: its stages run in
// reverse order, each undoing the forward stage's butterflies (their inverses up to a power of
// two: radix 2, 4 and 8 are exact; radix 3 and 5 keep double-single constants) and then its
// twiddles, and every exchange undoes the forward exchange.  So inverse(forward(x)) = N x up to
// arithmetic rounding, and n steps of inverse . update . forward equal inverse . update^n .
// forward: the rounding of the constants does not accumulate.
// Twiddle entries: float4 (p, u, s, 0).

__device__ __forceinline__ float2 lift_fwd(float2 a, float4 w) {
  float x = w.z * a.x, y = w.z * a.y;
  x = fmaf(w.x, y, x);
  y = fmaf(w.y, x, y);
  x = fmaf(w.x, y, x);
  return float2{x, y};
}
__device__ __forceinline__ float2 lift_inv(float2 a, float4 w) {
  float x = a.x, y = a.y;
  x = fmaf(-w.x, y, x);
  y = fmaf(-w.y, x, y);
  x = fmaf(-w.x, y, x);
  return float2{w.z * x, w.z * y};
}
// Fixed rotations by -pi/4 and +pi/4 (radix 8): p = tan(pi/8) resp. -tan(pi/8), u = -+ sin(pi/4).
constexpr float LIFT_P8 = 0.41421356237309504880f;
constexpr float LIFT_U8 = 0.70710678118654752440f;
template <int SGN> __device__ __forceinline__ float2 rot8_fwd(float2 a) {  // rotation by SGN * pi/4
  float x = a.x, y = a.y;
  x = fmaf(-SGN * LIFT_P8, y, x);
  y = fmaf(SGN * LIFT_U8, x, y);
  x = fmaf(-SGN * LIFT_P8, y, x);
  return float2{x, y};
}
template <int SGN> __device__ __forceinline__ float2 rot8_inv(float2 a) {  // exact inverse of rot8_fwd<SGN>
  float x = a.x, y = a.y;
  x = fmaf(SGN * LIFT_P8, y, x);
  y = fmaf(-SGN * LIFT_U8, x, y);
  x = fmaf(SGN * LIFT_P8, y, x);
  return float2{x, y};
}

// Forward radix-8 butterfly (exp(-2 pi i / 8) kernel) with lifted rotations:
// e = DFT4(v0, v2, v4, v6), o = DFT4(v1, v3, v5, v7); o_k *= exp(-i pi k / 4) (k = 1: rotation by
// -pi/4; k = 2: -i, exact; k = 3: minus a rotation by +pi/4, the sign taken by the combination).
template <int S> __device__ __forceinline__ void bfly8_lf(float2* v) {
  float2 e[4] = {v[0], v[2 * S], v[4 * S], v[6 * S]};
  float2 o[4] = {v[S], v[3 * S], v[5 * S], v[7 * S]};
  bfly4<-1, 1>(e);
  bfly4<-1, 1>(o);
  o[1] = rot8_fwd<-1>(o[1]);
  o[2] = rot<-1>(o[2]);
  o[3] = rot8_fwd<+1>(o[3]);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    v[k * S] = cadd(e[k], o[k]);
    v[(k + 4) * S] = csub(e[k], o[k]);
  }
  v[3 * S] = csub(e[3], o[3]);
  v[7 * S] = cadd(e[3], o[3]);
}
// Its inverse times 8.
template <int S> __device__ __forceinline__ void ibfly8_lf(float2* v) {
  float2 e[4], o[4];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    e[k] = cadd(v[k * S], v[(k + 4) * S]);
    o[k] = csub(v[k * S], v[(k + 4) * S]);
  }
  e[3] = cadd(v[3 * S], v[7 * S]);
  o[3] = csub(v[7 * S], v[3 * S]);
  o[1] = rot8_inv<-1>(o[1]);
  o[2] = rot<+1>(o[2]);
  o[3] = rot8_inv<+1>(o[3]);
  bfly4<+1, 1>(e);
  bfly4<+1, 1>(o);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[2 * k * S] = e[k];
    v[(2 * k + 1) * S] = o[k];
  }
}
template <int R, int S> __device__ __forceinline__ void bfly_lf(float2* v) {
  if constexpr (R == 8) bfly8_lf<S>(v);
  else bfly<R, -1, S>(v);
}
// Inverse butterfly times R: radix 2 and 4 are symmetric with exact constants (the conjugate
// kernel inverts them); radix 3 and 5 too, to the double-single accuracy of their constants.
template <int R, int S> __device__ __forceinline__ void ibfly_lf(float2* v) {
  if constexpr (R == 8) ibfly8_lf<S>(v);
  else bfly<R, +1, S>(v);
}

// Stage s of the plan: NS = product of the radices of the stages before it.
__host__ __device__ constexpr int stage_ns(int N, int E, int S) {
  int ns = 1;
  for (int i = 0; i < S; ++i) ns *= pick_radix(N / ns, E);
  return ns;
}

// Forward transform of NL lines (as lines_fft with DIR = -1), lifted twiddles.
template <int N, int E, int NBAR, int NL, int NS = 1, int IX = 0, bool PP = false, int CNS = 0>
__device__ __forceinline__ void lines_fft_lf(float2 (*v)[E], float2* sm, int SS, int LS, int t, const float4* tw,
                                             float2* sm2 = nullptr, const float4* twr = nullptr) {
  if constexpr (NS < N) {
    constexpr int P = N / E;
    constexpr int R = pick_radix(N / NS, E);
    static_assert(R > 0, "no factorisation for this (N, E)");
    constexpr int B = E / R;
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int j = t + P * b;
      const int k = j % NS;
      if constexpr (NS > 1) {
        constexpr int OFF = tw_stage_off(N, E, NS);
#pragma unroll
        for (int r = 1; r < R; ++r) {
          const float4 w = NS == CNS ? twr[b * (R - 1) + r - 1] : tw[OFF + (r - 1) * NS + k];
#pragma unroll
          for (int l = 0; l < NL; ++l) v[l][b + r * B] = lift_fwd(v[l][b + r * B], w);
        }
      }
#pragma unroll
      for (int l = 0; l < NL; ++l) bfly_lf<R, B>(v[l] + b);
    }
    if constexpr (NS * R < N) {
      float2* xb = (PP && (IX & 1)) ? sm2 : sm;
      constexpr int NX = num_stages(N, E) - 1;
      if constexpr (!(PP && (IX > 0 || NX % 2 == 0))) fft_bar<NBAR>();
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const int j = t + P * b;
        const int k = j % NS;
        const int base = (j / NS) * NS * R + k;
#pragma unroll
        for (int l = 0; l < NL; ++l)
#pragma unroll
          for (int r = 0; r < R; ++r) xb[l * LS + xoff(base + r * NS, SS)] = v[l][b + r * B];
      }
      fft_bar<NBAR>();
#pragma unroll
      for (int l = 0; l < NL; ++l)
#pragma unroll
        for (int m = 0; m < E; ++m) v[l][m] = xb[l * LS + xoff(t + P * m, SS)];
      lines_fft_lf<N, E, NBAR, NL, NS * R, IX + 1, PP, CNS>(v, sm, SS, LS, t, tw, sm2, twr);
    }
  }
}

// The mirror of lines_fft_lf (times N): stage S = num_stages - 1 down to 0.  Thread t holds the
// frequencies t + P m on entry and the positions t + P m on exit, like lines_fft.  Exchanges
// (IX counts them in execution order) alternate between sm and sm2 under PP as in lines_fft.
template <int N, int E, int NBAR, int NL, int S = num_stages(N, E) - 1, int IX = 0, bool PP = false, int CNS = 0>
__device__ __forceinline__ void lines_ifft_lf(float2 (*v)[E], float2* sm, int SS, int LS, int t, const float4* tw,
                                              float2* sm2 = nullptr, const float4* twr = nullptr) {
  if constexpr (S >= 0) {
    constexpr int P = N / E;
    constexpr int NS = stage_ns(N, E, S);
    constexpr int R = pick_radix(N / NS, E);
    constexpr int B = E / R;
    constexpr int NX = num_stages(N, E) - 1;
    constexpr int IXN = (NS * R < N) ? IX + 1 : IX;
    if constexpr (NS * R < N) {
      // undo the exchange that followed this stage: natural positions out, the stage's in
      float2* xb = (PP && (IX & 1)) ? sm2 : sm;
      if constexpr (!(PP && (IX > 0 || NX % 2 == 0))) fft_bar<NBAR>();
#pragma unroll
      for (int l = 0; l < NL; ++l)
#pragma unroll
        for (int m = 0; m < E; ++m) xb[l * LS + xoff(t + P * m, SS)] = v[l][m];
      fft_bar<NBAR>();
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const int j = t + P * b;
        const int k = j % NS;
        const int base = (j / NS) * NS * R + k;
#pragma unroll
        for (int l = 0; l < NL; ++l)
#pragma unroll
          for (int r = 0; r < R; ++r) v[l][b + r * B] = xb[l * LS + xoff(base + r * NS, SS)];
      }
    }
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int j = t + P * b;
      const int k = j % NS;
#pragma unroll
      for (int l = 0; l < NL; ++l) ibfly_lf<R, B>(v[l] + b);
      if constexpr (NS > 1) {
        constexpr int OFF = tw_stage_off(N, E, NS);
#pragma unroll
        for (int r = 1; r < R; ++r) {
          const float4 w = NS == CNS ? twr[b * (R - 1) + r - 1] : tw[OFF + (r - 1) * NS + k];
#pragma unroll
          for (int l = 0; l < NL; ++l) v[l][b + r * B] = lift_inv(v[l][b + r * B], w);
        }
      }
    }
    lines_ifft_lf<N, E, NBAR, NL, S - 1, IXN, PP, CNS>(v, sm, SS, LS, t, tw, sm2, twr);
  }
}

}  // namespace mx

// Seeded synthetic input on the device: a random, real, divergence-free
// spectrum written straight into the packed half-spectrum layout.  This is
// an input generator (used for large benchmark grids where host generation
// is slow); it holds none of the scheme's arithmetic.
//
// Recipe (per component, E and H independent): complex Gaussian
// coefficients g_k (unit variance per real part) times the envelope
// exp(-|k|^2 / (2 sigma^2)), projected perpendicular to k, with k = 0 and
// the Nyquist planes set to zero, scaled by `amp`.  Hermitian symmetry of the
// kx = 0 column (a real plane) is enforced by drawing each (ky, kz) /
// (-ky, -kz) pair from the smaller of the two counters and conjugating the
// other.
//
// Random numbers: SplitMix64 (Steele, Lea & Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014) applied to
// seed ^ (counter * golden-ratio constant), two 53-bit uniforms per
// counter, Box-Muller for the Gaussian pair.
#include "mx_launch.h"

namespace mx {

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  x += 0x9e3779b97f4a7c15ULL;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ULL;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebULL;
  return x ^ (x >> 31);
}

__device__ __forceinline__ double2 gauss_pair(unsigned long long seed, unsigned long long ctr) {
  const unsigned long long a = splitmix64(seed ^ (ctr * 0x9e3779b97f4a7c15ULL));
  const unsigned long long b = splitmix64(a);
  const double u1 = ((double)(a >> 11) + 1.0) * (1.0 / 9007199254740993.0);  // (0, 1]
  const double u2 = (double)(b >> 11) * (1.0 / 9007199254740992.0);          // [0, 1)
  const double r = sqrt(-2.0 * log(u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  return make_double2(r * c, r * s);
}

template <typename T>
__global__ void k_gen_divfree(cx<T>* __restrict__ spec, long npts, GridParams g, unsigned long long seed, double sigma,
                              double amp) {
  using C = cx<T>;
  const long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npts) return;
  const int x = (int)(p % g.mx);
  const long r = p / g.mx;
  const int y = (int)(r % g.ny), z = (int)(r / g.ny);
  const bool nyq = (y == g.ny / 2) || (z == g.nz / 2);
  const int my = signed_index(y, g.ny), mz = signed_index(z, g.nz);
  const double kx = g.nu[0] * x, ky = g.nu[1] * my, kz = g.nu[2] * mz;
  const double k2 = kx * kx + ky * ky + kz * kz;
  // canonical counter of this mode (kx = 0 column: pair with its mirror)
  long pc = p;
  bool conj = false;
  if (x == 0) {
    const int ym = (g.ny - y) % g.ny, zm = (g.nz - z) % g.nz;
    const long pm = ((long)zm * g.ny + ym) * g.mx;
    if (pm < p) {
      pc = pm;
      conj = true;
    }
  }
  const double env = (nyq || k2 == 0.0) ? 0.0 : amp * exp(-k2 / (2.0 * sigma * sigma));
  for (int f = 0; f < 2; ++f) {  // f = 0: E, f = 1: H
    double2 u[3];
    for (int c = 0; c < 3; ++c) {
      u[c] = gauss_pair(seed, ((unsigned long long)(f * 3 + c) << 40) ^ (unsigned long long)pc);
      if (conj) u[c].y = -u[c].y;
    }
    if (k2 > 0.0) {  // project perpendicular to k (a real direction: keeps the symmetry)
      const double dr = (kx * u[0].x + ky * u[1].x + kz * u[2].x) / k2;
      const double di = (kx * u[0].y + ky * u[1].y + kz * u[2].y) / k2;
      u[0].x -= dr * kx; u[0].y -= di * kx;
      u[1].x -= dr * ky; u[1].y -= di * ky;
      u[2].x -= dr * kz; u[2].y -= di * kz;
    }
    for (int c = 0; c < 3; ++c) {
      // self-mirrored modes of the kx = 0 column (ky, kz in {0, N/2}) are k = 0
      // or Nyquist and carry env = 0, so every nonzero mode has a distinct mirror
      const double re = env * u[c].x, im = env * u[c].y;
      spec[(long)(f * 3 + c) * npts + p] = C{(T)re, (T)im};
    }
  }
}

template <typename T>
cudaError_t launch_gen_divfree(cx<T>* spec, long npts, const GridParams& g, unsigned long long seed, double sigma, double amp,
                               cudaStream_t s) {
  const long blocks = (npts + 255) / 256;
  k_gen_divfree<T><<<(unsigned)blocks, 256, 0, s>>>(spec, npts, g, seed, sigma, amp);
  return cudaGetLastError();
}

template cudaError_t launch_gen_divfree<float>(float2*, long, const GridParams&, unsigned long long, double, double, cudaStream_t);
template cudaError_t launch_gen_divfree<double>(double2*, long, const GridParams&, unsigned long long, double, double, cudaStream_t);

}  // namespace mx

// Allocation-free variant of the spectral pass, for callers that cannot
// call cudaMalloc: code that runs inside another framework's memory pool or
// allocator, code that must not add allocations while a stream is being
// recorded, or embedded hosts that hand the library fixed buffers and
// forbid it from growing device memory.  The caller passes the input and
// output spectra; the only other device memory the pass needs (per-block
// partial sums of the invariants, the block counter and the final record)
// lives in one file-scope __device__ array of fixed size, which every GPU
// that loads the library holds until the process exits.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "../../include/maxexp.h"
#include "mx_launch.h"

namespace {

// Scratch layout: [partials: MAX_BLOCKS x NSUM doubles][record: 16 doubles][counter].
constexpr int MAX_BLOCKS = 304;  // the spectral pass never launches more (2 per SM of a 152-SM GB300)
constexpr size_t PARTIAL_BYTES = (size_t)MAX_BLOCKS * mx::NSUM * sizeof(double);
constexpr size_t RECORD_OFF = PARTIAL_BYTES;
constexpr size_t COUNTER_OFF = RECORD_OFF + 16 * sizeof(double);
constexpr size_t SCRATCH_BYTES = COUNTER_OFF + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_dev_ptr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t scratch_ptr(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_dev_ptr[dev] = p;
  }
  *out = (unsigned char*)g_dev_ptr[dev];
  return cudaSuccess;
}

template <typename T>
cudaError_t launch(int mode, const void* src, void* dst, long npts, const mx::GridParams& g, double t, int blocks,
                   unsigned char* scratch, cudaStream_t s) {
  double* partials = (double*)scratch;
  double* record = (double*)(scratch + RECORD_OFF);
  unsigned* counter = (unsigned*)(scratch + COUNTER_OFF);
  // coefficient kind 2: computed per point in FP64, no table
  return mx::launch_spectral<T>(mode, 2, (const mx::cx<T>*)src, (mx::cx<T>*)dst, npts, g, nullptr, t, blocks, partials,
                                counter, record, s);
}

}  // namespace

extern "C" mx_status mx_spectral_update_noalloc(const void* spec_in, void* spec_out, int nx, int ny, int nz,
                                                const double lo[3], const double hi[3], double eps, double mu,
                                                int precision, double t, mx_invariants* inv_out, void* stream) {
  if (!spec_in || !lo || !hi) return MX_E_INVAL;
  // the pass moves whole 16-byte pieces (double2 points, float4 point pairs)
  if ((((uintptr_t)spec_in) | ((uintptr_t)spec_out)) & 15u) return MX_E_INVAL;
  if (nx < 2 || ny < 2 || nz < 2 || nx % 2 || ny % 2 || nz % 2) return MX_E_INVAL;
  if (!(eps > 0.0) || !(mu > 0.0) || !isfinite(eps) || !isfinite(mu) || !isfinite(t)) return MX_E_INVAL;
  if (precision != MX_FP64 && precision != MX_FP32) return MX_E_INVAL;
  for (int w = 0; w < 3; ++w)
    if (!isfinite(lo[w]) || !isfinite(hi[w]) || !(hi[w] > lo[w])) return MX_E_INVAL;
  const long long npts = (long long)(nx / 2) * ny * nz;
  if (npts >= (1LL << 31)) return MX_E_UNSUPPORTED_N;  // the pass indexes components with 32-bit offsets
  const int mode = spec_out ? (inv_out ? 2 : 1) : (inv_out ? 0 : -1);
  if (mode < 0) return MX_OK;
  const int blocks = mx::spectral_blocks(npts);
  if (blocks > MAX_BLOCKS) return MX_E_UNSUPPORTED_N;  // more partial sums than the scratch holds

  mx::GridParams g;
  g.nx = nx; g.ny = ny; g.nz = nz; g.mx = nx / 2;
  for (int w = 0; w < 3; ++w) g.nu[w] = 2.0 * M_PI / (hi[w] - lo[w]);
  g.qa[0] = g.qa[1] = g.qa[2] = 0;
  g.s0 = 0.0;
  mx::set_material(g, eps, mu);

  cudaStream_t s = (cudaStream_t)stream;
  // reading the invariants back needs a copy into host memory and a wait: neither can be recorded
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return MX_E_CUDA;
  if (cap != cudaStreamCaptureStatusNone && inv_out) return MX_E_INVAL;
  unsigned char* scratch = nullptr;
  if (scratch_ptr(&scratch) != cudaSuccess) return MX_E_CUDA;
  // the block counter and the wait-timeout flag after it must start at zero
  if (cudaMemsetAsync(scratch + COUNTER_OFF, 0, 2 * sizeof(unsigned), s) != cudaSuccess) return MX_E_CUDA;
  cudaError_t e = precision == MX_FP64 ? launch<double>(mode, spec_in, spec_out, npts, g, t, blocks, scratch, s)
                                       : launch<float>(mode, spec_in, spec_out, npts, g, t, blocks, scratch, s);
  if (e != cudaSuccess) return MX_E_CUDA;
  if (!inv_out) return MX_OK;
  double sums[16];
  unsigned flags[2];
  if (cudaMemcpyAsync(sums, scratch + RECORD_OFF, sizeof(sums), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return MX_E_CUDA;
  if (cudaMemcpyAsync(flags, scratch + COUNTER_OFF, sizeof(flags), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return MX_E_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return MX_E_CUDA;
  if (flags[1]) return MX_E_TIMEOUT;
  const double N = (double)nx * ny * nz, N2 = N * N;
  mx_invariants& r = *inv_out;
  memset(&r, 0, sizeof(r));
  r.t = t;
  r.step = 0;
  r.E1 = sums[0] / (2 * N2);
  r.E2 = sums[1] / (2 * N2);
  for (int w = 0; w < 3; ++w) {
    r.E3[w] = sums[2 + w] / (2 * N2);
    r.E4[w] = sums[5 + w] / (2 * N2);
    r.M1[w] = -sums[10 + w] / N2;
    r.M2[w] = -r.M1[w];
  }
  r.H1 = sums[8] / N2;
  r.H2 = sums[9] / N2;
  r.divE = sqrt(sums[13] > 0.0 ? sums[13] : 0.0) / N;
  r.divH = sqrt(sums[14] > 0.0 ? sums[14] : 0.0) / N;
  return MX_OK;
}

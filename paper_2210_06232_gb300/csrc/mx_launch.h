// Host-side launchers of the CUDA kernels (internal to libmaxexp).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "mx_kernels.cuh"

namespace mx {

// FFT lengths with a compiled plan: 2^a (1..512), 3*2^a (3..384), 5*2^a (5..320).
bool fft_len_supported(int n);

// Number of SMs of the current device (cached per process).
int num_sms();

// Every device (and pinned host) allocation of the library goes through these, so that a test
// can make the k-th one fail (mx_debug_fail_alloc) and check the callers' cleanup paths.
cudaError_t dev_alloc(void** p, size_t bytes);
cudaError_t host_alloc_pinned(void** p, size_t bytes);

// Twiddle tables: twv<T> entries exp(-2 pi i j / n) (FP32: hi + lo pairs).
// bps: persistent grid of bps blocks per SM; 0 = one block per tile.
// counter: the context's block counter (counter[1] = wait-timeout flag); with
// counter != nullptr rows of >= 32 complex values use the bulk-copy pipeline.
template <typename T>
cudaError_t launch_x_r2c(int M, const T* in_e, const T* in_h, cx<T>* out, long rows3, long nrows, const twv<T>* tw,
                         int bps, cudaStream_t s, unsigned* counter = nullptr);
template <typename T>
cudaError_t launch_x_c2r(int M, const cx<T>* in, T* out_e, T* out_h, long rows3, long nrows, const twv<T>* tw,
                         double scale, int bps, cudaStream_t s, unsigned* counter = nullptr);
// dir = -1 forward, +1 inverse (unnormalised).  counter set: tiles moved by the tensor-copy engine
// (where the layout allows); dbuf: two input stages that double as exchange buffers (lengths that are
// multiples of 16), else one input stage and a separate exchange buffer.
template <typename T>
cudaError_t launch_strided(int N, int dir, cx<T>* data, long inner, long outer, const twv<T>* tw, int bps,
                           cudaStream_t s, unsigned* counter = nullptr, bool dbuf = false);

// Spectral pass.  mode: 0 = invariants only, 1 = update only, 2 = update + invariants.
// coef_kind: 0 = Coef<T> table, 1 = CoefHL table (float only), 2 = direct Coef<T>, 3 = direct CoefHL.
template <typename T>
cudaError_t launch_spectral(int mode, int coef_kind, const cx<T>* src, cx<T>* dst, long npts, const GridParams& g,
                            const void* tab, double t, int blocks, double* partials, unsigned* counter, double* record,
                            cudaStream_t s);
// Fill a coefficient table (coef_kind 0 or 1) for time t.
template <typename T>
cudaError_t launch_coef_table(int coef_kind, void* tab, int nq, const GridParams& g, double t, cudaStream_t s);

// Seeded random divergence-free spectrum (input generator), packed layout.
template <typename T>
cudaError_t launch_gen_divfree(cx<T>* spec, long npts, const GridParams& g, unsigned long long seed, double sigma,
                               double amp, cudaStream_t s);

// Fused z forward -> update (+ invariants when record != nullptr) -> z inverse
// of the literal form, in place on a spectrum after the x and y passes.
// coef_kind as for launch_spectral (table kinds need `tab`, direct kinds ignore it).
bool zfused_supported(int nz, bool fp64);
// Values per thread of the line FFT plans: the FFT passes (length n) and the fused z pass
// (0 when it has no plan for n); the twiddle tables are laid out for these plans.
int fft_line_E(int n);
int zfused_line_E(int n, bool fp64);
// Columns per tile of the fused z pass for length n.
int zfused_tile_cols(int n, bool fp64);
template <typename T>
// pipelined: tensor-copy tiles (when the layout allows), else per-thread loads and stores.
cudaError_t launch_z_fused(int coef_kind, cx<T>* data, const GridParams& g, const void* tab, double t,
                           const twv<T>* tw, int grid, bool pipelined, double* partials, unsigned* counter,
                           double* record, cudaStream_t s);

// Blocks used by the spectral pass for npts points (fixed per size: makes
// the invariant reduction order independent of what else runs).
int spectral_blocks(long npts);

}  // namespace mx

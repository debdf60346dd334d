/*
 * maxexp — exponential-integrator Fourier pseudospectral solver for the
 * periodic 3D Maxwell equations on one NVIDIA GB300 (sm_103a).
 *
 * The method is the fully discrete scheme of Wang & Jiang, "Time exponential
 * integrator Fourier pseudospectral methods with high accuracy and multiple
 * conservation laws for three-dimensional Maxwell's equations"
 * (arXiv 2210.06232): Def. 2.3, Alg. 1 (initial values: 3D DFT of the six
 * field components), Alg. 2 (exact per-wavevector exponential of the
 * spectral curl, Prop. 2.1-2.2, then the inverse 3D DFT), and the discrete
 * invariants of Sec. 4 (Thm 4.1 energies, Thm 4.3 helicities, Thm 4.4
 * momenta, Thm 4.6 divergence).
 *
 * Conventions shared by every call
 *  - Every function returns an mx_status and never aborts.  A CUDA error met
 *    while enqueuing work is returned as MX_E_CUDA and latched in the
 *    context: every later call on that context returns it again.
 *  - Field arrays: E and H are each 3 components x [Nz][Ny][Nx] values,
 *    x fastest (the vector ordering of Sec. 2.2, index
 *    Nx*Ny*(l-1) + Nx*(k-1) + j), component order (x, y, z).  The element
 *    type is double for MX_FP64 contexts and float for MX_FP32 contexts.
 *  - Host pointers are read or written before the call returns.  Device
 *    pointers are borrowed: the caller keeps ownership and keeps them valid
 *    until mx_sync returns.  All device work is ordered on the context's
 *    stream.
 *  - The library owns every device buffer it allocates and frees it in
 *    mx_destroy.
 */
#ifndef MAXEXP_H
#define MAXEXP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mx_ctx mx_ctx;

typedef enum {
  MX_OK = 0,
  MX_E_INVAL = 1,           /* bad argument (odd N, eps <= 0, non-finite h, NULL pointer, ...) */
  MX_E_UNSUPPORTED_N = 2,   /* grid size without a compiled FFT plan */
  MX_E_NOMEM = 3,           /* device allocation failed */
  MX_E_CUDA = 4,            /* CUDA error (latched) */
  MX_E_TIMEOUT = 5,         /* a bounded device wait gave up */
  MX_E_STATE = 6            /* call out of order (e.g. step before load) */
} mx_status;

typedef enum { MX_FP64 = 0, MX_FP32 = 1 } mx_precision;

/*
 * Forms of one time step (all compute the same map, Def. 2.3 with
 * Delta t = h, up to rounding):
 *  MX_FORM_LITERAL  : the state is the six physical fields; every step runs
 *                     Alg. 1 step 4 (forward 3D real DFT), Alg. 2 steps 1-4
 *                     with t_end = h, and Alg. 2 step 5 (inverse 3D DFT).
 *  MX_FORM_SPECTRAL : the state is the spectrum of the fields at load time
 *                     (Alg. 1, run once by mx_load_fields); step n writes the
 *                     spectrum at t_n = n h as R(t_n) applied to it (Alg. 2
 *                     steps 1-4 with t_end = t_n, phase c|k|t_n taken in
 *                     FP64).  Physical fields are produced by mx_read_fields
 *                     (Alg. 2 step 5).
 *  MX_FORM_XY       : the state is the spectrum of the fields in x and y (the
 *                     first two transforms of Alg. 1, run by mx_load_fields)
 *                     with z in physical space; every step runs the z
 *                     transform, Alg. 2 steps 1-4 with t_end = h and the
 *                     inverse z transform in one pass over HBM (the literal
 *                     step without its x and y transforms, which cancel
 *                     between steps).  mx_read_fields runs the inverse y and
 *                     x transforms on a copy, so the state is unchanged.  nz
 *                     must have a fused plan (2^a, 3*2^a in FP32; 2^a in
 *                     FP64), otherwise MX_E_UNSUPPORTED_N.
 */
typedef enum { MX_FORM_LITERAL = 0, MX_FORM_SPECTRAL = 1, MX_FORM_XY = 2 } mx_form;

/*
 * Discrete invariants of Sec. 4 at one time level.  E3..E6, M1, M2 hold the
 * k = 1, 2, 3 (x, y, z) members of each family.  divE and divH are the
 * discrete L2 norms ||D~.(eps E)||_N and ||D~.(mu H)||_N of Thm 4.6, with
 * <u,v>_N = (1/(Nx Ny Nz)) sum u v.  E5 and E6 vanish identically for real
 * fields (D_k is antisymmetric) and are returned as 0.  M2 = -M1 exactly
 * (B_k^T = -B_k).  Helicity H2 is the time-derivative helicity printed with
 * the label H_1 in Thm 4.3.
 */
typedef struct {
  double t;          /* time of the record */
  long long step;    /* step index n (0 = load time) */
  double E1, E2, E3[3], E4[3], E5[3], E6[3];
  double H1, H2;
  double M1[3], M2[3];
  double divE, divH;
} mx_invariants;

/*
 * Create a solver context.
 *  nx, ny, nz : even grid sizes >= 2 (Def. 2.3 Step 1).  Each of nx/2, ny,
 *               nz must be 2^a, 3*2^a or 5*2^a and at most 512 (ny, nz) or
 *               256 (nx/2); otherwise MX_E_UNSUPPORTED_N.
 *  lo, hi     : domain [lo_w, hi_w] per axis (x, y, z), hi_w > lo_w; the
 *               collocation points are lo_w + (j-1)(hi_w - lo_w)/N_w.
 *  eps, mu    : permittivity and permeability, positive (eq. maxsys).
 *  precision  : MX_FP64 or MX_FP32 (arithmetic and storage of the fields;
 *               phases and invariant sums are FP64 in both).
 *  form       : MX_FORM_LITERAL, MX_FORM_SPECTRAL or MX_FORM_XY.
 *  stream     : a cudaStream_t to order all work on, or NULL for the
 *               legacy default stream.
 * On success *out owns all device memory of the solver (its size is
 * mx_footprint_bytes); on failure *out is NULL.
 */
mx_status mx_create(mx_ctx** out, int nx, int ny, int nz, const double lo[3], const double hi[3], double eps, double mu,
                    int precision, int form, void* stream);

/* Device bytes a context of this shape would allocate (HBM budgeting). */
mx_status mx_footprint_bytes(int nx, int ny, int nz, int precision, int form, size_t* bytes);

/*
 * Load the initial fields E0, H0 at the collocation points (Def. 2.3
 * Step 2) and run Alg. 1 (forward 3D DFT).  Resets time to 0 and the
 * invariant record list to the record of t = 0.
 *  E, H      : 3 x [Nz][Ny][Nx] each, element type of the precision.
 *  on_device : 0 = host pointers (copied), 1 = device pointers (borrowed
 *              until mx_sync).
 */
mx_status mx_load_fields(mx_ctx* ctx, const void* E, const void* H, int on_device);

/*
 * Advance nsteps steps of size h (any real h, including negative: the
 * scheme has no step restriction, Sec. 2.5).  When invariants_every > 0 the
 * invariants of the state after every step n with n % invariants_every == 0
 * are appended to the record list; 0 records none.  Work is enqueued on the
 * context stream; the call does not wait for it.
 */
mx_status mx_step(mx_ctx* ctx, double h, long long nsteps, int invariants_every);

/*
 * Enqueue-only variants for host buffers that are pinned (page-locked):
 * the copy, transform and record are placed on the context stream and the
 * call returns without waiting; the host buffer must stay valid and
 * unmodified (load) or unread (read) until mx_sync.
 */
mx_status mx_load_fields_async(mx_ctx* ctx, const void* E, const void* H);
mx_status mx_read_fields_async(mx_ctx* ctx, void* E, void* H);

/*
 * Write the fields at the current time (Def. 2.3 Step 4).
 *  E, H      : 3 x [Nz][Ny][Nx] each, element type of the precision.
 *  on_device : 0 = host pointers (the call waits for the copy), 1 = device
 *              pointers (written in stream order; mx_sync to wait).
 */
mx_status mx_read_fields(mx_ctx* ctx, void* E, void* H, int on_device);

/*
 * Copy up to max invariant records (oldest first, starting at load time)
 * to out; *n_written receives the count.  Waits for the stream.  With
 * max == 0 nothing is copied (out may be NULL) and *n_written receives the
 * number of records held.
 */
mx_status mx_read_invariants(mx_ctx* ctx, mx_invariants* out, long long max, long long* n_written);

/*
 * Load a seeded random, real, divergence-free initial state directly in
 * Fourier space (an input generator for large grids, not part of the
 * scheme): per component complex Gaussian coefficients times
 * exp(-|k|^2 / (2 sigma^2)), projected perpendicular to k, k = 0 and the
 * Nyquist planes zero, scaled so each field component has RMS about 1.
 * E and H are independent.  Resets time and records like mx_load_fields.
 * The same (seed, sigma, grid) gives the same fields on every device.
 */
mx_status mx_load_random_divfree(mx_ctx* ctx, unsigned long long seed, double sigma);

/*
 * FFT schedule autotuner (no counterpart in the paper: it picks kernels and
 * launch shapes).  Each transform pass of this grid shape (x R2C, y forward,
 * z forward, z inverse, y inverse, x C2R and, for a literal-form context with
 * a fused z plan, the fused z pass) is timed on the context's own work
 * buffers with every candidate schedule: the kernel variant (tiles moved by
 * the bulk/tensor-copy engine where the layout allows; per-thread loads with
 * a register prefetch; for the y and z passes also the copy engine with two
 * input stages that double as exchange buffers) and the persistent grid (1,
 * 2, 4, 8 blocks per SM, 0 = one block per tile for the second variant; 1 or
 * 2 for the fused z pass).  The fastest is kept in a process-wide table keyed
 * by (pass, precision, nx, ny, nz) and used by every context of that shape.
 * Waits for the stream.  Skipped (MX_OK) while the stream is being captured,
 * or for a loaded literal-form context (its state lives in the buffers the
 * timing overwrites); a spectral-form context keeps its state.  Untuned
 * passes use the copy-engine variant with 4 blocks per SM (y and z passes of
 * lines of 512 or more: the two-stage variant; fused z: 2 blocks per SM).
 */
mx_status mx_autotune(mx_ctx* ctx);
/* The schedules in use, sched[0..6] for the seven passes in the order above
 * (n >= 7): blocks per SM + 16 * variant (0: copy-engine tiles, 1: register
 * prefetch, 2: two-stage copy-engine tiles). */
mx_status mx_schedule(mx_ctx* ctx, int* sched, int n);
/* Set the schedules of this grid shape and precision (the process-wide table
 * mx_autotune fills), sched[0..6] coded as mx_schedule reports them, for every
 * context of the shape: a tuned table saved earlier, or one variant forced for
 * a test.  MX_E_INVAL (nothing set) for an unknown variant, the two-stage
 * variant on a pass other than y and z, a copy-engine variant with 0 blocks per
 * SM, or a fused z pass with other than 1 or 2 blocks per SM. */
mx_status mx_set_schedule(mx_ctx* ctx, const int* sched, int n);

/*
 * Batched form (no counterpart in the paper, which solves one problem at a
 * time): n independent instances, each its own grid, domain, eps, mu and
 * step size h, all in the spectral form and one precision, advanced
 * together.  mx_batch_step(b, K, every) advances every instance K steps of
 * its own h with ONE persistent cooperative kernel launch (per step: the
 * coefficient tables of all instances, a grid barrier, the exponential
 * update of all instances over one chunk list, a grid barrier); the launch
 * is captured once per K into a CUDA graph and replayed.  Each instance is a
 * context (mx_batch_instance) for loading, reading fields and invariants and
 * autotuning.  An instance's fields and invariants are bit-identical whether
 * it runs alone or in any batch.  Device memory: the instances' contexts
 * plus about 1 KB of invariant partial sums per 512-point chunk (FP32).
 */
typedef struct mx_batch mx_batch;
typedef struct {
  int nx, ny, nz;           /* even grid sizes, as for mx_create */
  double lo[3], hi[3];      /* domain */
  double eps, mu;           /* positive */
  double h;                 /* step size of this instance */
} mx_instance_desc;

mx_status mx_batch_create(mx_batch** out, const mx_instance_desc* inst, int n, int precision, void* stream);
/*
 * The same in either form.  form = MX_FORM_LITERAL: every instance is a
 * literal-form context (state = the physical fields; each step the 3D R2C,
 * the fused z pass with the update and invariants, the 3D C2R), autotuned
 * at creation for its shape (mx_autotune); mx_batch_step(b, K, every) runs
 * the K steps of all instances as parallel branches of one CUDA graph (one
 * stream per instance), captured once per (K, every, step phases) and
 * replayed; the records the graph writes are appended to each instance's
 * list after the launch.  Instances are bit-identical alone or in any batch.
 * form = MX_FORM_XY: the same with xy-resident contexts (each step one fused
 * z pass per instance); every instance's nz needs a fused plan, otherwise
 * MX_E_UNSUPPORTED_N.
 * mx_batch_create is mx_batch_create_form with MX_FORM_SPECTRAL.
 */
mx_status mx_batch_create_form(mx_batch** out, const mx_instance_desc* inst, int n, int precision, int form,
                               void* stream);
mx_status mx_batch_size(mx_batch* b, int* n);
/* Context of instance i (owned by the batch: do not destroy it). */
mx_status mx_batch_instance(mx_batch* b, int i, mx_ctx** ctx);
/* mx_load_random_divfree on every instance, instance i with seed + i. */
mx_status mx_batch_load_random(mx_batch* b, unsigned long long seed, double sigma);
/* Advance every instance nsteps steps; records invariants as mx_step does. */
mx_status mx_batch_step(mx_batch* b, long long nsteps, int invariants_every);
/* Wait for the batch; MX_E_TIMEOUT if a bounded device wait gave up. */
mx_status mx_batch_sync(mx_batch* b);
/* 1 when the steps are replayed from a captured CUDA graph, 0 before the
 * first step, -e when capture was refused with CUDA error e (steps are then
 * launched directly).  A batch created with a NULL stream uses a stream of
 * its own (the legacy default stream cannot be captured). */
mx_status mx_batch_graph_used(mx_batch* b, int* used);
/* Blocks and threads per block of the spectral form's persistent launch (0, 0 for the literal
 * form, which launches each instance's passes). */
mx_status mx_batch_launch_shape(mx_batch* b, int* blocks, int* threads);
void mx_batch_destroy(mx_batch* b);

/*
 * Serving form (no counterpart in the paper): a request loop that solves
 * problems of different grids, domains, eps/mu, precisions and end times as
 * they arrive.  A worker thread admits queued requests in arrival order while
 * the HBM budget and `max_active` allow, each into a resident spectral-form
 * context from a pool keyed by (precision, grid, domain) or newly created
 * (idle pooled contexts are destroyed, least recently used first, when a new
 * shape needs memory; the budget counts active and pooled contexts by
 * mx_footprint_bytes).  Every context has its own CUDA stream, so requests
 * admitted while others run overlap on the device.  A request runs
 * mx_load_fields (host E0, H0), mx_step(t_end / nsteps, nsteps, ...) and
 * mx_read_fields (host E_out, H_out); with nsteps = 1 it is the paper's
 * single step of size t_end (Sec. 2.5).  Host buffers are borrowed until the
 * request is done and should be pinned (page-locked): pageable buffers make
 * the copies block the worker.  A request that can never fit the budget
 * fails with MX_E_NOMEM.  Latency is completion minus submission (host
 * steady clock).
 */
typedef struct mx_server mx_server;
typedef struct {
  int nx, ny, nz;
  double lo[3], hi[3];
  double eps, mu;
  int precision;            /* MX_FP32 or MX_FP64 */
  double t_end;             /* final time */
  long long nsteps;         /* >= 1 steps of size t_end / nsteps */
  int invariants_every;     /* record every k steps; 0: t = 0 and t_end only */
  const void* E0;           /* host, 3 x [nz][ny][nx] of the precision */
  const void* H0;
  void* E_out;              /* host, receives the fields at t_end */
  void* H_out;
} mx_request;
typedef struct {
  long long submitted, admitted, completed, rejected, queued, active, pooled_contexts;
  size_t hbm_in_use, hbm_high_water, hbm_budget;
  /* device concurrency since creation: the most requests admitted and not yet
   * finished at once; busy_s = seconds with at least one; mean_concurrent = their
   * time-weighted mean count over busy_s; request_s_sum = the sum over finished
   * requests of admission-to-completion seconds (> busy_s when requests overlap) */
  long long max_concurrent;
  double mean_concurrent, busy_s, request_s_sum;
} mx_server_info;

mx_status mx_server_create(mx_server** out, size_t hbm_budget_bytes, int max_active);
mx_status mx_server_submit(mx_server* s, const mx_request* req, long long* id);
/* state: 0 queued, 1 running, 2 done, < 0 failed with status -state. */
mx_status mx_server_poll(mx_server* s, long long id, int* state);
/* Wait up to timeout_s seconds; MX_E_TIMEOUT if the request is not done. */
mx_status mx_server_wait(mx_server* s, long long id, double timeout_s, int* state);
/* Invariant records (max == 0: count only) and latency of a done request;
 * release != 0 forgets the request. */
mx_status mx_server_result(mx_server* s, long long id, mx_invariants* inv, long long max, long long* n,
                           double* latency_s, int release);
mx_status mx_server_stats(mx_server* s, mx_server_info* out);
/* Waits for running requests, then frees every context. */
void mx_server_destroy(mx_server* s);

/* Kernel classes timed by mx_profile. */
typedef enum {
  MX_K_X_R2C = 0,     /* real rows -> packed half spectrum along x */
  MX_K_X_C2R = 1,     /* packed half spectrum -> real rows along x */
  MX_K_Y_FFT = 2,     /* complex DFT along y (forward or inverse) */
  MX_K_Z_FFT = 3,     /* complex DFT along z (forward or inverse) */
  MX_K_SPECTRAL = 4,  /* per-k exponential update and/or invariant sums */
  MX_K_TABLE = 5,     /* per-|k|^2 coefficient table */
  MX_K_GEN = 6,       /* input generator */
  MX_K_ZFUSED = 7,    /* z DFT + update + inverse z DFT in one pass */
  MX_K_COUNT = 8
} mx_kernel_kind;

/*
 * Per-kernel timing: with enable != 0, every kernel the context launches is
 * bracketed by CUDA events on the context stream (clears earlier samples).
 * mx_profile_read waits for the stream and fills ms[MX_K_COUNT] with the
 * summed device time and launches[MX_K_COUNT] with the launch counts since
 * the last read, then clears them.
 */
mx_status mx_profile(mx_ctx* ctx, int enable);
mx_status mx_profile_read(mx_ctx* ctx, double* ms, long long* launches);

/*
 * Allocation-free spectral pass.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc (code running inside
 * another framework's memory pool, code that must not allocate while a
 * stream is being recorded, embedded hosts that forbid the library from
 * growing device memory).  It applies the exact exponential R(t) to a
 * caller-owned packed half spectrum and/or reduces its invariants, without
 * a context and without allocating anything.
 *  spec_in   : device, 6 x [nz][ny][nx/2] complex (E_x, E_y, E_z, H_x, H_y,
 *              H_z; element = 2 x double for MX_FP64, 2 x float for MX_FP32),
 *              the unnormalised 3D DFT of real fields with column kx = 0
 *              holding the kx = 0 plane in its real part and the kx = nx/2
 *              plane in its imaginary part.
 *              Must start on a 16-byte boundary.
 *  spec_out  : device, same layout and alignment; receives R(t) spec_in
 *              (may equal spec_in).  NULL: no update, invariants of spec_in
 *              only.
 *  inv_out   : host; receives the invariants of the written spectrum (of
 *              spec_in when spec_out is NULL), t = t, step = 0.  NULL: none.
 *              When given, the call waits for the stream, so it cannot be
 *              made while the stream is being captured (MX_E_INVAL); the
 *              update alone (inv_out NULL) enqueues only a memset and one
 *              kernel.
 *  nx..mu, precision : as for mx_create (any even sizes >= 2).
 *  stream    : cudaStream_t or NULL.
 * Device memory: besides spec_in and spec_out the pass uses one static
 * device array of about 40 KB (partial sums of at most 304 blocks, a block
 * counter and one record), present on every device that loads the library.
 * Coefficients are computed per point in FP64 (no table), so the pass is
 * slower than mx_step.  Errors: MX_E_INVAL for bad arguments (including a
 * spectrum pointer that is not 16-byte aligned, checked before anything is
 * enqueued, and inv_out during a stream capture), MX_E_UNSUPPORTED_N when
 * (nx/2) * ny * nz >= 2^31, MX_E_CUDA otherwise.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the array: calls that overlap on the GPU (concurrent
 * streams or threads) race and must be serialised by the caller.
 */
mx_status mx_spectral_update_noalloc(const void* spec_in, void* spec_out, int nx, int ny, int nz, const double lo[3],
                                     const double hi[3], double eps, double mu, int precision, double t,
                                     mx_invariants* inv_out, void* stream);

/*
 * Failure injection for tests (no counterpart in the paper; the library's
 * error paths are exercised on the host, without a GPU fault).
 *
 * mx_debug_fail_alloc(k), k >= 0: the k-th device or pinned-host allocation
 * the library makes from now on (0 = the next one, counted across all
 * contexts, batches and servers of the process) fails once, as if the
 * memory were exhausted; the caller sees MX_E_NOMEM with everything it had
 * allocated released.  k < 0 disarms.  Process-wide; not for production use.
 *
 * mx_debug_wait_limit(ctx, tries): the waits of the context's fused z pass
 * for its tensor-copied tiles give up after `tries` tries (0: at once)
 * instead of the default bound; tries < 0 restores the default.  A wait
 * that gives up makes its block leave the pass (after the copy it issued
 * has landed) and latches MX_E_TIMEOUT, which mx_sync and every later call
 * on the context return.  Lets a test reach the timeout path without a
 * fault or a hang.
 */
mx_status mx_debug_fail_alloc(long long k);
mx_status mx_debug_wait_limit(mx_ctx* ctx, long long tries);

/*
 * Arithmetic peak of the current device (no counterpart in the paper: the
 * denominator of the ALU rooflines of the FP64 forms): FMA throughput of
 * the FP64 (precision MX_FP64) or FP32 pipe in flop/s (an FMA counts two),
 * best of five timed launches of independent FMA chains on every SM.
 * Allocates and frees a small output buffer; waits for the device.
 */
mx_status mx_fma_peak(int precision, double* flops_per_s);

/* Measurement of what HBM delivers for the access pattern of the fused z pass
 * (no counterpart in the paper): buf holds a spectrum [6][nz][ny][mx] of
 * complex FP32 (device memory, 16-byte aligned, left unchanged: every tile is
 * read into shared memory by tensor copy and written back in place), moved in
 * tiles of `cols` columns x nz x (24 / cols) components by one persistent
 * block per SM, the next tile's copy in flight while a tile is stored.  The
 * rows of a tile are cols x 8 bytes (cols = 4: 32 bytes, the fused pass's
 * tiles; 8: 64; 16: 128) at a stride of one z plane.  *gbs = bytes read and
 * written per launch / the best of `reps` timed launches (after one warm-up).
 * MX_E_INVAL for a null or misaligned buffer, cols other than 4, 8, 16, mx not
 * a multiple of cols, nz outside 2..512 or reps < 1; MX_E_TIMEOUT if a copy
 * wait gave up. */
mx_status mx_tile_stream(void* buf, int mx, int ny, int nz, int cols, int reps, double* gbs);

/*
 * DFT-as-GEMM evaluation (a measurement, not a step of the method; the
 * paper's cost model, Sec. 2.5, puts the time in the transforms): applies
 * `reps` radix-8 stages (twiddle by fixed unit-modulus / sqrt(8) factors,
 * then an 8-point DFT, exp(-2 pi i / 8) kernel) to tiles of 128 independent
 * 8-point vectors held on chip, and reports the kernel time.
 *  variant 0 : FMA pipe, the register butterfly of the line FFTs.
 *  variant 1, 3, 6 : tensor cores (tcgen05.mma, kind::tf32, 128 x 16 x 16
 *            per tile, result in tensor memory) with 1, 3 or 6 products of
 *            TF32-split operands (1: TF32 accuracy; 6: about FP32's).
 *  in, out : device, [tiles * 128][8] complex FP32 (interleaved), 16-byte
 *            aligned; caller-owned.
 *  ms      : host; kernel time from CUDA events on the legacy stream.
 * Allocates and frees a small constant buffer; waits for the device.
 * Errors: MX_E_INVAL (arguments), MX_E_TIMEOUT (a wait for the tensor core
 * gave up), MX_E_CUDA.
 */
mx_status mx_dft8_stage_eval(int variant, const void* in, void* out, long long tiles, int reps, double* ms);

/* Current time and step count of the context. */
mx_status mx_time(mx_ctx* ctx, double* t, long long* step);

/* Wait for all work of the context; returns a latched error if any. */
mx_status mx_sync(mx_ctx* ctx);

/* Static description of a status code. */
const char* mx_strerror(mx_status status);

/* Release the context and all its device memory (NULL is ignored). */
void mx_destroy(mx_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* MAXEXP_H */

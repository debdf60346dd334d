// C ABI of libmaxexp: context, plans, device buffers and the step driver.
// The public contract is documented in include/maxexp.h.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/maxexp.h"
#include "mx_launch.h"

using mx::GridParams;

#include <atomic>

namespace mx {

// Allocation fault injection (mx_debug_fail_alloc): when g_fail_at >= 0, the allocation with that
// index (counted from the arming call) fails once with cudaErrorMemoryAllocation.
static std::atomic<long long> g_fail_at{-1};
static std::atomic<long long> g_alloc_index{0};

static bool injected_failure() {
  if (g_fail_at.load(std::memory_order_relaxed) < 0) return false;
  const long long i = g_alloc_index.fetch_add(1);
  long long k = i;
  return g_fail_at.compare_exchange_strong(k, -1);  // one-shot
}

cudaError_t dev_alloc(void** p, size_t bytes) {
  *p = nullptr;
  if (injected_failure()) return cudaErrorMemoryAllocation;
  return cudaMalloc(p, bytes);
}

cudaError_t host_alloc_pinned(void** p, size_t bytes) {
  *p = nullptr;
  if (injected_failure()) return cudaErrorMemoryAllocation;
  return cudaMallocHost(p, bytes);
}

}  // namespace mx

#include "mx_ctx.h"

namespace {

constexpr int REC_STRIDE = 16;  // doubles per invariant record (NSUM used)

bool len_ok(int n) {
  if (n < 1 || n > 512) return false;
  int m = n;
  while (m % 2 == 0) m /= 2;
  return m == 1 || m == 3 || m == 5;
}

mx_status cuda_fail(mx_ctx* c, cudaError_t e) {
  if (e == cudaSuccess) return MX_OK;
  if (c) c->err = MX_E_CUDA;
  return MX_E_CUDA;
}

#define MX_CHECK(c, expr)                                      \
  do {                                                         \
    cudaError_t _e = (expr);                                   \
    if (_e != cudaSuccess) {                                   \
      if (_e == cudaErrorMemoryAllocation) return MX_E_NOMEM;  \
      return cuda_fail((c), _e);                               \
    }                                                          \
  } while (0)

// exp(-2 pi i j / n) for j < n in long double (at least 64-bit significands: the FP32 tables keep
// hi + lo pairs, the lifting constants are taken from the angle), reduced to the first quadrant
// exactly when 4 | n.
using ldvec = std::vector<long double>;
void twiddles(int n, ldvec& re, ldvec& im) {
  const long double PI = 3.141592653589793238462643383279502884L;
  re.resize(n);
  im.resize(n);
  for (int j = 0; j < n; ++j) {
    long double c, s;
    if (n % 4 == 0) {
      const int q = (4 * j) / n, r = 4 * j - q * n;  // angle = (q + r/n) * pi/2
      const long double a = (PI / 2.0L) * ((long double)r / (long double)n);
      const long double ca = cosl(a), sa = sinl(a);
      switch (q) {
        case 0: c = ca; s = sa; break;
        case 1: c = -sa; s = ca; break;
        case 2: c = -ca; s = -sa; break;
        default: c = sa; s = -ca; break;
      }
    } else {
      const long double a = 2.0L * PI * (long double)j / (long double)n;
      c = cosl(a);
      s = sinl(a);
    }
    re[j] = c;
    im[j] = -s;
  }
}

// Appends the stage-major twiddle table of the length-n line FFT with E values per
// thread (mx::tw_stage_off): stage (NS, R), entry [r-1][k] = exp(-2 pi i r k / (NS R)).
void stage_twiddles(int n, int E, ldvec& re, ldvec& im) {
  ldvec wr, wi;
  twiddles(n, wr, wi);
  for (int ns = 1; ns < n;) {
    const int r = mx::pick_radix(n / ns, E);
    if (r <= 0) return;
    if (ns > 1)
      for (int q = 1; q < r; ++q)
        for (int k = 0; k < ns; ++k) {
          const long j = ((long)q * k * (n / (ns * r))) % n;
          re.push_back(wr[j]);
          im.push_back(wi[j]);
        }
    ns *= r;
  }
}

// Per-axis tables of the FFT kernels:
//   x (line of nx reals = M = nx/2 complex): exp(-2 pi i k / nx) for k < M (packing),
//     then the stage table of the M-point FFT;
//   y: the stage table of the ny-point FFT;
//   z: the stage table of the nz-point FFT, then that of the fused z pass's plan
//     (starting at entry *zf_off).
void axis_twiddles(int axis, int n, bool fp64, ldvec& re, ldvec& im, int* zf_off) {
  re.clear();
  im.clear();
  if (axis == 0) {
    const int M = n / 2;
    ldvec wr, wi;
    twiddles(n, wr, wi);
    re.assign(wr.begin(), wr.begin() + M);
    im.assign(wi.begin(), wi.begin() + M);
    stage_twiddles(M, mx::fft_line_E(M), re, im);
    return;
  }
  stage_twiddles(n, mx::fft_line_E(n), re, im);
  if (axis == 2) {
    *zf_off = (int)re.size();
    const int ez = mx::zfused_line_E(n, fp64);
    if (ez > 0) stage_twiddles(n, ez, re, im);
  }
}

// FP64 entries: lifting constants dd2 (p, u, sign, 0) of every twiddle.  FP32 entries: float4
// hi + lo pairs, except the fused z pass's lifting constants (p, u, sign, 0).
cudaError_t upload_twiddles(mx_ctx* c, int axis, int n, void** dst) {
  ldvec re, im;
  int zf_off = 0;
  axis_twiddles(axis, n, c->prec == MX_FP64, re, im, &zf_off);
  if (axis == 2) c->twz_zf = zf_off;
  n = std::max<int>(1, (int)re.size());
  re.resize(n, 1.0L);
  im.resize(n, 0.0L);
  if (c->prec == MX_FP64) {
    cudaError_t e = mx::dev_alloc(dst, (size_t)n * sizeof(mx::dd2));
    if (e != cudaSuccess) return e;
    // lifting constants (p, u, sign, 0) of the rotation by the twiddle's angle (mx_fft.cuh, twmul)
    std::vector<mx::dd2> h(n);
    for (int j = 0; j < n; ++j) {
      const long double PI = 3.141592653589793238462643383279502884L;
      long double a = atan2l(im[j], re[j]);
      double sg = 1.0;
      if (a > PI / 2) a -= PI, sg = -1.0;
      else if (a < -PI / 2) a += PI, sg = -1.0;
      h[j] = mx::dd2{(double)(-tanl(0.5L * a)), (double)sinl(a), sg, 0.0};
    }
    return cudaMemcpy(*dst, h.data(), n * sizeof(mx::dd2), cudaMemcpyHostToDevice);
  }
  cudaError_t e = mx::dev_alloc(dst, (size_t)n * sizeof(float4));
  if (e != cudaSuccess) return e;
  std::vector<float4> h(n);
  // the fused z pass's entries (from twz_zf on) are lifting constants (p, u, s, 0) of the rotation by
  // the twiddle's angle a: s = -1 when |a| > pi/2 (a rotation by a -+ pi of the negated value),
  // p = -tan(a'/2), u = sin a' for the remaining angle a' (mx_fft.cuh, lines_fft_lf)
  const int lift_from = axis == 2 ? c->twz_zf : n;
  for (int j = 0; j < n; ++j) {
    if (j >= lift_from && (int)re.size() > lift_from) {
      const long double PI = 3.141592653589793238462643383279502884L;
      long double a = atan2l(im[j], re[j]);
      float sg = 1.f;
      if (a > PI / 2) a -= PI, sg = -1.f;
      else if (a < -PI / 2) a += PI, sg = -1.f;
      h[j] = make_float4((float)(-tanl(0.5L * a)), (float)sinl(a), sg, 0.f);
      continue;
    }
    const float rh = (float)re[j], ih = (float)im[j];
    h[j] = make_float4(rh, ih, (float)(re[j] - (long double)rh), (float)(im[j] - (long double)ih));
  }
  return cudaMemcpy(*dst, h.data(), n * sizeof(float4), cudaMemcpyHostToDevice);
}

// |k|^2 = s0 (a_x m_x^2 + a_y m_y^2 + a_z m_z^2) with small integers a_w when the
// nu_w^2 are commensurate; q then indexes a table of coefficients.
bool commensurate(const double nu[3], const int mmax[3], double* s0, int qa[3], int* nq) {
  double v[3] = {nu[0] * nu[0], nu[1] * nu[1], nu[2] * nu[2]};
  const double smin = std::min(v[0], std::min(v[1], v[2]));
  for (int d = 1; d <= 64; ++d) {
    bool ok = true;
    long long a[3];
    for (int w = 0; w < 3; ++w) {
      const double r = v[w] / smin * d;
      a[w] = llround(r);
      if (a[w] < 1 || fabs(r - (double)a[w]) > 1e-12 * r) ok = false;
    }
    if (!ok) continue;
    long long q = 1;
    for (int w = 0; w < 3; ++w) q += a[w] * (long long)mmax[w] * mmax[w];
    if (q > (1LL << 24)) return false;
    *s0 = smin / d;
    for (int w = 0; w < 3; ++w) qa[w] = (int)a[w];
    *nq = (int)q;
    return true;
  }
  return false;
}

int coef_kind(const mx_ctx* c) {
  // 0 Coef<T> table, 1 CoefHL table, 2 Coef<T> direct, 3 CoefHL direct
  // the repeated-step forms keep the coefficients as double-single pairs in FP32
  const bool hl = (c->prec == MX_FP32 && (c->form == MX_FORM_LITERAL || c->form == MX_FORM_XY));
  return (c->table ? 0 : 2) + (hl ? 1 : 0);
}

}  // namespace

mx_status mx_ensure_records(mx_ctx* c, long long more) {
  if (c->rec_n + more <= c->rec_cap) return MX_OK;
  long long cap = std::max<long long>(c->rec_n + more, std::max<long long>(64, 2 * c->rec_cap));
  double* nr = nullptr;
  MX_CHECK(c, mx::dev_alloc((void**)&nr, (size_t)cap * REC_STRIDE * sizeof(double)));
  if (c->rec && c->rec_n)
    MX_CHECK(c, cudaMemcpyAsync(nr, c->rec, (size_t)c->rec_n * REC_STRIDE * sizeof(double), cudaMemcpyDeviceToDevice,
                                c->stream));
  MX_CHECK(c, cudaStreamSynchronize(c->stream));
  if (c->rec) cudaFree(c->rec);
  c->rec = nr;
  c->rec_cap = cap;
  return MX_OK;
}

namespace {

mx_status ensure_records(mx_ctx* c, long long more) { return mx_ensure_records(c, more); }

double* next_record(mx_ctx* c, double t, long long step) {
  double* r = c->rec + (size_t)c->rec_n * REC_STRIDE;
  c->rec_t.push_back(t);
  c->rec_step.push_back(step);
  ++c->rec_n;
  return r;
}

template <typename T> using C2 = mx::cx<T>;

// ------------------------------------------------------------ FFT autotuner
//
// Each transform pass of a grid shape has a schedule: the kernel variant (0:
// tiles brought in and out by the bulk/tensor-copy engine where the layout
// allows, 1: per-thread loads with a register prefetch, 2: strided passes
// only, as 0 with two input stages that double as exchange buffers) and the
// persistent grid size in blocks per SM (0 = one block per tile), coded as
// bps + 16 * variant.  mx_autotune times the candidates on the context's own
// buffers and keeps the fastest in a process-wide table keyed by (pass,
// precision, grid shape); untuned passes use the default.
enum Pass { P_X_R2C = 0, P_Y_FWD, P_Z_FWD, P_Z_INV, P_Y_INV, P_X_C2R, P_Z_FUSED, P_COUNT };
constexpr int kCandidates[] = {1, 2, 4, 8, 16 + 0, 16 + 1, 16 + 2, 16 + 4, 16 + 8};
constexpr int kStridedCandidates[] = {1, 2, 4, 8, 16 + 0, 16 + 1, 16 + 2, 16 + 4, 16 + 8, 32 + 1, 32 + 2, 32 + 4};
constexpr int kFusedCandidates[] = {1, 2, 16 + 1, 16 + 2};  // at most 2 blocks per SM (partial sums)
constexpr int kDefaultSchedule = 4;
constexpr int kDefaultLongStrided = 32 + 4;  // strided passes of lines of 512 and more
constexpr int kDefaultFused = 2;
std::mutex g_tune_mu;
std::map<long long, int> g_tune;

long long tune_key(const mx_ctx* c, int pass) {
  return ((((long long)pass * 2 + c->prec) * 1024 + c->nx) * 1024 + c->ny) * 1024 + c->nz;
}
bool strided_pass(int pass) { return pass == P_Y_FWD || pass == P_Z_FWD || pass == P_Z_INV || pass == P_Y_INV; }
int default_schedule(const mx_ctx* c, int pass) {
  if (pass == P_Z_FUSED) return kDefaultFused;
  const int len = (pass == P_Y_FWD || pass == P_Y_INV) ? c->ny : c->nz;
  return strided_pass(pass) && len >= 512 ? kDefaultLongStrided : kDefaultSchedule;
}
int pass_schedule(const mx_ctx* c, int pass) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tune.find(tune_key(c, pass));
  return it == g_tune.end() ? default_schedule(c, pass) : it->second;
}
int sched_bps(int code) { return code & 15; }
bool sched_pipelined(int code) { return (code >> 4) != 1; }
bool sched_dbuf(int code) { return (code >> 4) == 2; }
int pass_bps(const mx_ctx* c, int pass) { return sched_bps(pass_schedule(c, pass)); }
// the completion counter turns the pipelined variants on (and is their timeout flag)
unsigned* pass_pipe(const mx_ctx* c, int pass) { return sched_pipelined(pass_schedule(c, pass)) ? c->counter : nullptr; }
bool pass_dbuf(const mx_ctx* c, int pass) { return sched_dbuf(pass_schedule(c, pass)); }

// Event pair around one kernel launch when profiling is on.
struct ProfScope {
  mx_ctx* c;
  size_t slot;
  bool on;
  ProfScope(mx_ctx* ctx, int kind) : c(ctx), slot(0), on(ctx->prof_on) {
    if (!on) return;
    slot = c->prof_used++;
    while (c->prof_ev.size() < 2 * c->prof_used) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) {
        on = false;
        --c->prof_used;
        return;
      }
      c->prof_ev.push_back(e);
    }
    if (c->prof_kind.size() < c->prof_used) c->prof_kind.resize(c->prof_used);
    c->prof_kind[slot] = kind;
    cudaEventRecord(c->prof_ev[2 * slot], c->stream);
  }
  ~ProfScope() {
    if (on) cudaEventRecord(c->prof_ev[2 * slot + 1], c->stream);
  }
};

template <typename T>
cudaError_t forward3(mx_ctx* c, const T* e, const T* h, void* spec, bool with_z = true) {
  const long long rows = (long long)c->ny * c->nz;
  C2<T>* s = (C2<T>*)spec;
  cudaError_t err;
  {
    ProfScope ps(c, MX_K_X_R2C);
    err = mx::launch_x_r2c<T>(c->mx, e, h, s, 3 * rows, 6 * rows, (const mx::twv<T>*)c->twx, pass_bps(c, P_X_R2C),
                              c->stream, pass_pipe(c, P_X_R2C));
  }
  if (err != cudaSuccess) return err;
  {
    ProfScope ps(c, MX_K_Y_FFT);
    err = mx::launch_strided<T>(c->ny, -1, s, c->mx, 6LL * c->nz, (const mx::twv<T>*)c->twy, pass_bps(c, P_Y_FWD),
                                c->stream, pass_pipe(c, P_Y_FWD), pass_dbuf(c, P_Y_FWD));
  }
  if (err != cudaSuccess || !with_z) return err;
  ProfScope ps(c, MX_K_Z_FFT);
  return mx::launch_strided<T>(c->nz, -1, s, (long)c->mx * c->ny, 6, (const mx::twv<T>*)c->twz, pass_bps(c, P_Z_FWD),
                               c->stream, pass_pipe(c, P_Z_FWD), pass_dbuf(c, P_Z_FWD));
}

template <typename T>
cudaError_t inverse3(mx_ctx* c, void* spec, T* e, T* h, bool with_z = true) {
  const long long rows = (long long)c->ny * c->nz;
  C2<T>* s = (C2<T>*)spec;
  cudaError_t err = cudaSuccess;
  if (with_z) {
    ProfScope ps(c, MX_K_Z_FFT);
    err = mx::launch_strided<T>(c->nz, +1, s, (long)c->mx * c->ny, 6, (const mx::twv<T>*)c->twz, pass_bps(c, P_Z_INV),
                                c->stream, pass_pipe(c, P_Z_INV), pass_dbuf(c, P_Z_INV));
  }
  if (err != cudaSuccess) return err;
  {
    ProfScope ps(c, MX_K_Y_FFT);
    err = mx::launch_strided<T>(c->ny, +1, s, c->mx, 6LL * c->nz, (const mx::twv<T>*)c->twy, pass_bps(c, P_Y_INV),
                                c->stream, pass_pipe(c, P_Y_INV), pass_dbuf(c, P_Y_INV));
  }
  if (err != cudaSuccess) return err;
  const double scale = 1.0 / (double)c->ns;
  ProfScope ps(c, MX_K_X_C2R);
  return mx::launch_x_c2r<T>(c->mx, s, e, h, 3 * rows, 6 * rows, (const mx::twv<T>*)c->twx, scale, pass_bps(c, P_X_C2R),
                             c->stream, pass_pipe(c, P_X_C2R));
}

template <typename T>
cudaError_t ensure_table(mx_ctx* c, double t);

// Grid of the fused z pass: bps blocks per SM over its tiles (at most the partial-sum slots).
int zfused_grid(const mx_ctx* c, int bps) {
  const int tx = std::max(1, mx::zfused_tile_cols(c->nz, c->prec == MX_FP64));
  const long tiles = (long)c->ny * ((c->mx + tx - 1) / tx);
  const long cap = std::min<long>((long)mx::num_sms() * std::max(bps, 1), c->pblocks);
  return (int)std::min<long>(std::max<long>(tiles, 1), cap);
}

// One launch of `pass` with schedule `code` on the context's work buffers (contents are scratch).
template <typename T>
cudaError_t run_pass(mx_ctx* c, int pass, int code) {
  const long long rows = (long long)c->ny * c->nz;
  const size_t fb = (size_t)3 * c->ns * c->es;
  T* e = (T*)c->phys;
  T* h = (T*)((char*)c->phys + fb);
  C2<T>* s = (C2<T>*)c->spec;
  const int bps = sched_bps(code);
  unsigned* pipe = sched_pipelined(code) ? c->counter : nullptr;
  const bool dbuf = sched_dbuf(code);
  switch (pass) {
    case P_X_R2C:
      return mx::launch_x_r2c<T>(c->mx, e, h, s, 3 * rows, 6 * rows, (const mx::twv<T>*)c->twx, bps, c->stream, pipe);
    case P_Y_FWD:
      return mx::launch_strided<T>(c->ny, -1, s, c->mx, 6LL * c->nz, (const mx::twv<T>*)c->twy, bps, c->stream, pipe, dbuf);
    case P_Z_FWD:
      return mx::launch_strided<T>(c->nz, -1, s, (long)c->mx * c->ny, 6, (const mx::twv<T>*)c->twz, bps, c->stream, pipe,
                                   dbuf);
    case P_Z_INV:
      return mx::launch_strided<T>(c->nz, +1, s, (long)c->mx * c->ny, 6, (const mx::twv<T>*)c->twz, bps, c->stream, pipe,
                                   dbuf);
    case P_Y_INV:
      return mx::launch_strided<T>(c->ny, +1, s, c->mx, 6LL * c->nz, (const mx::twv<T>*)c->twy, bps, c->stream, pipe, dbuf);
    case P_X_C2R:
      return mx::launch_x_c2r<T>(c->mx, s, e, h, 3 * rows, 6 * rows, (const mx::twv<T>*)c->twx, 1.0, bps, c->stream, pipe);
    case P_Z_FUSED: {  // literal form: coefficients of an arbitrary step, invariants not recorded
      cudaError_t err = ensure_table<T>(c, 0.01);
      if (err != cudaSuccess) return err;
      return mx::launch_z_fused<T>(coef_kind(c), s, c->g, c->tab, 0.01, (const mx::twv<T>*)c->twz + c->twz_zf,
                                   zfused_grid(c, bps), sched_pipelined(code), c->partials, c->counter, nullptr,
                                   c->stream);
    }
  }
  return cudaErrorInvalidValue;
}

template <typename T>
mx_status tune_t(mx_ctx* c) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  MX_CHECK(c, cudaStreamIsCapturing(c->stream, &cap));
  if (cap != cudaStreamCaptureStatusNone) return MX_OK;  // never time inside a capture
  // the passes below overwrite the work buffers: the spectral state at t_n is recomputed on demand
  // literal state lives in `phys`, xy-resident state in `spec`
  if ((c->form == MX_FORM_LITERAL || c->form == MX_FORM_XY) && c->loaded) return MX_OK;
  cudaEvent_t e0, e1;
  MX_CHECK(c, cudaEventCreate(&e0));
  MX_CHECK(c, cudaEventCreate(&e1));
  const bool fused =
      (c->form == MX_FORM_LITERAL || c->form == MX_FORM_XY) && mx::zfused_supported(c->nz, c->prec == MX_FP64);
  for (int pass = 0; pass < P_COUNT; ++pass) {
    if (pass == P_Z_FUSED && !fused) continue;
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      if (g_tune.count(tune_key(c, pass))) continue;
    }
    float best = 1e30f;
    int best_code = default_schedule(c, pass);
    const int* cand = pass == P_Z_FUSED ? kFusedCandidates : strided_pass(pass) ? kStridedCandidates : kCandidates;
    const int ncand = pass == P_Z_FUSED     ? (int)(sizeof(kFusedCandidates) / sizeof(int))
                      : strided_pass(pass) ? (int)(sizeof(kStridedCandidates) / sizeof(int))
                                           : (int)(sizeof(kCandidates) / sizeof(int));
    for (int ci = 0; ci < ncand; ++ci) {
      const int code = cand[ci];
      MX_CHECK(c, run_pass<T>(c, pass, code));  // warm-up (module load, attributes)
      MX_CHECK(c, cudaEventRecord(e0, c->stream));
      for (int r = 0; r < 3; ++r) MX_CHECK(c, run_pass<T>(c, pass, code));
      MX_CHECK(c, cudaEventRecord(e1, c->stream));
      MX_CHECK(c, cudaEventSynchronize(e1));
      float ms = 0.f;
      MX_CHECK(c, cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) best = ms, best_code = code;
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[tune_key(c, pass)] = best_code;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->spec_valid = false;
  return MX_OK;
}

template <typename T>
cudaError_t ensure_table(mx_ctx* c, double t) {
  if (!c->table) return cudaSuccess;
  const int kind = coef_kind(c);
  if (kind == c->tab_kind && t == c->tab_t) return cudaSuccess;
  c->tab_kind = kind;
  c->tab_t = t;
  ProfScope ps(c, MX_K_TABLE);
  return mx::launch_coef_table<T>(kind, c->tab, c->nq, c->g, t, c->stream);
}

// One spectral pass: dst = R(t) src (mode 1/2) or invariants of src (mode 0).
template <typename T>
cudaError_t spectral_pass(mx_ctx* c, int mode, const void* src, void* dst, double t, double* record) {
  if (mode != 0) {
    cudaError_t e = ensure_table<T>(c, t);
    if (e != cudaSuccess) return e;
  }
  ProfScope ps(c, MX_K_SPECTRAL);
  return mx::launch_spectral<T>(mode, coef_kind(c), (const C2<T>*)src, (C2<T>*)dst, c->nh, c->g, c->tab, t, c->sblocks,
                                c->partials, c->counter, record, c->stream);
}

template <typename T>
mx_status load_t(mx_ctx* c, const void* E, const void* H, int on_device, bool wait = true) {
  const size_t fb = (size_t)3 * c->ns * c->es;
  const T *e = (const T*)E, *h = (const T*)H;
  if (!on_device || c->form == MX_FORM_LITERAL) {
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    MX_CHECK(c, cudaMemcpyAsync(c->phys, E, fb, kind, c->stream));
    MX_CHECK(c, cudaMemcpyAsync((char*)c->phys + fb, H, fb, kind, c->stream));
    e = (const T*)c->phys;
    h = (const T*)((const char*)c->phys + fb);
  }
  // the record of t = 0 comes from the full 3D spectrum (xy-resident form: in the work buffer)
  void* target = c->form == MX_FORM_LITERAL ? c->spec : c->spec0;
  MX_CHECK(c, forward3<T>(c, e, h, target));
  if (c->form == MX_FORM_XY) MX_CHECK(c, forward3<T>(c, e, h, c->spec, false));  // the state: x and y only
  c->rec_n = 0;
  c->rec_t.clear();
  c->rec_step.clear();
  mx_status st = ensure_records(c, 1);
  if (st != MX_OK) return st;
  MX_CHECK(c, spectral_pass<T>(c, 0, target, nullptr, 0.0, next_record(c, 0.0, 0)));
  if (!on_device && wait) MX_CHECK(c, cudaStreamSynchronize(c->stream));
  c->t = 0.0;
  c->step = 0;
  c->loaded = true;
  c->spec_valid = false;
  return MX_OK;
}

template <typename T>
mx_status load_random_t(mx_ctx* c, unsigned long long seed, double sigma) {
  // amplitude so that each field component has RMS ~ 1 on the grid:
  // rms^2 = amp^2 * (sum_k env_k^2) * E|g|^2 (2) * (2/3 left after projection) / N_S^2,
  // with sum_k env^2 separable over the three axes.
  const int n[3] = {c->nx, c->ny, c->nz};
  double sum = 1.0;
  for (int w = 0; w < 3; ++w) {
    double sw = 0.0;
    for (int m = -n[w] / 2 + 1; m <= n[w] / 2 - 1; ++m) {
      const double k = c->g.nu[w] * m;
      sw += exp(-k * k / (sigma * sigma));
    }
    sum *= sw;
  }
  const double amp = (double)c->ns / sqrt(std::max(sum, 1e-300) * 4.0 / 3.0);
  void* target = c->form == MX_FORM_LITERAL ? c->spec : c->spec0;
  {
    ProfScope ps(c, MX_K_GEN);
    MX_CHECK(c, mx::launch_gen_divfree<T>((C2<T>*)target, c->nh, c->g, seed, sigma, amp, c->stream));
  }
  c->rec_n = 0;
  c->rec_t.clear();
  c->rec_step.clear();
  mx_status st = ensure_records(c, 1);
  if (st != MX_OK) return st;
  MX_CHECK(c, spectral_pass<T>(c, 0, target, nullptr, 0.0, next_record(c, 0.0, 0)));
  if (c->form != MX_FORM_SPECTRAL) {
    const size_t fb = (size_t)3 * c->ns * c->es;
    T* e = (T*)c->phys;
    T* h = (T*)((char*)c->phys + fb);
    MX_CHECK(c, inverse3<T>(c, target, e, h));
    if (c->form == MX_FORM_XY) MX_CHECK(c, forward3<T>(c, e, h, c->spec, false));  // the state: x and y only
  }
  c->t = 0.0;
  c->step = 0;
  c->loaded = true;
  c->spec_valid = false;
  return MX_OK;
}

template <typename T>
mx_status step_t(mx_ctx* c, double h, long long nsteps, int every) {
  long long nrec = 0;
  if (every > 0)
    for (long long i = 1; i <= nsteps; ++i)
      if ((c->step + i) % every == 0) ++nrec;
  mx_status st = ensure_records(c, nrec);
  if (st != MX_OK) return st;
  const size_t fb = (size_t)3 * c->ns * c->es;
  const double t0 = c->t;
  const long long n0 = c->step;
  for (long long i = 1; i <= nsteps; ++i) {
    const long long n = n0 + i;
    const double tn = t0 + (double)i * h;
    const bool inv = every > 0 && (n % every == 0);
    double* record = inv ? next_record(c, tn, n) : nullptr;
    if (c->form == MX_FORM_LITERAL) {
      T* e = (T*)c->phys;
      T* hh = (T*)((char*)c->phys + fb);
      if (mx::zfused_supported(c->nz, c->prec == MX_FP64)) {
        // x, y forward; fused z forward -> update -> z inverse; y, x inverse: 5 passes
        MX_CHECK(c, forward3<T>(c, e, hh, c->spec, false));
        MX_CHECK(c, ensure_table<T>(c, h));
        {
          ProfScope ps(c, MX_K_ZFUSED);
          const int code = pass_schedule(c, P_Z_FUSED);
          MX_CHECK(c, mx::launch_z_fused<T>(coef_kind(c), (C2<T>*)c->spec, c->g, c->tab, h, (const mx::twv<T>*)c->twz + c->twz_zf,
                                            zfused_grid(c, sched_bps(code)), sched_pipelined(code), c->partials,
                                            c->counter, record, c->stream));
        }
        MX_CHECK(c, inverse3<T>(c, c->spec, e, hh, false));
      } else {
        MX_CHECK(c, forward3<T>(c, e, hh, c->spec));
        MX_CHECK(c, spectral_pass<T>(c, inv ? 2 : 1, c->spec, c->spec, h, record));
        MX_CHECK(c, inverse3<T>(c, c->spec, e, hh));
      }
    } else if (c->form == MX_FORM_XY) {
      // one pass: z forward -> update -> z inverse (output scaled by 1/nz) on the x-y spectrum
      MX_CHECK(c, ensure_table<T>(c, h));
      ProfScope ps(c, MX_K_ZFUSED);
      const int code = pass_schedule(c, P_Z_FUSED);
      MX_CHECK(c, mx::launch_z_fused<T>(coef_kind(c), (C2<T>*)c->spec, c->g, c->tab, h,
                                        (const mx::twv<T>*)c->twz + c->twz_zf, zfused_grid(c, sched_bps(code)),
                                        sched_pipelined(code), c->partials, c->counter, record, c->stream));
    } else {
      MX_CHECK(c, spectral_pass<T>(c, inv ? 2 : 1, c->spec0, c->spec, tn, record));
      c->spec_valid = true;
    }
  }
  c->t = t0 + (double)nsteps * h;
  c->step = n0 + nsteps;
  return MX_OK;
}

template <typename T>
mx_status read_t(mx_ctx* c, void* E, void* H, int on_device, bool wait = true) {
  const size_t fb = (size_t)3 * c->ns * c->es;
  if (c->form == MX_FORM_LITERAL) {
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    MX_CHECK(c, cudaMemcpyAsync(E, c->phys, fb, kind, c->stream));
    MX_CHECK(c, cudaMemcpyAsync(H, (char*)c->phys + fb, fb, kind, c->stream));
  } else if (c->form == MX_FORM_XY) {
    // the inverse y and x passes on a copy of the state
    MX_CHECK(c, cudaMemcpyAsync(c->spec0, c->spec, (size_t)6 * c->nh * c->cs, cudaMemcpyDeviceToDevice, c->stream));
    T* e = on_device ? (T*)E : (T*)c->phys;
    T* h = on_device ? (T*)H : (T*)((char*)c->phys + fb);
    {
      ProfScope ps(c, MX_K_Y_FFT);
      MX_CHECK(c, mx::launch_strided<T>(c->ny, +1, (C2<T>*)c->spec0, c->mx, 6LL * c->nz, (const mx::twv<T>*)c->twy,
                                        pass_bps(c, P_Y_INV), c->stream, pass_pipe(c, P_Y_INV), pass_dbuf(c, P_Y_INV)));
    }
    {
      const long long rows = (long long)c->ny * c->nz;
      ProfScope ps(c, MX_K_X_C2R);
      // the z transforms of every step carried their 1/nz: the x pass scales by 1/(nx ny)
      MX_CHECK(c, mx::launch_x_c2r<T>(c->mx, (C2<T>*)c->spec0, e, h, 3 * rows, 6 * rows, (const mx::twv<T>*)c->twx,
                                      1.0 / ((double)c->nx * c->ny), pass_bps(c, P_X_C2R), c->stream, pass_pipe(c, P_X_C2R)));
    }
    if (!on_device) {
      MX_CHECK(c, cudaMemcpyAsync(E, c->phys, fb, cudaMemcpyDeviceToHost, c->stream));
      MX_CHECK(c, cudaMemcpyAsync(H, (char*)c->phys + fb, fb, cudaMemcpyDeviceToHost, c->stream));
    }
  } else {
    if (!c->spec_valid) MX_CHECK(c, spectral_pass<T>(c, 1, c->spec0, c->spec, c->t, nullptr));
    T* e = on_device ? (T*)E : (T*)c->phys;
    T* h = on_device ? (T*)H : (T*)((char*)c->phys + fb);
    MX_CHECK(c, inverse3<T>(c, c->spec, e, h));
    c->spec_valid = false;  // the inverse passes ran in place
    if (!on_device) {
      MX_CHECK(c, cudaMemcpyAsync(E, c->phys, fb, cudaMemcpyDeviceToHost, c->stream));
      MX_CHECK(c, cudaMemcpyAsync(H, (char*)c->phys + fb, fb, cudaMemcpyDeviceToHost, c->stream));
    }
  }
  if (!on_device && wait) MX_CHECK(c, cudaStreamSynchronize(c->stream));
  return MX_OK;
}

size_t footprint(int nx, int ny, int nz, int prec, int form, int nq) {
  const size_t es = prec == MX_FP64 ? 8 : 4;
  const size_t ns = (size_t)nx * ny * nz;
  size_t b = 6 * ns * es;                  // phys
  b += 6 * ns * es;                        // spec (nh complex == ns reals)
  if (form != MX_FORM_LITERAL) b += 6 * ns * es;  // spec0 (xy-resident form: the work copy of reads)
  b += (size_t)nq * 32;                    // table
  b += (size_t)(nx + ny + 2 * nz) * 16;   // twiddles (16-byte entries)
  b += (size_t)152 * 4 * 16 * sizeof(double) + 64 * REC_STRIDE * sizeof(double) + 256;
  return b;
}

void grid_info(int nx, int ny, int nz, const double lo[3], const double hi[3], double nu[3], int mmax[3]) {
  for (int w = 0; w < 3; ++w) nu[w] = 2.0 * M_PI / (hi[w] - lo[w]);
  mmax[0] = nx / 2 - 1;
  mmax[1] = ny / 2 - 1;
  mmax[2] = nz / 2 - 1;
}

}  // namespace

extern "C" {

const char* mx_strerror(mx_status s) {
  switch (s) {
    case MX_OK: return "ok";
    case MX_E_INVAL: return "invalid argument";
    case MX_E_UNSUPPORTED_N: return "unsupported grid size (need nx/2 <= 256 and ny, nz <= 512, each of the form 2^a, 3*2^a or 5*2^a; nx even)";
    case MX_E_NOMEM: return "device allocation failed";
    case MX_E_CUDA: return "CUDA error";
    case MX_E_TIMEOUT: return "device wait timed out";
    case MX_E_STATE: return "call out of order";
  }
  return "unknown status";
}

mx_status mx_footprint_bytes(int nx, int ny, int nz, int precision, int form, size_t* bytes) {
  if (!bytes || nx < 2 || ny < 2 || nz < 2 || nx % 2 || ny % 2 || nz % 2) return MX_E_INVAL;
  if (precision != MX_FP64 && precision != MX_FP32) return MX_E_INVAL;
  if (form != MX_FORM_LITERAL && form != MX_FORM_SPECTRAL && form != MX_FORM_XY) return MX_E_INVAL;
  // worst-case table size for a cubic-cell grid
  const long long nq = 1 + (long long)(nx / 2 - 1) * (nx / 2 - 1) + (long long)(ny / 2 - 1) * (ny / 2 - 1) +
                       (long long)(nz / 2 - 1) * (nz / 2 - 1);
  *bytes = footprint(nx, ny, nz, precision, form, (int)std::min<long long>(nq, 1 << 24));
  return MX_OK;
}

mx_status mx_create(mx_ctx** out, int nx, int ny, int nz, const double lo[3], const double hi[3], double eps, double mu,
                    int precision, int form, void* stream) {
  if (!out) return MX_E_INVAL;
  *out = nullptr;
  if (!lo || !hi) return MX_E_INVAL;
  if (nx < 2 || ny < 2 || nz < 2 || nx % 2 || ny % 2 || nz % 2) return MX_E_INVAL;
  if (!(eps > 0.0) || !(mu > 0.0) || !isfinite(eps) || !isfinite(mu)) return MX_E_INVAL;
  for (int w = 0; w < 3; ++w)
    if (!isfinite(lo[w]) || !isfinite(hi[w]) || !(hi[w] > lo[w])) return MX_E_INVAL;
  if (precision != MX_FP64 && precision != MX_FP32) return MX_E_INVAL;
  if (form != MX_FORM_LITERAL && form != MX_FORM_SPECTRAL && form != MX_FORM_XY) return MX_E_INVAL;
  if (!len_ok(nx / 2) || nx / 2 > 256 || !len_ok(ny) || !len_ok(nz)) return MX_E_UNSUPPORTED_N;
  if (6LL * nz > 65535) return MX_E_UNSUPPORTED_N;
  // the xy-resident form steps with the fused z pass only
  if (form == MX_FORM_XY && !mx::zfused_supported(nz, precision == MX_FP64)) return MX_E_UNSUPPORTED_N;

  mx_ctx* c = new mx_ctx();
  c->nx = nx; c->ny = ny; c->nz = nz; c->mx = nx / 2;
  for (int w = 0; w < 3; ++w) { c->lo[w] = lo[w]; c->hi[w] = hi[w]; }
  c->eps = eps; c->mu = mu; c->prec = precision; c->form = form;
  c->stream = (cudaStream_t)stream;
  c->es = precision == MX_FP64 ? 8 : 4;
  c->cs = 2 * c->es;
  c->ns = (long long)nx * ny * nz;
  c->nh = (long long)c->mx * ny * nz;
  int mmax[3];
  GridParams& g = c->g;
  g.nx = nx; g.ny = ny; g.nz = nz; g.mx = c->mx;
  grid_info(nx, ny, nz, lo, hi, g.nu, mmax);
  mx::set_material(g, eps, mu);
  if (form == MX_FORM_XY) {  // the fused pass's output is the state: its inverse z transform carries 1/nz
    g.zscale = 1.0 / nz;
    g.zscalef = (float)g.zscale;
  }
  g.s0 = 0.0; g.qa[0] = g.qa[1] = g.qa[2] = 0;
  c->nq = 0;
  c->table = commensurate(g.nu, mmax, &g.s0, g.qa, &c->nq);
  c->sblocks = mx::spectral_blocks(c->nh);

  auto fail = [&](mx_status s) {
    mx_destroy(c);
    return s;
  };
  const size_t field_bytes = (size_t)6 * c->ns * c->es;
  if (mx::dev_alloc(&c->phys, field_bytes) != cudaSuccess) return fail(MX_E_NOMEM);
  if (mx::dev_alloc(&c->spec, field_bytes) != cudaSuccess) return fail(MX_E_NOMEM);
  if (form != MX_FORM_LITERAL && mx::dev_alloc(&c->spec0, field_bytes) != cudaSuccess) return fail(MX_E_NOMEM);
  if (c->table && mx::dev_alloc(&c->tab, (size_t)c->nq * 32) != cudaSuccess) return fail(MX_E_NOMEM);
  // partial sums for up to 2 blocks per SM of any pass that reduces invariants
  c->pblocks = std::max(c->sblocks, 2 * mx::num_sms());
  if (mx::dev_alloc((void**)&c->partials, (size_t)c->pblocks * mx::NSUM * sizeof(double)) != cudaSuccess) return fail(MX_E_NOMEM);
  if (mx::dev_alloc((void**)&c->counter, 64) != cudaSuccess) return fail(MX_E_NOMEM);
  if (cudaMemset(c->counter, 0, 64) != cudaSuccess) return fail(MX_E_CUDA);
  if (upload_twiddles(c, 0, nx, &c->twx) != cudaSuccess) return fail(MX_E_NOMEM);
  if (upload_twiddles(c, 1, ny, &c->twy) != cudaSuccess) return fail(MX_E_NOMEM);
  if (upload_twiddles(c, 2, nz, &c->twz) != cudaSuccess) return fail(MX_E_NOMEM);
  if (ensure_records(c, 64) != MX_OK) return fail(MX_E_NOMEM);
  *out = c;
  return MX_OK;
}

mx_status mx_load_fields(mx_ctx* c, const void* E, const void* H, int on_device) {
  if (!c || !E || !H) return MX_E_INVAL;
  if (c->err != MX_OK) return c->err;
  return c->prec == MX_FP64 ? load_t<double>(c, E, H, on_device) : load_t<float>(c, E, H, on_device);
}

// Host-buffer load and read that only enqueue (the caller waits on the stream):
// used by the server, whose host buffers are pinned.
mx_status mx_load_fields_async(mx_ctx* c, const void* E, const void* H) {
  if (!c || !E || !H) return MX_E_INVAL;
  if (c->err != MX_OK) return c->err;
  return c->prec == MX_FP64 ? load_t<double>(c, E, H, 0, false) : load_t<float>(c, E, H, 0, false);
}
mx_status mx_read_fields_async(mx_ctx* c, void* E, void* H) {
  if (!c || !E || !H) return MX_E_INVAL;
  if (c->err != MX_OK) return c->err;
  if (!c->loaded) return MX_E_STATE;
  return c->prec == MX_FP64 ? read_t<double>(c, E, H, 0, false) : read_t<float>(c, E, H, 0, false);
}

mx_status mx_load_random_divfree(mx_ctx* c, unsigned long long seed, double sigma) {
  if (!c || !(sigma > 0.0) || !isfinite(sigma)) return MX_E_INVAL;
  if (c->err != MX_OK) return c->err;
  return c->prec == MX_FP64 ? load_random_t<double>(c, seed, sigma) : load_random_t<float>(c, seed, sigma);
}

mx_status mx_autotune(mx_ctx* c) {
  if (!c) return MX_E_INVAL;
  if (c->err != MX_OK) return c->err;
  return c->prec == MX_FP64 ? tune_t<double>(c) : tune_t<float>(c);
}

mx_status mx_schedule(mx_ctx* c, int* sched, int n) {
  if (!c || !sched || n < P_COUNT) return MX_E_INVAL;
  for (int p = 0; p < P_COUNT; ++p) sched[p] = pass_schedule(c, p);
  return MX_OK;
}

mx_status mx_set_schedule(mx_ctx* c, const int* sched, int n) {
  if (!c || !sched || n < P_COUNT) return MX_E_INVAL;
  for (int p = 0; p < P_COUNT; ++p) {
    const int code = sched[p], bps = code & 15, variant = code >> 4;
    if (code < 0 || variant > 2) return MX_E_INVAL;
    if (variant == 2 && !strided_pass(p)) return MX_E_INVAL;
    if (p == P_Z_FUSED && (variant > 1 || bps < 1 || bps > 2)) return MX_E_INVAL;  // partial-sum slots
    if (variant != 1 && bps == 0) return MX_E_INVAL;  // copy-engine variants are persistent
  }
  std::lock_guard<std::mutex> lock(g_tune_mu);
  for (int p = 0; p < P_COUNT; ++p) g_tune[tune_key(c, p)] = sched[p];
  return MX_OK;
}

mx_status mx_profile(mx_ctx* c, int enable) {
  if (!c) return MX_E_INVAL;
  if (c->err != MX_OK) return c->err;
  c->prof_on = enable != 0;
  c->prof_used = 0;
  return MX_OK;
}

mx_status mx_profile_read(mx_ctx* c, double* ms, long long* launches) {
  if (!c || !ms || !launches) return MX_E_INVAL;
  if (c->err != MX_OK) return c->err;
  MX_CHECK(c, cudaStreamSynchronize(c->stream));
  for (int k = 0; k < MX_K_COUNT; ++k) {
    ms[k] = 0.0;
    launches[k] = 0;
  }
  for (size_t i = 0; i < c->prof_used; ++i) {
    float v = 0.f;
    MX_CHECK(c, cudaEventElapsedTime(&v, c->prof_ev[2 * i], c->prof_ev[2 * i + 1]));
    ms[c->prof_kind[i]] += v;
    launches[c->prof_kind[i]] += 1;
  }
  c->prof_used = 0;
  return MX_OK;
}

mx_status mx_step(mx_ctx* c, double h, long long nsteps, int invariants_every) {
  if (!c) return MX_E_INVAL;
  if (c->err != MX_OK) return c->err;
  if (!isfinite(h) || nsteps < 0 || invariants_every < 0) return MX_E_INVAL;
  if (!c->loaded) return MX_E_STATE;
  if (nsteps == 0) return MX_OK;
  return c->prec == MX_FP64 ? step_t<double>(c, h, nsteps, invariants_every)
                            : step_t<float>(c, h, nsteps, invariants_every);
}

mx_status mx_read_fields(mx_ctx* c, void* E, void* H, int on_device) {
  if (!c || !E || !H) return MX_E_INVAL;
  if (c->err != MX_OK) return c->err;
  if (!c->loaded) return MX_E_STATE;
  return c->prec == MX_FP64 ? read_t<double>(c, E, H, on_device) : read_t<float>(c, E, H, on_device);
}

mx_status mx_read_invariants(mx_ctx* c, mx_invariants* out, long long max, long long* n_written) {
  if (!c || !n_written || max < 0 || (max > 0 && !out)) return MX_E_INVAL;
  if (c->err != MX_OK) return c->err;
  *n_written = 0;
  if (max == 0) {
    *n_written = c->rec_n;
    return MX_OK;
  }
  const long long n = std::min(max, c->rec_n);
  if (n == 0) return MX_OK;
  std::vector<double> raw((size_t)n * REC_STRIDE);
  MX_CHECK(c, cudaMemcpyAsync(raw.data(), c->rec, raw.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  MX_CHECK(c, cudaStreamSynchronize(c->stream));
  const double N = (double)c->ns, N2 = N * N;
  for (long long i = 0; i < n; ++i) {
    const double* s = raw.data() + (size_t)i * REC_STRIDE;
    mx_invariants& r = out[i];
    memset(&r, 0, sizeof(r));
    r.t = c->rec_t[i];
    r.step = c->rec_step[i];
    r.E1 = s[0] / (2 * N2);
    r.E2 = s[1] / (2 * N2);
    for (int w = 0; w < 3; ++w) {
      r.E3[w] = s[2 + w] / (2 * N2);
      r.E4[w] = s[5 + w] / (2 * N2);
      r.M1[w] = -s[10 + w] / N2;
      r.M2[w] = -r.M1[w];
    }
    r.H1 = s[8] / N2;
    r.H2 = s[9] / N2;
    r.divE = sqrt(std::max(s[13], 0.0)) / N;
    r.divH = sqrt(std::max(s[14], 0.0)) / N;
  }
  *n_written = n;
  return MX_OK;
}

mx_status mx_time(mx_ctx* c, double* t, long long* step) {
  if (!c) return MX_E_INVAL;
  if (t) *t = c->t;
  if (step) *step = c->step;
  return MX_OK;
}

mx_status mx_debug_fail_alloc(long long k) {
  if (k < 0) {
    mx::g_fail_at.store(-1);
    return MX_OK;
  }
  mx::g_alloc_index.store(0);
  mx::g_fail_at.store(k);
  return MX_OK;
}

mx_status mx_debug_wait_limit(mx_ctx* c, long long tries) {
  if (!c) return MX_E_INVAL;
  c->g.wait_tries = (tries < 0 || tries > (long long)mx::MBAR_TRIES) ? mx::MBAR_TRIES : (unsigned)tries;
  return MX_OK;
}

mx_status mx_sync(mx_ctx* c) {
  if (!c) return MX_E_INVAL;
  if (c->err != MX_OK) return c->err;
  MX_CHECK(c, cudaStreamSynchronize(c->stream));
  // counter[1] is set by a kernel whose bounded wait gave up
  unsigned flag = 0;
  MX_CHECK(c, cudaMemcpy(&flag, c->counter + 1, sizeof(flag), cudaMemcpyDeviceToHost));
  if (flag) {
    c->err = MX_E_TIMEOUT;
    return c->err;
  }
  return MX_OK;
}

void mx_destroy(mx_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
  void* bufs[] = {c->phys, c->spec, c->spec0, c->tab, c->twx, c->twy, c->twz, c->partials, c->counter, c->rec};
  for (void* b : bufs)
    if (b) cudaFree(b);
  delete c;
}

}  // extern "C"

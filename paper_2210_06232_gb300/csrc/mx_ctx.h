// Internal: the solver context behind the opaque mx_ctx handle (shared by
// the C-ABI translation units; not part of the public interface).
#pragma once
#include <math.h>

#include <vector>

#include "../../include/maxexp.h"
#include "mx_launch.h"

struct mx_ctx {
  int nx, ny, nz, mx;
  double lo[3], hi[3];
  double eps, mu;
  int prec, form;
  cudaStream_t stream;
  mx::GridParams g;
  bool table;  // commensurate |k|^2 -> coefficient table
  int nq;
  size_t es, cs;  // real / complex element bytes
  long long ns, nh;
  void* phys = nullptr;   // 6 * ns reals: literal state; staging for host I/O
  void* spec = nullptr;   // 6 * nh complex: literal work spectrum; spectral state at t_n
  void* spec0 = nullptr;  // spectral form: spectrum at load time
  void* tab = nullptr;
  void* twx = nullptr;
  void* twy = nullptr;
  void* twz = nullptr;
  int twz_zf = 0;  // entry of twz where the fused z pass's table starts
  double* partials = nullptr;
  unsigned* counter = nullptr;
  int sblocks;
  int pblocks;  // capacity of `partials` in blocks
  double* rec = nullptr;
  long long rec_cap = 0, rec_n = 0;
  std::vector<double> rec_t;
  std::vector<long long> rec_step;
  bool loaded = false;
  bool spec_valid = false;  // spectral form: `spec` holds the state at `t`
  double t = 0.0;
  long long step = 0;
  int tab_kind = -1;
  double tab_t = NAN;
  mx_status err = MX_OK;
  // per-kernel event timing (mx_profile)
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_ev;
  std::vector<int> prof_kind;
  size_t prof_used = 0;
};


// Grow the device record array so `more` records fit after the current ones.
mx_status mx_ensure_records(mx_ctx* c, long long more);


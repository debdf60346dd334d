// Batched forms (C ABI): independent instances of different grids, eps, mu
// and step sizes, advanced together.
//  * spectral form: each instance a spectral-form context, all advanced by one
//    persistent cooperative launch per mx_batch_step call; the launch (with
//    the upload of the per-instance descriptors) is captured once per step
//    count into a CUDA graph and replayed.
//  * literal form: each instance a literal-form context whose transform
//    passes run the schedules the autotuner picked for its shape; the K steps
//    of every instance (x, y, fused z, y, x passes per step) are captured as
//    parallel branches of one CUDA graph (one stream per instance, forked from
//    and joined to the batch stream) and replayed, so the small instances'
//    passes overlap on the device.  The graph writes each instance's
//    invariant records into a region of its own, copied after every replay to
//    the instance's record list.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "mx_batch.cuh"
#include "mx_ctx.h"

struct mx_batch {
  int n = 0;
  int prec = MX_FP32;
  cudaStream_t stream = nullptr;
  std::vector<mx_ctx*> ctx;
  std::vector<double> h;
  mx::BInst* h_inst = nullptr;  // pinned: read by the graph's copy node at launch
  mx::BInst* d_inst = nullptr;
  double* cpart = nullptr;
  double* segpart = nullptr;
  mx::QK* qk = nullptr;  // FP32: per table entry, (0.5 c)|k|, |k|, |k|^2
  unsigned* bar = nullptr;
  unsigned total_chunks = 0, total_q = 0, total_segs = 0;
  int grid = 0;
  bool use_graph = true;
  int graph_err = 0;                       // CUDA error of a refused capture (0: none)
  bool own_stream = false;
  std::map<int, cudaGraphExec_t> graphs;  // nsteps -> executable graph
  mx_status err = MX_OK;
  // literal form
  int form = MX_FORM_SPECTRAL;
  std::vector<cudaStream_t> lstreams;      // one per instance
  std::vector<cudaEvent_t> ldone;          // one per instance (join)
  cudaEvent_t fork = nullptr;
  std::vector<double*> grec;               // record region of the graph, per instance
  std::vector<long long> grec_cap;         // its capacity (records)
  std::map<std::string, cudaGraphExec_t> lgraphs;  // (K, every, step phases) -> graph
};

namespace {

template <typename T> void* batch_kernel() { return (void*)mx::k_batch_steps<T>; }

cudaError_t launch_batch(mx_batch* b, int nsteps) {
  mx::BatchArgs a;
  a.inst = b->d_inst;
  a.ninst = b->n;
  a.total_chunks = b->total_chunks;
  a.total_q = b->total_q;
  a.nsteps = nsteps;
  a.total_segs = b->total_segs;
  a.cpart = b->cpart;
  a.segpart = b->segpart;
  a.qk = b->qk;
  a.bar = b->bar;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(b->grid);
  cfg.blockDim = dim3(mx::BT_THREADS);
  cfg.dynamicSmemBytes = b->prec == MX_FP64 ? mx::bt_smem_bytes<double>() : mx::bt_smem_bytes<float>();
  cfg.stream = b->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (b->prec == MX_FP64) return cudaLaunchKernelEx(&cfg, mx::k_batch_steps<double>, a);
  return cudaLaunchKernelEx(&cfg, mx::k_batch_steps<float>, a);
}

// Descriptor upload + launch, on the batch stream.
cudaError_t enqueue_step(mx_batch* b, int nsteps) {
  cudaError_t e = cudaMemcpyAsync(b->d_inst, b->h_inst, sizeof(mx::BInst) * b->n, cudaMemcpyHostToDevice, b->stream);
  if (e != cudaSuccess) return e;
  return launch_batch(b, nsteps);
}

mx_status fail(mx_batch* b, cudaError_t e) {
  if (e == cudaSuccess) return MX_OK;
  b->err = MX_E_CUDA;
  return MX_E_CUDA;
}

// Literal form: the K steps of every instance, each on its own stream forked from and joined to
// the batch stream (inside a capture: parallel graph branches).  Records go to each instance's
// graph region (c->rec pointed there for the duration; the caller restores the context state).
mx_status enqueue_literal(mx_batch* b, long long k, int every) {
  if (cudaEventRecord(b->fork, b->stream) != cudaSuccess) return MX_E_CUDA;
  for (int i = 0; i < b->n; ++i) {
    mx_ctx* c = b->ctx[i];
    if (cudaStreamWaitEvent(b->lstreams[i], b->fork, 0) != cudaSuccess) return MX_E_CUDA;
    c->stream = b->lstreams[i];
    const mx_status st = mx_step(c, b->h[i], k, every);
    c->stream = b->stream;
    if (st != MX_OK) return st;
    if (cudaEventRecord(b->ldone[i], b->lstreams[i]) != cudaSuccess) return MX_E_CUDA;
    if (cudaStreamWaitEvent(b->stream, b->ldone[i], 0) != cudaSuccess) return MX_E_CUDA;
  }
  return MX_OK;
}

struct CtxState {
  double* rec;
  long long rec_n, rec_cap;
  std::vector<double> rec_t;
  std::vector<long long> rec_step;
  double t;
  long long step;
  bool prof_on;
};

mx_status step_literal(mx_batch* b, long long k, int every) {
  std::vector<long long> nrec(b->n, 0);
  std::string key = std::to_string(k) + ":" + std::to_string(every);
  for (int i = 0; i < b->n; ++i) {
    mx_ctx* c = b->ctx[i];
    if (c->err != MX_OK) return c->err;
    if (every > 0) {
      nrec[i] = (c->step + k) / every - c->step / every;
      key += ":" + std::to_string(c->step % every);
    }
    if (nrec[i] > b->grec_cap[i]) {  // the graph region of this instance (graphs captured before refer to the old one)
      for (auto& kv : b->lgraphs) cudaGraphExecDestroy(kv.second);
      b->lgraphs.clear();
      if (cudaStreamSynchronize(b->stream) != cudaSuccess) return MX_E_CUDA;
      if (b->grec[i]) cudaFree(b->grec[i]);
      b->grec[i] = nullptr;
      b->grec_cap[i] = 0;
      if (mx::dev_alloc((void**)&b->grec[i], (size_t)nrec[i] * 16 * sizeof(double)) != cudaSuccess) return MX_E_NOMEM;
      b->grec_cap[i] = nrec[i];
    }
  }
  // the contexts as the graph sees them: records into the graph regions, the table recomputed
  // inside the graph, no profiling events
  std::vector<CtxState> saved(b->n);
  auto redirect = [&]() {
    for (int i = 0; i < b->n; ++i) {
      mx_ctx* c = b->ctx[i];
      saved[i] = CtxState{c->rec, c->rec_n, c->rec_cap, c->rec_t, c->rec_step, c->t, c->step, c->prof_on};
      c->rec = b->grec[i];
      c->rec_n = 0;
      c->rec_cap = b->grec_cap[i];
      c->rec_t.clear();
      c->rec_step.clear();
      c->prof_on = false;
      c->tab_t = NAN;
    }
  };
  auto restore = [&]() {
    for (int i = 0; i < b->n; ++i) {
      mx_ctx* c = b->ctx[i];
      c->rec = saved[i].rec;
      c->rec_n = saved[i].rec_n;
      c->rec_cap = saved[i].rec_cap;
      c->rec_t.swap(saved[i].rec_t);
      c->rec_step.swap(saved[i].rec_step);
      c->t = saved[i].t;
      c->step = saved[i].step;
      c->prof_on = saved[i].prof_on;
    }
  };
  mx_status st = MX_OK;
  if (b->use_graph) {
    auto it = b->lgraphs.find(key);
    if (it == b->lgraphs.end()) {
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      redirect();
      cudaError_t ce = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
      if (ce == cudaSuccess) {
        st = enqueue_literal(b, k, every);
        ce = cudaStreamEndCapture(b->stream, &graph);
      }
      restore();
      if (st == MX_OK && ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (st != MX_OK || ce != cudaSuccess) {
        cudaGetLastError();  // capture refused: launch directly from now on
        b->graph_err = ce != cudaSuccess ? (int)ce : (int)cudaErrorUnknown;
        b->use_graph = false;
        st = MX_OK;
      } else {
        it = b->lgraphs.emplace(key, exec).first;
      }
    }
    if (b->use_graph && cudaGraphLaunch(it->second, b->stream) != cudaSuccess) return MX_E_CUDA;
  }
  if (!b->use_graph) {
    redirect();
    st = enqueue_literal(b, k, every);
    restore();
    if (st != MX_OK) return st;
  }
  // records of this call: from the graph regions to the instances' record lists
  for (int i = 0; i < b->n; ++i) {
    mx_ctx* c = b->ctx[i];
    const long long n0 = c->step;
    if (nrec[i] > 0) {
      st = mx_ensure_records(c, nrec[i]);
      if (st != MX_OK) return st;
      if (cudaMemcpyAsync(c->rec + (size_t)c->rec_n * 16, b->grec[i], (size_t)nrec[i] * 16 * sizeof(double),
                          cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess)
        return MX_E_CUDA;
      for (long long N = (n0 / every + 1) * every; N <= n0 + k; N += every) {
        c->rec_t.push_back(c->t + (double)(N - n0) * b->h[i]);
        c->rec_step.push_back(N);
        ++c->rec_n;
      }
    }
    c->t += (double)k * b->h[i];
    c->step += k;
    c->tab_t = b->h[i];  // the graph left the table of h in place
    c->tab_kind = -1;    // (recomputed by the next direct step of the instance)
  }
  return MX_OK;
}

}  // namespace

extern "C" {

mx_status mx_batch_create(mx_batch** out, const mx_instance_desc* inst, int n, int precision, void* stream) {
  return mx_batch_create_form(out, inst, n, precision, MX_FORM_SPECTRAL, stream);
}

mx_status mx_batch_create_form(mx_batch** out, const mx_instance_desc* inst, int n, int precision, int form,
                               void* stream) {
  if (!out) return MX_E_INVAL;
  *out = nullptr;
  if (!inst || n < 1 || n > 4096) return MX_E_INVAL;
  if (precision != MX_FP64 && precision != MX_FP32) return MX_E_INVAL;
  if (form != MX_FORM_SPECTRAL && form != MX_FORM_LITERAL && form != MX_FORM_XY) return MX_E_INVAL;
  mx_batch* b = new mx_batch();
  b->n = n;
  b->prec = precision;
  b->form = form;
  b->stream = (cudaStream_t)stream;
  if (!b->stream) {  // the legacy default stream cannot be captured into a graph: use an own stream
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return MX_E_CUDA;
    }
    b->own_stream = true;
  }
  stream = b->stream;
  auto bail = [&](mx_status s) {
    mx_batch_destroy(b);
    return s;
  };
  if (form != MX_FORM_SPECTRAL) {  // literal or xy-resident: a graph of every instance's own passes
    for (int i = 0; i < n; ++i) {
      if (!isfinite(inst[i].h)) return bail(MX_E_INVAL);
      mx_ctx* c = nullptr;
      mx_status st = mx_create(&c, inst[i].nx, inst[i].ny, inst[i].nz, inst[i].lo, inst[i].hi, inst[i].eps, inst[i].mu,
                               precision, form, stream);
      if (st != MX_OK) return bail(st);
      b->ctx.push_back(c);
      b->h.push_back(inst[i].h);
      st = mx_autotune(c);  // the pass schedules of this shape (cached per process; before any load)
      if (st != MX_OK) return bail(st);
      cudaStream_t ls = nullptr;
      cudaEvent_t ev = nullptr;
      if (cudaStreamCreateWithFlags(&ls, cudaStreamNonBlocking) != cudaSuccess) return bail(MX_E_CUDA);
      b->lstreams.push_back(ls);
      if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return bail(MX_E_CUDA);
      b->ldone.push_back(ev);
    }
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) return bail(MX_E_CUDA);
    b->grec.assign(n, nullptr);
    b->grec_cap.assign(n, 0);
    *out = b;
    return MX_OK;
  }
  const unsigned ch = precision == MX_FP64 ? mx::bt_ch<double>() : mx::bt_ch<float>();
  unsigned long long chunks = 0, q = 0;
  for (int i = 0; i < n; ++i) {
    if (!isfinite(inst[i].h)) return bail(MX_E_INVAL);
    mx_ctx* c = nullptr;
    mx_status st = mx_create(&c, inst[i].nx, inst[i].ny, inst[i].nz, inst[i].lo, inst[i].hi, inst[i].eps, inst[i].mu,
                             precision, MX_FORM_SPECTRAL, stream);
    if (st != MX_OK) return bail(st);
    b->ctx.push_back(c);
    b->h.push_back(inst[i].h);
    chunks += ((unsigned long long)c->nh + ch - 1) / ch;
    q += c->table ? (unsigned long long)c->nq : 0ULL;
  }
  if (chunks >= (1ULL << 31) || q >= (1ULL << 31)) return bail(MX_E_UNSUPPORTED_N);
  b->total_chunks = (unsigned)chunks;
  b->total_q = (unsigned)q;
  if (mx::host_alloc_pinned((void**)&b->h_inst, sizeof(mx::BInst) * n) != cudaSuccess) return bail(MX_E_NOMEM);
  if (mx::dev_alloc((void**)&b->d_inst, sizeof(mx::BInst) * n) != cudaSuccess) return bail(MX_E_NOMEM);
  if (mx::dev_alloc((void**)&b->cpart, (size_t)b->total_chunks * mx::BT_CWARPS * 16 * sizeof(double)) != cudaSuccess)
    return bail(MX_E_NOMEM);
  if (mx::dev_alloc((void**)&b->bar, 64) != cudaSuccess) return bail(MX_E_NOMEM);
  if (cudaMemset(b->bar, 0, 64) != cudaSuccess) return bail(MX_E_CUDA);
  // descriptors that do not change between calls
  unsigned c0 = 0, q0 = 0, s0 = 0;
  for (int i = 0; i < n; ++i) {
    mx_ctx* c = b->ctx[i];
    mx::BInst& d = b->h_inst[i];
    memset(&d, 0, sizeof(d));
    d.g = c->g;
    d.src = c->spec0;
    d.dst = c->spec;
    d.tab = c->table ? c->tab : nullptr;
    d.nq = c->table ? c->nq : 0;
    d.npts = (unsigned)c->nh;
    d.chunk0 = c0;
    d.nchunks = (unsigned)((c->nh + ch - 1) / ch);
    d.q0 = q0;
    d.seg0 = s0;
    d.nseg = (d.nchunks + mx::BT_SEGC - 1) / mx::BT_SEGC;
    d.h = b->h[i];
    c0 += d.nchunks;
    q0 += (unsigned)d.nq;
    s0 += d.nseg;
  }
  b->total_segs = s0;
  if (mx::dev_alloc((void**)&b->segpart, (size_t)2 * b->total_segs * mx::NSUM * sizeof(double)) != cudaSuccess)
    return bail(MX_E_NOMEM);
  if (precision == MX_FP32 && b->total_q > 0) {
    // what phase A's coefficients take from |k| alone, as coef_direct forms it
    std::vector<mx::QK> qk(b->total_q);
    for (int i = 0; i < n; ++i) {
      const mx::BInst& d = b->h_inst[i];
      for (int qi = 0; qi < d.nq; ++qi) {
        const double k2 = d.g.s0 * (double)qi, kabs = std::sqrt(k2);
        qk[d.q0 + qi] = mx::QK{0.5 * d.g.c * kabs, (float)kabs, (float)k2};
      }
    }
    if (mx::dev_alloc((void**)&b->qk, qk.size() * sizeof(mx::QK)) != cudaSuccess) return bail(MX_E_NOMEM);
    if (cudaMemcpy(b->qk, qk.data(), qk.size() * sizeof(mx::QK), cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(MX_E_CUDA);
  }
  // co-resident grid for the cooperative launch
  const void* kern = precision == MX_FP64 ? batch_kernel<double>() : batch_kernel<float>();
  const size_t smem = precision == MX_FP64 ? mx::bt_smem_bytes<double>() : mx::bt_smem_bytes<float>();
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return bail(MX_E_CUDA);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, mx::BT_THREADS, smem) != cudaSuccess || per_sm < 1)
    return bail(MX_E_CUDA);
  const long long cap = (long long)mx::num_sms() * std::min(per_sm, 2);
  b->grid = (int)std::max<long long>(1, std::min<long long>(cap, b->total_chunks));
  *out = b;
  return MX_OK;
}

mx_status mx_batch_size(mx_batch* b, int* n) {
  if (!b || !n) return MX_E_INVAL;
  *n = b->n;
  return MX_OK;
}

mx_status mx_batch_instance(mx_batch* b, int i, mx_ctx** ctx) {
  if (!b || !ctx || i < 0 || i >= b->n) return MX_E_INVAL;
  *ctx = b->ctx[i];
  return MX_OK;
}

mx_status mx_batch_load_random(mx_batch* b, unsigned long long seed, double sigma) {
  if (!b) return MX_E_INVAL;
  if (b->err != MX_OK) return b->err;
  for (int i = 0; i < b->n; ++i) {
    mx_status st = mx_load_random_divfree(b->ctx[i], seed + (unsigned long long)i, sigma);
    if (st != MX_OK) return st;
  }
  return MX_OK;
}

mx_status mx_batch_step(mx_batch* b, long long nsteps, int invariants_every) {
  if (!b || nsteps < 0 || nsteps > (1LL << 30) || invariants_every < 0) return MX_E_INVAL;
  if (b->err != MX_OK) return b->err;
  if (nsteps == 0) return MX_OK;
  for (int i = 0; i < b->n; ++i)
    if (!b->ctx[i]->loaded) return MX_E_STATE;
  if (b->form != MX_FORM_SPECTRAL) {
    const mx_status st = step_literal(b, nsteps, invariants_every);
    if (st != MX_OK && st != MX_E_INVAL && st != MX_E_STATE) b->err = st;
    return st;
  }
  // the pinned descriptors may still be read by the previous launch's copy node
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return fail(b, cudaErrorUnknown);
  // per-call descriptor fields; record capacity
  std::vector<long long> nrec(b->n, 0);
  for (int i = 0; i < b->n; ++i) {
    mx_ctx* c = b->ctx[i];
    if (c->err != MX_OK) return c->err;
    if (invariants_every > 0) nrec[i] = (c->step + nsteps) / invariants_every - c->step / invariants_every;
    mx_status st = mx_ensure_records(c, nrec[i]);
    if (st != MX_OK) return st;
    mx::BInst& d = b->h_inst[i];
    d.n0 = c->step;
    d.t0 = c->t;
    d.every = invariants_every;
    d.rec = c->rec + (size_t)c->rec_n * 16;
  }
  const int k = (int)nsteps;
  cudaError_t e = cudaSuccess;
  if (b->use_graph) {
    auto it = b->graphs.find(k);
    if (it == b->graphs.end()) {
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      cudaError_t ce = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
      if (ce == cudaSuccess) {
        const cudaError_t le = enqueue_step(b, k);
        ce = cudaStreamEndCapture(b->stream, &graph);
        if (ce == cudaSuccess) ce = le;
      }
      if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (ce != cudaSuccess) {
        cudaGetLastError();  // capture refused: launch directly from now on
        b->graph_err = (int)ce;
        b->use_graph = false;
      } else {
        it = b->graphs.emplace(k, exec).first;
      }
    }
    if (b->use_graph) e = cudaGraphLaunch(it->second, b->stream);
  }
  if (!b->use_graph) e = enqueue_step(b, k);
  if (e != cudaSuccess) return fail(b, e);
  for (int i = 0; i < b->n; ++i) {
    mx_ctx* c = b->ctx[i];
    const long long n0 = c->step;
    if (invariants_every > 0)
      for (long long N = (n0 / invariants_every + 1) * invariants_every; N <= n0 + nsteps; N += invariants_every) {
        c->rec_t.push_back(c->t + (double)(N - n0) * b->h[i]);
        c->rec_step.push_back(N);
        ++c->rec_n;
      }
    c->t += (double)nsteps * b->h[i];
    c->step += nsteps;
    c->spec_valid = true;
    c->tab_t = NAN;  // the batch wrote the tables for its last step
  }
  return MX_OK;
}

mx_status mx_batch_sync(mx_batch* b) {
  if (!b) return MX_E_INVAL;
  if (b->err != MX_OK) return b->err;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return fail(b, cudaErrorUnknown);
  if (b->form != MX_FORM_SPECTRAL) {
    for (int i = 0; i < b->n; ++i) {
      const mx_status st = mx_sync(b->ctx[i]);  // latched errors and timed-out waits of the instance
      if (st != MX_OK) {
        b->err = st;
        return st;
      }
    }
    return MX_OK;
  }
  unsigned flags[3] = {0, 0, 0};
  if (cudaMemcpy(flags, b->bar, sizeof(flags), cudaMemcpyDeviceToHost) != cudaSuccess) return fail(b, cudaErrorUnknown);
  if (flags[2]) {
    b->err = MX_E_TIMEOUT;
    return b->err;
  }
  return MX_OK;
}

mx_status mx_batch_launch_shape(mx_batch* b, int* blocks, int* threads) {
  if (!b || !blocks || !threads) return MX_E_INVAL;
  *blocks = b->form != MX_FORM_SPECTRAL ? 0 : b->grid;
  *threads = b->form != MX_FORM_SPECTRAL ? 0 : mx::BT_THREADS;
  return MX_OK;
}

mx_status mx_batch_graph_used(mx_batch* b, int* used) {
  if (!b || !used) return MX_E_INVAL;
  *used = b->graph_err ? -b->graph_err : (b->use_graph && (!b->graphs.empty() || !b->lgraphs.empty()));
  return MX_OK;
}

void mx_batch_destroy(mx_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  for (auto& kv : b->lgraphs) cudaGraphExecDestroy(kv.second);
  for (cudaStream_t ls : b->lstreams) cudaStreamDestroy(ls);
  for (cudaEvent_t ev : b->ldone) cudaEventDestroy(ev);
  if (b->fork) cudaEventDestroy(b->fork);
  for (double* r : b->grec)
    if (r) cudaFree(r);
  for (mx_ctx* c : b->ctx) mx_destroy(c);
  if (b->h_inst) cudaFreeHost(b->h_inst);
  if (b->d_inst) cudaFree(b->d_inst);
  if (b->cpart) cudaFree(b->cpart);
  if (b->segpart) cudaFree(b->segpart);
  if (b->qk) cudaFree(b->qk);
  if (b->bar) cudaFree(b->bar);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
}

}  // extern "C"

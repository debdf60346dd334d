// Batched spectral form (C ABI): independent instances of different grids,
// eps, mu and step sizes, each a spectral-form context, advanced together by
// one persistent cooperative launch per mx_batch_step call.  The launch
// (with the upload of the per-instance descriptors) is captured once per
// step count into a CUDA graph and replayed.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
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
  unsigned* bar = nullptr;
  unsigned total_chunks = 0, total_q = 0, total_segs = 0;
  int grid = 0;
  bool use_graph = true;
  int graph_err = 0;                       // CUDA error of a refused capture (0: none)
  bool own_stream = false;
  std::map<int, cudaGraphExec_t> graphs;  // nsteps -> executable graph
  mx_status err = MX_OK;
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

}  // namespace

extern "C" {

mx_status mx_batch_create(mx_batch** out, const mx_instance_desc* inst, int n, int precision, void* stream) {
  if (!out) return MX_E_INVAL;
  *out = nullptr;
  if (!inst || n < 1 || n > 4096) return MX_E_INVAL;
  if (precision != MX_FP64 && precision != MX_FP32) return MX_E_INVAL;
  mx_batch* b = new mx_batch();
  b->n = n;
  b->prec = precision;
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
  if (mx::dev_alloc((void**)&b->cpart, (size_t)b->total_chunks * mx::BT_CWARPS * mx::NSUM * sizeof(double)) != cudaSuccess)
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
    d.nseg = (d.nchunks * mx::BT_CWARPS + mx::BT_SEG - 1) / mx::BT_SEG;
    d.h = b->h[i];
    c0 += d.nchunks;
    q0 += (unsigned)d.nq;
    s0 += d.nseg;
  }
  b->total_segs = s0;
  if (mx::dev_alloc((void**)&b->segpart, (size_t)2 * b->total_segs * mx::NSUM * sizeof(double)) != cudaSuccess)
    return bail(MX_E_NOMEM);
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
  unsigned flags[3] = {0, 0, 0};
  if (cudaMemcpy(flags, b->bar, sizeof(flags), cudaMemcpyDeviceToHost) != cudaSuccess) return fail(b, cudaErrorUnknown);
  if (flags[2]) {
    b->err = MX_E_TIMEOUT;
    return b->err;
  }
  return MX_OK;
}

mx_status mx_batch_graph_used(mx_batch* b, int* used) {
  if (!b || !used) return MX_E_INVAL;
  *used = b->graph_err ? -b->graph_err : (b->use_graph && !b->graphs.empty());
  return MX_OK;
}

void mx_batch_destroy(mx_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  for (mx_ctx* c : b->ctx) mx_destroy(c);
  if (b->h_inst) cudaFreeHost(b->h_inst);
  if (b->d_inst) cudaFree(b->d_inst);
  if (b->cpart) cudaFree(b->cpart);
  if (b->segpart) cudaFree(b->segpart);
  if (b->bar) cudaFree(b->bar);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
}

}  // extern "C"

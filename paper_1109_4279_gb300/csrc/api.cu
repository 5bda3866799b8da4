// The C-ABI of libqcdgb (include/qcdgb.h): argument checking, host/device
// staging, context lifetime and kernel instrumentation.
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "internal.h"

namespace qcd {

static thread_local std::string g_last_error;
std::atomic<long long> g_launches{0};

int cuda_fail(cudaError_t e, const char* where) {
  g_last_error = std::string(cudaGetErrorString(e)) + " at " + where;
  return QCD_ERR_CUDA;
}

int rec_alloc(Rec& r, int prec, int nreal, long long V) {
  rec_free(r);
  const size_t data = (size_t)V * chunks(prec, nreal) * 16;
  const size_t norm = (prec == P16 || prec == PB16) ? (size_t)V * sizeof(float) : 0;
  void* p = nullptr;
  if (cudaMalloc(&p, data + norm) != cudaSuccess) {
    cudaGetLastError();
    return QCD_ERR_NOMEM;
  }
  r.prec = prec;
  r.nreal = nreal;
  r.data = p;
  r.norm = norm ? (float*)((char*)p + data) : nullptr;
  r.bytes = data + norm;
  return QCD_OK;
}

void rec_free(Rec& r) {
  if (r.data) cudaFree(r.data);
  r = Rec();
}

Workspace* ensure_ws(qcd_ctx* c) {
  if (!c->ws) c->ws = new (std::nothrow) Workspace();
  return c->ws;
}

ProfScope::ProfScope(qcd_ctx* ctx, int kernel, cudaStream_t st, double bytes, double flops) : c(ctx), k(kernel), s(st) {
  if (!c->prof) return;
  cudaEvent_t e0;
  if (c->event_pool.size() >= 2) {
    e0 = c->event_pool.back();
    c->event_pool.pop_back();
    e1 = c->event_pool.back();
    c->event_pool.pop_back();
  } else {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
  }
  cudaEventRecord(e0, s);
  c->timers[k].pending.emplace_back(e0, e1);
  c->timers[k].bytes += bytes;
  c->timers[k].flops += flops;
}

ProfScope::~ProfScope() {
  if (!c->prof || !e1) return;
  cudaEventRecord(e1, s);
  c->timers[k].launches += 1;
}

static void prof_collect(qcd_ctx* c) {
  for (auto& t : c->timers) {
    for (auto& pr : t.pending) {
      cudaEventSynchronize(pr.second);
      float ms = 0;
      if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) t.total_ms += ms;
      c->event_pool.push_back(pr.first);
      c->event_pool.push_back(pr.second);
    }
    t.pending.clear();
  }
}

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace qcd

using namespace qcd;

extern "C" {

void qcd_solver_defaults(qcd_solver_params* sp) {
  if (!sp) return;
  sp->tol = 1e-10;
  sp->nkv = 16;
  sp->max_restarts = 100;
  sp->precond = QCD_PRECOND_SAP;
  sp->ncy = 4;
  sp->nmr = 4;
  sp->sap_prec = QCD_PREC_F32;
  sp->outer_prec = QCD_PREC_F64;
  sp->inner_tol = 1e-5;
  sp->solver = QCD_SOLVER_FGCR;
  sp->ndefl = 4;
  sp->cg_fallback = 0;
  sp->cg_max_iter = 20000;
  sp->zero_guess = 0;
  sp->residual_prec = QCD_PREC_DF64;
}

const char* qcd_status_string(int st) {
  switch (st) {
    case QCD_OK: return "ok";
    case QCD_ERR_ARG: return "invalid argument";
    case QCD_ERR_GEOMETRY: return "block extents must be even, divide the lattice, and give an even block count per direction";
    case QCD_ERR_CUDA: return "CUDA runtime error";
    case QCD_ERR_NOMEM: return "device allocation failed";
    case QCD_ERR_STATE: return "call out of order (gauge field or clover term missing)";
    case QCD_ERR_NOT_SU3: return "a link is not in SU(3)";
    case QCD_ERR_SINGULAR_CLOVER: return "a clover block is singular";
    case QCD_NOT_CONVERGED: return "not converged within max_restarts";
    case QCD_STAGNATED: return "stagnated: restart cycles stopped reducing the true residual";
    case QCD_NAN: return "NaN or Inf in the recursion";
    case QCD_ERR_UNSUPPORTED: return "unsupported precision or block shape";
    case QCD_ERR_TOO_LARGE: return "size beyond the entry point's fixed limit";
    case QCD_ERR_TIMEOUT: return "a kernel's bounded wait ran out";
    default: return "unknown status";
  }
}

const char* qcd_last_error(void) { return g_last_error.c_str(); }

long long qcd_launch_count(void) { return g_launches.load(); }

int qcd_create(qcd_ctx** out, const qcd_params* p) {
  if (!out || !p) return QCD_ERR_ARG;
  *out = nullptr;
  for (int mu = 0; mu < 4; ++mu)
    if (!(p->bc[mu] == 1.0 || p->bc[mu] == -1.0)) return QCD_ERR_ARG;
  qcd_ctx* c = new (std::nothrow) qcd_ctx();
  if (!c) return QCD_ERR_NOMEM;
  c->p = *p;
  int st = setup_geometry(c);
  if (st == QCD_OK) {
    if (cudaMalloc(&c->d_scalars, 64 * 1024) != cudaSuccess || cudaMallocHost(&c->h_scalars, 64 * 1024) != cudaSuccess ||
        cudaMemset(c->d_scalars, 0, 64 * 1024) != cudaSuccess)
      st = QCD_ERR_NOMEM;
  }
  if (st != QCD_OK) {
    qcd_destroy(c);
    return st;
  }
  *out = c;
  return QCD_OK;
}

void qcd_destroy(qcd_ctx* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  workspace_free(c);
  for (int p = 0; p < 5; ++p) {
    if (c->U[p]) cudaFree(c->U[p]);
    rec_free(c->A[p]);
    rec_free(c->Ahat[p]);
  }
  for (auto st : c->streams) cudaStreamDestroy(st);
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  if (c->deliver_stream) cudaStreamDestroy(c->deliver_stream);
  c->streams.clear();
  if (c->d_tables) cudaFree(c->d_tables);
  if (c->d_scalars) cudaFree(c->d_scalars);
  if (c->h_scalars) cudaFreeHost(c->h_scalars);
  for (auto& t : c->timers)
    for (auto& pr : t.pending) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
  for (auto e : c->event_pool) cudaEventDestroy(e);
  delete c;
}

int qcd_load_gauge(qcd_ctx* c, const double* U, int is_device, void* stream) {
  if (!c || !U) return QCD_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)c->V * 4 * 9 * 16;
  if (is_device) return load_gauge_device(c, U, s);
  void* tmp = nullptr;
  if (cudaMalloc(&tmp, bytes) != cudaSuccess) {
    cudaGetLastError();
    return QCD_ERR_NOMEM;
  }
  int st = QCD_OK;
  cudaError_t e = cudaMemcpyAsync(tmp, U, bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) st = cuda_fail(e, "gauge upload");
  if (st == QCD_OK) st = load_gauge_device(c, (const double*)tmp, s);
  cudaStreamSynchronize(s);
  cudaFree(tmp);
  return st;
}

int qcd_build_clover(qcd_ctx* c, void* stream) {
  if (!c) return QCD_ERR_ARG;
  return build_clover(c, (cudaStream_t)stream);
}

int qcd_apply_D(qcd_ctx* c, const double* in, double* out, int dagger, int prec, int nrhs, void* stream) {
  if (!c || !in || !out || nrhs < 1 || prec < 0 || prec > 4) return QCD_ERR_ARG;
  if (!c->clover_built) return QCD_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  Rec a, b;
  int st = rec_alloc(a, prec, 24, c->V * nrhs);
  if (st == QCD_OK) st = rec_alloc(b, prec, 24, c->V * nrhs);
  if (st == QCD_OK) st = import_spinor(c, in, a, nrhs, s);
  if (st == QCD_OK) st = dirac_apply(c, a, b, dagger, s, nrhs);
  if (st == QCD_OK) st = export_spinor(c, b, out, nrhs, s);
  cudaStreamSynchronize(s);
  rec_free(a);
  rec_free(b);
  return st;
}

// streams of a context for batched right-hand sides (created once)
static int ctx_streams(qcd_ctx* c, int n) {
  while ((int)c->streams.size() < n) {
    cudaStream_t s;
    QCD_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    c->streams.push_back(s);
  }
  return QCD_OK;
}

static Workspace* rhs_workspace(qcd_ctx* c, int k) {
  if (k == 0) return ensure_ws(c);
  while ((int)c->batch_ws.size() < k) {
    Workspace* w = new (std::nothrow) Workspace();
    if (!w) return nullptr;
    c->batch_ws.push_back(w);
  }
  return c->batch_ws[k - 1];
}

// order: the problems' streams wait for `s`, and `s` waits for them afterwards
static int fork_streams(cudaStream_t s, std::vector<Problem>& probs) {
  cudaEvent_t e;
  QCD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  cudaEventRecord(e, s);
  for (auto& p : probs)
    if (p.s != s) cudaStreamWaitEvent(p.s, e, 0);
  cudaEventDestroy(e);
  return QCD_OK;
}

static int join_streams(cudaStream_t s, std::vector<Problem>& probs) {
  for (size_t i = 0; i < probs.size(); ++i) {
    Problem& p = probs[i];
    if (p.s == s || (i > 0 && probs[i - 1].s == p.s)) continue;  // each stream once
    cudaEvent_t e;
    QCD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    cudaEventRecord(e, p.s);
    cudaStreamWaitEvent(s, e, 0);
    cudaEventDestroy(e);
  }
  return QCD_OK;
}

// solve a set of problems whose b/x are lexicographic device or host arrays
static int solve_problems(std::vector<Problem>& probs, const double* const* b, double* const* x, bool dev,
                          const qcd_solver_params& sp, qcd_solve_info* info, cudaStream_t s) {
  if (sp.solver < QCD_SOLVER_FGCR || sp.solver > QCD_SOLVER_CG_EO || sp.cg_fallback < 0 || sp.cg_fallback > 2)
    return QCD_ERR_ARG;
  const int n = (int)probs.size();
  std::vector<double*> stage(n, nullptr);
  int st = QCD_OK;
  for (int k = 0; k < n && st == QCD_OK; ++k) {
    Problem& p = probs[k];
    for (Rec* f : {&p.w->b, &p.w->x})
      if (!f->data) st = rec_alloc(*f, P64, 24, p.c->V);
    if (st != QCD_OK) break;
    p.b = p.w->b;
    p.x = p.w->x;
    const size_t fbytes = (size_t)p.c->V * 24 * sizeof(double);
    const double* bd = b[k];
    const double* xd = x[k];
    if (!dev) {
      // lexicographic staging of b and x for host buffers, kept by the
      // problem's workspace across calls
      Workspace& w = *p.w;
      if (w.stage_bytes < 2 * fbytes) {
        if (w.stage) cudaFree(w.stage);
        w.stage = nullptr;
        w.stage_bytes = 0;
        if (cudaMalloc(&w.stage, 2 * fbytes) != cudaSuccess) {
          cudaGetLastError();
          w.stage = nullptr;
          st = QCD_ERR_NOMEM;
          break;
        }
        w.stage_bytes = 2 * fbytes;
      }
      stage[k] = w.stage;
      st = upload_spinor(p.c, b[k], stage[k], p.b, s);
      if (st == QCD_OK && !sp.zero_guess) st = upload_spinor(p.c, x[k], stage[k] + p.c->V * 24, p.x, s);
    } else {
      st = import_spinor(p.c, bd, p.b, 1, s);
      if (st == QCD_OK && !sp.zero_guess) st = import_spinor(p.c, xd, p.x, 1, s);
    }
    if (st == QCD_OK && sp.zero_guess) {
      const cudaError_t e = cudaMemsetAsync(p.x.data, 0, fbytes, s);  // FP64 block-major, same size
      if (e != cudaSuccess) st = cuda_fail(e, "solve zero guess");
    }
    // FGCR hands each restart's updated x to the caller's field at once; the
    // export at the end is then needed only if x changed after the last one
    if (sp.solver == QCD_SOLVER_FGCR) {
      p.dlv_lex = x[k];
      p.dlv_stage = dev ? nullptr : stage[k] + p.c->V * 24;
    }
  }
  if (st == QCD_OK) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    fork_streams(s, probs);
    bool prof = false;
    for (auto& p : probs) prof |= p.c->prof;
    // captured iteration graphs are replayed unless kernels are being timed
    // one by one (the profiler's events would be baked into the graphs)
    st = run_solver(probs, sp, !prof);
    join_streams(s, probs);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (auto& p : probs) p.info.time_ms = ms;
    for (int k = 0; k < n; ++k) {
      Problem& p = probs[k];
      int e2 = QCD_OK;
      // s follows the last delivery (its writes to the caller's field end first)
      if (p.dlv_event && cudaStreamWaitEvent(s, p.dlv_event, 0) != cudaSuccess) e2 = QCD_ERR_CUDA;
      if (e2 == QCD_OK && !p.delivered)
        e2 = dev ? export_spinor(p.c, p.x, x[k], 1, s) : download_spinor(p.c, p.x, stage[k] + p.c->V * 24, x[k], s);
      if (e2 != QCD_OK && p.status == QCD_OK) p.status = p.info.status = e2;
      if (e2 != QCD_OK && st == QCD_OK) st = e2;
    }
  }
  cudaStreamSynchronize(s);
  for (auto& p : probs)
    if (p.dlv_event) cudaEventDestroy(p.dlv_event);
  for (int k = 0; k < n; ++k) {

    if (info) info[k] = probs[k].info;
  }
  return st;
}

// nrhs > 1 right-hand sides of one lattice by FGCR, all iterated by the same
// launches: one workspace holds their fields back to back
static int solve_tile(qcd_ctx* c, const double* b, double* x, int nrhs, bool dev, const qcd_solver_params& sp,
                      qcd_solve_info* info, cudaStream_t s) {
  if (!c->tile_ws) c->tile_ws = new (std::nothrow) Workspace();
  Workspace* w = c->tile_ws;
  if (!w) return QCD_ERR_NOMEM;
  if (sp.nkv < 1 || sp.nkv > 64) return QCD_ERR_ARG;
  QCD_TRY(ws_prepare(c, *w, sp, s, nrhs));
  const size_t fbytes = (size_t)c->V * 24 * sizeof(double) * nrhs;
  const double* bd = b;
  double* xd = x;
  if (!dev) {  // lexicographic staging of b and x, kept by the workspace across calls
    if (w->stage_bytes < 2 * fbytes) {
      if (w->stage) cudaFree(w->stage);
      w->stage = nullptr;
      w->stage_bytes = 0;
      if (cudaMalloc(&w->stage, 2 * fbytes) != cudaSuccess) {
        cudaGetLastError();
        w->stage = nullptr;
        return QCD_ERR_NOMEM;
      }
      w->stage_bytes = 2 * fbytes;
    }
    QCD_CUDA(cudaMemcpyAsync(w->stage, b, fbytes, cudaMemcpyHostToDevice, s));
    if (!sp.zero_guess)
      QCD_CUDA(cudaMemcpyAsync(w->stage + c->V * 24 * nrhs, x, fbytes, cudaMemcpyHostToDevice, s));
    bd = w->stage;
    xd = w->stage + c->V * 24 * nrhs;
  }
  QCD_TRY(import_spinor(c, bd, w->b, nrhs, s));
  if (sp.zero_guess)
    QCD_CUDA(cudaMemsetAsync(w->x.data, 0, w->x.bytes, s));
  else
    QCD_TRY(import_spinor(c, xd, w->x, nrhs, s));
  // the iterations run on the context's own stream, ordered after and before
  // the caller's: a stream the library owns can always be captured into graphs
  // (the legacy default stream cannot)
  QCD_TRY(ctx_streams(c, 1));
  const cudaStream_t ws = c->streams[0];
  std::vector<Problem> probs(nrhs);
  Group G;
  G.c = c;
  G.w = w;
  G.s = ws;
  G.rt = sap_tile(c, nrhs);
  for (int q = 0; q < nrhs; ++q) {
    probs[q].c = c;
    probs[q].w = w;
    probs[q].s = ws;
    probs[q].b = rhs_view(w->b, q, c->V);
    probs[q].x = rhs_view(w->x, q, c->V);
    G.rhs.push_back(&probs[q]);
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  std::vector<Group> groups(1, G);
  int st = QCD_OK;
  if (sp.solver != QCD_SOLVER_FGCR || sp.cg_fallback < 0 || sp.cg_fallback > 2) st = QCD_ERR_ARG;
  if (st == QCD_OK) st = fork_streams(s, probs);
  if (st == QCD_OK) st = fgcr_groups(groups, sp, !c->prof);
  join_streams(s, probs);
  if (st != QCD_OK && sp.cg_fallback) {
    // CG from the iterate of every right-hand side that stagnated or ran out of
    // restarts, one after another in the single-right-hand-side workspace
    std::vector<Problem> fb;
    Workspace* w1 = ensure_ws(c);
    for (int q = 0; q < nrhs; ++q)
      if (probs[q].status == QCD_STAGNATED || probs[q].status == QCD_NOT_CONVERGED) {
        fb.push_back(probs[q]);
        fb.back().w = w1;
      }
    if (w1 && !fb.empty()) {
      cg_batch(fb, sp, true);
      size_t i = 0;
      for (int q = 0; q < nrhs; ++q)
        if (probs[q].status == QCD_STAGNATED || probs[q].status == QCD_NOT_CONVERGED) probs[q] = fb[i++];
    }
    st = QCD_OK;
    for (auto& p : probs)
      if (p.status != QCD_OK && st == QCD_OK) st = p.status;
  }
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int e2 = export_spinor(c, w->x, xd, nrhs, s);
  if (e2 == QCD_OK && !dev) {
    const cudaError_t e = cudaMemcpyAsync(x, xd, fbytes, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) e2 = cuda_fail(e, "solve download");
  }
  cudaStreamSynchronize(s);
  for (int q = 0; q < nrhs; ++q) {
    probs[q].info.time_ms = ms;
    if (e2 != QCD_OK && probs[q].status == QCD_OK) probs[q].status = probs[q].info.status = e2;
    if (info) info[q] = probs[q].info;
  }
  return st != QCD_OK ? st : e2;
}

int qcd_solve(qcd_ctx* c, const double* b, double* x, int nrhs, const qcd_solver_params* sp_in, qcd_solve_info* info,
              void* stream) {
  NvtxRange nv("qcd_solve");
  if (!c || !b || !x || nrhs < 1) return QCD_ERR_ARG;
  if (!c->clover_built) return QCD_ERR_STATE;
  qcd_solver_params sp;
  if (sp_in) sp = *sp_in; else qcd_solver_defaults(&sp);
  cudaStream_t s = (cudaStream_t)stream;
  const bool dev = is_device_ptr(b);
  if (dev != is_device_ptr(x)) return QCD_ERR_ARG;
  if (nrhs > 1 && sp.solver == QCD_SOLVER_FGCR) return solve_tile(c, b, x, nrhs, dev, sp, info, s);
  QCD_TRY(ctx_streams(c, nrhs));
  std::vector<Problem> probs(nrhs);
  std::vector<const double*> bs(nrhs);
  std::vector<double*> xs(nrhs);
  for (int k = 0; k < nrhs; ++k) {
    probs[k].c = c;
    probs[k].w = rhs_workspace(c, k);
    if (!probs[k].w) return QCD_ERR_NOMEM;
    probs[k].s = c->streams[k];  // a context stream (capturable), forked from and joined to s
    bs[k] = b + (size_t)k * c->V * 24;
    xs[k] = x + (size_t)k * c->V * 24;
  }
  return solve_problems(probs, bs.data(), xs.data(), dev, sp, info, s);
}

int qcd_solve_dagger(qcd_ctx* c, const double* b, double* x, const qcd_solver_params* sp_in, qcd_solve_info* info,
                     void* stream) {
  NvtxRange nv("qcd_solve_dagger");
  if (!c || !b || !x) return QCD_ERR_ARG;
  if (!c->clover_built) return QCD_ERR_STATE;
  qcd_solver_params sp;
  if (sp_in) sp = *sp_in; else qcd_solver_defaults(&sp);
  cudaStream_t s = (cudaStream_t)stream;
  Workspace* w = ensure_ws(c);
  if (!w) return QCD_ERR_NOMEM;
  for (Rec* f : {&w->b, &w->x})
    if (!f->data) QCD_TRY(rec_alloc(*f, P64, 24, c->V));
  // D^+ x = b  <=>  D (g5 x) = g5 b
  QCD_TRY(import_spinor(c, b, w->b, 1, s));
  if (sp.zero_guess)
    QCD_CUDA(cudaMemsetAsync(w->x.data, 0, (size_t)c->V * 24 * sizeof(double), s));
  else
    QCD_TRY(import_spinor(c, x, w->x, 1, s));
  QCD_TRY(blas_gamma5(c, (const double*)w->b.data, (double*)w->b.data, 0, s));
  QCD_TRY(blas_gamma5(c, (const double*)w->x.data, (double*)w->x.data, 0, s));
  int st = solve_one(c, w->b, w->x, sp, info, s);
  int e = blas_gamma5(c, (const double*)w->x.data, (double*)w->x.data, 0, s);
  if (e == QCD_OK) e = export_spinor(c, w->x, x, 1, s);
  cudaStreamSynchronize(s);
  return st != QCD_OK ? st : e;
}

int qcd_solve_batch(qcd_ctx** ctxs, int n, const double* const* b, double* const* x, const qcd_solver_params* sp_in,
                    qcd_solve_info* info, void* stream) {
  NvtxRange nv("qcd_solve_batch");
  if (!ctxs || !b || !x || n < 1) return QCD_ERR_ARG;
  qcd_solver_params sp;
  if (sp_in) sp = *sp_in; else qcd_solver_defaults(&sp);
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<Problem> probs(n);
  for (int i = 0; i < n; ++i) {
    qcd_ctx* c = ctxs[i];
    if (!c || !b[i] || !x[i]) return QCD_ERR_ARG;
    if (!c->clover_built) return QCD_ERR_STATE;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == c) return QCD_ERR_ARG;  // one right-hand side per context (use qcd_solve's nrhs)
    if (!is_device_ptr(b[i]) || !is_device_ptr(x[i])) return QCD_ERR_ARG;
    QCD_TRY(ctx_streams(c, 1));
    probs[i].c = c;
    probs[i].w = ensure_ws(c);
    if (!probs[i].w) return QCD_ERR_NOMEM;
    probs[i].s = c->streams[0];  // a context stream (capturable), forked from and joined to s
  }
  return solve_problems(probs, b, x, true, sp, info, s);
}

int qcd_force(qcd_ctx* c, const double* x, const double* y, double* F, void* stream) {
  if (!c || !x || !y || !F) return QCD_ERR_ARG;
  if (!c->clover_built) return QCD_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  Rec xi, yi;
  int st = rec_alloc(xi, P64, 24, c->V);
  if (st == QCD_OK) st = rec_alloc(yi, P64, 24, c->V);
  if (st == QCD_OK) st = import_spinor(c, x, xi, 1, s);
  if (st == QCD_OK) st = import_spinor(c, y, yi, 1, s);
  if (st == QCD_OK) st = force_apply(c, xi, yi, F, s);
  cudaStreamSynchronize(s);
  rec_free(xi);
  rec_free(yi);
  return st;
}

int qcd_gradient(qcd_ctx* c, const double* phi, double* dL_dphi, double* dL_dtheta, double* x_out, double* y_out,
                 const qcd_solver_params* sp_in, void* stream) {
  NvtxRange nv("qcd_gradient");
  if (!c || !phi) return QCD_ERR_ARG;
  if (!c->clover_built) return QCD_ERR_STATE;
  qcd_solver_params sp;
  if (sp_in) sp = *sp_in; else qcd_solver_defaults(&sp);
  cudaStream_t s = (cudaStream_t)stream;
  Workspace* w = ensure_ws(c);
  if (!w) return QCD_ERR_NOMEM;
  for (Rec* f : {&w->b, &w->x})
    if (!f->data) QCD_TRY(rec_alloc(*f, P64, 24, c->V));
  const size_t fbytes = (size_t)c->V * 24 * sizeof(double);
  Rec xk, yk;
  int st = rec_alloc(xk, P64, 24, c->V);
  if (st == QCD_OK) st = rec_alloc(yk, P64, 24, c->V);
  // x = D^-1 phi
  if (st == QCD_OK) st = import_spinor(c, phi, w->b, 1, s);
  if (st == QCD_OK) st = cudaMemsetAsync(xk.data, 0, fbytes, s) == cudaSuccess ? QCD_OK : QCD_ERR_CUDA;
  if (st == QCD_OK) st = solve_one(c, w->b, xk, sp, nullptr, s);
  // y = D^-+ phi = g5 D^-1 g5 phi
  if (st == QCD_OK) st = blas_gamma5(c, (const double*)w->b.data, (double*)w->b.data, 0, s);
  if (st == QCD_OK) st = cudaMemsetAsync(yk.data, 0, fbytes, s) == cudaSuccess ? QCD_OK : QCD_ERR_CUDA;
  if (st == QCD_OK) st = solve_one(c, w->b, yk, sp, nullptr, s);
  if (st == QCD_OK) st = blas_gamma5(c, (const double*)yk.data, (double*)yk.data, 0, s);
  if (st == QCD_OK && dL_dtheta) st = force_apply(c, xk, yk, dL_dtheta, s);
  if (st == QCD_OK && x_out) st = export_spinor(c, xk, x_out, 1, s);
  if (st == QCD_OK && y_out) st = export_spinor(c, yk, y_out, 1, s);
  if (st == QCD_OK && dL_dphi) {
    // dL/dphi = x + y
    double one[2] = {1.0, 0.0};
    double* d_one = c->d_scalars + 64;
    if (cudaMemcpyAsync(d_one, one, sizeof(one), cudaMemcpyHostToDevice, s) != cudaSuccess) st = QCD_ERR_CUDA;
    const double* lst[1] = {(const double*)yk.data};
    if (st == QCD_OK) st = blas_multi_axpy(c, lst, 1, d_one, (double*)xk.data, s);
    if (st == QCD_OK) st = export_spinor(c, xk, dL_dphi, 1, s);
  }
  cudaStreamSynchronize(s);
  rec_free(xk);
  rec_free(yk);
  return st;
}

int qcd_field_create(qcd_ctx* c, int prec, qcd_field** out) { return qcd_field_create_n(c, prec, 1, out); }

int qcd_field_create_n(qcd_ctx* c, int prec, int nrhs, qcd_field** out) {
  if (!c || !out || prec < 0 || prec > 3 || nrhs < 1) return QCD_ERR_ARG;
  qcd_field* f = new (std::nothrow) qcd_field();
  if (!f) return QCD_ERR_NOMEM;
  f->ctx = c;
  f->nrhs = nrhs;
  int st = rec_alloc(f->rec, prec, 24, c->V * nrhs);
  if (st) {
    delete f;
    return st;
  }
  QCD_CUDA(cudaMemset(f->rec.data, 0, f->rec.bytes));
  *out = f;
  return QCD_OK;
}

void qcd_field_free(qcd_field* f) {
  if (!f) return;
  rec_free(f->rec);
  delete f;
}

int qcd_field_import(qcd_ctx* c, qcd_field* f, const double* in, void* stream) {
  if (!c || !f || !in || f->ctx != c) return QCD_ERR_ARG;
  return import_spinor(c, in, f->rec, f->nrhs, (cudaStream_t)stream);
}

int qcd_field_export(qcd_ctx* c, const qcd_field* f, double* out, void* stream) {
  if (!c || !f || !out || f->ctx != c) return QCD_ERR_ARG;
  return export_spinor(c, f->rec, out, f->nrhs, (cudaStream_t)stream);
}

int qcd_apply_D_field(qcd_ctx* c, const qcd_field* in, qcd_field* out, int dagger, void* stream) {
  if (!c || !in || !out || in->ctx != c || out->ctx != c || in == out || in->nrhs != out->nrhs) return QCD_ERR_ARG;
  if (!c->clover_built) return QCD_ERR_STATE;
  return dirac_apply(c, in->rec, out->rec, dagger, (cudaStream_t)stream, in->nrhs);
}

int qcd_sap_apply(qcd_ctx* c, const double* eta, double* psi, int ncy, int nmr, int sap_prec, void* stream) {
  if (!c || !eta || !psi || ncy < 1 || nmr < 0 || sap_prec < 0 || sap_prec > 3) return QCD_ERR_ARG;
  if (!c->clover_built) return QCD_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  Workspace* w = ensure_ws(c);
  if (!w) return QCD_ERR_NOMEM;
  for (Rec* f : {&w->b, &w->x})
    if (!f->data) QCD_TRY(rec_alloc(*f, P64, 24, c->V));
  QCD_TRY(import_spinor(c, eta, w->b, 1, s));
  QCD_CUDA(cudaMemsetAsync(c->d_scalars + 128, 0, sizeof(double), s));  // staging time-out flag
  QCD_TRY(sap_apply(c, w->sap, w->b, w->x, ncy, nmr, sap_prec, s));
  QCD_TRY(export_spinor(c, w->x, psi, 1, s));
  int timed_out = 0;
  QCD_CUDA(cudaMemcpyAsync(&timed_out, c->d_scalars + 128, sizeof(int), cudaMemcpyDeviceToHost, s));
  QCD_CUDA(cudaStreamSynchronize(s));
  return timed_out ? QCD_ERR_TIMEOUT : QCD_OK;
}

int qcd_sap_apply_n(qcd_ctx* c, const double* eta, double* psi, int nrhs, int rt, int ncy, int nmr, int sap_prec,
                    void* stream) {
  if (!c || !eta || !psi || nrhs < 1 || rt < 0 || ncy < 1 || nmr < 0 || sap_prec < 0 || sap_prec > 3)
    return QCD_ERR_ARG;
  if (!c->clover_built) return QCD_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  Rec a, b;
  SapWork w;
  int st = rec_alloc(a, P64, 24, c->V * nrhs);
  if (st == QCD_OK) st = rec_alloc(b, P64, 24, c->V * nrhs);
  if (st == QCD_OK) st = import_spinor(c, eta, a, nrhs, s);
  if (st == QCD_OK && cudaMemsetAsync(c->d_scalars + 128, 0, sizeof(double), s) != cudaSuccess) st = QCD_ERR_CUDA;
  Batch B;
  B.n = nrhs;
  if (st == QCD_OK) st = sap_apply(c, w, a, b, ncy, nmr, sap_prec, s, B, rt > nrhs ? nrhs : rt);
  if (st == QCD_OK) st = export_spinor(c, b, psi, nrhs, s);
  int timed_out = 0;
  if (st == QCD_OK && cudaMemcpyAsync(&timed_out, c->d_scalars + 128, sizeof(int), cudaMemcpyDeviceToHost, s) !=
                          cudaSuccess)
    st = QCD_ERR_CUDA;
  cudaStreamSynchronize(s);
  rec_free(a);
  rec_free(b);
  rec_free(w.rho);
  rec_free(w.psi);
  if (w.faces) cudaFree(w.faces);
  if (st == QCD_OK && timed_out) st = QCD_ERR_TIMEOUT;
  return st;
}

int qcd_set_launch(qcd_ctx* c, int prec, int threads, int tps) {
  if (!c || prec < 0 || prec > 4) return QCD_ERR_ARG;
  if (tps != 1 && tps != 2) return QCD_ERR_ARG;
  if (tps == 2 && prec != QCD_PREC_F16 && prec != QCD_PREC_BF16) return QCD_ERR_UNSUPPORTED;
  // the double-float operator is compiled for CTAs of at most 256 threads
  if (threads < 32 || threads > (prec == QCD_PREC_DF64 ? 256 : 1024) || threads % 32) return QCD_ERR_ARG;
  ++c->gen;  // captured graphs hold the launch shape
  c->dirac_threads[prec] = threads;
  c->dirac_tps[prec] = tps;
  return QCD_OK;
}

int qcd_get_launch(const qcd_ctx* c, int prec, int* threads, int* tps) {
  if (!c || prec < 0 || prec > 4) return QCD_ERR_ARG;
  if (threads) *threads = c->dirac_tps[prec] == 2 ? 256 : c->dirac_threads[prec];
  if (tps) *tps = c->dirac_tps[prec];
  return QCD_OK;
}

int qcd_set_sap_tile(qcd_ctx* c, int rt) {
  if (!c || rt < 0 || rt > 64) return QCD_ERR_ARG;
  ++c->gen;
  c->sap_rt = rt;
  return QCD_OK;
}

int qcd_get_sap_tile(qcd_ctx* c, int nrhs) {
  if (!c || nrhs < 1) return QCD_ERR_ARG;
  return sap_tile(c, nrhs);
}

int qcd_debug_set(qcd_ctx* c, int what, long long value) {
  if (!c) return QCD_ERR_ARG;
  ++c->gen;  // captured SAP launches hold the hook values
  switch (what) {
    case QCD_DEBUG_SAP_WAIT_CYCLES:
      if (value < 1 || value > (1ll << 31)) return QCD_ERR_ARG;
      c->dbg_sap_wait_cycles = value;
      return QCD_OK;
    case QCD_DEBUG_SAP_EXTRA_TX:
      if (value < 0 || value > 4096) return QCD_ERR_ARG;
      c->dbg_sap_extra_tx = (int)value;
      return QCD_OK;
    default:
      return QCD_ERR_ARG;
  }
}

int qcd_convert_check(const double* in64, const float* in32, float* out32, double* out64, long long n, void* stream) {
  if (n < 0 || (n > 0 && (!in64 || !in32 || !out32 || !out64))) return QCD_ERR_ARG;
  QCD_TRY(convert_check(in64, in32, out32, out64, n, (cudaStream_t)stream));
  return QCD_OK;
}

int qcd_profile_enable(qcd_ctx* c, int on) {
  if (!c) return QCD_ERR_ARG;
  c->prof = on != 0;
  return QCD_OK;
}

int qcd_profile_reset(qcd_ctx* c) {
  if (!c) return QCD_ERR_ARG;
  prof_collect(c);
  for (auto& t : c->timers) {
    t.launches = 0;
    t.total_ms = 0;
    t.bytes = t.flops = 0;
  }
  return QCD_OK;
}

int qcd_profile_get(qcd_ctx* c, int kernel, long long* launches, double* total_ms, double* bytes, double* flops) {
  if (!c || kernel < 0 || kernel >= QCD_KERNEL_COUNT) return QCD_ERR_ARG;
  prof_collect(c);
  const Timer& t = c->timers[kernel];
  if (launches) *launches = t.launches;
  if (total_ms) *total_ms = t.total_ms;
  if (bytes) *bytes = t.launches ? t.bytes / (double)t.launches : 0.0;  // averages over the launches
  if (flops) *flops = t.launches ? t.flops / (double)t.launches : 0.0;
  return QCD_OK;
}

}  // extern "C"

// Host-side internals of libqcdgb: the context, resident fields, launchers.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/qcdgb.h"
#include "qcd.cuh"

namespace qcd {

// record a CUDA error message for qcd_last_error and return QCD_ERR_CUDA
int cuda_fail(cudaError_t e, const char* where);

#define QCD_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

// every kernel launch is counted (qcd_launch_count) and checked
extern std::atomic<long long> g_launches;
#define QCD_LAUNCHED()                                  \
  do {                                                  \
    g_launches.fetch_add(1, std::memory_order_relaxed); \
    QCD_CUDA(cudaGetLastError());                       \
  } while (0)

#define QCD_TRY(call)          \
  do {                         \
    int st_ = (call);          \
    if (st_ != QCD_OK) return st_; \
  } while (0)

inline int chunks(int prec, int nreal) {
  int w = (prec == P64 || prec == PDF) ? 2 : (prec == P32 ? 4 : 8);
  return (nreal + w - 1) / w;
}

// a device field of N-real records per site in one precision
struct Rec {
  int prec = -1;
  int nreal = 0;
  void* data = nullptr;
  float* norm = nullptr;  // per-site scale for 16-bit storage
  size_t bytes = 0;       // data + norm
  FieldPtr ptr() const { return FieldPtr{data, norm}; }
};

struct Timer {  // CUDA-event timing of one kernel class
  long long launches = 0;
  double total_ms = 0;
  double bytes = 0, flops = 0;  // summed algorithmic bytes and flops of the timed launches
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
};

// SAP work fields: residual (SAP storage precision), accumulated solution
// (FP32, FP64 for the FP64 variant) and the face buffers
struct SapWork {
  Rec rho, psi;
  void* faces = nullptr;
  size_t faces_bytes = 0;
  int prec = -1;
  int nr = 1;  // right-hand sides (entry points that allocate b and x themselves use one) the fields hold (back to back)
};

// Right-hand sides of one launch, held back to back: the vector fields of RHS
// r start r field lengths after RHS 0's, its scalars ss doubles and its
// partial sums ps doubles after RHS 0's.  Kernels run a grid dimension over
// the right-hand sides; a masked-out RHS is skipped (its outputs keep their
// previous contents).
struct Batch {
  int n = 1;                  // right-hand sides
  long long ss = 0;           // doubles between consecutive RHS scalar blocks
  long long ps = 0;           // doubles between consecutive RHS partial-sum blocks
  const int* mask = nullptr;  // device flags: RHS r runs iff mask[r] != 0 (null: every RHS runs)
  const int* k = nullptr;     // device per-RHS vector counts (solution update, back substitution)
};

// What a captured FGCR iteration depends on beyond the workspace's own
// fields: every solver parameter the iteration's launches read, and the
// generation of the context's operator data (gauge copies, clover records,
// launch shapes, test hooks), which changes whenever those are reallocated or
// altered.  A captured graph is replayed only while its key is unchanged.
struct GraphKey {
  unsigned long long gen = ~0ull;
  int nkv = -1, precond = -1, ncy = -1, nmr = -1, sap_prec = -1, outer_prec = -1, nr = -1, rt = -1;
  bool operator==(const GraphKey& o) const {
    return gen == o.gen && nkv == o.nkv && precond == o.precond && ncy == o.ncy && nmr == o.nmr &&
           sap_prec == o.sap_prec && outer_prec == o.outer_prec && nr == o.nr && rt == o.rt;
  }
  bool operator!=(const GraphKey& o) const { return !(*this == o); }
};

// solver work fields of nr right-hand sides (FP64 internal layout unless
// stated; the fields of the nr right-hand sides back to back).  Every buffer a
// solve touches is allocated by ws_prepare, so the iteration itself never
// allocates (and can be captured in a CUDA graph).
struct Workspace {
  SapWork sap;
  int nkv = 0;
  int nr = 1;  // right-hand sides (entry points that allocate b and x themselves use one)
  Rec b, x, r, rho, tmp64;
  int rprec = P64;    // precision of rho and chi_k: P64, P32 (refinement scheme) or PDF (double-float)
  int pprec = P64;    // precision of phi_k: rprec, but P32 with the double-float recursion and SAP
  std::vector<Rec> phi, chi;
  // scalars of right-hand side q start q * ss doubles after these (right-hand side 0's)
  double* d_scal = nullptr;  // nr blocks of ss doubles holding the arrays below
  long long ss = 0;
  double* d_a1 = nullptr;  // [nkv][nkv] complex, first Gram-Schmidt pass
  double* d_a2 = nullptr;  // [nkv][nkv] complex, second pass
  double* d_cr = nullptr;  // [nkv][3]: |chi_k|^2, (chi_k, rho_k)
  double* d_rn = nullptr;  // [nkv + 8] residual norms
  double* d_gam = nullptr; // [nkv] complex
  double* d_gs = nullptr;  // [nkv][8] Gram-Schmidt norms and pass results
  double* d_part = nullptr;  // reduction partial sums, ps doubles per right-hand side
  long long ps = 0;
  double* h_pin = nullptr; // pinned host mirror for scalars read back: nr rows of nkv + 8
  int* d_mask = nullptr;   // per right-hand side: take part in the current launch (batched solves)
  int* h_mask = nullptr;   // pinned staging of the mask
  int* d_k = nullptr;      // per right-hand side: Krylov vectors of the finished cycle
  int* h_k = nullptr;      // pinned staging of those counts
  // FGMRES-DR: Arnoldi basis V (m + 1), preconditioned vectors Z (m), k + 1
  // spare fields for the deflated restart, pinned host copy of H's columns
  std::vector<Rec> drV, drZ, drT;
  // CG on the normal equations: r, p, t = D p, q = D^+ t; device scalars, pinned mirror
  std::vector<Rec> cgv;
  double* d_cg = nullptr;
  double* h_cg = nullptr;
  // device staging of lexicographic b and x when the caller passes host buffers
  double* stage = nullptr;
  size_t stage_bytes = 0;
  double* h_hcol = nullptr;
  double* d_hnorm = nullptr;
  // one captured CUDA graph per FGCR iteration index, valid while graph_key
  // equals the key of the current solve (parameters and context generation)
  std::vector<cudaGraphExec_t> graphs;
  std::vector<char> graph_warm;  // iteration k ran eagerly under graph_key (its kernels are loaded)
  GraphKey graph_key;
};
}  // namespace qcd

struct qcd_field {
  qcd_ctx* ctx;
  int nrhs = 1;  // fields back to back
  qcd::Rec rec;
};

struct qcd_ctx {
  qcd_params p;
  qcd::Geom g;  // host copy; r2y/j2r are device pointers
  int* d_tables = nullptr;
  long long V = 0;
  int nblk = 0;
  bool gauge_loaded = false, clover_built = false;
  // gauge field and clover in each storage precision (built lazily); index
  // PDF: the double-float copies of the df64 operator
  void* U[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  size_t U_bytes[5] = {0, 0, 0, 0, 0};
  qcd::Rec A[5];     // clover (4 + m0 + c_sw term), 72 reals per site
  qcd::Rec Ahat[5];  // SAP block clover: A on even sites, A^-1 on odd sites
  qcd::Workspace* ws = nullptr;
  qcd::Workspace* tile_ws = nullptr;       // right-hand sides solved together by batched launches
  std::vector<qcd::Workspace*> batch_ws;  // extra right-hand sides of a multi-RHS solve (one workspace each)
  std::vector<cudaStream_t> streams;      // one stream per right-hand side of a batch
  cudaStream_t copy_stream = nullptr;     // host transfers overlapped with the layout kernels
  cudaStream_t deliver_stream = nullptr;  // early delivery of solutions (Problem::dlv_lex)
  // instrumentation
  bool prof = false;
  qcd::Timer timers[QCD_KERNEL_COUNT];
  std::vector<cudaEvent_t> event_pool;
  // launch shape chosen by the autotuner
  int dirac_threads[5] = {256, 256, 256, 256, 256};  // CTA size of the operator kernel per precision
  int sap_rt = 0;  // right-hand sides per CTA of batched SAP launches (0: sap_tile's default)
  int dirac_tps[5] = {1, 1, 1, 1, 1};  // threads per site of the operator kernel (2: 16-bit storage only)
  double* d_scalars = nullptr;  // small device array for coefficients
  double* h_scalars = nullptr;  // pinned host mirror
  // test hooks (qcd_debug_set): budget of the SAP staging wait, and bytes its
  // barrier expects beyond the copies (a count that never arrives)
  long long dbg_sap_wait_cycles = 1ll << 31;
  int dbg_sap_extra_tx = 0;
  // bumped whenever device operator data or a launch setting that captured
  // graphs bake in changes (gauge load, clover build, lazily built copies,
  // autotuning, test hooks): graphs captured under another generation are
  // discarded instead of replayed
  unsigned long long gen = 0;
};

namespace qcd {

// ---- instrumentation (api.cu)
// NVTX range around a solver phase (header-only NVTX; a no-op unless a
// profiler is attached): the phases appear by name in the profiler's timeline
// and can select kernels for a capture
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

struct ProfScope {
  qcd_ctx* c;
  int k;
  cudaStream_t s;
  cudaEvent_t e1 = nullptr;
  ProfScope(qcd_ctx* ctx, int kernel, cudaStream_t st, double bytes, double flops);
  ~ProfScope();
};

// ---- memory helpers (api.cu)
int rec_alloc(Rec& r, int prec, int nreal, long long V);
void rec_free(Rec& r);
Workspace* ensure_ws(qcd_ctx* c);

// ---- layout.cu
int setup_geometry(qcd_ctx* c);
int import_spinor(qcd_ctx* c, const double* lex, const Rec& out, int nrhs, cudaStream_t s);
int export_spinor(qcd_ctx* c, const Rec& in, double* lex, int nrhs, cudaStream_t s);
// one lattice's field between host memory and the internal layout through a
// device staging field, copies and layout kernels overlapped slab by slab
int upload_spinor(qcd_ctx* c, const double* host, double* stage, const Rec& out, cudaStream_t s);
int download_spinor(qcd_ctx* c, const Rec& in, double* stage, double* host, cudaStream_t s);
int load_gauge_device(qcd_ctx* c, const double* lex_dev, cudaStream_t s);
int ensure_gauge(qcd_ctx* c, int prec, cudaStream_t s);
// convert records between precisions (same layout family)
int convert_rec(qcd_ctx* c, const Rec& in, const Rec& out, cudaStream_t s);
// out32 = FP32 of in64, out64 = FP64 of in32 through the integer-pipe conversions
int convert_check(const double* in64, const float* in32, float* out32, double* out64, long long n, cudaStream_t s);

// ---- clover.cu
int build_clover(qcd_ctx* c, cudaStream_t s);
int ensure_clover(qcd_ctx* c, int prec, cudaStream_t s);

// ---- dirac.cu
// out = D in (dagger: D^+); fields in one precision
// nrhs > 1: in/out hold nrhs fields back to back (V sites apart)
// mask (device, nrhs flags, may be null): right-hand sides whose flag is 0 are skipped
int dirac_apply(qcd_ctx* c, const Rec& in, const Rec& out, int dagger, cudaStream_t s, int nrhs = 1,
                const int* mask = nullptr);
// r = b - D x and |r|^2 (FP64), for each right-hand side of B (fields V sites apart)
int residual64(qcd_ctx* c, double* part, const Rec& b, const Rec& x, const Rec& r, double* d_norm2, cudaStream_t s,
               const Batch& B = Batch());
// the same residual with D x in double-float arithmetic (x split into tmp, a
// double-float field of B.n right-hand sides, unless presplit says tmp holds
// the split already); the FGCR restart of the double-float recursion
int residual_df(qcd_ctx* c, double* part, const Rec& b, const Rec& x, const Rec& r, const Rec& tmp, double* d_norm2,
                cudaStream_t s, const Batch& B = Batch(),
                bool presplit = false);
// even/odd split (FP64): on the sites of parity par,
//   pre = 1: out = c1 M x + c2 H y;  pre = 0: out = M (c1 x + c2 H y),
// H the hopping term of D (of D^+ with dagger) from the other parity, M the
// block clover Ahat (A_ee / A_oo^-1) if use_m, else 1
int eo_apply(qcd_ctx* c, const Rec& x, const Rec& y, const Rec& out, int par, int dagger, int pre, int use_m,
             double c1, double c2, cudaStream_t s);
// out_e = Dhat x_e (dagger: Dhat^+ x_e), Dhat = A_ee - H_eo A_oo^-1 H_oe; tmp: odd-site scratch
int schur_apply(qcd_ctx* c, const Rec& x, const Rec& tmp, const Rec& out, int dagger, cudaStream_t s);

// ---- sap.cu
// work fields for nr right-hand sides (back to back)
int sap_prepare(qcd_ctx* c, SapWork& w, int prec, cudaStream_t s, int nr = 1);
// right-hand sides per CTA of a SAP launch over nr of them
int sap_tile(qcd_ctx* c, int nr);
// psi = M_SAP eta for each right-hand side of B; rt right-hand sides per CTA
// share one staging of the block's links and clover (rt < 1: sap_tile)
int sap_apply(qcd_ctx* c, SapWork& w, const Rec& eta64, const Rec& psi64, int ncy, int nmr, int prec, cudaStream_t s,
              const Batch& B = Batch(), int rt = 0);

// ---- blas.cu: fields of 24 reals per site, R = double (FP64 layout) or
// float (FP32 layout, the recursion of the mixed-precision scheme).
// Gram-Schmidt building blocks.  cond (optional) = {|chi|^2, |chi'|^2}: the
// call is skipped unless |chi'|^2 < |chi|^2 / 2 (second pass, DGKS criterion).
// d_out[j] = (v_j, w) for j < k (complex); d_norm (optional) = |w|^2
template <typename R>
int blas_multidot(qcd_ctx* c, double* part, const R* const* v, int k, const R* w, double* d_out, cudaStream_t s,
                  const double* cond = nullptr, double* d_norm = nullptr, const Batch& B = Batch());
// w -= sum_j coef[j] v_j (coef on device, complex); then d_out[j] = (v_j, w) for j < k
template <typename R>
int blas_axpy_dot(qcd_ctx* c, double* part, const R* const* v, int k, const double* d_coef, R* w, double* d_out,
                  cudaStream_t s, const Batch& B = Batch());
// w -= sum_j coef[j] v_j; d_out = {|w|^2, (w, rho)}
template <typename R>
int blas_axpy_norm_dot(qcd_ctx* c, double* part, const R* const* v, int k, const double* d_coef, R* w, const R* rho,
                       double* d_out, cudaStream_t s, const double* cond = nullptr, const Batch& B = Batch());
// gs = {|chi|^2, pass-1 {|chi'|^2, (chi', rho)}, pass-2 {...}}: picks the final
// coefficients into cr, chi /= |chi|, rho -= (chi, rho) chi, d_out = |rho|^2
template <typename R>
int blas_normalise_update(qcd_ctx* c, double* part, R* chi, R* rho, const double* d_gs, int two_pass, double* d_cr,
                          double* d_out, cudaStream_t s, const Batch& B = Batch());
// x += sum_j gamma_j phi_j (gamma on device)
template <typename R>
int blas_multi_axpy(qcd_ctx* c, const R* const* phi, int k, const double* d_gamma, R* x, cudaStream_t s,
                    const Batch& B = Batch());
// iterative refinement: x64 += sqrt(*d_rn2) sum_j gamma_j phi_j (FP32 phi_j)
int blas_refine_update(qcd_ctx* c, const float* const* phi, int k, const double* d_gamma, const double* d_rn2,
                       double* x, cudaStream_t s, const Batch& B = Batch());
// out32 = r64 / sqrt(*d_rn2)
int blas_demote_normalised(qcd_ctx* c, const double* r, const double* d_rn2, float* out, cudaStream_t s,
                           const Batch& B = Batch());
// x /= |x| (FP64) with |x|^2 from the Gram-Schmidt results (pass 2 when it
// ran); *d_hnorm = |x| before the scaling
int blas_gs_normalise(qcd_ctx* c, double* x, const double* d_gs, int two_pass, double* d_hnorm, cudaStream_t s);
// CG on the normal equations (FP64): x += a p, r -= a q with a = *d_rr / *d_tt,
// *d_rr_new = |r|^2; and p = r + (*d_rr_new / *d_rr) p
int blas_cg_update(qcd_ctx* c, double* part, double* x, double* r, const double* p, const double* q,
                   const double* d_rr, const double* d_tt, double* d_rr_new, cudaStream_t s);
int blas_cg_direction(qcd_ctx* c, double* p, const double* r, const double* d_rr_new, const double* d_rr,
                      cudaStream_t s);
// the double-float recursion (Prec PDF): the same Gram-Schmidt building blocks
// on fields of float4 (re hi, re lo, im hi, im lo), V * 12 per right-hand side
int blas_df_multidot(qcd_ctx* c, double* part, const float4* const* v, int k, const float4* w, double* d_out,
                     cudaStream_t s, const double* cond, double* d_norm, const Batch& B = Batch());
int blas_df_axpy_norm_dot(qcd_ctx* c, double* part, const float4* const* v, int k, const double* d_coef, float4* w,
                          const float4* rho, double* d_out, cudaStream_t s, const double* cond,
                          const Batch& B = Batch());
int blas_df_normalise_update(qcd_ctx* c, double* part, float4* chi, float4* rho, const double* d_gs, int two_pass,
                             double* d_cr, double* d_out, cudaStream_t s, const Batch& B = Batch());
// x (FP64) += sum_j gamma_j phi_j for double-float phi_j (B.k: per-RHS counts)
int blas_df_update(qcd_ctx* c, const float4* const* phi, int k, const double* d_gamma, double* x, cudaStream_t s,
                   const Batch& B = Batch());
// the same with FP32 phi_j (FP32-exact fields: the SAP outputs of the
// double-float recursion), read at half the bytes
int blas_df_update32(qcd_ctx* c, const float4* const* phi, int k, const double* d_gamma, double* x, cudaStream_t s,
                     const Batch& B = Batch(), float* xs = nullptr);
// FP64 field <-> double-float field (same internal layout)
int blas_df_split(qcd_ctx* c, const double* in, float* out, cudaStream_t s, const Batch& B = Batch());
int blas_df_join(qcd_ctx* c, const float* in, double* out, cudaStream_t s, const Batch& B = Batch());
// norm2
template <typename R>
int blas_norm2(qcd_ctx* c, double* part, const R* v, double* d_out, cudaStream_t s, const Batch& B = Batch());
// y = g5 x (in place allowed)
int blas_gamma5(qcd_ctx* c, const double* x, double* y, int nsites_layout, cudaStream_t s);
// small dense solve of the FGCR triangular system on the device
int fgcr_backsub(const double* d_a1, const double* d_a2, const double* d_cr, int k, int ld, double* d_gamma,
                 cudaStream_t s, const Batch& B = Batch());
// out[j] = sum_p partials[p * stride + j], j < m (fixed order)
int reduce_partials(const double* partials, int nparts, int stride, int m, double* out, cudaStream_t s,
                    const Batch& B = Batch());

// ---- solver.cu
size_t partials_for(long long V);
// allocate the solver fields and scalars of nr right-hand sides (a change of
// nr reallocates everything)
int ws_prepare(qcd_ctx* c, Workspace& w, const qcd_solver_params& sp, cudaStream_t s, int nr = 1);
void ws_release(Workspace& w);
// the launch descriptor of a workspace's right-hand sides
Batch batch_of(const Workspace& w, const int* mask);
// one right-hand side of one lattice, solved in lock step with the others
struct Problem {
  qcd_ctx* c = nullptr;
  Workspace* w = nullptr;
  cudaStream_t s = nullptr;
  Rec b, x;  // FP64 internal fields (b is read, x holds the guess / solution)
  qcd_solve_info info{};
  // state of the solver loop
  double bn = 0, rn = 0;
  int kused = 0, slow = 0;
  bool active = true, cycle_done = false;
  int status = QCD_OK;
  // early delivery of the solution to the caller's lexicographic field (set
  // up by the API): after every restart update of x the field is exported on
  // the context's delivery stream -- through dlv_stage when dlv_lex is host
  // memory -- while the solver goes on to the residual; `delivered` says the
  // last delivery followed the last change of x, dlv_event marks its end
  double* dlv_lex = nullptr;
  double* dlv_stage = nullptr;
  bool delivered = false;
  cudaEvent_t dlv_event = nullptr;
};
// deliver p.x to p.dlv_lex now (ordered after s's work), off the solver's stream
int deliver_solution(Problem& p, cudaStream_t s);
// right-hand sides of one lattice that share a workspace and are iterated by
// the same launches (each kernel of an FGCR iteration runs over all of them);
// rhs[q]->b / ->x view right-hand side q of the workspace's fields
struct Group {
  qcd_ctx* c = nullptr;
  Workspace* w = nullptr;
  cudaStream_t s = nullptr;
  std::vector<Problem*> rhs;
  int rt = 1;  // right-hand sides per CTA of the SAP launches
  int nr() const { return (int)rhs.size(); }
};
// a view of right-hand side q of a workspace field
Rec rhs_view(const Rec& f, int q, long long V);
// FGCR (Sec. 4) on all groups in lock step: each iteration is enqueued for
// every group on its own stream (replayed from a CUDA graph when use_graphs),
// then one host synchronisation checks every residual.
int fgcr_groups(std::vector<Group>& groups, const qcd_solver_params& sp, bool use_graphs);
// FGCR on single-right-hand-side problems (one group each)
int fgcr_batch(std::vector<Problem>& probs, const qcd_solver_params& sp, bool use_graphs);
// FGMRES with deflated restarts (Sec. 4), FP64 recursion; problems one after another
int fgmres_dr_batch(std::vector<Problem>& probs, const qcd_solver_params& sp);
void dr_release(Workspace& w);
// CG on the normal equations (FP64), problems one after another; with
// fallback_only, only problems whose status is QCD_STAGNATED or
// QCD_NOT_CONVERGED run, from their current x
int cg_batch(std::vector<Problem>& probs, const qcd_solver_params& sp, bool fallback_only);
// dispatch on sp.solver (FGCR, FGMRES-DR, CG, even/odd CG) plus the CG fallback
int run_solver(std::vector<Problem>& probs, const qcd_solver_params& sp, bool use_graphs);
void cg_release(Workspace& w);
int solve_one(qcd_ctx* c, const Rec& b, const Rec& x, const qcd_solver_params& sp, qcd_solve_info* info,
              cudaStream_t s);
void workspace_free(qcd_ctx* c);

// ---- force.cu
int force_apply(qcd_ctx* c, const Rec& x, const Rec& y, double* F, cudaStream_t s);

}  // namespace qcd

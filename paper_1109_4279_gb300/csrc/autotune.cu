// Launch-shape and block-shape tuning by measurement.
//
// qcd_autotune: the operator kernel's CTA size per storage precision and, for
// 16-bit storage, one or two threads per site; for several right-hand sides
// the number of them one CTA of the SAP sweep solves per staging of its
// block.  Timed with CUDA events on resident fields, cached in a small JSON
// file.
// qcd_tune_block: the Schwarz block shape (Sec. 4/5), chosen by timing whole
// solves, since the shape changes both the kernel speed and the iteration
// count.
#include <cstdio>
#include <cstring>
#include <array>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "internal.h"

namespace qcd {

static std::string tune_key(qcd_ctx* c, int nrhs) {
  cudaDeviceProp prop;
  int dev = 0;
  cudaGetDevice(&dev);
  std::string name = "gpu";
  if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
  for (auto& ch : name)
    if (ch == '"' || ch == '\\') ch = '_';
  std::ostringstream k;
  k << name << "|" << c->p.dims[0] << "x" << c->p.dims[1] << "x" << c->p.dims[2] << "x" << c->p.dims[3] << "|b"
    << c->p.block[0] << "x" << c->p.block[1] << "x" << c->p.block[2] << "x" << c->p.block[3] << "|nrhs" << nrhs;
  return k.str();
}

// The cache holds one entry per line:
//   "key": [t64, t32, t16, tb16, tdf, tps16, tpsb16, sap_rt],
// the operator's CTA size per precision (double-float last), the threads per
// site of the 16-bit operators and the SAP right-hand-side tile (0: default)
static constexpr int kTuneFields = 8;

static bool tune_valid(const int v[kTuneFields]) {
  for (int i = 0; i < 4; ++i)
    if (v[i] != 128 && v[i] != 256 && v[i] != 512) return false;
  if (v[4] != 128 && v[4] != 256) return false;
  return (v[5] == 1 || v[5] == 2) && (v[6] == 1 || v[6] == 2) && v[7] >= 0 && v[7] <= 64;
}

static bool cache_lookup(const char* path, const std::string& key, int out[kTuneFields]) {
  if (!path) return false;
  std::ifstream f(path);
  std::string line;
  const std::string tag = "\"" + key + "\":";
  while (std::getline(f, line)) {
    const size_t p = line.find(tag);
    if (p == std::string::npos) continue;
    const size_t lb = line.find('[', p), rb = line.find(']', p);
    if (lb == std::string::npos || rb == std::string::npos) return false;
    int v[kTuneFields];
    if (sscanf(line.c_str() + lb + 1, "%d , %d , %d , %d , %d , %d , %d , %d", &v[0], &v[1], &v[2], &v[3], &v[4],
               &v[5], &v[6], &v[7]) != kTuneFields)
      return false;
    if (!tune_valid(v)) return false;
    for (int i = 0; i < kTuneFields; ++i) out[i] = v[i];
    return true;
  }
  return false;
}

static void cache_store(const char* path, const std::string& key, const int v[kTuneFields]) {
  if (!path) return;
  std::vector<std::string> entries;
  {
    std::ifstream f(path);
    std::string line;
    const std::string tag = "\"" + key + "\":";
    while (std::getline(f, line)) {
      if (line.find("\":") == std::string::npos || line.find(tag) != std::string::npos) continue;
      while (!line.empty() && (line.back() == ',' || line.back() == ' ')) line.pop_back();
      entries.push_back(line);
    }
  }
  std::ostringstream e;
  e << "  \"" << key << "\": [";
  for (int i = 0; i < kTuneFields; ++i) e << v[i] << (i + 1 < kTuneFields ? ", " : "]");
  entries.push_back(e.str());
  std::ofstream f(path, std::ios::trunc);
  f << "{\n";
  for (size_t i = 0; i < entries.size(); ++i) f << entries[i] << (i + 1 < entries.size() ? ",\n" : "\n");
  f << "}\n";
}

static void tune_apply(qcd_ctx* c, const int v[kTuneFields]) {
  for (int p = 0; p < 5; ++p) c->dirac_threads[p] = v[p];
  c->dirac_tps[P64] = c->dirac_tps[P32] = c->dirac_tps[PDF] = 1;
  c->dirac_tps[P16] = v[5];
  c->dirac_tps[PB16] = v[6];
  c->sap_rt = v[7];
}

// mean ms of reps calls of f() after one warm-up, CUDA events on s
template <typename F>
static float time_ms(cudaStream_t s, int reps, F f, int* st) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  *st = f();
  cudaEventRecord(e0, s);
  for (int it = 0; it < reps && *st == QCD_OK; ++it) *st = f();
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms / reps;
}

}  // namespace qcd

using namespace qcd;

extern "C" int qcd_autotune(qcd_ctx* c, int nrhs, const char* cache_path) {
  if (!c || nrhs < 1) return QCD_ERR_ARG;
  if (!c->clover_built) return QCD_ERR_STATE;
  const std::string key = tune_key(c, nrhs);
  int best[kTuneFields] = {256, 256, 256, 256, 256, 1, 1, 0};
  ++c->gen;  // the operator's launch shape changes under captured graphs
  if (cache_lookup(cache_path, key, best)) {
    tune_apply(c, best);
    return QCD_OK;
  }
  cudaStream_t s = nullptr;
  QCD_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  const bool prof = c->prof;
  c->prof = false;
  int st = QCD_OK;
  // operator: CTA size with one thread per site, for 16-bit storage also the
  // two-threads-per-site form
  const int cand[4][2] = {{128, 1}, {256, 1}, {512, 1}, {256, 2}};
  for (int p = P64; p <= PDF && st == QCD_OK; ++p) {
    Rec a, b;
    st = rec_alloc(a, p, 24, c->V * nrhs);
    if (st == QCD_OK) st = rec_alloc(b, p, 24, c->V * nrhs);
    if (st == QCD_OK && cudaMemsetAsync(a.data, 0, a.bytes, s) != cudaSuccess) st = QCD_ERR_CUDA;
    float best_ms = 1e30f;
    const int ncand = (p == P16 || p == PB16) ? 4 : (p == PDF ? 2 : 3);
    for (int k = 0; k < ncand && st == QCD_OK; ++k) {
      c->dirac_threads[p] = cand[k][0];
      c->dirac_tps[p] = cand[k][1];
      const float ms = time_ms(s, 5, [&] { return dirac_apply(c, a, b, 0, s, nrhs); }, &st);
      if (st == QCD_OK && ms < best_ms) {
        best_ms = ms;
        best[p] = cand[k][0];
        if (p == P16 || p == PB16) best[5 + (p - P16)] = cand[k][1];
      }
    }
    c->dirac_threads[p] = best[p];
    c->dirac_tps[p] = (p == P16 || p == PB16) ? best[5 + (p - P16)] : 1;
    rec_free(a);
    rec_free(b);
  }
  // SAP right-hand-side tile: FP16 block fields, 4 cycles of 4 MR steps
  if (st == QCD_OK && nrhs > 1) {
    SapWork w;
    Rec eta, psi;
    int s2 = sap_prepare(c, w, P16, s, nrhs);
    if (s2 == QCD_OK) s2 = rec_alloc(eta, P64, 24, c->V * nrhs);
    if (s2 == QCD_OK) s2 = rec_alloc(psi, P64, 24, c->V * nrhs);
    if (s2 == QCD_OK && cudaMemsetAsync(eta.data, 0, eta.bytes, s) != cudaSuccess) s2 = QCD_ERR_CUDA;
    if (s2 == QCD_OK) {
      Batch B;
      B.n = nrhs;
      float best_ms = 1e30f;
      const int rts[8] = {1, 2, 3, 4, 6, 8, 12, 16};
      for (int k = 0; k < 8 && rts[k] <= nrhs && s2 == QCD_OK; ++k) {
        const float ms = time_ms(s, 2, [&] { return sap_apply(c, w, eta, psi, 4, 4, P16, s, B, rts[k]); }, &s2);
        if (s2 == QCD_OK && ms < best_ms) {
          best_ms = ms;
          best[7] = rts[k];
        }
      }
    }
    // a SAP that does not fit this block shape leaves the default tile
    cudaStreamSynchronize(s);
    rec_free(eta);
    rec_free(psi);
    rec_free(w.rho);
    rec_free(w.psi);
    if (w.faces) cudaFree(w.faces);
    cudaGetLastError();
  }
  c->sap_rt = best[7];
  c->prof = prof;
  cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  if (st == QCD_OK) cache_store(cache_path, key, best);
  return st;
}

extern "C" int qcd_tune_block(const qcd_params* p, const double* U, const double* b, int is_device,
                              const qcd_solver_params* sp, const int* candidates, int n, int out_block[4],
                              double* times_ms) {
  if (!p || !U || !b || !out_block) return QCD_ERR_ARG;
  std::vector<std::array<int, 4>> cands;
  if (candidates) {
    if (n < 1) return QCD_ERR_ARG;
    for (int i = 0; i < n; ++i) cands.push_back({candidates[4 * i], candidates[4 * i + 1], candidates[4 * i + 2],
                                                 candidates[4 * i + 3]});
  } else {
    // even extents from {2, 4, 6, 8}, an even block count per direction,
    // 64 .. 512 sites per block (the SAP kernel's range)
    const int ext[4] = {2, 4, 6, 8};
    for (int a0 : ext)
      for (int a1 : ext)
        for (int a2 : ext)
          for (int a3 : ext) {
            const int bb[4] = {a0, a1, a2, a3};
            bool ok = true;
            int vb = 1;
            for (int mu = 0; mu < 4; ++mu) {
              if (p->dims[mu] % bb[mu] || (p->dims[mu] / bb[mu]) % 2) ok = false;
              vb *= bb[mu];
            }
            if (ok && vb >= 64 && vb <= 512 && (int)cands.size() < 64) cands.push_back({a0, a1, a2, a3});
          }
    if (cands.empty()) return QCD_ERR_GEOMETRY;
  }
  qcd_solver_params spl;
  if (sp) spl = *sp; else qcd_solver_defaults(&spl);
  const long long V = (long long)p->dims[0] * p->dims[1] * p->dims[2] * p->dims[3];
  const size_t fbytes = (size_t)V * 24 * sizeof(double);
  double* dx = nullptr;
  double* db = nullptr;
  double* dU = nullptr;
  int st = QCD_OK;
  if (cudaMalloc(&dx, fbytes) != cudaSuccess) st = QCD_ERR_NOMEM;
  if (st == QCD_OK && !is_device) {
    if (cudaMalloc(&db, fbytes) != cudaSuccess || cudaMalloc(&dU, (size_t)V * 4 * 9 * 16) != cudaSuccess)
      st = QCD_ERR_NOMEM;
    if (st == QCD_OK) {
      cudaMemcpy(db, b, fbytes, cudaMemcpyHostToDevice);
      cudaMemcpy(dU, U, (size_t)V * 4 * 9 * 16, cudaMemcpyHostToDevice);
    }
  }
  const double* Ub = is_device ? U : dU;
  const double* bb = is_device ? b : db;
  double best = 1e300;
  int tried = 0;
  for (size_t i = 0; i < cands.size() && st == QCD_OK; ++i) {
    qcd_params q = *p;
    for (int mu = 0; mu < 4; ++mu) q.block[mu] = cands[i][mu];
    qcd_ctx* c = nullptr;
    double t = -1;
    if (qcd_create(&c, &q) == QCD_OK && qcd_load_gauge(c, Ub, 1, nullptr) == QCD_OK &&
        qcd_build_clover(c, nullptr) == QCD_OK) {
      qcd_solve_info info;
      cudaMemset(dx, 0, fbytes);
      // first solve warms up (allocations, graphs); the second is timed
      if (qcd_solve(c, bb, dx, 1, &spl, &info, nullptr) == QCD_OK) {
        cudaMemset(dx, 0, fbytes);
        if (qcd_solve(c, bb, dx, 1, &spl, &info, nullptr) == QCD_OK) t = info.time_ms;
      }
    }
    if (c) qcd_destroy(c);
    cudaGetLastError();
    if (times_ms) times_ms[i] = t;
    ++tried;
    if (t > 0 && t < best) {
      best = t;
      for (int mu = 0; mu < 4; ++mu) out_block[mu] = cands[i][mu];
    }
  }
  if (dx) cudaFree(dx);
  if (db) cudaFree(db);
  if (dU) cudaFree(dU);
  if (st != QCD_OK) return st;
  return best < 1e300 ? tried : QCD_NOT_CONVERGED;
}

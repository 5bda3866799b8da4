// Launch-shape and block-shape tuning by measurement.
//
// qcd_autotune: CTA size of the operator kernel per storage precision, timed
// with CUDA events on resident fields, cached in a small JSON file.
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

// The cache holds one entry per line:  "key": [t64, t32, t16, tb16],
static bool cache_lookup(const char* path, const std::string& key, int out[4]) {
  if (!path) return false;
  std::ifstream f(path);
  std::string line;
  const std::string tag = "\"" + key + "\":";
  while (std::getline(f, line)) {
    const size_t p = line.find(tag);
    if (p == std::string::npos) continue;
    const size_t lb = line.find('[', p), rb = line.find(']', p);
    if (lb == std::string::npos || rb == std::string::npos) return false;
    int v[4];
    if (sscanf(line.c_str() + lb + 1, "%d , %d , %d , %d", &v[0], &v[1], &v[2], &v[3]) != 4) return false;
    for (int i = 0; i < 4; ++i) {
      if (v[i] != 128 && v[i] != 256 && v[i] != 512) return false;
      out[i] = v[i];
    }
    return true;
  }
  return false;
}

static void cache_store(const char* path, const std::string& key, const int v[4]) {
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
  e << "  \"" << key << "\": [" << v[0] << ", " << v[1] << ", " << v[2] << ", " << v[3] << "]";
  entries.push_back(e.str());
  std::ofstream f(path, std::ios::trunc);
  f << "{\n";
  for (size_t i = 0; i < entries.size(); ++i) f << entries[i] << (i + 1 < entries.size() ? ",\n" : "\n");
  f << "}\n";
}

}  // namespace qcd

using namespace qcd;

extern "C" int qcd_autotune(qcd_ctx* c, int nrhs, const char* cache_path) {
  if (!c || nrhs < 1) return QCD_ERR_ARG;
  if (!c->clover_built) return QCD_ERR_STATE;
  const std::string key = tune_key(c, nrhs);
  int best[4] = {256, 256, 256, 256};
  ++c->gen;  // the operator's launch shape changes under captured graphs
  if (cache_lookup(cache_path, key, best)) {
    for (int p = 0; p < 4; ++p) c->dirac_threads[p] = best[p];
    return QCD_OK;
  }
  cudaStream_t s = nullptr;
  QCD_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const bool prof = c->prof;
  c->prof = false;
  int st = QCD_OK;
  const int cand[3] = {128, 256, 512};
  for (int p = P64; p <= PB16 && st == QCD_OK; ++p) {
    Rec a, b;
    st = rec_alloc(a, p, 24, c->V * nrhs);
    if (st == QCD_OK) st = rec_alloc(b, p, 24, c->V * nrhs);
    if (st == QCD_OK && cudaMemsetAsync(a.data, 0, a.bytes, s) != cudaSuccess) st = QCD_ERR_CUDA;
    float best_ms = 1e30f;
    for (int k = 0; k < 3 && st == QCD_OK; ++k) {
      c->dirac_threads[p] = cand[k];
      st = dirac_apply(c, a, b, 0, s, nrhs);  // warm-up (also builds this precision's fields)
      cudaEventRecord(e0, s);
      for (int it = 0; it < 5 && st == QCD_OK; ++it) st = dirac_apply(c, a, b, 0, s, nrhs);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) {
        best_ms = ms;
        best[p] = cand[k];
      }
    }
    c->dirac_threads[p] = best[p];
    rec_free(a);
    rec_free(b);
  }
  c->prof = prof;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
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

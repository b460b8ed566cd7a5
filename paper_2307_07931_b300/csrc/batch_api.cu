// C ABI of the batched persistent relaxation: plan (size classes, autotuning,
// schedule, CUDA graph) and run. The kernel is in batch.cu.
#include "px_internal.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <sstream>
#include <string>
#include <vector>

namespace {

struct ClassCfg {
  int mode = px::MODE_BANDED;
  int ry = 8;
  int tb = 1;                // sweeps per cluster barrier (MODE_BANDED_T)
  double rate_per_sm = 0.0;  // measured cell updates / s per SM (0 = not measured)
  bool tuned = false;
};

std::string class_key(int dtype, int nx, int ny, int csize) {
  char b[64];
  snprintf(b, sizeof b, "%s:%dx%d@c%d", dtype == PX_F64 ? "f64" : "f32", nx, ny, csize);
  return b;
}

bool fits_whole(int nx, int ny, int dtype, size_t cap = 0) {
  return px::whole_bytes(nx, ny, dtype) <= (cap ? cap : px::batch_whole_smem());
}

// Shared bytes of a configured class.
size_t cfg_smem(const ClassCfg& k, int nx, int ny, int dtype) {
  if (k.mode == px::MODE_WHOLE) return px::whole_bytes(nx, ny, dtype);
  if (k.mode == px::MODE_BANDED_T) return px::banded_t_smem(dtype, k.tb);
  return 0;
}

// Mixed-precision plans: the FP64 and the FP32 instances run as two launches
// side by side, one CTA of each on every SM, so that the FP64-pipe-bound
// sweeps and the memory-bound FP32 sweeps overlap on the same SMs. A CTA of
// such a plan uses at most this much shared memory (two must fit an SM);
// classes whose fastest mode needs more are tuned again under the cap (key
// suffix "s").
constexpr size_t kCoSmem = 100 * 1024;
// Measured on B300 (1024-instance workload, 300 sweeps): FP64 launch alone
// 231.5 ms, FP32 launch alone 66.9 ms, side by side 244.0 ms, so the shorter
// launch adds about a fifth of its own time to the longer one.
constexpr double kCoOverlap = 0.2;

// Default rates per SM (cell updates / s) when a class was not measured: FP64
// is bound by the FP64 pipe (about 0.555e12 DFMA/s over 148 SMs, 6 per
// update); FP32 by shared memory (WHOLE) or L2 bandwidth (BANDED).
double default_rate(int dtype, int mode) {
  if (dtype == PX_F64) return 0.6e9;
  return mode == px::MODE_WHOLE ? 8e9 : 6e9;
}

std::string gpu_name(int dev) {
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
  return p.name;
}

// Tune cache: one JSON object, {"gpu": "...", "classes": {"f32:96x96@c2": {"mode": 0,
// "ry": 8, "tb": 1, "rate_per_sm": 1.2e10}, ...}}. Written and read only by this file.
void load_cache(const char* path, const std::string& gpu, std::map<std::string, ClassCfg>& out) {
  if (!path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  std::string s;
  char buf[4096];
  size_t n;
  while ((n = fread(buf, 1, sizeof buf, f)) > 0) s.append(buf, n);
  fclose(f);
  const std::string gk = "\"gpu\": \"" + gpu + "\"";
  if (s.find(gk) == std::string::npos) return;  // another GPU: ignore
  size_t pos = 0;
  while ((pos = s.find("\"f", pos)) != std::string::npos) {
    const size_t q = s.find('"', pos + 1);
    if (q == std::string::npos) break;
    const std::string key = s.substr(pos + 1, q - pos - 1);
    int mode = 0, ry = 0, tb = 0;
    double rate = 0;
    if (sscanf(s.c_str() + q + 1, ": {\"mode\": %d, \"ry\": %d, \"tb\": %d, \"rate_per_sm\": %lf}",
               &mode, &ry, &tb, &rate) == 4 && key.find(':') != std::string::npos &&
        mode >= px::MODE_WHOLE && mode <= px::MODE_BANDED_T && tb >= 1 && tb <= 8 &&
        (mode != px::MODE_BANDED_T || px::banded_t_ok(key[1] == '3' ? PX_F32 : PX_F64, tb))) {
      ClassCfg c;
      c.mode = mode;
      c.ry = ry;
      c.tb = tb;
      c.rate_per_sm = rate;
      c.tuned = true;
      out[key] = c;
    }
    pos = q + 1;
  }
}

void save_cache(const char* path, const std::string& gpu, const std::map<std::string, ClassCfg>& m) {
  if (!path) return;
  std::string tmp = std::string(path) + ".tmp";
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) return;
  fprintf(f, "{\"gpu\": \"%s\", \"classes\": {", gpu.c_str());
  bool first = true;
  for (const auto& kv : m) {
    if (!kv.second.tuned) continue;
    fprintf(f, "%s\n  \"%s\": {\"mode\": %d, \"ry\": %d, \"tb\": %d, \"rate_per_sm\": %.6e}",
            first ? "" : ",", kv.first.c_str(), kv.second.mode, kv.second.ry, kv.second.tb,
            kv.second.rate_per_sm);
    first = false;
  }
  fprintf(f, "\n}}\n");
  fclose(f);
  rename(tmp.c_str(), path);
}

}  // namespace

struct px_batch {
  px_ctx* ctx = nullptr;
  int n = 0, nsweeps = 0, every = 0, nrep = 0;
  double omega = 0;
  std::vector<px_grid> grids;
  std::vector<px::BInst> inst;       // host copy; pointers filled per run
  px::BInst* inst_dev = nullptr;
  px::BInst* inst_pinned = nullptr;
  int* idx_dev = nullptr;            // cl_off | cl_items | cta_off | cta_items
  void* scratch = nullptr;
  int nclusters = 0;
  size_t smem = 0;
  px::BParams params{};
  // a mixed-precision plan runs FP32 instances in a second launch beside the
  // FP64 one (params2, nclusters2, smem2); nclusters2 == 0 otherwise
  px::BParams params2{};
  int nclusters2 = 0;
  size_t smem2 = 0;
  cudaStream_t cap_stream = nullptr;
  cudaStream_t cap_stream2 = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::string desc;
};

namespace {

// Measures one class: every candidate (WHOLE in one CTA; BANDED with rows per
// task 4, 8, 16; for FP32 BANDED_T with 4 or 8 sweeps per barrier) runs on
// `copies` zero instances at once, one per cluster (or CTA for WHOLE), so the
// rate includes the memory traffic of a full device: a single instance alone
// stays in L2 and would make streaming modes look faster than they run in
// the batch. Keeps the fastest rate per SM.
px_status tune_class(px_ctx* c, int dtype, int nx, int ny, int sweeps, double omega, int C,
                     int clusters, size_t smem_cap, ClassCfg* out) {
  const int64_t ld = nx;
  const size_t es = dtype == PX_F64 ? 8 : 4;
  const size_t fb = ((size_t)ld * ny * es + 255) / 256 * 256;
  // concurrent copies: every cluster, within 4 GiB of fields
  const int copies = (int)std::max<int64_t>(1, std::min<int64_t>(clusters, ((int64_t)4 << 30) / (int64_t)(4 * fb)));
  void *mem = nullptr, *idx = nullptr, *ins = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  px_status st = PX_OK;
  struct Cand { int mode, ry, tb; };
  std::vector<Cand> cands;
  if (fits_whole(nx, ny, dtype, smem_cap)) cands.push_back({px::MODE_WHOLE, 0, 1});
  for (int ry : {4, 8, 16}) cands.push_back({px::MODE_BANDED, ry, 1});
  if (dtype == PX_F32)
    for (int tb : {4, 8})
      if (px::banded_t_smem(dtype, tb) <= smem_cap) cands.push_back({px::MODE_BANDED_T, 8, tb});
  double best = -1;
  cudaError_t e = cudaMalloc(&mem, 4 * fb * copies);  // per copy: phi, rho, scratch, -c rho
  if (e == cudaSuccess) e = cudaMemset(mem, 0, 4 * fb * copies);
  const int nidx = 2 * (copies * C + 2) + 2 * copies + 8;
  if (e == cudaSuccess) e = cudaMalloc(&idx, (size_t)nidx * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&ins, copies * sizeof(px::BInst));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  for (size_t k = 0; e == cudaSuccess && k < cands.size(); ++k) {
    const bool whole = cands[k].mode == px::MODE_WHOLE;
    // WHOLE: copies instances over the CTAs of ceil(copies / C) clusters
    const int ncl = whole ? (copies + C - 1) / C : copies;
    std::vector<px::BInst> I(copies);
    const double h = 1.0 / nx;
    for (int j = 0; j < copies; ++j) {
      char* base = (char*)mem + (size_t)j * 4 * fb;
      I[j] = px::BInst{};
      I[j].phi = base; I[j].rho = base + fb; I[j].scratch = base + 2 * fb;
      I[j].nx = nx; I[j].ny = ny; I[j].ld = ld; I[j].dtype = dtype;
      I[j].mode = cands[k].mode; I[j].ry = cands[k].ry; I[j].tb = cands[k].tb;
      I[j].c = omega * h * h / 4.0; I[j].ih2 = 1.0 / (h * h); I[j].resid = nullptr;
      I[j].a1 = 1.0 - omega; I[j].w4 = omega / 4.0;
      I[j].rhos = (I[j].mode == px::MODE_BANDED && dtype == PX_F64) ? base + 3 * fb : nullptr;
    }
    // cl_off | cl_items | cta_off | cta_items
    std::vector<int> ix;
    for (int q = 0; q <= ncl; ++q) ix.push_back(whole ? 0 : q);
    const size_t cl_items_at = ix.size();
    for (int q = 0; q < (whole ? 0 : copies); ++q) ix.push_back(q);
    const size_t cta_off_at = ix.size();
    for (int r = 0; r <= ncl * C; ++r) ix.push_back(whole ? std::min(r, copies) : 0);
    const size_t cta_items_at = ix.size();
    for (int q = 0; q < (whole ? copies : 0); ++q) ix.push_back(q);
    ix.push_back(0);
    e = cudaMemcpy(idx, ix.data(), ix.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ins, I.data(), copies * sizeof(px::BInst), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) break;
    px::BParams p{};
    p.inst = (px::BInst*)ins;
    p.cl_off = (int*)idx;
    p.cl_items = (int*)idx + cl_items_at;
    p.cta_off = (int*)idx + cta_off_at;
    p.cta_items = (int*)idx + cta_items_at;
    p.nsweeps = sweeps;
    p.every = 0;
    p.csize = C;
    const size_t smem = whole ? px::whole_bytes(nx, ny, dtype)
                              : (cands[k].mode == px::MODE_BANDED_T ? px::banded_t_smem(dtype, cands[k].tb) : 0);
    e = px::batch_launch(p, ncl, smem, 0);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, 0);
    if (e == cudaSuccess) e = px::batch_launch(p, ncl, smem, 0);
    if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) break;
    const double sms = whole ? copies : (double)copies * C;
    const double rate = (double)nx * ny * sweeps * copies / (ms * 1e-3) / sms;
    if (rate > best) {
      best = rate;
      out->mode = cands[k].mode;
      out->ry = whole ? 8 : cands[k].ry;
      out->tb = cands[k].tb;
      out->rate_per_sm = rate;
      out->tuned = true;
    }
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    st = px::ctx_fail(c, PX_ECUDA, (std::string("batch tuning: ") + cudaGetErrorString(e)).c_str());
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(mem); cudaFree(idx); cudaFree(ins);
  return st;
}

void destroy_batch(px_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->cap_stream2) cudaStreamDestroy(b->cap_stream2);
  if (b->inst_dev) cudaFree(b->inst_dev);
  if (b->inst_pinned) cudaFreeHost(b->inst_pinned);
  if (b->idx_dev) cudaFree(b->idx_dev);
  if (b->scratch) cudaFree(b->scratch);
  delete b;
}

}  // namespace

extern "C" {

px_status px_batch_plan(px_ctx* c, int n, const px_grid* grids, int nsweeps, double omega,
                        int report_every, const char* tune_cache, int tune, px_batch** out) {
  PX_NVTX_RANGE("px_batch_plan");
  if (!c) return PX_EINVAL;
  c->err.clear();
  if (!out) return px::ctx_fail(c, PX_EINVAL, "out is NULL");
  *out = nullptr;
  if (n <= 0 || !grids) return px::ctx_fail(c, PX_EINVAL, "need n > 0 grids");
  if (nsweeps < 0 || report_every < 0 || !std::isfinite(omega))
    return px::ctx_fail(c, PX_EINVAL, "bad nsweeps / report_every / omega");
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != c->device) cudaSetDevice(c->device);
  struct Restore { int p, d; ~Restore() { if (p >= 0 && p != d) cudaSetDevice(p); } } rs{prev, c->device};

  px_batch* b = new (std::nothrow) px_batch();
  if (!b) return px::ctx_fail(c, PX_ENOMEM, "host allocation failed");
  b->ctx = c;
  b->n = n;
  b->nsweeps = nsweeps;
  b->every = report_every;
  b->omega = omega;
  b->nrep = report_every > 0 ? (nsweeps + report_every - 1) / report_every : 0;
  b->grids.assign(grids, grids + n);

  // validate, and size the shared memory for every class that can run WHOLE
  size_t smem = 0;
  for (int i = 0; i < n; ++i) {
    px::FieldDesc f;
    px_status s = px::ctx_check_grid(c, &grids[i], &f);
    if (s != PX_OK) { destroy_batch(b); return s; }
    const int V = f.dtype == PX_F64 ? 2 : 4;
    if (f.ghost || f.nx < 1 || f.ny < 1 || f.nx % V || f.ld % V) {
      destroy_batch(b);
      return px::ctx_fail(c, PX_EUNSUPPORTED,
                          "batched instances must be unghosted, non-empty, with nx and ld "
                          "multiples of 4 (FP32) or 2 (FP64)");
    }
    if (fits_whole(f.nx, f.ny, f.dtype)) smem = std::max(smem, px::whole_bytes(f.nx, f.ny, f.dtype));
  }
  smem = (smem + 1023) / 1024 * 1024;
  // Candidate cluster sizes: every size of which one cluster fits. Each is
  // tuned (or read from the cache) and scheduled; the plan keeps the one with
  // the smallest predicted makespan. The largest BANDED instances matter most
  // here: one of them runs on a single cluster, so small clusters can leave it
  // as the critical path even when they cover more SMs. A launch holds one
  // CTA per SM at most, which leaves the second CTA slot of every SM to the
  // other launch of a mixed-precision plan.
  std::vector<std::pair<int, int>> cands;  // (cluster size, resident clusters)
  for (int cs = px::batch_max_cluster_size(); cs >= 2; cs /= 2) {
    int m = 0;
    cudaError_t e = px::batch_max_clusters(&m, smem, cs);
    if (e != cudaSuccess) { cudaGetLastError(); continue; }
    m = std::min(m, px::device_sm_count() / cs);
    if (m >= 1) cands.push_back({cs, m});
  }
  if (cands.empty()) {
    destroy_batch(b);
    return px::ctx_fail(c, PX_ECUDA, "no cluster of the batch kernel fits on this device");
  }
  bool has64 = false, has32 = false;
  for (int i = 0; i < n; ++i) (grids[i].dtype == PX_F64 ? has64 : has32) = true;
  const bool mixed = has64 && has32 && c->opt_batch_launches == 0 && px::batch_coresident(kCoSmem);

  // classes and their configuration, per candidate cluster size
  std::map<std::string, ClassCfg> cfg;
  std::map<std::string, int> count;
  for (auto& cand : cands) {
    for (int i = 0; i < n; ++i) {
      const px_grid& g = grids[i];
      const std::string k = class_key(g.dtype, g.nx, g.ny, cand.first);
      count[k]++;
      if (!cfg.count(k)) {
        ClassCfg d;
        d.mode = fits_whole(g.nx, g.ny, g.dtype) ? px::MODE_WHOLE : px::MODE_BANDED;
        d.ry = 8;
        d.rate_per_sm = default_rate(g.dtype, d.mode);
        cfg[k] = d;
      }
    }
  }
  const std::string gpu = gpu_name(c->device);
  std::map<std::string, ClassCfg> cached;
  load_cache(tune_cache, gpu, cached);
  int tuned_now = 0;
  auto tune_key = [&](const std::string& key, size_t cap, ClassCfg* out) -> px_status {
    auto it = cached.find(key);
    if (it != cached.end()) {
      *out = it->second;
      return PX_OK;
    }
    if (!tune) return PX_OK;
    int dt = key[1] == '6' ? PX_F64 : PX_F32;
    int nx = 0, ny = 0, cs = 0;
    sscanf(key.c_str() + 4, "%dx%d@c%d", &nx, &ny, &cs);
    ClassCfg t;
    int ncl_cs = 1;
    for (auto& cand : cands)
      if (cand.first == cs) ncl_cs = cand.second;
    px_status s = tune_class(c, dt, nx, ny, std::max(1, std::min(nsweeps, 40)), omega, cs,
                             ncl_cs, cap, &t);
    if (s != PX_OK) return s;
    *out = t;
    cached[key] = t;
    ++tuned_now;
    return PX_OK;
  };
  for (auto& kv : cfg) {
    px_status s = tune_key(kv.first, px::batch_whole_smem(), &kv.second);
    if (s != PX_OK) { destroy_batch(b); return s; }
  }
  // configurations under the co-resident cap (mixed plans only): the class's
  // own where it fits, else tuned again without the modes that do not. A
  // class over the cap with no measured configuration under it (no tuning,
  // none cached) leaves the plan to a single launch.
  std::map<std::string, ClassCfg> cocfg;
  bool co_ok = mixed;
  for (auto& kv : cfg) {
    if (!co_ok) break;
    int dt = kv.first[1] == '6' ? PX_F64 : PX_F32;
    int nx = 0, ny = 0, cs = 0;
    sscanf(kv.first.c_str() + 4, "%dx%d@c%d", &nx, &ny, &cs);
    if (cfg_smem(kv.second, nx, ny, dt) <= kCoSmem) {
      cocfg[kv.first] = kv.second;
      continue;
    }
    ClassCfg d;
    px_status s = tune_key(kv.first + "s", kCoSmem, &d);
    if (s != PX_OK) { destroy_batch(b); return s; }
    if (!d.tuned) co_ok = false;
    cocfg[kv.first] = d;
  }
  if (tuned_now) save_cache(tune_cache, gpu, cached);

  // schedule every candidate: longest first to the least loaded (seconds)
  struct Sched {
    int C = 0, ncl = 0;
    size_t smem = 0;
    double makespan = 0, total = 0;
    std::vector<std::vector<int>> cl_items, cta_items;
  };
  // instances `sub` on ncl_full clusters of C CTAs, configured by `conf`
  auto schedule = [&](int C, int ncl_full, const std::vector<int>& sub,
                      std::map<std::string, ClassCfg>& conf) {
    Sched S;
    S.C = C;
    // WHOLE classes decide the shared memory actually used (less is fine)
    size_t used = 0;
    for (int i : sub) {
      const ClassCfg& k = conf[class_key(grids[i].dtype, grids[i].nx, grids[i].ny, C)];
      used = std::max(used, cfg_smem(k, grids[i].nx, grids[i].ny, grids[i].dtype));
    }
    S.smem = (used + 1023) / 1024 * 1024;
    S.ncl = ncl_full;
    int m = 0;
    if (px::batch_max_clusters(&m, S.smem, C) == cudaSuccess && m > S.ncl) S.ncl = m;
    cudaGetLastError();
    S.ncl = std::min(S.ncl, std::max(1, px::device_sm_count() / C));
    std::vector<double> cl_load(S.ncl, 0.0), cta_load((size_t)S.ncl * C, 0.0);
    S.cl_items.assign(S.ncl, {});
    S.cta_items.assign((size_t)S.ncl * C, {});
    std::vector<std::pair<double, int>> banded, whole;
    for (int i : sub) {
      const px_grid& g = grids[i];
      const ClassCfg& k = conf[class_key(g.dtype, g.nx, g.ny, C)];
      const double work = (double)g.nx * g.ny * nsweeps / std::max(k.rate_per_sm, 1.0);
      if (k.mode != px::MODE_WHOLE) banded.push_back({work / C, i});
      else whole.push_back({work, i});
    }
    std::sort(banded.begin(), banded.end(), [](auto& x, auto& y) { return x.first > y.first; });
    std::sort(whole.begin(), whole.end(), [](auto& x, auto& y) { return x.first > y.first; });
    for (auto& w : banded) {
      const int k = (int)(std::min_element(cl_load.begin(), cl_load.end()) - cl_load.begin());
      cl_load[k] += w.first;
      S.cl_items[k].push_back(w.second);
    }
    for (int k = 0; k < S.ncl; ++k)
      for (int r = 0; r < C; ++r) cta_load[(size_t)k * C + r] = cl_load[k];
    for (auto& w : whole) {
      const int k = (int)(std::min_element(cta_load.begin(), cta_load.end()) - cta_load.begin());
      cta_load[k] += w.first;
      S.cta_items[k].push_back(w.second);
    }
    S.makespan = *std::max_element(cta_load.begin(), cta_load.end());
    for (double v : cta_load) S.total += v;
    return S;
  };
  struct Plan {
    Sched a, b;       // b: the FP32 launch of a mixed plan (b.ncl == 0 otherwise)
    double predicted = 0;
  };
  std::vector<int> all(n), sub64, sub32;
  for (int i = 0; i < n; ++i) {
    all[i] = i;
    (grids[i].dtype == PX_F64 ? sub64 : sub32).push_back(i);
  }
  std::vector<Plan> plans;
  for (auto& cand : cands) {
    Plan P;
    P.a = schedule(cand.first, cand.second, all, cfg);
    P.predicted = P.a.makespan;
    plans.push_back(std::move(P));
    if (co_ok) {
      Plan Q;
      Q.a = schedule(cand.first, cand.second, sub64, cocfg);
      Q.b = schedule(cand.first, cand.second, sub32, cocfg);
      const double hi = std::max(Q.a.makespan, Q.b.makespan), lo = std::min(Q.a.makespan, Q.b.makespan);
      Q.predicted = hi + kCoOverlap * lo;
      if (Q.a.smem <= kCoSmem && Q.b.smem <= kCoSmem) plans.push_back(std::move(Q));
    }
  }
  size_t pick = 0;
  for (size_t k = 1; k < plans.size(); ++k)
    if (plans[k].predicted < plans[pick].predicted * (1 - 1e-9)) pick = k;
  Plan& PL = plans[pick];
  const bool co = PL.b.ncl > 0;
  std::map<std::string, ClassCfg>& used_cfg = co ? cocfg : cfg;
  Sched& S = PL.a;
  const int C = S.C, ncl = S.ncl;
  smem = S.smem;
  b->nclusters = ncl;
  b->smem = smem;
  b->nclusters2 = co ? PL.b.ncl : 0;
  b->smem2 = co ? PL.b.smem : 0;

  size_t scratch_bytes = 0;
  std::vector<size_t> scr_off(n, 0), rhs_off(n, SIZE_MAX);
  b->inst.resize(n);
  for (int i = 0; i < n; ++i) {
    const px_grid& g = grids[i];
    const ClassCfg& k = used_cfg[class_key(g.dtype, g.nx, g.ny, C)];
    px::BInst& I = b->inst[i];
    I = px::BInst{};
    I.nx = g.nx; I.ny = g.ny; I.ld = g.ld; I.dtype = g.dtype; I.mode = k.mode; I.ry = k.ry;
    I.tb = k.tb;
    I.c = omega * g.h * g.h / 4.0;
    I.ih2 = 1.0 / (g.h * g.h);
    I.a1 = 1.0 - omega;
    I.w4 = omega / 4.0;
    if (k.mode != px::MODE_WHOLE) {
      const size_t fb = ((size_t)g.ld * g.ny * (g.dtype == PX_F64 ? 8 : 4) + 255) / 256 * 256;
      scr_off[i] = scratch_bytes;
      scratch_bytes += fb;
      if (g.dtype == PX_F64 && k.mode == px::MODE_BANDED) {  // -c rho for unreported sweeps
        rhs_off[i] = scratch_bytes;
        scratch_bytes += fb;
      }
    }
  }
  // index arrays of one launch: cl_off | cl_items | cta_off | cta_items
  std::vector<int> ix;
  struct Offs { size_t cl_off, cl_items, cta_off, cta_items; };
  auto append = [&](const Sched& T) {
    Offs o;
    o.cl_off = ix.size();
    ix.push_back(0);
    for (int k = 0; k < T.ncl; ++k) ix.push_back(ix[o.cl_off + k] + (int)T.cl_items[k].size());
    o.cl_items = ix.size();
    for (int k = 0; k < T.ncl; ++k) ix.insert(ix.end(), T.cl_items[k].begin(), T.cl_items[k].end());
    o.cta_off = ix.size();
    ix.push_back(0);
    for (int k = 0; k < T.ncl * T.C; ++k) ix.push_back(ix[o.cta_off + k] + (int)T.cta_items[k].size());
    o.cta_items = ix.size();
    for (int k = 0; k < T.ncl * T.C; ++k) ix.insert(ix.end(), T.cta_items[k].begin(), T.cta_items[k].end());
    ix.push_back(0);  // keep the arrays non-empty
    return o;
  };
  const Offs oa = append(S);
  const Offs ob = co ? append(PL.b) : Offs{};

  cudaError_t e = cudaMalloc(&b->idx_dev, ix.size() * sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(b->idx_dev, ix.data(), ix.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&b->inst_dev, n * sizeof(px::BInst));
  if (e == cudaSuccess) e = cudaMallocHost(&b->inst_pinned, n * sizeof(px::BInst));
  if (e == cudaSuccess && scratch_bytes) e = cudaMalloc(&b->scratch, scratch_bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    destroy_batch(b);
    return px::ctx_fail(c, PX_ENOMEM, "batch plan buffers");
  }
  for (int i = 0; i < n; ++i) {
    if (b->inst[i].mode != px::MODE_WHOLE) b->inst[i].scratch = (char*)b->scratch + scr_off[i];
    if (rhs_off[i] != SIZE_MAX) b->inst[i].rhos = (char*)b->scratch + rhs_off[i];
  }
  auto set_params = [&](px::BParams& P, const Offs& o) {
    P.inst = b->inst_dev;
    P.cl_off = b->idx_dev + o.cl_off;
    P.cl_items = b->idx_dev + o.cl_items;
    P.cta_off = b->idx_dev + o.cta_off;
    P.cta_items = b->idx_dev + o.cta_items;
    P.nsweeps = nsweeps;
    P.every = report_every;
    P.csize = C;
  };
  set_params(b->params, oa);
  if (co) set_params(b->params2, ob);

  // The launch (or the two side-by-side launches) is captured once into a
  // graph; runs replay it.
  e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess && co) e = cudaStreamCreateWithFlags(&b->cap_stream2, cudaStreamNonBlocking);
  cudaEvent_t fork = nullptr, join = nullptr;
  if (e == cudaSuccess && co) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  if (e == cudaSuccess && co) e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t el = cudaSuccess;
    if (co) {
      el = cudaEventRecord(fork, b->cap_stream);
      if (el == cudaSuccess) el = cudaStreamWaitEvent(b->cap_stream2, fork, 0);
    }
    if (el == cudaSuccess) el = px::batch_launch(b->params, ncl, smem, b->cap_stream);
    if (el == cudaSuccess && co) el = px::batch_launch(b->params2, b->nclusters2, b->smem2, b->cap_stream2);
    if (el == cudaSuccess && co) el = cudaEventRecord(join, b->cap_stream2);
    if (el == cudaSuccess && co) el = cudaStreamWaitEvent(b->cap_stream, join, 0);
    e = cudaStreamEndCapture(b->cap_stream, &b->graph);
    if (el != cudaSuccess) e = el;
  }
  if (fork) cudaEventDestroy(fork);
  if (join) cudaEventDestroy(join);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    std::string m = std::string("batch graph: ") + cudaGetErrorString(e);
    destroy_batch(b);
    return px::ctx_fail(c, PX_ECUDA, m.c_str());
  }

  // description
  std::ostringstream os;
  os << "{\"clusters\": " << ncl << ", \"cluster_size\": " << C << ", \"smem\": " << smem
     << ", \"predicted_ms\": " << PL.predicted * 1e3
     << ", \"balance\": " << (S.makespan > 0 ? S.total / (S.makespan * ncl * C) : 1.0)
     << ", \"launches\": " << (co ? 2 : 1);
  if (co)
    os << ", \"side_by_side\": {\"fp64_ms\": " << S.makespan * 1e3 << ", \"fp32_ms\": "
       << PL.b.makespan * 1e3 << ", \"fp32_clusters\": " << PL.b.ncl << ", \"fp32_smem\": "
       << PL.b.smem << ", \"smem_cap\": " << kCoSmem << "}";
  os << ", \"candidates\": [";
  for (size_t k = 0; k < plans.size(); ++k)
    os << (k ? ", " : "") << "{\"cluster_size\": " << plans[k].a.C << ", \"clusters\": "
       << plans[k].a.ncl << ", \"launches\": " << (plans[k].b.ncl > 0 ? 2 : 1)
       << ", \"predicted_ms\": " << plans[k].predicted * 1e3 << "}";
  os << "], \"classes\": {";
  const std::string suffix = "@c" + std::to_string(C);
  bool first = true;
  for (auto& kv : used_cfg) {
    if (kv.first.size() < suffix.size() ||
        kv.first.compare(kv.first.size() - suffix.size(), suffix.size(), suffix) != 0)
      continue;
    os << (first ? "" : ", ") << "\"" << kv.first << "\": {\"count\": " << count[kv.first]
       << ", \"mode\": \""
       << (kv.second.mode == px::MODE_WHOLE ? "whole"
                                            : kv.second.mode == px::MODE_BANDED ? "banded" : "banded_t")
       << "\", \"ry\": " << kv.second.ry << ", \"tb\": " << kv.second.tb
       << ", \"rate_per_sm\": " << kv.second.rate_per_sm
       << ", \"tuned\": " << (kv.second.tuned ? "true" : "false") << "}";
    first = false;
  }
  os << "}}";
  b->desc = os.str();
  *out = b;
  return PX_OK;
}

px_status px_batch_run(px_batch* b, void* const* phis, const void* const* rhos,
                       double* resid_dev, void* stream) {
  PX_NVTX_RANGE("px_batch_run");
  if (!b) return PX_EINVAL;
  px_ctx* c = b->ctx;
  c->err.clear();
  if (!phis || !rhos) return px::ctx_fail(c, PX_EINVAL, "phis / rhos is NULL");
  for (int i = 0; i < b->n; ++i) {
    const px_grid& g = b->grids[i];
    const size_t span = (size_t)((int64_t)(g.ny - 1) * g.ld + g.nx) * (g.dtype == PX_F64 ? 8 : 4);
    if (!phis[i] || !rhos[i]) return px::ctx_fail(c, PX_EINVAL, "NULL instance pointer");
    if ((((uintptr_t)phis[i]) & 15) || (((uintptr_t)rhos[i]) & 15))
      return px::ctx_fail(c, PX_EINVAL, "instance fields must be 16-byte aligned");
    const uintptr_t a = (uintptr_t)phis[i], r = (uintptr_t)rhos[i];
    if (a < r + span && r < a + span) return px::ctx_fail(c, PX_EINVAL, "phi overlaps rho");
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != c->device) cudaSetDevice(c->device);
  struct Restore { int p, d; ~Restore() { if (p >= 0 && p != d) cudaSetDevice(p); } } rs{prev, c->device};
  cudaStream_t st = (cudaStream_t)stream;
  // The previous run may still read the pinned table: wait for it first.
  cudaError_t e = cudaStreamSynchronize(st);
  for (int i = 0; i < b->n && e == cudaSuccess; ++i) {
    px::BInst I = b->inst[i];
    I.phi = phis[i];
    I.rho = rhos[i];
    I.resid = (resid_dev && b->nrep) ? resid_dev + (size_t)i * b->nrep : nullptr;
    b->inst_pinned[i] = I;
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->inst_dev, b->inst_pinned, b->n * sizeof(px::BInst),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && resid_dev && b->nrep)
    e = cudaMemsetAsync(resid_dev, 0, (size_t)b->n * b->nrep * sizeof(double), st);
  if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return px::ctx_fail(c, PX_ECUDA, (std::string("batch run: ") + cudaGetErrorString(e)).c_str());
  }
  return PX_OK;
}

const char* px_batch_describe(const px_batch* b) { return b ? b->desc.c_str() : ""; }

px_status px_batch_destroy(px_batch* b) {
  if (!b) return PX_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != b->ctx->device) cudaSetDevice(b->ctx->device);
  cudaDeviceSynchronize();
  const int dev = b->ctx->device;
  destroy_batch(b);
  if (prev >= 0 && prev != dev) cudaSetDevice(prev);
  return PX_OK;
}

}  // extern "C"

// C ABI of the fused periodic Poisson relaxation library (declared in
// include/protox.h). Validates every argument before any launch, plans the
// temporal-blocking launches of a relax call and ping-pongs between the
// caller's output and context scratch so that phi_in == phi_out works.
#include "../../include/protox.h"
#include "px_internal.cuh"

#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <limits>
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>


#ifdef PX_CHECKED
namespace px {
__device__ unsigned long long g_px_checked[2];  // violations, first (site << 48 | index)
}
#endif

namespace {

thread_local std::string g_create_err;

px_status fail(px_ctx* c, px_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf; else g_create_err = buf;
  return s;
}

px_status cuda_fail(px_ctx* c, cudaError_t e, const char* what) {
  return fail(c, e == cudaErrorMemoryAllocation ? PX_ENOMEM : PX_ECUDA, "%s: %s (%s)", what,
              cudaGetErrorName(e), cudaGetErrorString(e));
}

// Makes the context's device current for the scope of a call and restores the
// caller's device afterwards.
struct DeviceScope {
  int prev = -1;
  bool ok = true;
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceScope() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

size_t elem_size(int dtype) { return dtype == PX_F64 ? 8 : 4; }

px_status check_grid(px_ctx* c, const px_grid* g, px::FieldDesc* f) {
  if (!g) return fail(c, PX_EINVAL, "grid is NULL");
  if (g->dtype != PX_F64 && g->dtype != PX_F32)
    return fail(c, PX_EINVAL, "dtype %d is not PX_F64 or PX_F32", (int)g->dtype);
  if (g->ghost != 0 && g->ghost != 1) return fail(c, PX_EINVAL, "ghost must be 0 or 1");
  if (g->nx < 0 || g->ny < 0) return fail(c, PX_EINVAL, "negative extent %d x %d", g->nx, g->ny);
  if (g->nx > (1 << 29) || g->ny > (1 << 29))
    return fail(c, PX_EINVAL, "extent %d x %d above 2^29", g->nx, g->ny);
  if (g->ld < (int64_t)g->nx + 2 * g->ghost)
    return fail(c, PX_EINVAL, "ld %lld < nx + 2*ghost", (long long)g->ld);
  if (!(std::isfinite(g->h) && g->h > 0.0)) return fail(c, PX_EINVAL, "h must be finite and > 0");
  const double ih2 = 1.0 / (g->h * g->h);
  if (!std::isfinite(ih2)) return fail(c, PX_EINVAL, "1/h^2 overflows");
  const double rows = (double)g->ny + 2 * g->ghost;
  if (rows * (double)g->ld * elem_size(g->dtype) > 9.0e18)
    return fail(c, PX_EINVAL, "field too large");
  f->nx = g->nx;
  f->ny = g->ny;
  f->ld = g->ld;
  f->ghost = g->ghost;
  f->off = g->ghost ? g->ld + 1 : 0;
  f->dtype = g->dtype;
  f->h = g->h;
  f->family = c ? c->opt_fp32_family : 0;
  return PX_OK;
}

// Bytes from the field's base pointer to one past its last element.
size_t field_span(const px::FieldDesc& f) {
  const int64_t rows = f.ny + 2 * f.ghost;
  if (rows == 0 || f.nx == 0) return 0;
  return (size_t)(((rows - 1) * f.ld + f.nx + 2 * f.ghost) * (int64_t)elem_size(f.dtype));
}

bool overlap(const void* a, const void* b, size_t n) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return n > 0 && x < y + n && y < x + n;
}

// Whether [a, a + na) and [b, b + nb) share a byte.
bool overlap2(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return na > 0 && nb > 0 && x < y + nb && y < x + na;
}

px_status ensure_scratch(px_ctx* c, size_t bytes) {
  if (c->scratch_bytes >= bytes) return PX_OK;
  if (c->scratch) cudaFree(c->scratch);
  c->scratch = nullptr;
  c->scratch_bytes = 0;
  cudaError_t e = cudaMalloc(&c->scratch, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, PX_ENOMEM, "scratch of %zu bytes: %s", bytes, cudaGetErrorString(e));
  }
  c->scratch_bytes = bytes;
  return PX_OK;
}

int auto_tblock(const px::FieldDesc& f) {
  // FP64 is bound by the FP64 pipe at depth 1, so deeper blocking only adds
  // redundant halo work. FP32 is bound by HBM at depth 1 and by instruction
  // issue from depth 4 or so; measured on B300 (GLUP/s, 200 sweeps, a report
  // every sweep), depth 8 is the fastest from 128^2 up: on the register
  // wavefront 2406 vs 1989 at depth 4 (16384^2), 2067 vs 1679 (6144^2), 1431
  // vs 1019 (3072^2); on the two-row wavefront 997 (2048^2), 63 vs 42 at
  // depth 4 (256^2), 16 vs 5 at depth 1 (128^2).
  if (f.dtype == PX_F64) return 1;
  const int64_t cells = (int64_t)f.nx * f.ny;
  return cells >= (1 << 10) ? 8 : 1;
}


// Launch sizes of a relax call: T, T, ..., remainder, with T the requested or
// automatic depth (1 when the layout cannot use the tiled kernel). In place,
// the first launch must not write the buffer it reads: an odd launch count is
// made even by splitting a multi-sweep launch, else the input is staged into
// scratch first (*copy_first).
std::vector<int> plan_launches(const px::FieldDesc& f, bool vec, bool inplace, int nsweeps,
                               int tblock, bool* copy_first) {
  int T = tblock == 0 ? auto_tblock(f) : tblock;
  if (!vec) T = 1;
  std::vector<int> sizes;
  for (int left = nsweeps; left > 0; left -= T) sizes.push_back(left < T ? left : T);
  *copy_first = false;
  if (inplace && (sizes.size() % 2 == 1)) {
    size_t k = 0;
    while (k < sizes.size() && sizes[k] < 2) ++k;
    if (k < sizes.size()) {
      const int a = sizes[k];
      sizes[k] = 1;
      sizes.insert(sizes.begin() + (long)k + 1, a - 1);
    } else {
      *copy_first = true;
    }
  }
  return sizes;
}

}  // namespace

// Helpers shared with the context-free entry point in relax_static.cu. They
// report failures through the thread's context-free message (px_last_error(NULL)).
namespace px {
px_status ctx_fail(px_ctx* c, px_status st, const char* msg) { return fail(c, st, "%s", msg); }
px_status ctx_check_grid(px_ctx* c, const px_grid* g, FieldDesc* f) { return check_grid(c, g, f); }
px_status unbound_check_grid(const px_grid* g, FieldDesc* f) { return check_grid(nullptr, g, f); }
px_status unbound_fail(px_status s, const char* msg) { return fail(nullptr, s, "%s", msg); }
void unbound_clear() { g_create_err.clear(); }
size_t field_bytes(const FieldDesc& f) { return field_span(f); }
bool ranges_overlap(const void* a, const void* b, size_t n) { return overlap(a, b, n); }
bool ranges_overlap2(const void* a, size_t na, const void* b, size_t nb) {
  return overlap2(a, na, b, nb);
}
std::vector<int> plan_relax_launches(const FieldDesc& f, bool vec, bool inplace, int nsweeps,
                                     int tblock, bool* copy_first) {
  return plan_launches(f, vec, inplace, nsweeps, tblock, copy_first);
}
}  // namespace px

extern "C" {

const char* px_status_string(px_status s) {
  switch (s) {
    case PX_OK: return "PX_OK";
    case PX_EINVAL: return "PX_EINVAL";
    case PX_ECUDA: return "PX_ECUDA";
    case PX_ENOMEM: return "PX_ENOMEM";
    case PX_ENOCONV: return "PX_ENOCONV";
    case PX_ETIMEOUT: return "PX_ETIMEOUT";
    case PX_EMEAN: return "PX_EMEAN";
    case PX_ENAN: return "PX_ENAN";
    case PX_EUNSUPPORTED: return "PX_EUNSUPPORTED";
  }
  return "PX_UNKNOWN";
}

px_status px_create(px_ctx** out, int device) {
  if (!out) return fail(nullptr, PX_EINVAL, "out is NULL");
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(nullptr, PX_ECUDA, "cudaGetDeviceCount: %s", cudaGetErrorString(e));
  }
  if (device < 0 || device >= n) return fail(nullptr, PX_EINVAL, "device %d of %d", device, n);
  DeviceScope ds(device);
  if (!ds.ok) return fail(nullptr, PX_ECUDA, "cudaSetDevice(%d) failed", device);
  px_ctx* c = new (std::nothrow) px_ctx();
  if (!c) return fail(nullptr, PX_ENOMEM, "host allocation failed");
  c->device = device;
  e = cudaMalloc(&c->red, (8 + (size_t)px::sum_partials_count()) * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost(&c->red_host, 4 * sizeof(double));
  // load-balance words: one per resident warp at most (64 warps per SM)
  int sms = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) {
    c->sched_cap = 64 * sms;
    e = cudaMalloc(&c->sched, sizeof(unsigned long long) * (size_t)c->sched_cap);
  }
  if (e == cudaSuccess)
    e = cudaMemset(c->sched, 0, sizeof(unsigned long long) * (size_t)c->sched_cap);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (c->red) cudaFree(c->red);
    if (c->red_host) cudaFreeHost(c->red_host);
    if (c->sched) cudaFree(c->sched);
    delete c;
    return fail(nullptr, PX_ENOMEM, "context buffers: %s", cudaGetErrorString(e));
  }
  *out = c;
  return PX_OK;
}

px_status px_destroy(px_ctx* c) {
  if (!c) return PX_OK;
  DeviceScope ds(c->device);
  cudaDeviceSynchronize();
  if (c->scratch) cudaFree(c->scratch);
  if (c->ws) cudaFree(c->ws);
  if (c->red) cudaFree(c->red);
  if (c->red_host) cudaFreeHost(c->red_host);
  if (c->sched) cudaFree(c->sched);
  if (c->mg) cudaFree(c->mg);
  if (c->ewave) cudaFree(c->ewave);
  delete c;
  return PX_OK;
}

const char* px_last_error(const px_ctx* c) {
  return c ? c->err.c_str() : g_create_err.c_str();
}

int px_is_checked_build(void) {
#ifdef PX_CHECKED
  return 1;
#else
  return 0;
#endif
}

px_status px_checked_faults(px_ctx* c, uint64_t* count, uint64_t* first) {
  if (!c || !count) return PX_EINVAL;
  c->err.clear();
#ifdef PX_CHECKED
  DeviceScope ds(c->device);
  unsigned long long h[2] = {0, 0};
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(h, px::g_px_checked, sizeof h);
  const unsigned long long z[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(px::g_px_checked, z, sizeof z);
  if (e != cudaSuccess) return cuda_fail(c, e, "checked-build fault word");
  *count = h[0];
  if (first) *first = h[1];
  return PX_OK;
#else
  *count = 0;
  if (first) *first = 0;
  return fail(c, PX_EUNSUPPORTED, "bounds checks are compiled only into the checked build");
#endif
}

px_status px_set_option(px_ctx* c, int option, int value) {
  if (!c) return PX_EINVAL;
  c->err.clear();
  switch (option) {
    case PX_OPT_FP32_FAMILY:
      if (value < 0 || value > 4) return fail(c, PX_EINVAL, "FP32 family %d not in 0..4", value);
      c->opt_fp32_family = value;
      return PX_OK;
    case PX_OPT_RB_SWEEPS_PER_LAUNCH:
      if (value < 0 || value > 4)
        return fail(c, PX_EINVAL, "red-black sweeps per launch %d not in 0..4", value);
      c->opt_rb_sweeps = value;
      return PX_OK;
    case PX_OPT_BATCH_LAUNCHES:
      if (value < 0 || value > 1) return fail(c, PX_EINVAL, "batch launches option %d not in 0..1", value);
      c->opt_batch_launches = value;
      return PX_OK;
    case PX_OPT_RB_FP64_PASSES:
      if (value < 0 || value > 2)
        return fail(c, PX_EINVAL, "FP64 red-black passes option %d not in 0..2", value);
      c->opt_rb_fp64_passes = value;
      return PX_OK;
    case PX_OPT_MG_PROLONG:
      if (value < 0 || value > 1)
        return fail(c, PX_EINVAL, "multigrid interpolation option %d not in 0..1", value);
      c->opt_mg_prolong = value;
      return PX_OK;
  }
  return fail(c, PX_EINVAL, "unknown option %d", option);
}

px_status px_get_option(const px_ctx* c, int option, int* value) {
  if (!c || !value) return PX_EINVAL;
  switch (option) {
    case PX_OPT_FP32_FAMILY: *value = c->opt_fp32_family; return PX_OK;
    case PX_OPT_RB_SWEEPS_PER_LAUNCH: *value = c->opt_rb_sweeps; return PX_OK;
    case PX_OPT_BATCH_LAUNCHES: *value = c->opt_batch_launches; return PX_OK;
    case PX_OPT_RB_FP64_PASSES: *value = c->opt_rb_fp64_passes; return PX_OK;
    case PX_OPT_MG_PROLONG: *value = c->opt_mg_prolong; return PX_OK;
  }
  return PX_EINVAL;
}

px_status px_apply_stencil(px_ctx* c, const px_grid* g, const void* phi, void* lphi,
                           void* stream) {
  PX_NVTX_RANGE("px_apply_stencil");
  if (!c) return PX_EINVAL;
  c->err.clear();
  px::FieldDesc f;
  px_status s = check_grid(c, g, &f);
  if (s != PX_OK) return s;
  if (f.nx == 0 || f.ny == 0) return PX_OK;
  if (!phi || !lphi) return fail(c, PX_EINVAL, "NULL field pointer");
  if (overlap(phi, lphi, field_span(f))) return fail(c, PX_EINVAL, "phi and lphi overlap");
  DeviceScope ds(c->device);
  cudaError_t e = px::launch_apply_stencil(f, phi, lphi, (cudaStream_t)stream);
  return e == cudaSuccess ? PX_OK : cuda_fail(c, e, "apply_stencil launch");
}

px_status px_relax_n(px_ctx* c, const px_grid* g, const void* phi_in, void* phi_out,
                     const void* rho, double omega, int nsweeps, int tblock,
                     double* resid_dev, int report_every, void* stream) {
  PX_NVTX_RANGE("px_relax_n");
  if (!c) return PX_EINVAL;
  c->err.clear();
  px::FieldDesc f;
  px_status s = check_grid(c, g, &f);
  if (s != PX_OK) return s;
  if (nsweeps < 0) return fail(c, PX_EINVAL, "nsweeps %d < 0", nsweeps);
  if (report_every < 0) return fail(c, PX_EINVAL, "report_every %d < 0", report_every);
  if (tblock < 0 || tblock > 8) return fail(c, PX_EINVAL, "tblock %d not in 0..8", tblock);
  if (!std::isfinite(omega)) return fail(c, PX_EINVAL, "omega must be finite");
  const bool reports = resid_dev && report_every > 0 && nsweeps > 0;
  const int nrep = reports ? (nsweeps + report_every - 1) / report_every : 0;
  const bool empty = f.nx == 0 || f.ny == 0;
  const size_t span = field_span(f);
  const bool inplace = phi_in == phi_out;
  if (!empty) {
    if (!phi_in || !phi_out || !rho) return fail(c, PX_EINVAL, "NULL field pointer");
    if (!inplace && overlap(phi_in, phi_out, span))
      return fail(c, PX_EINVAL, "phi_in and phi_out overlap without being equal");
    if (overlap(rho, phi_out, span)) return fail(c, PX_EINVAL, "rho overlaps phi_out");
    if (reports && overlap2(resid_dev, sizeof(double) * (size_t)nrep, phi_out, span))
      return fail(c, PX_EINVAL, "resid_dev overlaps phi_out");
  }
  DeviceScope ds(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (reports) {
    cudaError_t e = cudaMemsetAsync(resid_dev, 0, sizeof(double) * (size_t)nrep, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "clear resid_dev");
  }
  if (empty) return PX_OK;

  if (nsweeps == 0) {
    if (inplace) return PX_OK;
    cudaError_t e = px::launch_copy_field(f, phi_in, phi_out, st);
    return e == cudaSuccess ? PX_OK : cuda_fail(c, e, "copy launch");
  }

  const bool vec = px::vector_ok(f, phi_in, phi_out, rho);
  bool copy_first = false;
  std::vector<int> sizes = plan_launches(f, vec, inplace, nsweeps, tblock, &copy_first);
  const size_t L = sizes.size();
  if (L >= 2 || copy_first) {
    // Scratch uses the caller's layout (same pitch and ghost offset), and
    // cudaMalloc returns 256-byte aligned memory, so alignment is preserved.
    s = ensure_scratch(c, span);
    if (s != PX_OK) return s;
  }
  void* scratch = c->scratch;
  const void* src = phi_in;
  if (copy_first) {
    cudaError_t e = px::launch_copy_field(f, phi_in, scratch, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "copy launch");
    src = scratch;
  }
  const bool vec_all = vec && (L < 2 && !copy_first ? true : px::vector_ok(f, scratch, scratch, scratch));
  int s0 = 0;
  for (size_t k = 0; k < L; ++k) {
    void* dst = ((L - 1 - k) % 2 == 0) ? phi_out : scratch;
    cudaError_t e = px::launch_relax(f, src, dst, rho, omega, sizes[k], vec_all,
                                     reports ? resid_dev : nullptr, s0, report_every,
                                     c->sched, c->sched_cap, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "relax launch");
    s0 += sizes[k];
    src = dst;
  }
  return PX_OK;
}

// Red-black sweeps per launch of the FP32 register wavefront (1..4): the
// context option PX_OPT_RB_SWEEPS_PER_LAUNCH, else 3. Measured at 16384^2
// with a report every sweep: 496, 984, 1542 and 1525 GLUP/s for 1..4 (four
// sweeps need two halo lanes per side and one CTA of 12 warps per SM).
static int rb_sweeps(const px_ctx* c) { return c->opt_rb_sweeps > 0 ? c->opt_rb_sweeps : 3; }

// FP64 vector layouts take one fused launch per red-black sweep unless the
// context option PX_OPT_RB_FP64_PASSES = 2 asks for the two passes. Measured at
// 16384^2: 54.8 GLUP/s fused against 50.2 in two passes with a report every
// sweep, 75.8 against 51.1 without reports.
static bool rb_fused(const px_ctx* c, const px::FieldDesc& f, bool vec) {
  return f.dtype == 0 && vec && c->opt_rb_fp64_passes != 2;
}

// One red-black sweep src -> dst (src != dst): fused, or a red pass (out of
// place) and a black pass (in place on dst).
static cudaError_t rb_sweep(const px::FieldDesc& f, const void* src, void* dst, const void* rho,
                            double omega, bool fused, bool vec, double* slot, cudaStream_t st) {
  if (fused)
    return px::launch_rbsor_fused(f, (const double*)src, (double*)dst, (const double*)rho, omega,
                                  slot, st);
  cudaError_t e = px::launch_rbsor_pass(f, src, dst, rho, omega, true, vec, slot, st);
  if (e == cudaSuccess) e = px::launch_rbsor_pass(f, dst, dst, rho, omega, false, vec, nullptr, st);
  return e;
}

px_status px_rbsor_n(px_ctx* c, const px_grid* g, const void* phi_in, void* phi_out,
                     const void* rho, double omega, int nsweeps, double* resid_dev,
                     int report_every, void* stream) {
  PX_NVTX_RANGE("px_rbsor_n");
  if (!c) return PX_EINVAL;
  c->err.clear();
  px::FieldDesc f;
  px_status s = check_grid(c, g, &f);
  if (s != PX_OK) return s;
  if (f.ghost) return fail(c, PX_EUNSUPPORTED, "red-black SOR takes unghosted layouts");
  if (f.nx % 2 || f.ny % 2)
    return fail(c, PX_EINVAL, "red-black SOR needs even nx and ny (got %d x %d)", f.nx, f.ny);
  if (nsweeps < 0) return fail(c, PX_EINVAL, "nsweeps %d < 0", nsweeps);
  if (report_every < 0) return fail(c, PX_EINVAL, "report_every %d < 0", report_every);
  if (!std::isfinite(omega)) return fail(c, PX_EINVAL, "omega must be finite");
  const bool reports = resid_dev && report_every > 0 && nsweeps > 0;
  const int nrep = reports ? (nsweeps + report_every - 1) / report_every : 0;
  const bool empty = f.nx == 0 || f.ny == 0;
  const size_t span = field_span(f);
  const bool inplace = phi_in == phi_out;
  if (!empty) {
    if (!phi_in || !phi_out || !rho) return fail(c, PX_EINVAL, "NULL field pointer");
    if (!inplace && overlap(phi_in, phi_out, span))
      return fail(c, PX_EINVAL, "phi_in and phi_out overlap without being equal");
    if (overlap(rho, phi_out, span)) return fail(c, PX_EINVAL, "rho overlaps phi_out");
    if (reports && overlap2(resid_dev, sizeof(double) * (size_t)nrep, phi_out, span))
      return fail(c, PX_EINVAL, "resid_dev overlaps phi_out");
  }
  DeviceScope ds(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (reports) {
    cudaError_t e = cudaMemsetAsync(resid_dev, 0, sizeof(double) * (size_t)nrep, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "clear resid_dev");
  }
  if (empty) return PX_OK;
  if (nsweeps == 0) {
    if (inplace) return PX_OK;
    cudaError_t e = px::launch_copy_field(f, phi_in, phi_out, st);
    return e == cudaSuccess ? PX_OK : cuda_fail(c, e, "copy launch");
  }
  // FP32 vector layouts run rb_sweeps() sweeps per launch of the register
  // wavefront; FP64 vector layouts one fused launch per sweep (out of place);
  // other layouts each sweep as a red pass (out of place) and a black pass (in
  // place on its output). Launch outputs alternate
  // between phi_out and scratch: out of place so that the last lands in
  // phi_out (phi_in is never written), in place starting with scratch, an odd
  // launch count ending with a copy back.
  const bool reg_ok = f.dtype == 1 && px::vector_ok(f, phi_in, phi_out, rho);
  const int D = reg_ok ? rb_sweeps(c) : 1;
  const int L = (nsweeps + D - 1) / D;
  if (inplace || L >= 2) {
    s = ensure_scratch(c, span);
    if (s != PX_OK) return s;
  }
  void* scratch = c->scratch;
  const bool vec = px::vector_ok(f, phi_in, phi_out, rho) &&
                   (!scratch || px::vector_ok(f, scratch, scratch, scratch));
  const bool reg = reg_ok && vec;
  const bool fused = rb_fused(c, f, vec);
  const void* src = phi_in;
  for (int i = 0, done = 0; i < L; ++i) {
    void* dst = inplace ? (i % 2 == 0 ? scratch : phi_out) : ((L - 1 - i) % 2 == 0 ? phi_out : scratch);
    const int n = std::min(D, nsweeps - done);
    cudaError_t e = cudaSuccess;
    if (reg) {
      e = px::launch_rbsor_reg(f, (const float*)src, (float*)dst, (const float*)rho, omega, n,
                               reports ? resid_dev : nullptr, done, report_every, c->sched,
                               c->sched_cap, st);
    } else {
      double* slot = reports && done % report_every == 0 ? resid_dev + done / report_every : nullptr;
      e = rb_sweep(f, src, dst, rho, omega, fused, vec, slot, st);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "red-black SOR launch");
    done += n;
    src = dst;
  }
  if (src != phi_out) {
    cudaError_t e = px::launch_copy_field(f, src, phi_out, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "copy launch");
  }
  return PX_OK;
}

namespace {

// n red-black sweeps alternating between the buffers a and b, from *cur (one
// of them); *cur ends on the buffer that holds the result. With slot, the
// residual of the first sweep's input state is folded into *slot. With pl
// (FP32 vector layouts only, n > 0), the first launch adds the interpolated
// coarse correction to *cur's values as it loads them.
cudaError_t rb_sweeps_ab(px_ctx* c, const px::FieldDesc& f, void* a, void* b, void** cur,
                         const void* rho, double omega, int n, double* slot, cudaStream_t st,
                         const px::Prolong* pl = nullptr) {
  const bool vec = px::vector_ok(f, a, b, rho);
  const bool reg = f.dtype == 1 && vec;
  const bool fused = rb_fused(c, f, vec);
  const int D = reg ? rb_sweeps(c) : 1;
  for (int done = 0; done < n;) {
    const int k = std::min(D, n - done);
    void* src = *cur;
    void* dst = src == a ? b : a;
    double* s = done == 0 ? slot : nullptr;
    cudaError_t e;
    if (reg) {
      e = px::launch_rbsor_reg(f, (const float*)src, (float*)dst, (const float*)rho, omega, k, s,
                               0, n, c->sched, c->sched_cap, st, done == 0 ? pl : nullptr);
    } else {
      e = rb_sweep(f, src, dst, rho, omega, fused, vec, s, st);
    }
    if (e != cudaSuccess) return e;
    *cur = dst;
    done += k;
  }
  return cudaSuccess;
}

}  // namespace

px_status px_mg_solve(px_ctx* c, const px_grid* g, void* phi, const void* rho, int ncycles,
                      int nu1, int nu2, double omega, int coarse_sweeps, int max_levels,
                      double* resid_dev, void* stream) {
  PX_NVTX_RANGE("px_mg_solve");
  if (!c) return PX_EINVAL;
  c->err.clear();
  px::FieldDesc f;
  px_status s = check_grid(c, g, &f);
  if (s != PX_OK) return s;
  if (f.ghost) return fail(c, PX_EUNSUPPORTED, "multigrid takes unghosted layouts");
  if (f.nx % 2 || f.ny % 2)
    return fail(c, PX_EINVAL, "multigrid needs even nx and ny (got %d x %d)", f.nx, f.ny);
  if (ncycles < 0 || nu1 < 0 || nu2 < 0 || coarse_sweeps < 0 || max_levels < 0)
    return fail(c, PX_EINVAL, "negative ncycles, nu1, nu2, coarse_sweeps or max_levels");
  if (!std::isfinite(omega)) return fail(c, PX_EINVAL, "omega must be finite");
  const bool empty = f.nx == 0 || f.ny == 0;
  const size_t span = field_span(f);
  const size_t nrep = resid_dev ? (size_t)ncycles + 1 : 0;
  if (!empty) {
    if (!phi || !rho) return fail(c, PX_EINVAL, "NULL field pointer");
    if (overlap(rho, phi, span)) return fail(c, PX_EINVAL, "rho overlaps phi");
    if (resid_dev && overlap2(resid_dev, sizeof(double) * nrep, phi, span))
      return fail(c, PX_EINVAL, "resid_dev overlaps phi");
  }
  // levels: halve both extents while both halves stay even
  std::vector<px::FieldDesc> lv(1, f);
  while (!empty && lv.back().nx % 4 == 0 && lv.back().ny % 4 == 0 &&
         (max_levels == 0 || (int)lv.size() < max_levels)) {
    px::FieldDesc q = lv.back();
    q.nx /= 2;
    q.ny /= 2;
    q.ld = q.nx;
    q.off = 0;
    q.h *= 2.0;
    lv.push_back(q);
  }
  const int L = (int)lv.size();
  const int nc = std::max(lv.back().nx, lv.back().ny);
  const int cs = coarse_sweeps > 0 ? coarse_sweeps : (nc <= 2 ? 1 : 2 * nc * nc);
  DeviceScope ds(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (resid_dev) {
    cudaError_t e = cudaMemsetAsync(resid_dev, 0, sizeof(double) * nrep, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "clear resid_dev");
  }
  if (empty) return PX_OK;
  // buffers: level 0 is phi, the context scratch and rho; every coarser level
  // has its right-hand side r and two states, 256-byte aligned
  s = ensure_scratch(c, span);
  if (s != PX_OK) return s;
  const size_t es = f.dtype == 0 ? 8 : 4;
  auto level_bytes = [&](int l) {
    return ((size_t)lv[l].nx * lv[l].ny * es + 255) & ~(size_t)255;
  };
  size_t total = 0;
  for (int l = 1; l < L; ++l) total += 3 * level_bytes(l);
  if (total > c->mg_bytes) {
    if (c->mg) cudaFree(c->mg);
    c->mg = nullptr;
    c->mg_bytes = 0;
    cudaError_t e = cudaMalloc(&c->mg, total);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(c, PX_ENOMEM, "multigrid levels of %zu bytes: %s", total, cudaGetErrorString(e));
    }
    c->mg_bytes = total;
  }
  std::vector<void*> A(L), B(L), R(L), cur(L);
  A[0] = phi;
  B[0] = c->scratch;
  R[0] = const_cast<void*>(rho);
  char* base = (char*)c->mg;
  for (int l = 1; l < L; ++l) {
    const size_t one = level_bytes(l);
    R[l] = base;
    A[l] = base + one;
    B[l] = base + 2 * one;
    base += 3 * one;
  }
  auto chk = [&](cudaError_t e) -> px_status {
    return e == cudaSuccess ? PX_OK : cuda_fail(c, e, "multigrid launch");
  };
  for (int k = 0; k < ncycles; ++k) {
    double* rep = resid_dev ? resid_dev + k : nullptr;  // residual of the cycle's input
    cur[0] = phi;
    for (int l = 0; l + 1 < L; ++l) {
      double* pre = l == 0 && nu1 > 0 ? rep : nullptr;
      s = chk(rb_sweeps_ab(c, lv[l], A[l], B[l], &cur[l], R[l], omega, nu1, pre, st));
      if (s != PX_OK) return s;
      double* rr = l == 0 && nu1 == 0 ? rep : nullptr;
      s = chk(px::launch_mg_restrict(lv[l], cur[l], R[l], R[l + 1], A[l + 1], lv[l + 1].ld, rr,
                                     st));
      if (s != PX_OK) return s;
      cur[l + 1] = A[l + 1];
    }
    s = chk(rb_sweeps_ab(c, lv[L - 1], A[L - 1], B[L - 1], &cur[L - 1], R[L - 1], omega, cs,
                         L == 1 ? rep : nullptr, st));
    if (s != PX_OK) return s;
    for (int l = L - 2; l >= 0; --l) {
      // on levels that the FP32 register wavefront smooths, the interpolation
      // and correction ride in the first post-smoothing launch's loads (one
      // read and one write of the level fewer); elsewhere a pass of their own
      const bool fold = nu2 > 0 && c->opt_mg_prolong != 1 && lv[l].dtype == 1 &&
                        px::vector_ok(lv[l], A[l], B[l], R[l]);
      const px::Prolong pl{(const float*)cur[l + 1], lv[l + 1].ld, lv[l + 1].nx, lv[l + 1].ny};
      if (!fold) {
        s = chk(px::launch_mg_prolong(lv[l], cur[l + 1], lv[l + 1].ld, cur[l], st));
        if (s != PX_OK) return s;
      }
      s = chk(rb_sweeps_ab(c, lv[l], A[l], B[l], &cur[l], R[l], omega, nu2, nullptr, st,
                           fold ? &pl : nullptr));
      if (s != PX_OK) return s;
    }
    if (cur[0] != phi) {
      s = chk(px::launch_copy_field(f, cur[0], phi, st));
      if (s != PX_OK) return s;
    }
  }
  if (resid_dev) {
    // the final state's residual in the storage precision: the residual and
    // restriction pass (its coarse outputs land in level-1 buffers that no
    // one reads), or, on a single level, the FP64 residual pass
    if (L >= 2) {
      s = chk(px::launch_mg_restrict(f, phi, rho, R[1], A[1], lv[1].ld, resid_dev + ncycles, st));
      if (s != PX_OK) return s;
    } else {
      s = chk(px::launch_residual_norm(f, phi, rho, c->red, st));
      if (s != PX_OK) return s;
      cudaError_t e = cudaMemcpyAsync(resid_dev + ncycles, c->red, sizeof(double),
                                      cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return cuda_fail(c, e, "copy final residual");
    }
  }
  return PX_OK;
}

px_status px_relax3_n(px_ctx* c, const px_grid3* g, const void* phi_in, void* phi_out,
                      const void* rho, double omega, int nsweeps, double* resid_dev,
                      int report_every, void* stream) {
  PX_NVTX_RANGE("px_relax3_n");
  if (!c) return PX_EINVAL;
  c->err.clear();
  if (!g) return fail(c, PX_EINVAL, "grid is NULL");
  if (g->dtype != PX_F64 && g->dtype != PX_F32)
    return fail(c, PX_EINVAL, "dtype %d is not PX_F64 or PX_F32", (int)g->dtype);
  if (g->nx < 0 || g->ny < 0 || g->nz < 0)
    return fail(c, PX_EINVAL, "negative extent %d x %d x %d", g->nx, g->ny, g->nz);
  if (g->nx > (1 << 29) || g->ny > (1 << 22) || g->nz > (1 << 22))
    return fail(c, PX_EINVAL, "extent %d x %d x %d too large", g->nx, g->ny, g->nz);
  if (g->ld < g->nx) return fail(c, PX_EINVAL, "ld %lld < nx", (long long)g->ld);
  if (g->ny > 0 && g->lp < (int64_t)(g->ny - 1) * g->ld + g->nx)
    return fail(c, PX_EINVAL, "lp %lld < (ny - 1) * ld + nx", (long long)g->lp);
  if (!(std::isfinite(g->h) && g->h > 0.0) || !std::isfinite(1.0 / (g->h * g->h)))
    return fail(c, PX_EINVAL, "h must be finite and > 0 with a finite 1/h^2");
  if (nsweeps < 0 || report_every < 0) return fail(c, PX_EINVAL, "negative nsweeps or report_every");
  if (!std::isfinite(omega)) return fail(c, PX_EINVAL, "omega must be finite");
  px::Field3 f{g->nx, g->ny, g->nz, g->ld, g->lp, g->dtype, g->h};
  const bool empty = f.nx == 0 || f.ny == 0 || f.nz == 0;
  const size_t es = elem_size(g->dtype);
  const double spand = empty ? 0.0 : ((double)(f.nz - 1) * f.lp + (double)(f.ny - 1) * f.ld + f.nx) * es;
  if (spand > 9.0e18) return fail(c, PX_EINVAL, "field too large");
  const size_t span = (size_t)spand;
  const bool reports = resid_dev && report_every > 0 && nsweeps > 0;
  const int nrep = reports ? (nsweeps + report_every - 1) / report_every : 0;
  const bool inplace = phi_in == phi_out;
  if (!empty) {
    if (!phi_in || !phi_out || !rho) return fail(c, PX_EINVAL, "NULL field pointer");
    if (!inplace && overlap(phi_in, phi_out, span))
      return fail(c, PX_EINVAL, "phi_in and phi_out overlap without being equal");
    if (overlap(rho, phi_out, span)) return fail(c, PX_EINVAL, "rho overlaps phi_out");
    if (reports && overlap2(resid_dev, sizeof(double) * (size_t)nrep, phi_out, span))
      return fail(c, PX_EINVAL, "resid_dev overlaps phi_out");
  }
  DeviceScope ds(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (reports) {
    cudaError_t e = cudaMemsetAsync(resid_dev, 0, sizeof(double) * (size_t)nrep, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "clear resid_dev");
  }
  if (empty) return PX_OK;
  if (nsweeps == 0) {
    if (inplace) return PX_OK;
    cudaError_t e = px::launch_copy3(f, phi_in, phi_out, st);
    return e == cudaSuccess ? PX_OK : cuda_fail(c, e, "copy launch");
  }
  // sweeps alternate between phi_out and scratch: out of place so that the
  // last lands in phi_out, in place starting with scratch (an odd count ends
  // with a copy back)
  if (inplace || nsweeps >= 2) {
    px_status s = ensure_scratch(c, span);
    if (s != PX_OK) return s;
  }
  void* scratch = c->scratch;
  const bool vec = px::vector_ok3(f, phi_in, phi_out, rho) &&
                   (!scratch || px::vector_ok3(f, scratch, scratch, scratch));
  const void* src = phi_in;
  for (int k = 0; k < nsweeps; ++k) {
    void* dst = inplace ? (k % 2 == 0 ? scratch : phi_out)
                        : ((nsweeps - 1 - k) % 2 == 0 ? phi_out : scratch);
    double* slot = reports && k % report_every == 0 ? resid_dev + k / report_every : nullptr;
    cudaError_t e = px::launch_relax3(f, src, dst, rho, omega, vec, slot, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "3D relax launch");
    src = dst;
  }
  if (src != phi_out) {
    cudaError_t e = px::launch_copy3(f, src, phi_out, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "copy launch");
  }
  return PX_OK;
}

px_status px_relax_plan(px_ctx* c, const px_grid* g, const void* phi_in,
                        const void* phi_out, const void* rho, int nsweeps, int tblock,
                        int* tblock_used, int* launches) {
  if (!c) return PX_EINVAL;
  c->err.clear();
  px::FieldDesc f;
  px_status s = check_grid(c, g, &f);
  if (s != PX_OK) return s;
  if (nsweeps < 0 || tblock < 0 || tblock > 8) return fail(c, PX_EINVAL, "bad nsweeps/tblock");
  const bool vec = px::vector_ok(f, phi_in, phi_out, rho);
  bool copy_first = false;
  std::vector<int> sizes = plan_launches(f, vec, phi_in == phi_out, nsweeps, tblock, &copy_first);
  int tb = 0;
  for (int v : sizes) tb = v > tb ? v : tb;
  if (tblock_used) *tblock_used = tb;
  if (launches) *launches = (int)sizes.size();
  return PX_OK;
}

px_status px_residual_norm_async(px_ctx* c, const px_grid* g, const void* phi,
                                 const void* rho, double* out_dev, void* stream) {
  PX_NVTX_RANGE("px_residual_norm_async");
  if (!c) return PX_EINVAL;
  c->err.clear();
  px::FieldDesc f;
  px_status s = check_grid(c, g, &f);
  if (s != PX_OK) return s;
  if (!out_dev) return fail(c, PX_EINVAL, "out_dev is NULL");
  if ((f.nx && f.ny) && (!phi || !rho)) return fail(c, PX_EINVAL, "NULL field pointer");
  DeviceScope ds(c->device);
  cudaError_t e = px::launch_residual_norm(f, phi, rho, out_dev, (cudaStream_t)stream);
  return e == cudaSuccess ? PX_OK : cuda_fail(c, e, "residual_norm launch");
}

px_status px_residual_norm(px_ctx* c, const px_grid* g, const void* phi, const void* rho,
                           double* out_host, double* rho_norm_host, void* stream) {
  PX_NVTX_RANGE("px_residual_norm");
  if (!c) return PX_EINVAL;
  if (!out_host) return fail(c, PX_EINVAL, "out_host is NULL");
  px_status s = px_residual_norm_async(c, g, phi, rho, c->red, stream);
  if (s != PX_OK) return s;
  DeviceScope ds(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(c->red_host, c->red, 2 * sizeof(double),
                                  cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(c, e, "residual_norm sync");
  *out_host = c->red_host[0];
  if (rho_norm_host) *rho_norm_host = c->red_host[1];
  return PX_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// 2D Euler finite-volume steps (euler.cu).
namespace {

px_status check_euler(px_ctx* c, const px_euler_grid* g, px::EulerDesc* d) {
  if (!g) return fail(c, PX_EINVAL, "grid is NULL");
  if (g->dtype != PX_F64 && g->dtype != PX_F32)
    return fail(c, PX_EINVAL, "dtype %d is not PX_F64 or PX_F32", (int)g->dtype);
  if (g->nx < 0 || g->ny < 0 || g->nx > (1 << 29) || g->ny > (1 << 29))
    return fail(c, PX_EINVAL, "extent %d x %d not in 0..2^29", g->nx, g->ny);
  if (g->ld < g->nx) return fail(c, PX_EINVAL, "ld %lld < nx", (long long)g->ld);
  const int64_t plane = g->ny > 0 ? (int64_t)(g->ny - 1) * g->ld + g->nx : 0;
  if (g->cs < plane) return fail(c, PX_EINVAL, "cs %lld < (ny - 1) * ld + nx", (long long)g->cs);
  if (!(std::isfinite(g->dx) && g->dx > 0 && std::isfinite(g->dy) && g->dy > 0))
    return fail(c, PX_EINVAL, "dx and dy must be finite and > 0");
  if ((double)g->cs * 4.0 * elem_size(g->dtype) > 9.0e18) return fail(c, PX_EINVAL, "field too large");
  d->nx = g->nx;
  d->ny = g->ny;
  d->ld = g->ld;
  d->cs = g->cs;
  d->dtype = g->dtype;
  d->dx = g->dx;
  d->dy = g->dy;
  return PX_OK;
}

size_t euler_span(const px::EulerDesc& d) {
  if (d.nx == 0 || d.ny == 0) return 0;
  return (size_t)((3 * d.cs + (int64_t)(d.ny - 1) * d.ld + d.nx) * (int64_t)elem_size(d.dtype));
}

}  // namespace

extern "C" {

px_status px_euler_step(px_ctx* c, const px_euler_grid* g, const void* u_in, void* u_out,
                        double gamma, double cfl, int nsteps, double dt_fixed, double* dt_dev,
                        void* stream) {
  PX_NVTX_RANGE("px_euler_step");
  if (!c) return PX_EINVAL;
  c->err.clear();
  px::EulerDesc d;
  px_status s = check_euler(c, g, &d);
  if (s != PX_OK) return s;
  if (!(std::isfinite(gamma) && gamma > 1.0)) return fail(c, PX_EINVAL, "gamma must be > 1");
  if (nsteps < 0) return fail(c, PX_EINVAL, "nsteps %d < 0", nsteps);
  if (!(std::isfinite(dt_fixed) && dt_fixed >= 0.0)) return fail(c, PX_EINVAL, "dt_fixed must be >= 0");
  if (dt_fixed == 0.0 && !(std::isfinite(cfl) && cfl > 0.0))
    return fail(c, PX_EINVAL, "cfl must be finite and > 0 when dt_fixed is 0");
  const size_t span = euler_span(d);
  if (span == 0 || nsteps == 0) {
    if (span > 0 && u_in != u_out) {
      if (!u_in || !u_out) return fail(c, PX_EINVAL, "NULL field pointer");
      if (overlap(u_in, u_out, span)) return fail(c, PX_EINVAL, "u_in and u_out overlap");
      DeviceScope ds(c->device);
      cudaError_t e = cudaMemcpyAsync(u_out, u_in, span, cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "copy");
    }
    return PX_OK;
  }
  if (!u_in || !u_out) return fail(c, PX_EINVAL, "NULL field pointer");
  if (u_in != u_out && overlap(u_in, u_out, span))
    return fail(c, PX_EINVAL, "u_in and u_out overlap without being equal");
  if (dt_dev && overlap2(dt_dev, sizeof(double) * (size_t)nsteps, u_out, span))
    return fail(c, PX_EINVAL, "dt_dev overlaps u_out");
  DeviceScope ds(c->device);
  s = ensure_scratch(c, span);
  if (s != PX_OK) return s;
  if (!c->ewave) {
    cudaError_t e = cudaMalloc(&c->ewave, 2 * sizeof(double));
    if (e != cudaSuccess) {
      c->ewave = nullptr;
      return cuda_fail(c, e, "wave-speed slots");
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  const bool adaptive = dt_fixed == 0.0;
  if (adaptive) {
    cudaError_t e = cudaMemsetAsync(c->ewave, 0, sizeof(double), st);
    if (e == cudaSuccess) e = px::launch_euler_wave(d, u_in, gamma, c->ewave, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "wave-speed launch");
  }
  const void* src = u_in;
  for (int k = 0; k < nsteps; ++k) {
    double* cur = adaptive ? c->ewave + (k & 1) : nullptr;
    double* next = adaptive ? c->ewave + ((k + 1) & 1) : nullptr;
    cudaError_t e = px::launch_euler_step(d, src, u_out, c->scratch, gamma, cfl, dt_fixed, cur,
                                          next, dt_dev ? dt_dev + k : nullptr, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "Euler step launch");
    src = u_out;
  }
  return PX_OK;
}

px_status px_euler_conserved(px_ctx* c, const px_euler_grid* g, const void* w, void* u,
                             double gamma, void* stream) {
  PX_NVTX_RANGE("px_euler_conserved");
  if (!c) return PX_EINVAL;
  c->err.clear();
  px::EulerDesc d;
  px_status s = check_euler(c, g, &d);
  if (s != PX_OK) return s;
  if (!(std::isfinite(gamma) && gamma > 1.0)) return fail(c, PX_EINVAL, "gamma must be > 1");
  const size_t span = euler_span(d);
  if (span == 0) return PX_OK;
  if (!w || !u) return fail(c, PX_EINVAL, "NULL field pointer");
  if (overlap(w, u, span)) return fail(c, PX_EINVAL, "w and u overlap");
  DeviceScope ds(c->device);
  cudaError_t e = px::launch_euler_conserved(d, w, u, gamma, (cudaStream_t)stream);
  return e == cudaSuccess ? PX_OK : cuda_fail(c, e, "conversion launch");
}

}  // extern "C"

// ---------------------------------------------------------------------------
namespace {

px_status sync_norms(px_ctx* c, const px::FieldDesc& f, const void* phi, const void* rho,
                     cudaStream_t st, double* R, double* P) {
  cudaError_t e = px::launch_residual_norm(f, phi, rho, c->red, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->red_host, c->red, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(c, e, "solve residual check");
  *R = c->red_host[0];
  *P = c->red_host[1];
  return PX_OK;
}

}  // namespace

extern "C" px_status px_solve(px_ctx* c, const px_grid* g, void* phi, const void* rho,
                              const px_solve_opts* o, px_solve_info* info, void* stream) {
  PX_NVTX_RANGE("px_solve");
  if (!c) return PX_EINVAL;
  c->err.clear();
  const auto t0 = std::chrono::steady_clock::now();
  px::FieldDesc f;
  px_status s = check_grid(c, g, &f);
  if (s != PX_OK) return s;
  if (!o) return fail(c, PX_EINVAL, "opts is NULL");
  if (o->mode != PX_SOLVE_PLAIN && o->mode != PX_SOLVE_REFINE)
    return fail(c, PX_EINVAL, "unknown solve mode %d", o->mode);
  if (o->mode == PX_SOLVE_REFINE && f.dtype != PX_F64)
    return fail(c, PX_EINVAL, "refinement needs FP64 phi and rho");
  if (!std::isfinite(o->omega) || !(o->rtol >= 0.0) || o->max_sweeps < 0 ||
      o->tblock < 0 || o->tblock > 8 || o->timeout_ms < 0 || o->reserved != 0)
    return fail(c, PX_EINVAL, "bad solve options");
  if (o->mode == PX_SOLVE_PLAIN && o->check_every <= 0)
    return fail(c, PX_EINVAL, "check_every must be > 0");
  if (o->mode == PX_SOLVE_REFINE && o->inner_sweeps <= 0)
    return fail(c, PX_EINVAL, "inner_sweeps must be > 0");
  if (f.nx == 0 || f.ny == 0) {
    if (info) *info = px_solve_info{0, 0, 0, 0.0, 0.0};
    return PX_OK;
  }
  if (!phi || !rho) return fail(c, PX_EINVAL, "NULL field pointer");
  const size_t span = field_span(f);
  if (overlap(phi, rho, span)) return fail(c, PX_EINVAL, "phi and rho overlap");
  DeviceScope ds(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  px_solve_info inf{0, 0, 0, 0.0, 0.0};
  auto finish = [&](px_status rc) {
    inf.wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                      .count();
    if (info) *info = inf;
    return rc;
  };

  if (o->check_mean) {
    cudaError_t e = px::launch_field_sum(f, rho, c->red + 8, c->red + 3, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->red_host + 3, c->red + 3, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return finish(cuda_fail(c, e, "mean of rho"));
    double R = 0, P = 0;
    s = sync_norms(c, f, phi, rho, st, &R, &P);
    if (s != PX_OK) return finish(s);
    const double mean = c->red_host[3] / ((double)f.nx * (double)f.ny);
    if (!(std::fabs(mean) <= 1e-12 * P))
      return finish(fail(c, PX_EMEAN, "mean of rho %.3e exceeds 1e-12 * ||rho||_inf (%.3e)", mean, P));
  }

  // REFINE workspace: two unghosted FP32 fields with a 16-byte aligned pitch.
  const int64_t ld32 = ((int64_t)f.nx + 3) / 4 * 4;
  px_grid g32{f.nx, f.ny, ld32, 0, PX_F32, f.h};
  float *r32 = nullptr, *e32 = nullptr;
  if (o->mode == PX_SOLVE_REFINE) {
    const size_t one = (size_t)ld32 * (size_t)f.ny * sizeof(float);
    const size_t need = 2 * ((one + 255) / 256 * 256);
    if (c->ws_bytes < need) {
      if (c->ws) cudaFree(c->ws);
      c->ws = nullptr;
      c->ws_bytes = 0;
      cudaError_t e = cudaMalloc(&c->ws, need);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return finish(fail(c, PX_ENOMEM, "solve workspace of %zu bytes", need));
      }
      c->ws_bytes = need;
    }
    r32 = (float*)c->ws;
    e32 = (float*)((char*)c->ws + need / 2);
  }

  // After one plain launch of a block (which allocates any scratch), a full
  // block (PLAIN: check_every sweeps; REFINE: one cycle) is captured once on a
  // private stream into a CUDA graph and replayed on the caller's stream.
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int blocks_done = 0;
  struct GraphGuard {
    cudaStream_t* s; cudaGraph_t* g; cudaGraphExec_t* x;
    ~GraphGuard() {
      if (*x) cudaGraphExecDestroy(*x);
      if (*g) cudaGraphDestroy(*g);
      if (*s) cudaStreamDestroy(*s);
    }
  } guard{&cap, &graph, &gexec};
  const int full = o->mode == PX_SOLVE_PLAIN ? o->check_every : o->inner_sweeps;
  auto enqueue_block = [&](cudaStream_t qs, int n) -> px_status {
    if (o->mode == PX_SOLVE_PLAIN)
      return px_relax_n(c, g, phi, phi, rho, o->omega, n, o->tblock, nullptr, 0, qs);
    cudaError_t e = px::launch_refine_residual(f, phi, rho, c->red, r32, e32, ld32, c->red + 2, qs);
    if (e != cudaSuccess) return cuda_fail(c, e, "refine residual");
    px_status s2 = px_relax_n(c, &g32, e32, e32, r32, o->omega, n, o->tblock, nullptr, 0, qs);
    if (s2 != PX_OK) return s2;
    e = px::launch_refine_update(f, phi, e32, ld32, c->red + 2, qs);
    return e == cudaSuccess ? PX_OK : cuda_fail(c, e, "refine update");
  };
  auto run_block = [&](int n) -> px_status {
    if (n != full || blocks_done == 0) {
      ++blocks_done;
      return enqueue_block(st, n);
    }
    if (!gexec) {
      cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return cuda_fail(c, e, "solve graph capture");
      px_status s2 = enqueue_block(cap, n);
      e = cudaStreamEndCapture(cap, &graph);
      if (s2 != PX_OK) return s2;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&gexec, graph, 0);
      if (e != cudaSuccess) return cuda_fail(c, e, "solve graph instantiate");
    }
    ++blocks_done;
    cudaError_t e = cudaGraphLaunch(gexec, st);
    return e == cudaSuccess ? PX_OK : cuda_fail(c, e, "solve graph launch");
  };

  const double inf_d = std::numeric_limits<double>::infinity();
  for (;;) {
    double R = 0, P = 0;
    s = sync_norms(c, f, phi, rho, st, &R, &P);
    if (s != PX_OK) return finish(s);
    inf.checks++;
    inf.rel_resid = P > 0 ? R / P : (R == 0 ? 0.0 : inf_d);
    if (!std::isfinite(R) || !std::isfinite(P))
      return finish(fail(c, PX_ENAN, "residual is %g (rho norm %g)", R, P));
    if (inf.rel_resid <= o->rtol || R == 0.0) return finish(PX_OK);
    if (inf.sweeps >= o->max_sweeps)
      return finish(fail(c, PX_ENOCONV, "%lld sweeps, relative residual %.3e > %.3e",
                         (long long)inf.sweeps, inf.rel_resid, o->rtol));
    if (o->timeout_ms > 0) {
      const double ms = std::chrono::duration<double, std::milli>(
                            std::chrono::steady_clock::now() - t0).count();
      if (ms > (double)o->timeout_ms)
        return finish(fail(c, PX_ETIMEOUT, "timeout after %.0f ms", ms));
    }
    const int64_t left = o->max_sweeps - inf.sweeps;
    const int n = (int)std::min<int64_t>(full, left);
    s = run_block(n);
    if (s != PX_OK) return finish(s);
    inf.sweeps += n;
    if (o->mode == PX_SOLVE_REFINE) inf.cycles++;
  }
}

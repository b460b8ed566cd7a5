// px_relax_n_static: the fused relaxation of px_relax_n for callers that must
// not allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is off limits or unsafe, for
// example a real-time loop that may not block on the allocator, an
// application whose own pool owns all device memory, or a plug-in that may
// not create library contexts (px_create allocates). Such a caller still
// passes its own phi_in, phi_out, rho and report buffers; the only working
// memory the sweeps need beyond them, the ping-pong field of a multi-launch
// relax, comes from the fixed array below.
//
// The array lives in this library's device image, so every GPU on which the
// library's kernels are loaded holds its 16 MiB until the process exits. Host
// code may not use its name as a pointer (on the host it names a stand-in, not
// device memory), so its device address is looked up with
// cudaGetSymbolAddress while that device is current, and cached per device
// together with the identity of the device's current context: a context that
// was destroyed and recreated (cudaDeviceReset) gets a fresh lookup instead
// of a stale address.
#include "px_internal.cuh"

#include <cuda.h>

#include <cmath>
#include <cstdio>
#include <mutex>

namespace {

constexpr size_t kStaticScratchBytes = (size_t)16 << 20;  // 16 MiB

static __device__ __align__(256) unsigned char px_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_ptr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};  // context id the address belongs to

// Unique id of the calling thread's current context (never reused within a
// process), through the driver entry points the runtime resolves; 0 if the
// driver does not provide them, in which case the address is looked up on
// every call.
unsigned long long current_ctx_id() {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool resolved = false;
  if (!resolved) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
    cudaGetLastError();
    resolved = true;
  }
  if (!get_current || !get_id) return 0;
  CUcontext cx = nullptr;
  unsigned long long id = 0;
  if (get_current(&cx) != CUDA_SUCCESS || !cx || get_id(cx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of the static scratch on the current device, looked up on the
// first call for that device and context.
px_status static_scratch(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return px::unbound_fail(PX_ECUDA, "px_relax_n_static: no current CUDA device");
  }
  if (dev < 0 || dev >= kMaxDevices)
    return px::unbound_fail(PX_EUNSUPPORTED, "px_relax_n_static: device index above 63");
  std::lock_guard<std::mutex> lock(g_setup_mu);
  const unsigned long long cid = current_ctx_id();
  if (!g_scratch_ptr[dev] || cid == 0 || cid != g_scratch_ctx[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, px_static_scratch);  // binds the primary context if none is
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      char msg[256];
      snprintf(msg, sizeof msg, "px_relax_n_static: cudaGetSymbolAddress failed: %s",
               cudaGetErrorString(e));
      return px::unbound_fail(PX_ECUDA, msg);
    }
    g_scratch_ptr[dev] = p;
    g_scratch_ctx[dev] = cid != 0 ? cid : current_ctx_id();
  }
  *out = g_scratch_ptr[dev];
  return PX_OK;
}

px_status launch_error(cudaError_t e, const char* what) {
  cudaGetLastError();
  char msg[256];
  snprintf(msg, sizeof msg, "px_relax_n_static: %s: %s", what, cudaGetErrorString(e));
  return px::unbound_fail(PX_ECUDA, msg);
}

}  // namespace

extern "C" px_status px_relax_n_static(const px_grid* g, const void* phi_in, void* phi_out,
                                       const void* rho, double omega, int nsweeps,
                                       int tblock, double* resid_dev, int report_every,
                                       void* stream) {
  PX_NVTX_RANGE("px_relax_n_static");
  px::unbound_clear();
  px::FieldDesc f;
  px_status s = px::unbound_check_grid(g, &f);
  if (s != PX_OK) return s;
  const size_t span = px::field_bytes(f);
  if (span > kStaticScratchBytes) {
    char msg[256];
    snprintf(msg, sizeof msg,
             "px_relax_n_static: the field spans %zu bytes but the static scratch holds "
             "%zu bytes (16 MiB); use px_relax_n for larger fields",
             span, kStaticScratchBytes);
    return px::unbound_fail(PX_EINVAL, msg);
  }
  if (nsweeps < 0 || report_every < 0 || tblock < 0 || tblock > 8 || !std::isfinite(omega))
    return px::unbound_fail(PX_EINVAL,
                            "px_relax_n_static: need nsweeps >= 0, report_every >= 0, "
                            "tblock in 0..8 and a finite omega");
  const bool reports = resid_dev && report_every > 0 && nsweeps > 0;
  const int nrep = reports ? (nsweeps + report_every - 1) / report_every : 0;
  const bool empty = f.nx == 0 || f.ny == 0;
  const bool inplace = phi_in == phi_out;
  if (!empty) {
    if (!phi_in || !phi_out || !rho)
      return px::unbound_fail(PX_EINVAL, "px_relax_n_static: NULL field pointer");
    if (!inplace && px::ranges_overlap(phi_in, phi_out, span))
      return px::unbound_fail(PX_EINVAL,
                              "px_relax_n_static: phi_in and phi_out overlap without being equal");
    if (px::ranges_overlap(rho, phi_out, span))
      return px::unbound_fail(PX_EINVAL, "px_relax_n_static: rho overlaps phi_out");
    if (reports && px::ranges_overlap2(resid_dev, sizeof(double) * (size_t)nrep, phi_out, span))
      return px::unbound_fail(PX_EINVAL, "px_relax_n_static: resid_dev overlaps phi_out");
  }
  void* scratch = nullptr;
  s = static_scratch(&scratch);
  if (s != PX_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  if (reports) {
    cudaError_t e = cudaMemsetAsync(resid_dev, 0, sizeof(double) * (size_t)nrep, st);
    if (e != cudaSuccess) return launch_error(e, "clear resid_dev");
  }
  if (empty) return PX_OK;

  if (nsweeps == 0) {
    if (inplace) return PX_OK;
    cudaError_t e = px::launch_copy_field(f, phi_in, phi_out, st);
    return e == cudaSuccess ? PX_OK : launch_error(e, "copy launch");
  }
  // The scratch field takes the caller's layout (pitch and ghost offset); the
  // array's 256-byte alignment keeps the vector path available. Nothing in it
  // must start at zero: every cell a launch reads from it was written by the
  // launch before.
  const bool vec = px::vector_ok(f, phi_in, phi_out, rho) &&
                   px::vector_ok(f, scratch, scratch, scratch);
  bool copy_first = false;
  const std::vector<int> sizes =
      px::plan_relax_launches(f, vec, inplace, nsweeps, tblock, &copy_first);
  const size_t L = sizes.size();
  const void* src = phi_in;
  if (copy_first) {
    cudaError_t e = px::launch_copy_field(f, phi_in, scratch, st);
    if (e != cudaSuccess) return launch_error(e, "copy launch");
    src = scratch;
  }
  int s0 = 0;
  for (size_t k = 0; k < L; ++k) {
    void* dst = ((L - 1 - k) % 2 == 0) ? phi_out : scratch;
    cudaError_t e = px::launch_relax(f, src, dst, rho, omega, sizes[k], vec,
                                     reports ? resid_dev : nullptr, s0, report_every,
                                     nullptr, 0, st);
    if (e != cudaSuccess) return launch_error(e, "relax launch");
    s0 += sizes[k];
    src = dst;
  }
  return PX_OK;
}

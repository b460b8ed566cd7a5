// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

namespace px {

// NVTX range around a library call (header-only NVTX: no effect and no
// library dependency unless a profiler attaches), named after the call.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
#define PX_NVTX_RANGE(name) ::px::NvtxRange px_nvtx_range_(name)

constexpr int kWarp = 32;

// Bounds checks of the checked build (compiled with -DPX_CHECKED; the
// sanitizer's stand-in): an index outside [lo, hi) is counted in a device
// word, the first one recorded (site << 48 | index), and the access skipped.
// In the normal build the check is the constant true and costs nothing.
#ifdef PX_CHECKED
extern __device__ unsigned long long g_px_checked[2];
__device__ __forceinline__ bool in_range(int site, int64_t v, int64_t lo, int64_t hi) {
  if (v >= lo && v < hi) return true;
  if (atomicAdd(&g_px_checked[0], 1ull) == 0ull)
    g_px_checked[1] = ((unsigned long long)site << 48) | ((unsigned long long)v & 0xffffffffffffull);
  return false;
}
#define PX_IN_RANGE(site, v, lo, hi) ::px::in_range((site), (int64_t)(v), (int64_t)(lo), (int64_t)(hi))
#else
#define PX_IN_RANGE(site, v, lo, hi) true
#endif

// Periodic index for i in [-n, 2n).
__device__ __forceinline__ int wrap1(int i, int n) {
  return i < 0 ? i + n : (i >= n ? i - n : i);
}
// Periodic index for any i.
__device__ __forceinline__ int wrapn(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

// Non-negative floats / doubles (and +NaN) order like their bit patterns read
// as unsigned integers, so a max-norm reduces with integer max.
// |v| as bits by clearing the sign bit on the integer pipe (keeps the FP64 pipe,
// the bound of the FP64 sweep, free of the residual's absolute value). The mask
// is inline PTX: written in C++ the compiler recognises it as a floating-point
// absolute value, and for doubles that costs one FP64-pipe operation per cell
// (measured: 4 DADD + 3 DFMA per reported cell update instead of 3 + 3).
__device__ __forceinline__ uint32_t absbits(float v) {
  uint32_t b;
  asm("and.b32 %0, %1, 0x7fffffff;" : "=r"(b) : "r"(__float_as_uint(v)));
  return b;
}
__device__ __forceinline__ uint64_t absbits(double v) {
  uint64_t b;
  asm("and.b64 %0, %1, 0x7fffffffffffffff;" : "=l"(b) : "l"(__double_as_longlong(v)));
  return b;
}
__device__ __forceinline__ uint32_t umax(uint32_t a, uint32_t b) { return a > b ? a : b; }
__device__ __forceinline__ uint64_t umax(uint64_t a, uint64_t b) { return a > b ? a : b; }

__device__ __forceinline__ uint32_t warp_max(uint32_t v) {
  return __reduce_max_sync(0xffffffffu, v);
}
__device__ __forceinline__ uint64_t warp_max(uint64_t v) {
  uint32_t hi = (uint32_t)(v >> 32), lo = (uint32_t)v;
  uint32_t mhi = __reduce_max_sync(0xffffffffu, hi);
  uint32_t mlo = __reduce_max_sync(0xffffffffu, hi == mhi ? lo : 0u);
  return ((uint64_t)mhi << 32) | mlo;
}

// Widen a max-bits value of the storage type to the bits of the equal double.
__device__ __forceinline__ uint64_t to_f64_bits(uint32_t b) {
  return (uint64_t)__double_as_longlong((double)__uint_as_float(b));
}
__device__ __forceinline__ uint64_t to_f64_bits(uint64_t b) { return b; }

__device__ __forceinline__ void atomic_max_bits(double* slot, uint64_t bits) {
  atomicMax(reinterpret_cast<unsigned long long*>(slot), (unsigned long long)bits);
}

template <typename T> struct MaxBits;
template <> struct MaxBits<float> { using type = uint32_t; };
template <> struct MaxBits<double> { using type = uint64_t; };

// Coefficients of one sweep in the storage type:
//   s = (W + E) + (S + N) - 4 C;  r = s / h^2 - rho;  C' = C + c r,  c = omega h^2 / 4.
template <typename T> struct Coef {
  T c;    // omega h^2 / 4
  T ih2;  // 1 / h^2
};

// One launch's residual-report window: state index s0 + t is reported into
// resid[(s0 + t) / every] when every > 0 and (s0 + t) % every == 0.
struct Reports {
  double* resid;
  int s0;
  int every;
  __host__ __device__ __forceinline__ bool due(int t) const {
    return resid != nullptr && ((s0 + t) % every) == 0;
  }
  __host__ __device__ __forceinline__ double* slot(int t) const { return resid + (s0 + t) / every; }
};

// ---------------------------------------------------------------------------
// Host-side launchers (relax.cu, stencil.cu). All return the cudaError_t of
// the launch; arguments were validated by the API layer.
struct FieldDesc {
  int nx, ny;
  int64_t ld;
  int64_t off;   // element offset of interior cell (0, 0)
  int ghost;
  int dtype;     // 0 = f64, 1 = f32
  double h;
  int family = 0;  // FP32 kernel family for depth >= 2 (PX_OPT_FP32_FAMILY; 0 = automatic)
};

// Whether the vectorised kernels may run on this layout / these pointers.
bool vector_ok(const FieldDesc& f, const void* a, const void* b, const void* c);

// One launch of `tb` fused sweeps (tb in 1..8) reading src, writing dst.
// sched: sched_cap zero-initialised 64-bit words for the dynamic load balance
// of the FP32 depth-3/4 kernel (left all-exhausted on exit, so reusable by the
// next launch in stream order), or NULL for static shares.
cudaError_t launch_relax(const FieldDesc& f, const void* src, void* dst,
                         const void* rho, double omega, int tb, bool vec,
                         double* resid, int s0, int every, unsigned long long* sched,
                         int sched_cap, cudaStream_t st);

// One pass of a red-black SOR sweep (rbsor.cu): red_pass = src -> dst with the
// input-state residual folded into *slot (if not NULL); else black cells of
// dst updated in place.
// `sweeps` (1..4) red-black SOR sweeps in one launch of the FP32 register
// wavefront (two stages per sweep: red, then black); src != dst, vector
// layout (vector_ok), nx and ny even. Reports as launch_relax (sweep s0 first).
// Multigrid interpolation folded into a red-black launch of the FP32 register
// wavefront: every input row is corrected by the bilinear interpolation of the
// coarse correction e (nxc x nyc cells, row pitch ldc) as it is loaded, with the
// operations of the separate interpolation pass (so bitwise its result).
struct Prolong {
  const float* e;
  int64_t ldc;
  int nxc, nyc;
};
cudaError_t launch_rbsor_reg(const FieldDesc& f, const float* src, float* dst, const float* rho,
                             double omega, int sweeps, double* resid, int s0, int every,
                             unsigned long long* sched, int sched_cap, cudaStream_t st,
                             const Prolong* pl = nullptr);

// 3D fields (relax3.cu): unghosted, contiguous x, pitches ld (rows) and lp
// (planes) in elements.
struct Field3 {
  int nx, ny, nz;
  int64_t ld, lp;
  int dtype;  // 0 = f64, 1 = f32
  double h;
};
bool vector_ok3(const Field3& f, const void* a, const void* b, const void* c);
// One fused 3D sweep src -> dst (src != dst); folds the input state's
// residual max-norm into *slot when slot is not NULL.
cudaError_t launch_relax3(const Field3& f, const void* src, void* dst, const void* rho,
                          double omega, bool vec, double* slot, cudaStream_t st);
cudaError_t launch_copy3(const Field3& f, const void* src, void* dst, cudaStream_t st);

// Multigrid transfers (mg.cu). launch_mg_restrict: for the fine field f
// (phi, rho), writes the block means of r = rho - L phi to rc and zeros to ec
// (coarse row pitch ldc); folds max |r| into *slot when slot is not NULL.
// launch_mg_prolong: adds the bilinear interpolation of the coarse e (pitch
// ldc) to the fine phi described by f. Both need even nx and ny.
cudaError_t launch_mg_restrict(const FieldDesc& f, const void* phi, const void* rho, void* rc,
                               void* ec, int64_t ldc, double* slot, cudaStream_t st);
cudaError_t launch_mg_prolong(const FieldDesc& f, const void* e, int64_t ldc, void* phi,
                              cudaStream_t st);

cudaError_t launch_rbsor_pass(const FieldDesc& f, const void* src, void* dst, const void* rho,
                              double omega, bool red_pass, bool vec, double* slot,
                              cudaStream_t st);
// One red-black sweep src -> dst (out of place) in one launch: FP64, 16-byte
// vector layouts; bitwise the red pass followed by the black pass.
cudaError_t launch_rbsor_fused(const FieldDesc& f, const double* src, double* dst,
                               const double* rho, double omega, double* slot, cudaStream_t st);

cudaError_t launch_apply_stencil(const FieldDesc& f, const void* phi, void* out,
                                 cudaStream_t st);
// out2[0] = max|rho - L phi| (FP64), out2[1] = max|rho|; out2 zero-filled here.
cudaError_t launch_residual_norm(const FieldDesc& f, const void* phi, const void* rho,
                                 double* out2, cudaStream_t st);
// Copy the interior (and, for ghost layout, refill ghosts) of src into dst.
cudaError_t launch_copy_field(const FieldDesc& f, const void* src, void* dst,
                              cudaStream_t st);

// 2D Euler finite-volume fields (euler.cu): four component planes (rho,
// rho u, rho v, E) of ny rows of nx cells, row pitch ld, plane pitch cs.
struct EulerDesc {
  int nx, ny;
  int64_t ld, cs;
  int dtype;  // 0 = f64, 1 = f32
  double dx, dy;
};
// Max over cells of (|u| + c) / dx + (|v| + c) / dy folded into *slot (atomic max).
cudaError_t launch_euler_wave(const EulerDesc& g, const void* u, double gamma, double* slot,
                              cudaStream_t st);
// One SSP-RK2 step u0 -> out through the stage field s1 (two launches). dt is
// dt_fixed if > 0, else cfl / *wave_cur; stage 1 writes dt to *dt_out (if not
// null) and zeroes *wave_next, stage 2 folds the new state's max wave speed
// into *wave_next (if not null). out may equal u0.
cudaError_t launch_euler_step(const EulerDesc& g, const void* u0, void* out, void* s1, double gamma,
                              double cfl, double dt_fixed, double* wave_cur, double* wave_next,
                              double* dt_out, cudaStream_t st);
// Conserved variables from primitive planes (rho, u, v, p).
cudaError_t launch_euler_conserved(const EulerDesc& g, const void* w, void* u, double gamma,
                                   cudaStream_t st);

int device_sm_count();
// Current device index clamped to 0..63, for the per-device caches of the
// launchers (occupancy, function attributes, symbol addresses).
int dev_index();

// Iterative refinement (stencil.cu). phi/rho FP64 with layout f; r32/e32 are
// unghosted FP32 fields of pitch ld32. norm[0] = ||rho - L phi||_inf > 0.
cudaError_t launch_refine_residual(const FieldDesc& f, const void* phi, const void* rho,
                                   const double* norm, float* r32, float* e32, int64_t ld32,
                                   double* inv_scale, cudaStream_t st);
cudaError_t launch_refine_update(const FieldDesc& f, void* phi, const float* e32, int64_t ld32,
                                 const double* inv_scale, cudaStream_t st);
// Deterministic FP64 sum of a field's interior into *out (partials: sum_partials_count()).
int sum_partials_count();
cudaError_t launch_field_sum(const FieldDesc& f, const void* a, double* partials, double* out,
                             cudaStream_t st);

}  // namespace px

#include <string>
#include <vector>
#include "../../include/protox.h"

// The library context (opaque in the C ABI).
struct px_ctx {
  int device = 0;
  void* scratch = nullptr;   // ping-pong field buffer
  size_t scratch_bytes = 0;
  double* red = nullptr;     // device aux block: [0,1] norms, [2] scale, [3] sum, [8..] partials
  double* red_host = nullptr;  // pinned mirror of red[0..3]
  void* ws = nullptr;        // solve workspace: FP32 r and e fields
  size_t ws_bytes = 0;
  unsigned long long* sched = nullptr;  // load-balance words of the relax kernels
  int sched_cap = 0;
  void* mg = nullptr;        // multigrid levels 1..L-1: right-hand side and two states each
  size_t mg_bytes = 0;
  double* ewave = nullptr;   // Euler: max wave speeds of the current and next state
  int opt_fp32_family = 0;   // PX_OPT_FP32_FAMILY (0 = automatic)
  int opt_rb_sweeps = 0;     // PX_OPT_RB_SWEEPS_PER_LAUNCH (0 = automatic)
  int opt_batch_launches = 0;  // PX_OPT_BATCH_LAUNCHES (0 = automatic, 1 = one launch)
  int opt_rb_fp64_passes = 0;  // PX_OPT_RB_FP64_PASSES (0 = automatic, 1 fused, 2 two passes)
  int opt_mg_prolong = 0;      // PX_OPT_MG_PROLONG (0 = automatic: fused, 1 = separate pass)
  std::string err;
};


namespace px {

// Validation and planning of api.cu, for entry points without a context;
// failures set the message returned by px_last_error(NULL).
px_status unbound_check_grid(const px_grid* g, FieldDesc* f);
px_status unbound_fail(px_status s, const char* msg);
// Clears the calling thread's context-free error message (px_last_error(NULL)).
void unbound_clear();
size_t field_bytes(const FieldDesc& f);
bool ranges_overlap(const void* a, const void* b, size_t n);
bool ranges_overlap2(const void* a, size_t na, const void* b, size_t nb);
std::vector<int> plan_relax_launches(const FieldDesc& f, bool vec, bool inplace, int nsweeps,
                                     int tblock, bool* copy_first);
// Error reporting and grid validation on a context (api.cu).
px_status ctx_fail(px_ctx* c, px_status st, const char* msg);
px_status ctx_check_grid(px_ctx* c, const px_grid* g, FieldDesc* f);

// Batched persistent kernel (batch.cu).
enum { MODE_WHOLE = 0, MODE_BANDED = 1, MODE_BANDED_T = 2 };

struct BInst {
  void* phi;
  const void* rho;
  void* scratch;  // BANDED ping-pong partner
  void* rhos;     // BANDED FP64: the scaled right-hand side -c rho (same layout), or null
  int nx, ny;
  int64_t ld;
  int dtype, mode, ry, tb;  // tb: sweeps per cluster barrier of MODE_BANDED_T
  double c, ih2;
  double a1, w4;  // 1 - omega and omega / 4: the update without the residual
  double* resid;  // this instance's reports, or null
};

struct BParams {
  BInst* inst;
  const int* cl_off;
  const int* cl_items;
  const int* cta_off;
  const int* cta_items;
  int nsweeps, every;
  int csize;  // CTAs per cluster
};

size_t whole_bytes(int nx, int ny, int dtype);
cudaError_t batch_max_clusters(int* n, size_t smem, int csize);
cudaError_t batch_launch(const BParams& p, int nclusters, size_t smem, cudaStream_t st);
int batch_max_cluster_size();
// Whether two CTAs of the batch kernel with `smem` dynamic shared bytes fit on one SM.
bool batch_coresident(size_t smem);
size_t batch_whole_smem();
// Shared bytes of the tiles of a MODE_BANDED_T instance of dtype at depth tb.
size_t banded_t_smem(int dtype, int tb);
// Whether MODE_BANDED_T supports dtype at depth tb (FP32, 4 or 8 sweeps).
bool banded_t_ok(int dtype, int tb);

}  // namespace px

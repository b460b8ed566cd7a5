// Laplacian application, FP64 residual max-norm and periodic field copy.
//
// These run once per solve check rather than once per sweep, so they use one
// thread per cell with a grid-stride loop on any layout (ghosted or not, any
// pitch). The residual norm evaluates in FP64 with the taps summed as
// ((W + E) + (S + N)) - 4 C and r = (s * (1/h^2)) - rho without contraction,
// which reproduces the plain evaluation of the max-norm check of Sec. IV
// (OL rule ||.||_inf with a = h) exactly for FP64 fields.
#include "px_internal.cuh"

#include <algorithm>

namespace px {

namespace {

template <typename T>
__device__ __forceinline__ void store_all_images(T* O, int x, int j, int nx, int ny,
                                                 int64_t ld, int ghost, T v) {
  O[(int64_t)j * ld + x] = v;
  if (!ghost) return;
  int xs[3] = {x, 0, 0}, ys[3] = {j, 0, 0};
  int nxs = 1, nys = 1;
  if (x == 0) xs[nxs++] = nx;
  if (x == nx - 1) xs[nxs++] = -1;
  if (j == 0) ys[nys++] = ny;
  if (j == ny - 1) ys[nys++] = -1;
  for (int a = 0; a < nys; ++a)
    for (int b = 0; b < nxs; ++b)
      if (a | b) O[(int64_t)ys[a] * ld + xs[b]] = v;
}

template <typename T>
__global__ void apply_stencil_k(const T* __restrict__ phi, T* __restrict__ out, int nx,
                                int ny, int64_t ld, int ghost, T ih2) {
  const int64_t n = (int64_t)nx * ny;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(c / nx), i = (int)(c - (int64_t)j * nx);
    const T* row = phi + (int64_t)j * ld;
    const T C = row[i];
    const T W = row[wrap1(i - 1, nx)], E = row[wrap1(i + 1, nx)];
    const T S = phi[(int64_t)wrap1(j - 1, ny) * ld + i];
    const T N = phi[(int64_t)wrap1(j + 1, ny) * ld + i];
    const T s = fma((T)-4, C, (W + E) + (S + N));
    store_all_images<T>(out, i, j, nx, ny, ld, ghost, s * ih2);
  }
}

// A thread owns one column and strides over rows (gridDim.y), so no cell
// index needs a division; the arithmetic is the oracle's FP64 order.
template <typename T>
__global__ void residual_norm_k(const T* __restrict__ phi, const T* __restrict__ rho, int nx,
                                int ny, int64_t ld, double ih2, double* __restrict__ out2) {
  uint64_t mr = 0, mp = 0;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nx) {
    const int iw = i == 0 ? nx - 1 : i - 1, ie = i + 1 == nx ? 0 : i + 1;
    for (int j = blockIdx.y; j < ny; j += gridDim.y) {
      const T* row = phi + (int64_t)j * ld;
      const double C = (double)row[i];
      const double W = (double)row[iw], E = (double)row[ie];
      const double S = (double)phi[(int64_t)(j == 0 ? ny - 1 : j - 1) * ld + i];
      const double N = (double)phi[(int64_t)(j + 1 == ny ? 0 : j + 1) * ld + i];
      const double s = __dsub_rn(__dadd_rn(__dadd_rn(W, E), __dadd_rn(S, N)), __dmul_rn(4.0, C));
      const double rv = (double)rho[(int64_t)j * ld + i];
      const double r = __dsub_rn(__dmul_rn(ih2, s), rv);
      mr = umax(mr, absbits(r));
      mp = umax(mp, absbits(rv));
    }
  }
  __shared__ uint64_t sm[2][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  mr = warp_max(mr);
  mp = warp_max(mp);
  if (lane == 0) { sm[0][warp] = mr; sm[1][warp] = mp; }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t a = 0, b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a = umax(a, sm[0][w]); b = umax(b, sm[1][w]); }
    atomic_max_bits(out2, a);
    atomic_max_bits(out2 + 1, b);
  }
}

template <typename T>
__global__ void copy_field_k(const T* __restrict__ src, T* __restrict__ dst, int nx, int ny,
                             int64_t ld, int ghost) {
  // Writes every cell of the layout: interior, plus ghosts (periodic images)
  // when ghost = 1. Reads only interior cells of src.
  const int wx = nx + 2 * ghost, wy = ny + 2 * ghost;
  const int64_t n = (int64_t)wx * wy;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(c / wx) - ghost, i = (int)(c - (int64_t)(c / wx) * wx) - ghost;
    dst[(int64_t)j * ld + i] = src[(int64_t)wrap1(j, ny) * ld + wrap1(i, nx)];
  }
}

int grid_for(int64_t n, int threads) {
  const int64_t cap = (int64_t)device_sm_count() * 8;
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, cap));
}

}  // namespace

cudaError_t launch_apply_stencil(const FieldDesc& f, const void* phi, void* out,
                                 cudaStream_t st) {
  const int64_t n = (int64_t)f.nx * f.ny;
  const int blocks = grid_for(n, 256);
  const double ih2 = 1.0 / (f.h * f.h);
  if (f.dtype == 0)
    apply_stencil_k<double><<<blocks, 256, 0, st>>>((const double*)phi + f.off,
                                                    (double*)out + f.off, f.nx, f.ny, f.ld,
                                                    f.ghost, ih2);
  else
    apply_stencil_k<float><<<blocks, 256, 0, st>>>((const float*)phi + f.off,
                                                   (float*)out + f.off, f.nx, f.ny, f.ld,
                                                   f.ghost, (float)ih2);
  return cudaGetLastError();
}

cudaError_t launch_residual_norm(const FieldDesc& f, const void* phi, const void* rho,
                                 double* out2, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out2, 0, 2 * sizeof(double), st);
  if (e != cudaSuccess) return e;
  if (f.nx == 0 || f.ny == 0) return cudaSuccess;
  const int bx = (f.nx + 255) / 256;
  const int by = (int)std::max<int64_t>(
      1, std::min<int64_t>({(int64_t)f.ny, 65535, (int64_t)device_sm_count() * 8 / bx}));
  const dim3 blocks(bx, by);
  const double ih2 = 1.0 / (f.h * f.h);
  if (f.dtype == 0)
    residual_norm_k<double><<<blocks, 256, 0, st>>>((const double*)phi + f.off,
                                                    (const double*)rho + f.off, f.nx, f.ny,
                                                    f.ld, ih2, out2);
  else
    residual_norm_k<float><<<blocks, 256, 0, st>>>((const float*)phi + f.off,
                                                   (const float*)rho + f.off, f.nx, f.ny,
                                                   f.ld, ih2, out2);
  return cudaGetLastError();
}

cudaError_t launch_copy_field(const FieldDesc& f, const void* src, void* dst,
                              cudaStream_t st) {
  const int64_t n = (int64_t)(f.nx + 2 * f.ghost) * (f.ny + 2 * f.ghost);
  const int blocks = grid_for(n, 256);
  if (f.dtype == 0)
    copy_field_k<double><<<blocks, 256, 0, st>>>((const double*)src + f.off,
                                                 (double*)dst + f.off, f.nx, f.ny, f.ld,
                                                 f.ghost);
  else
    copy_field_k<float><<<blocks, 256, 0, st>>>((const float*)src + f.off, (float*)dst + f.off,
                                                f.nx, f.ny, f.ld, f.ghost);
  return cudaGetLastError();
}

}  // namespace px

// ---------------------------------------------------------------------------
// Iterative refinement around FP32-storage sweeps. The outer loop works in FP64:
//   r = rho - L phi (FP64, same evaluation as the residual norm), scaled by the
//   exact power of two s = 2^-ilogb(R) with R = ||r||_inf, stored as FP32;
//   the FP32 sweeps solve L e = s r from e = 0;
//   phi += e / s (FP64; the division by a power of two is exact).
namespace px {
namespace {

__global__ void refine_residual_k(const double* __restrict__ phi, const double* __restrict__ rho,
                                  int nx, int ny, int64_t ld, double ih2,
                                  const double* __restrict__ norm, float* __restrict__ r32,
                                  float* __restrict__ e32, int64_t ld32,
                                  double* __restrict__ inv_scale) {
  const double R = norm[0];
  const int ex = ilogb(R);
  const double s = ldexp(1.0, -ex);
  if (blockIdx.x == 0 && threadIdx.x == 0) *inv_scale = ldexp(1.0, ex);
  const int64_t n = (int64_t)nx * ny;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(c / nx), i = (int)(c - (int64_t)j * nx);
    const double* row = phi + (int64_t)j * ld;
    const double C = row[i];
    const double W = row[wrap1(i - 1, nx)], E = row[wrap1(i + 1, nx)];
    const double S = phi[(int64_t)wrap1(j - 1, ny) * ld + i];
    const double N = phi[(int64_t)wrap1(j + 1, ny) * ld + i];
    const double s5 = __dsub_rn(__dadd_rn(__dadd_rn(W, E), __dadd_rn(S, N)), __dmul_rn(4.0, C));
    const double r = __dsub_rn(rho[(int64_t)j * ld + i], __dmul_rn(ih2, s5));
    r32[(int64_t)j * ld32 + i] = __double2float_rn(r * s);
    e32[(int64_t)j * ld32 + i] = 0.0f;
  }
}

__global__ void refine_update_k(double* __restrict__ phi, const float* __restrict__ e32, int nx,
                                int ny, int64_t ld, int64_t ld32, int ghost,
                                const double* __restrict__ inv_scale) {
  const double is = *inv_scale;
  const int64_t n = (int64_t)nx * ny;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(c / nx), i = (int)(c - (int64_t)j * nx);
    const double v = __dadd_rn(phi[(int64_t)j * ld + i], (double)e32[(int64_t)j * ld32 + i] * is);
    store_all_images<double>(phi, i, j, nx, ny, ld, ghost, v);
  }
}

// Deterministic FP64 sum: fixed grid, per-block partials, one block sums them
// in index order.
constexpr int kSumBlocks = 512;
template <typename T>
__global__ void sum_partials_k(const T* __restrict__ a, int nx, int ny, int64_t ld,
                               double* __restrict__ partials) {
  const int64_t n = (int64_t)nx * ny;
  double acc = 0.0;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(c / nx), i = (int)(c - (int64_t)j * nx);
    acc += (double)a[(int64_t)j * ld + i];
  }
  __shared__ double sm[256];
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = sm[0];
}

__global__ void sum_final_k(const double* __restrict__ partials, int n, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += partials[k];
    *out = s;
  }
}

}  // namespace

cudaError_t launch_refine_residual(const FieldDesc& f, const void* phi, const void* rho,
                                   const double* norm, float* r32, float* e32, int64_t ld32,
                                   double* inv_scale, cudaStream_t st) {
  const int64_t n = (int64_t)f.nx * f.ny;
  refine_residual_k<<<grid_for(n, 256), 256, 0, st>>>(
      (const double*)phi + f.off, (const double*)rho + f.off, f.nx, f.ny, f.ld,
      1.0 / (f.h * f.h), norm, r32, e32, ld32, inv_scale);
  return cudaGetLastError();
}

cudaError_t launch_refine_update(const FieldDesc& f, void* phi, const float* e32, int64_t ld32,
                                 const double* inv_scale, cudaStream_t st) {
  const int64_t n = (int64_t)f.nx * f.ny;
  refine_update_k<<<grid_for(n, 256), 256, 0, st>>>((double*)phi + f.off, e32, f.nx, f.ny, f.ld,
                                                    ld32, f.ghost, inv_scale);
  return cudaGetLastError();
}

int sum_partials_count() { return kSumBlocks; }

cudaError_t launch_field_sum(const FieldDesc& f, const void* a, double* partials, double* out,
                             cudaStream_t st) {
  if (f.dtype == 0)
    sum_partials_k<double><<<kSumBlocks, 256, 0, st>>>((const double*)a + f.off, f.nx, f.ny, f.ld,
                                                       partials);
  else
    sum_partials_k<float><<<kSumBlocks, 256, 0, st>>>((const float*)a + f.off, f.nx, f.ny, f.ld,
                                                      partials);
  sum_final_k<<<1, 32, 0, st>>>(partials, kSumBlocks, out);
  return cudaGetLastError();
}

}  // namespace px

// Grid-transfer kernels of the geometric multigrid V-cycle (multigrid with a
// red-black SOR smoother is what the paper builds on Proto's operators, Sec.
// VI; the cycle is the textbook cell-centred one).
//
//  * mg_restrict: residual and restriction in one pass. For every coarse cell
//    (J, I) it evaluates r = rho - L_h phi at the four fine cells of its 2 x 2
//    block (periodic wrap in the loads) and writes their mean
//    ((r00 + r01) + (r10 + r11)) / 4 to the coarse right-hand side; it also
//    writes the coarse starting state e = 0, and can fold max |r| into a
//    report slot (the residual of the fine state it reads).
//  * mg_prolong: bilinear interpolation of the coarse correction between cell
//    centres, added to the fine state. Fine cell (2J + b, 2I + a) lies a
//    quarter of a coarse cell from centre (J, I) towards its x neighbour
//    I - 1 (a = 0) or I + 1 (a = 1), and likewise in y, so it receives
//    9/16 e(J, I) + 3/16 (e(J, I') + e(J', I)) + 1/16 e(J', I').
//    Levels that the FP32 register wavefront smooths do this inside the first
//    post-smoothing launch instead (prolong_add in relax.cu, the same
//    expressions); this pass serves FP64 and layouts off the 16-byte grid.
// A thread owns one coarse cell; a block covers 32 coarse columns x 8 coarse
// rows and strides over rows, so neighbouring threads share fine rows through
// L1. Per-cell arithmetic (FMA form, storage type T):
//   s = fma(-4, C, (W + E) + (U + D)), r = fma(-s, 1/h^2, rho).
#include "px_internal.cuh"

#include <algorithm>

namespace px {
namespace {

template <typename T>
__device__ __forceinline__ T fine_resid(T C, T W, T E, T U, T D, T rh, T ih2) {
  return fma(-fma((T)-4, C, (W + E) + (U + D)), ih2, rh);
}

template <typename T>
__global__ void __launch_bounds__(256)
mg_restrict_k(const T* __restrict__ phi, const T* __restrict__ rho, int nx, int ny, int64_t ld,
              T ih2, T* __restrict__ rc, T* __restrict__ ec, int64_t ldc,
              double* __restrict__ slot) {
  using MB = typename MaxBits<T>::type;
  const int nxc = nx / 2, nyc = ny / 2;
  const int I = blockIdx.x * 32 + threadIdx.x;
  MB mx = 0;
  if (I < nxc) {
    const int i0 = 2 * I, i1 = i0 + 1;
    const int im = i0 == 0 ? nx - 1 : i0 - 1, ip = i1 + 1 == nx ? 0 : i1 + 1;
    for (int J = blockIdx.y * 8 + threadIdx.y; J < nyc; J += gridDim.y * 8) {
      const int j0 = 2 * J, j1 = j0 + 1;
      const int jm = j0 == 0 ? ny - 1 : j0 - 1, jp = j1 + 1 == ny ? 0 : j1 + 1;
      const T* Rm = phi + (int64_t)jm * ld;
      const T* R0 = phi + (int64_t)j0 * ld;
      const T* R1 = phi + (int64_t)j1 * ld;
      const T* Rp = phi + (int64_t)jp * ld;
      const T* H0 = rho + (int64_t)j0 * ld;
      const T* H1 = rho + (int64_t)j1 * ld;
      const T c00 = R0[i0], c01 = R0[i1], c10 = R1[i0], c11 = R1[i1];
      const T a = fine_resid(c00, R0[im], c01, Rm[i0], c10, H0[i0], ih2);
      const T b = fine_resid(c01, c00, R0[ip], Rm[i1], c11, H0[i1], ih2);
      const T c = fine_resid(c10, R1[im], c11, c00, Rp[i0], H1[i0], ih2);
      const T d = fine_resid(c11, c10, R1[ip], c01, Rp[i1], H1[i1], ih2);
      rc[(int64_t)J * ldc + I] = ((a + b) + (c + d)) * (T)0.25;
      ec[(int64_t)J * ldc + I] = (T)0;
      if (slot) mx = umax(umax(mx, umax(absbits(a), absbits(b))), umax(absbits(c), absbits(d)));
    }
  }
  if (slot) {
    __shared__ MB red[8];
    const int t = threadIdx.y * 32 + threadIdx.x;
    mx = warp_max(mx);
    if ((t & 31) == 0) red[t >> 5] = mx;
    __syncthreads();
    if (t == 0) {
      MB m = 0;
      for (int w = 0; w < 8; ++w) m = umax(m, red[w]);
      atomic_max_bits(slot, to_f64_bits(m));
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256)
mg_prolong_k(const T* __restrict__ e, int nxc, int nyc, int64_t ldc, T* __restrict__ phi,
             int64_t ld) {
  const int I = blockIdx.x * 32 + threadIdx.x;
  if (I >= nxc) return;
  const int il = I == 0 ? nxc - 1 : I - 1, ir = I + 1 == nxc ? 0 : I + 1;
  for (int J = blockIdx.y * 8 + threadIdx.y; J < nyc; J += gridDim.y * 8) {
    const int ju = J == 0 ? nyc - 1 : J - 1, jd = J + 1 == nyc ? 0 : J + 1;
    const T* Eu = e + (int64_t)ju * ldc;
    const T* E0 = e + (int64_t)J * ldc;
    const T* Ed = e + (int64_t)jd * ldc;
    const T c = (T)0.5625 * E0[I];
    const T xl = E0[il], xr = E0[ir], yu = Eu[I], yd = Ed[I];
    const T q = (T)0.1875, o = (T)0.0625;
    T* F0 = phi + (int64_t)(2 * J) * ld + 2 * I;
    T* F1 = F0 + ld;
    F0[0] += fma(o, Eu[il], fma(q, xl + yu, c));
    F0[1] += fma(o, Eu[ir], fma(q, xr + yu, c));
    F1[0] += fma(o, Ed[il], fma(q, xl + yd, c));
    F1[1] += fma(o, Ed[ir], fma(q, xr + yd, c));
  }
}

dim3 coarse_grid(int nxc, int nyc) {
  const int bx = (nxc + 31) / 32;
  const int by = (int)std::max<int64_t>(
      1, std::min<int64_t>({(int64_t)(nyc + 7) / 8, 65535,
                            std::max<int64_t>(1, (int64_t)device_sm_count() * 8 / bx)}));
  return dim3(bx, by);
}

}  // namespace

cudaError_t launch_mg_restrict(const FieldDesc& f, const void* phi, const void* rho, void* rc,
                               void* ec, int64_t ldc, double* slot, cudaStream_t st) {
  const int nxc = f.nx / 2, nyc = f.ny / 2;
  if (nxc == 0 || nyc == 0) return cudaSuccess;
  const dim3 grid = coarse_grid(nxc, nyc), block(32, 8);
  const double ih2 = 1.0 / (f.h * f.h);
  if (f.dtype == 0)
    mg_restrict_k<double><<<grid, block, 0, st>>>((const double*)phi, (const double*)rho, f.nx,
                                                  f.ny, f.ld, ih2, (double*)rc, (double*)ec, ldc,
                                                  slot);
  else
    mg_restrict_k<float><<<grid, block, 0, st>>>((const float*)phi, (const float*)rho, f.nx,
                                                 f.ny, f.ld, (float)ih2, (float*)rc, (float*)ec,
                                                 ldc, slot);
  return cudaGetLastError();
}

cudaError_t launch_mg_prolong(const FieldDesc& f, const void* e, int64_t ldc, void* phi,
                              cudaStream_t st) {
  const int nxc = f.nx / 2, nyc = f.ny / 2;
  if (nxc == 0 || nyc == 0) return cudaSuccess;
  const dim3 grid = coarse_grid(nxc, nyc), block(32, 8);
  if (f.dtype == 0)
    mg_prolong_k<double><<<grid, block, 0, st>>>((const double*)e, nxc, nyc, ldc, (double*)phi,
                                                 f.ld);
  else
    mg_prolong_k<float><<<grid, block, 0, st>>>((const float*)e, nxc, nyc, ldc, (float*)phi,
                                                f.ld);
  return cudaGetLastError();
}

}  // namespace px

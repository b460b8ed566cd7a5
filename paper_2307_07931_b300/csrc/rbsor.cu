// Red-black SOR sweeps (the relaxation the paper names as the smoother of
// Proto's multigrid, Sec. VI; standard definition): one sweep updates, in
// place, first every red cell ((x + y) even) and then every black cell, each
// with the Jacobi per-point update phi <- phi + c (s / h^2 - rho),
// c = omega h^2 / 4, s the unscaled 5-point tap sum of the current state.
//
// Two passes per sweep (FP64 storage, and FP32 layouts that the register
// wavefront does not take; FP32 vector layouts run the wavefront in relax.cu):
//  * red pass, src -> dst (out of place): every cell of src is read once; red
//    cells are updated, black cells copied; with a report, the residual of the
//    input state of every cell is folded into the report slot (integer max of
//    the sign-cleared bits, NaN-sticky), otherwise only red cells are
//    evaluated;
//  * black pass, dst in place: black cells are updated from their (now new)
//    red neighbours; only black cells are evaluated and stored. A black update
//    reads only red cells and its own cell, none of which another thread
//    writes in this pass.
// A thread owns a column group of V cells (V = 2: one 16-byte FP64 vector,
// one red and one black cell; V = 1: the general path for any pitch and
// alignment) and walks rows with a stride of gridDim.y, so no index needs a
// division. The FP64 pipe bounds the FP64 sweep, so a cell is evaluated only
// where its value is used: 6 FP64 operations per updated cell plus 5 per
// reported black cell.
// The per-cell arithmetic is the one of the Jacobi kernels (FMA form):
//   q = (W + E) + (S + N), s = fma(-4, C, q), r = fma(s, 1/h^2, -rho),
//   C' = fma(c, r, C).
#include "px_internal.cuh"

#include <algorithm>

namespace px {
namespace {

template <typename T>
__device__ __forceinline__ T rb_resid(T w, T e, T n, T s, T c, T rh, Coef<T> k) {
  return fma(fma((T)-4, c, (w + e) + (n + s)), k.ih2, -rh);
}

// colour 0 = red ((x + y) even), 1 = black. src and dst are the same array in
// the black pass (no __restrict__ on them).
template <typename T, int V, int kColour, bool kRep>
__global__ void __launch_bounds__(256)
rb_pass(const T* src, T* dst, const T* __restrict__ rho, int nx, int ny, int64_t ld, Coef<T> k,
        double* __restrict__ slot) {
  static_assert(V == 1 || (V == 2 && sizeof(T) == 8), "one cell or one FP64 pair per thread");
  using MB = typename MaxBits<T>::type;
  const int groups = nx / V;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  MB mx = 0;
  if (g < groups) {
    const int x0 = g * V;
    const int xw = x0 == 0 ? nx - 1 : x0 - 1, xe = x0 + V == nx ? 0 : x0 + V;
    for (int j = blockIdx.y; j < ny; j += gridDim.y) {
      const T* rc = src + (int64_t)j * ld;
      const T* ru = src + (int64_t)(j == 0 ? ny - 1 : j - 1) * ld;
      const T* rd = src + (int64_t)(j + 1 == ny ? 0 : j + 1) * ld;
      const T* rr = rho + (int64_t)j * ld;
      T* out = dst + (int64_t)j * ld;
      const int vu = (x0 + j + kColour) & 1;  // V = 2: the cell of this pass's colour
      if constexpr (V == 1) {
        if (kColour == 1 && vu) continue;  // black pass: red cells stay
        const T c = rc[x0];
        if (kRep || !vu) {
          const T r = rb_resid(rc[xw], rc[xe], ru[x0], rd[x0], c, rr[x0], k);
          if (kRep) mx = umax(mx, absbits(r));
          if (!vu) {
            out[x0] = fma(k.c, r, c);
            continue;
          }
        }
        out[x0] = c;  // red pass: black cells are copied
      } else {
        const double2 c = *reinterpret_cast<const double2*>(rc + x0);
        const double2 u = *reinterpret_cast<const double2*>(ru + x0);
        const double2 d = *reinterpret_cast<const double2*>(rd + x0);
        const double2 rh = *reinterpret_cast<const double2*>(rr + x0);
        const T wl = rc[xw], er = rc[xe];
        double2 o = c;
        if (kRep) {
          const T r0 = rb_resid(wl, c.y, u.x, d.x, c.x, rh.x, k);
          const T r1 = rb_resid(c.x, er, u.y, d.y, c.y, rh.y, k);
          mx = umax(mx, umax(absbits(r0), absbits(r1)));
          if (vu) o.y = fma(k.c, r1, c.y);
          else o.x = fma(k.c, r0, c.x);
        } else if (vu) {
          o.y = fma(k.c, rb_resid(c.x, er, u.y, d.y, c.y, rh.y, k), c.y);
        } else {
          o.x = fma(k.c, rb_resid(wl, c.y, u.x, d.x, c.x, rh.x, k), c.x);
        }
        if (kColour == 0) *reinterpret_cast<double2*>(out + x0) = o;
        else if (vu) out[x0 + 1] = o.y;
        else out[x0] = o.x;
      }
    }
  }
  if (kRep) {
    __shared__ MB red[8];
    mx = warp_max(mx);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      MB m = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = umax(m, red[w]);
      atomic_max_bits(slot, to_f64_bits(m));
    }
  }
}

template <typename T, int V>
cudaError_t launch_rb_t(const FieldDesc& f, const T* src, T* dst, const T* rho, double omega,
                        bool red_pass, double* slot, cudaStream_t st) {
  Coef<T> k;
  k.c = (T)(omega * f.h * f.h / 4.0);
  k.ih2 = (T)(1.0 / (f.h * f.h));
  const int groups = f.nx / V;
  const int bx = (groups + 255) / 256;
  // about 16 CTAs per SM, rows split over gridDim.y (at most 65535)
  const int by = (int)std::max<int64_t>(
      1, std::min<int64_t>({(int64_t)f.ny, 65535, (int64_t)device_sm_count() * 16 / bx}));
  const dim3 grid(bx, by);
  if (red_pass) {
    if (slot)
      rb_pass<T, V, 0, true><<<grid, 256, 0, st>>>(src, dst, rho, f.nx, f.ny, f.ld, k, slot);
    else
      rb_pass<T, V, 0, false><<<grid, 256, 0, st>>>(src, dst, rho, f.nx, f.ny, f.ld, k, nullptr);
  } else {
    rb_pass<T, V, 1, false><<<grid, 256, 0, st>>>(dst, dst, rho, f.nx, f.ny, f.ld, k, nullptr);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rbsor_pass(const FieldDesc& f, const void* src, void* dst, const void* rho,
                              double omega, bool red_pass, bool vec, double* slot,
                              cudaStream_t st) {
  if (f.dtype == 0)
    return vec ? launch_rb_t<double, 2>(f, (const double*)src, (double*)dst, (const double*)rho,
                                        omega, red_pass, slot, st)
               : launch_rb_t<double, 1>(f, (const double*)src, (double*)dst, (const double*)rho,
                                        omega, red_pass, slot, st);
  return launch_rb_t<float, 1>(f, (const float*)src, (float*)dst, (const float*)rho, omega,
                               red_pass, slot, st);
}

}  // namespace px

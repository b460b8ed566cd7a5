// Red-black SOR sweeps (the relaxation the paper names as the smoother of
// Proto's multigrid, Sec. VI; standard definition): one sweep updates, in
// place, first every red cell ((x + y) even) and then every black cell, each
// with the Jacobi per-point update phi <- phi + c (s / h^2 - rho),
// c = omega h^2 / 4, s the unscaled 5-point tap sum of the current state.
//
// FP64 16-byte vector layouts run one fused launch per sweep (rb_fused_f64
// below); FP32 vector layouts the register wavefront in relax.cu. Other
// layouts take two passes per sweep:
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

// Fused red-black sweep for FP64 vector layouts: one launch per sweep, src ->
// dst out of place (src is never written), so every value a thread needs is an
// input value or a new red value it can compute from input values alone. A
// warp owns a strip of kRbOwn = 30 column pairs (x0, x0 + 1), x0 even, and a
// segment [j0, j1) of rows; lanes 0 and 31 hold the pairs on either side of
// the strip (periodic images at the grid's edges) and compute their new red
// values only for the black updates of their neighbours. Walking down the
// segment, the warp computes the black values of row j from the new red
// values of rows j - 1 .. j + 1 and, independently, the new red values of row
// j + 2 from input rows j + 1 .. j + 3 (in row j the red cell is x0 for even j,
// x0 + 1 for odd j); rows j0 - 1 and j1 get their red values computed by both
// segments that need them. Per cell the operations and their order are those
// of rb_pass, so the two forms agree bitwise. With a report the residual of
// the input state of both cells of every pair of the segment's rows is folded
// in (the black cell's from the input rows): 17 FP64 operations per pair and
// row as in the two passes (12 without), plus the two halo lanes of 32, with
// one pass over HBM (24 bytes per cell) instead of two.
constexpr int kRbOwn = 30;

struct RbRow {
  double2 v;      // the lane's pair (x0, x0 + 1)
  double el, er;  // lane 0: cell x0 - 1; lane 31: cell x0 + 2
};

template <bool kRep>
__global__ void __launch_bounds__(256, 2)
rb_fused_f64(const double* __restrict__ src, double* __restrict__ dst,
             const double* __restrict__ rho, int nx, int ny, int64_t ld, int nstrips, int ry,
             int nseg, Coef<double> k, double* __restrict__ slot) {
  const int lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const int np = nx >> 1;
  const int ntasks = nstrips * nseg;
  uint64_t mx = 0;

  for (int task = gw; task < ntasks; task += nw) {
    const int strip = task % nstrips, seg = task / nstrips;
    const int pu = strip * kRbOwn - 1 + lane;  // pair index before the periodic wrap
    const int x0 = 2 * wrapn(pu, np);
    const bool own = lane >= 1 && lane <= kRbOwn && pu < np;
    const int xl = x0 == 0 ? nx - 1 : x0 - 1;
    const int xr = x0 + 2 == nx ? 0 : x0 + 2;
    const int j0 = seg * ry, j1 = min(j0 + ry, ny);

    // rows j0 - 2 .. j1 + 1 lie in [-ny, 2 ny) (ny >= 2), where wrap1 is exact
    auto load = [&](int j, RbRow& r) {
      const int jw = wrap1(j, ny);
      const double* rp = src + (int64_t)jw * ld;
      if (PX_IN_RANGE(31, jw, 0, ny) && PX_IN_RANGE(32, x0, 0, nx - 1))
        r.v = *reinterpret_cast<const double2*>(rp + x0);
      if (lane == 0) r.el = rp[xl];
      if (lane == 31) r.er = rp[xr];
    };
    auto load_rho = [&](int j) {
      const int jw = wrap1(j, ny);
      double2 r = make_double2(0.0, 0.0);
      if (PX_IN_RANGE(33, jw, 0, ny))
        r = *reinterpret_cast<const double2*>(rho + (int64_t)jw * ld + x0);
      return r;
    };
    // the new red value of row j from input rows u, c, d; with rep, the
    // residuals of both cells of the pair are folded into mx
    auto red = [&](const RbRow& u, const RbRow& c, const RbRow& d, double2 rh, int j, bool rep) {
      double left = __shfl_up_sync(0xffffffffu, c.v.y, 1);
      double right = __shfl_down_sync(0xffffffffu, c.v.x, 1);
      if (lane == 0) left = c.el;
      if (lane == 31) right = c.er;
      double rn;
      if ((j & 1) == 0) {
        const double r = rb_resid(left, c.v.y, u.v.x, d.v.x, c.v.x, rh.x, k);
        rn = fma(k.c, r, c.v.x);
        if (kRep && rep) {
          const double b = rb_resid(c.v.x, right, u.v.y, d.v.y, c.v.y, rh.y, k);
          mx = umax(mx, umax(absbits(r), absbits(b)));
        }
      } else {
        const double r = rb_resid(c.v.x, right, u.v.y, d.v.y, c.v.y, rh.y, k);
        rn = fma(k.c, r, c.v.y);
        if (kRep && rep) {
          const double b = rb_resid(left, c.v.y, u.v.x, d.v.x, c.v.x, rh.x, k);
          mx = umax(mx, umax(absbits(r), absbits(b)));
        }
      }
      return rn;
    };

    // Each step j computes the black values of row j (from new red values of
    // rows j - 1 .. j + 1, computed earlier) and the new red values of row j + 2:
    // two independent chains of FP64 operations per step.
    RbRow ra, rb, rc, rd, re;
    load(j0 - 2, ra);
    load(j0 - 1, rb);
    load(j0, rc);
    load(j0 + 1, rd);
    load(j0 + 2, re);
    double2 rh0 = load_rho(j0), rh1 = load_rho(j0 + 1), rh2 = rh1;
    double rm = red(ra, rb, rc, load_rho(j0 - 1), j0 - 1, false);  // new red of row j0 - 1
    double r0 = red(rb, rc, rd, rh0, j0, true);                      // row j0
    double rp = red(rc, rd, re, rh1, j0 + 1, j0 + 1 < j1);           // row j0 + 1
    RbRow cj = rc, cj1 = rd, cj2 = re, cj3;
    if (j0 + 3 <= j1 + 1) load(j0 + 3, cj3);
    if (j0 + 2 <= j1) rh2 = load_rho(j0 + 2);

    for (int j = j0; j < j1; ++j) {
      // input rows j0 - 2 .. j1 + 1 and rho rows j0 - 1 .. j1 are used
      RbRow nxt;
      double2 rh3 = rh2;
      if (j + 4 <= j1 + 1) load(j + 4, nxt);
      if (j + 3 <= j1) rh3 = load_rho(j + 3);
      double rpp = rp;
      if (j + 2 <= j1) rpp = red(cj1, cj2, cj3, rh2, j + 2, j + 2 < j1);  // new red of row j + 2
      const double rw = __shfl_up_sync(0xffffffffu, r0, 1);   // new red of cell x0 - 1
      const double rv = __shfl_down_sync(0xffffffffu, r0, 1); // new red of cell x0 + 2
      double2 o;
      if ((j & 1) == 0) {
        o.x = r0;
        o.y = fma(k.c, rb_resid(r0, rv, rm, rp, cj.v.y, rh0.y, k), cj.v.y);
      } else {
        o.x = fma(k.c, rb_resid(rw, r0, rm, rp, cj.v.x, rh0.x, k), cj.v.x);
        o.y = r0;
      }
      if (own && PX_IN_RANGE(34, j, 0, ny) && PX_IN_RANGE(32, x0, 0, nx - 1))
        *reinterpret_cast<double2*>(dst + (int64_t)j * ld + x0) = o;
      cj = cj1;
      cj1 = cj2;
      cj2 = cj3;
      cj3 = nxt;
      rm = r0;
      r0 = rp;
      rp = rpp;
      rh0 = rh1;
      rh1 = rh2;
      rh2 = rh3;
    }
  }

  if constexpr (kRep) {
    __shared__ uint64_t red_mx[8];
    mx = warp_max(mx);
    if (lane == 0) red_mx[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint64_t m = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = umax(m, red_mx[w]);
      atomic_max_bits(slot, m);
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

cudaError_t launch_rbsor_fused(const FieldDesc& f, const double* src, double* dst,
                               const double* rho, double omega, double* slot, cudaStream_t st) {
  Coef<double> k;
  k.c = omega * f.h * f.h / 4.0;
  k.ih2 = 1.0 / (f.h * f.h);
  const int np = f.nx / 2;
  const int nstrips = (np + kRbOwn - 1) / kRbOwn;
  // Rows per warp task: 64 on large grids (two recomputed red rows per task);
  // fewer on small grids so that there are about four warp tasks per resident
  // warp slot of the device (two CTAs of eight warps per SM).
  const int64_t target = (int64_t)device_sm_count() * 16 * 4;
  const int ry = (int)std::max<int64_t>(1, std::min<int64_t>(64, (int64_t)f.ny * nstrips / target));
  const int nseg = (f.ny + ry - 1) / ry;
  const int64_t ntasks = (int64_t)nstrips * nseg;
  static int blocks_by_dev[64][2] = {};
  int& blocks_per_sm = blocks_by_dev[dev_index()][slot ? 1 : 0];
  if (blocks_per_sm == 0) {
    cudaError_t e = slot ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                               &blocks_per_sm, rb_fused_f64<true>, 256, 0)
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                               &blocks_per_sm, rb_fused_f64<false>, 256, 0);
    if (e != cudaSuccess) return e;
    if (blocks_per_sm < 1) blocks_per_sm = 1;
  }
  const int64_t resident = (int64_t)blocks_per_sm * device_sm_count();
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((ntasks + 7) / 8, resident));
  if (slot)
    rb_fused_f64<true><<<blocks, 256, 0, st>>>(src, dst, rho, f.nx, f.ny, f.ld, nstrips, ry, nseg,
                                               k, slot);
  else
    rb_fused_f64<false><<<blocks, 256, 0, st>>>(src, dst, rho, f.nx, f.ny, f.ld, nstrips, ry,
                                                nseg, k, nullptr);
  return cudaGetLastError();
}

}  // namespace px

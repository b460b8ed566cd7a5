// Fused 3D periodic Poisson sweep (the paper's Eq. "jacobi" in D = 3
// dimensions, 7-point Laplacian): per cell, in the storage type T,
//   q  = ((W + E) + (S + N)) + (B + T)     (x, y and z neighbours)
//   s  = fma(-6, C, q)
//   r  = fma(s, 1/h^2, -rho)               (residual of the input state)
//   C' = fma(omega h^2 / 6, r, C)          (weighted Jacobi)
// and the max-norm of r, in one pass.
//
// relax3_k: a CTA owns a tile of 32 V x 8 cells in x and y (V = 16 bytes per
// element, or 1 on the general path) and a segment of planes, and marches up
// the segment one plane per step. Each thread keeps its V cells of planes
// k-1, k, k+1 in registers; plane k of the tile, plus the rows above and
// below it, goes through a double-buffered shared-memory tile so that a warp
// reads its y neighbours there (one CTA barrier per plane); x neighbours come
// from warp shuffles and, for the two edge lanes, scalar loads. Every thread
// loads real cells (columns and rows are wrapped to their periodic images
// when the tile runs past the grid), so every residual it evaluates is exact;
// only owned cells are stored. Loads for plane k+1 are issued before the
// arithmetic of plane k. DRAM traffic is one read of phi and rho and one write
// per cell, plus the two halo rows per 8 rows that L2 serves from the
// neighbouring tiles.
#include "px_internal.cuh"

#include <algorithm>

namespace px {
namespace {

constexpr int kTY = 8;  // rows (warps) per tile

template <typename T, int V>
__device__ __forceinline__ void ld_v(T (&v)[V], const T* p) {
  if constexpr (V * sizeof(T) == 16) {
    using VT = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    *reinterpret_cast<VT*>(v) = *reinterpret_cast<const VT*>(p);
  } else {
#pragma unroll
    for (int i = 0; i < V; ++i) v[i] = p[i];
  }
}

template <typename T, int V>
__device__ __forceinline__ void st_v(T* p, const T (&v)[V]) {
  if constexpr (V * sizeof(T) == 16) {
    using VT = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    *reinterpret_cast<VT*>(p) = *reinterpret_cast<const VT*>(v);
  } else {
#pragma unroll
    for (int i = 0; i < V; ++i) p[i] = v[i];
  }
}

template <typename T, int V, bool kRep>
__global__ void __launch_bounds__(256)
relax3_k(const T* __restrict__ phi, T* __restrict__ out, const T* __restrict__ rho, int nx,
         int ny, int nz, int64_t ld, int64_t lp, int seg, Coef<T> k, double* __restrict__ slot) {
  constexpr int TX = 32 * V;
  __shared__ __align__(16) T sm[2][kTY + 2][TX];
  using MB = typename MaxBits<T>::type;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int z0 = blockIdx.z * seg;
  if (z0 >= nz) return;  // the whole CTA: no barrier is skipped by part of it
  const int z1 = min(z0 + seg, nz);
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * kTY;
  const int xs = x0 + lane * V;                  // first column of the thread
  const int xc = wrapn(xs, nx);                  // its periodic image
  const int yr = wrapn(y0 + w, ny);              // the warp's row (image)
  const bool own = xs < nx && y0 + w < ny;
  // the halo row that this warp brings in: above the tile (warp 0) or below
  // it (the last warp)
  const bool halo = w == 0 || w == kTY - 1;
  const int yh = w == 0 ? wrapn(y0 - 1, ny) : wrapn(y0 + kTY, ny);
  const int xw = wrapn(x0 - 1, nx), xe = wrapn(x0 + TX, nx);
  auto cell = [&](int z, int y, int x) { return (int64_t)z * lp + (int64_t)y * ld + x; };

  T prv[V], cur[V], nxt[V], rh[V], hl[V];
  T eW = 0, eE = 0;
  {
    const int zm = z0 == 0 ? nz - 1 : z0 - 1, zp = z0 + 1 == nz ? 0 : z0 + 1;
    ld_v<T, V>(prv, phi + cell(zm, yr, xc));
    ld_v<T, V>(cur, phi + cell(z0, yr, xc));
    ld_v<T, V>(nxt, phi + cell(zp, yr, xc));
    ld_v<T, V>(rh, rho + cell(z0, yr, xc));
    if (halo) ld_v<T, V>(hl, phi + cell(z0, yh, xc));
    if (lane == 0) eW = phi[cell(z0, yr, xw)];
    if (lane == 31) eE = phi[cell(z0, yr, xe)];
  }
  MB mx = 0;
  for (int z = z0; z < z1; ++z) {
    T (*S)[TX] = sm[z & 1];
    st_v<T, V>(&S[w + 1][lane * V], cur);
    if (w == 0) st_v<T, V>(&S[0][lane * V], hl);
    if (w == kTY - 1) st_v<T, V>(&S[kTY + 1][lane * V], hl);
    __syncthreads();
    // loads for plane z + 1, in flight during the arithmetic of plane z
    T nn[V], rhn[V], hln[V];
    T eWn = 0, eEn = 0;
    const bool more = z + 1 < z1;
    if (more) {
      const int zq = z + 1, zqq = z + 2 >= nz ? z + 2 - nz : z + 2;
      ld_v<T, V>(nn, phi + cell(zqq, yr, xc));
      ld_v<T, V>(rhn, rho + cell(zq, yr, xc));
      if (halo) ld_v<T, V>(hln, phi + cell(zq, yh, xc));
      if (lane == 0) eWn = phi[cell(zq, yr, xw)];
      if (lane == 31) eEn = phi[cell(zq, yr, xe)];
    }
    T up[V], dn[V];
    ld_v<T, V>(up, &S[w][lane * V]);
    ld_v<T, V>(dn, &S[w + 2][lane * V]);
    const T wl = __shfl_up_sync(0xffffffffu, cur[V - 1], 1);
    const T er = __shfl_down_sync(0xffffffffu, cur[0], 1);
    T o[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const T W = v == 0 ? (lane == 0 ? eW : wl) : cur[v - 1];
      const T E = v == V - 1 ? (lane == 31 ? eE : er) : cur[v + 1];
      const T q = ((W + E) + (up[v] + dn[v])) + (prv[v] + nxt[v]);
      const T s = fma((T)-6, cur[v], q);
      const T r = fma(s, k.ih2, -rh[v]);
      if (kRep) mx = umax(mx, absbits(r));
      o[v] = fma(k.c, r, cur[v]);
    }
    if (own) st_v<T, V>(out + cell(z, yr, xs), o);
    if (more) {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        prv[v] = cur[v];
        cur[v] = nxt[v];
        nxt[v] = nn[v];
        rh[v] = rhn[v];
        if (halo) hl[v] = hln[v];
      }
      eW = eWn;
      eE = eEn;
    }
  }
  if (kRep) {
    __shared__ MB red[8];
    mx = warp_max(mx);
    if (lane == 0) red[w] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      MB m = 0;
      for (int i = 0; i < 8; ++i) m = umax(m, red[i]);
      atomic_max_bits(slot, to_f64_bits(m));
    }
  }
}

template <typename T, int V>
cudaError_t launch3_t(const Field3& f, const T* src, T* dst, const T* rho, double omega,
                      double* slot, cudaStream_t st) {
  constexpr int TX = 32 * V;
  Coef<T> k;
  k.c = (T)(omega * f.h * f.h / 6.0);
  k.ih2 = (T)(1.0 / (f.h * f.h));
  const int64_t bx = (f.nx + TX - 1) / TX, by = (f.ny + kTY - 1) / kTY;
  if (by > 65535) return cudaErrorInvalidConfiguration;
  // enough CTAs for about eight per SM; planes split into segments for that
  const int64_t want = (int64_t)device_sm_count() * 8;
  const int64_t segs = std::max<int64_t>(1, std::min<int64_t>(f.nz, (want + bx * by - 1) / (bx * by)));
  const int seg = (int)((f.nz + segs - 1) / segs);
  const int bz = (f.nz + seg - 1) / seg;
  if (bx > 0x7fffffffLL || bz > 65535) return cudaErrorInvalidConfiguration;
  const dim3 grid((unsigned)bx, (unsigned)by, (unsigned)bz);
  if (slot)
    relax3_k<T, V, true><<<grid, 256, 0, st>>>(src, dst, rho, f.nx, f.ny, f.nz, f.ld, f.lp, seg,
                                               k, slot);
  else
    relax3_k<T, V, false><<<grid, 256, 0, st>>>(src, dst, rho, f.nx, f.ny, f.nz, f.ld, f.lp,
                                                seg, k, nullptr);
  return cudaGetLastError();
}

template <typename T>
__global__ void copy3_k(const T* __restrict__ src, T* __restrict__ dst, int nx, int ny, int nz,
                        int64_t ld, int64_t lp) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= nx) return;
  for (int64_t r = blockIdx.y; r < (int64_t)ny * nz; r += gridDim.y) {
    const int z = (int)(r / ny), y = (int)(r - (int64_t)z * ny);
    const int64_t c = (int64_t)z * lp + (int64_t)y * ld + x;
    dst[c] = src[c];
  }
}

}  // namespace

bool vector_ok3(const Field3& f, const void* a, const void* b, const void* c) {
  const int V = f.dtype == 0 ? 2 : 4;
  if (f.nx % V || f.ld % V || f.lp % V) return false;
  auto al = [](const void* p) { return ((uintptr_t)p & 15u) == 0; };
  return al(a) && al(b) && al(c);
}

cudaError_t launch_relax3(const Field3& f, const void* src, void* dst, const void* rho,
                          double omega, bool vec, double* slot, cudaStream_t st) {
  if (f.dtype == 0)
    return vec ? launch3_t<double, 2>(f, (const double*)src, (double*)dst, (const double*)rho,
                                      omega, slot, st)
               : launch3_t<double, 1>(f, (const double*)src, (double*)dst, (const double*)rho,
                                      omega, slot, st);
  return vec ? launch3_t<float, 4>(f, (const float*)src, (float*)dst, (const float*)rho, omega,
                                   slot, st)
             : launch3_t<float, 1>(f, (const float*)src, (float*)dst, (const float*)rho, omega,
                                   slot, st);
}

cudaError_t launch_copy3(const Field3& f, const void* src, void* dst, cudaStream_t st) {
  const int bx = (f.nx + 255) / 256;
  const int by = (int)std::max<int64_t>(
      1, std::min<int64_t>({(int64_t)f.ny * f.nz, 65535, (int64_t)device_sm_count() * 8}));
  if (f.dtype == 0)
    copy3_k<double><<<dim3(bx, by), 256, 0, st>>>((const double*)src, (double*)dst, f.nx, f.ny,
                                                  f.nz, f.ld, f.lp);
  else
    copy3_k<float><<<dim3(bx, by), 256, 0, st>>>((const float*)src, (float*)dst, f.nx, f.ny,
                                                 f.nz, f.ld, f.lp);
  return cudaGetLastError();
}

}  // namespace px

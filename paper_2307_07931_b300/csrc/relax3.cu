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
// the segment one plane per step. Planes stream through a ring of five
// shared-memory slots filled by cp.async (each thread copies its own row
// pieces; warps 0 and 7 also the rows above and below the tile, lanes 0 and 31
// the x-edge values), two planes beyond the three a step reads, so that the
// loads of a plane are in flight for two steps; one CTA barrier per plane
// makes the copies visible. A step reads planes z-1, z, z+1 of its own cells,
// rows y-1 and y+1 of plane z from the slot, and x neighbours by warp
// shuffles. Every thread copies real cells (columns and rows are wrapped to
// their periodic images when the tile runs past the grid), so every residual
// it evaluates is exact; only owned cells are stored. DRAM traffic is one read
// of phi and rho and one write per cell, plus the two halo rows per 8 rows
// that L2 serves from the neighbouring tiles.
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

// One 4-, 8- or 16-byte asynchronous copy global -> shared.
template <int B>
__device__ __forceinline__ void cp_async(void* sdst, const void* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  if constexpr (B == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gsrc) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(sa), "l"(gsrc), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

constexpr int kRing = 5;      // plane slots
constexpr int kAhead = 2;     // planes in flight beyond the one the step needs
// At step z the ring holds planes z-1 .. z+1 (read) and z+2 .. z+1+kAhead (in
// flight); plane z+2+kAhead refills the slot of plane z-1 after the step's
// reads of it. In that slot a step reads only the pieces each thread copies
// itself (its own row of plane z-1), and every other read of the slot
// happened before this step's barrier.
static_assert(kRing >= kAhead + 3, "ring too small for the planes a step holds");

// One plane slot: phi rows y0 - 1 .. y0 + kTY (kTY + 2 rows of TX), rho rows
// y0 .. y0 + kTY - 1, and the x-edge values (left of lane 0, right of lane 31)
// of the kTY own rows.
template <typename T, int V>
struct Slot3 {
  static constexpr int TX = 32 * V;
  static constexpr int kPhi = (kTY + 2) * TX, kRho = kTY * TX, kEdge = 2 * kTY;
  static constexpr int kElems = kPhi + kRho + ((kEdge * (int)sizeof(T) + 15) / 16) * 16 / (int)sizeof(T);
};

template <typename T, int V, bool kRep>
__global__ void __launch_bounds__(256)
relax3_k(const T* __restrict__ phi, T* __restrict__ out, const T* __restrict__ rho, int nx,
         int ny, int nz, int64_t ld, int64_t lp, int seg, Coef<T> k, double* __restrict__ slot) {
  using SL = Slot3<T, V>;
  constexpr int TX = SL::TX;
  extern __shared__ __align__(16) unsigned char smem3[];
  T* const ring = reinterpret_cast<T*>(smem3);
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
  const bool halo = w == 0 || w == kTY - 1;      // warp 0: row above, last: row below
  const int yh = w == 0 ? wrapn(y0 - 1, ny) : wrapn(y0 + kTY, ny);
  const int hrow = w == 0 ? 0 : kTY + 1;
  const int xw = wrapn(x0 - 1, nx), xe = wrapn(x0 + TX, nx);
  auto cell = [&](int z, int y, int x) { return (int64_t)z * lp + (int64_t)y * ld + x; };
  auto slot_of = [&](int p) { return ring + (size_t)((p - z0 + 1) % kRing) * SL::kElems; };
  // this thread's copies of plane p (needed iff p <= z1), then one commit group
  auto fetch = [&](int p) {
    if (p <= z1) {
      const int zz = p < 0 ? p + nz : (p >= nz ? p - nz : p);
      T* S = slot_of(p);
      cp_async<V * sizeof(T)>(S + (w + 1) * TX + lane * V, phi + cell(zz, yr, xc));
      if (p < z1) cp_async<V * sizeof(T)>(S + SL::kPhi + w * TX + lane * V, rho + cell(zz, yr, xc));
      if (halo) cp_async<V * sizeof(T)>(S + hrow * TX + lane * V, phi + cell(zz, yh, xc));
      if (lane == 0) cp_async<sizeof(T)>(S + SL::kPhi + SL::kRho + 2 * w, phi + cell(zz, yr, xw));
      if (lane == 31) cp_async<sizeof(T)>(S + SL::kPhi + SL::kRho + 2 * w + 1, phi + cell(zz, yr, xe));
    }
    cp_commit();
  };
  // prologue: planes z0 - 1 .. z0 + 1 (the first step's) and kAhead more
  for (int p = z0 - 1; p <= z0 + 1 + kAhead; ++p) fetch(p);
  MB mx = 0;
  for (int z = z0; z < z1; ++z) {
    cp_wait<kAhead>();  // plane z + 1 (and all before it) has landed
    __syncthreads();
    const T* Sb = slot_of(z - 1);
    const T* Sc = slot_of(z);
    const T* St = slot_of(z + 1);
    T b[V], c[V], t[V], up[V], dn[V], rh[V];
    ld_v<T, V>(b, Sb + (w + 1) * TX + lane * V);
    ld_v<T, V>(c, Sc + (w + 1) * TX + lane * V);
    ld_v<T, V>(t, St + (w + 1) * TX + lane * V);
    ld_v<T, V>(up, Sc + w * TX + lane * V);
    ld_v<T, V>(dn, Sc + (w + 2) * TX + lane * V);
    ld_v<T, V>(rh, Sc + SL::kPhi + w * TX + lane * V);
    const T eW = Sc[SL::kPhi + SL::kRho + 2 * w], eE = Sc[SL::kPhi + SL::kRho + 2 * w + 1];
    fetch(z + 2 + kAhead);  // into the slot of plane z - 1, after this thread's read of it
    const T wl = __shfl_up_sync(0xffffffffu, c[V - 1], 1);
    const T er = __shfl_down_sync(0xffffffffu, c[0], 1);
    T o[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const T W = v == 0 ? (lane == 0 ? eW : wl) : c[v - 1];
      const T E = v == V - 1 ? (lane == 31 ? eE : er) : c[v + 1];
      const T q = ((W + E) + (up[v] + dn[v])) + (b[v] + t[v]);
      const T s = fma((T)-6, c[v], q);
      const T r = fma(s, k.ih2, -rh[v]);
      if (kRep) mx = umax(mx, absbits(r));
      o[v] = fma(k.c, r, c[v]);
    }
    if (own) st_v<T, V>(out + cell(z, yr, xs), o);
  }
  cp_wait<0>();
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
  const size_t smem = (size_t)kRing * Slot3<T, V>::kElems * sizeof(T);
  static int occ_by_dev[64][2] = {};
  int (&occ)[2] = occ_by_dev[dev_index()];
  const int ri = slot ? 1 : 0;
  if (occ[ri] == 0) {
    auto kern = slot ? relax3_k<T, V, true> : relax3_k<T, V, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[ri], kern, 256, smem);
    if (e != cudaSuccess) return e;
    if (occ[ri] < 1) return cudaErrorInvalidConfiguration;
  }
  Coef<T> k;
  k.c = (T)(omega * f.h * f.h / 6.0);
  k.ih2 = (T)(1.0 / (f.h * f.h));
  const int64_t bx = (f.nx + TX - 1) / TX, by = (f.ny + kTY - 1) / kTY;
  if (by > 65535) return cudaErrorInvalidConfiguration;
  // planes split into segments: minimise (waves of CTAs) x (planes per CTA +
  // the ring's two-plane restart), so that the tiles fill the resident slots
  const int64_t resident = (int64_t)occ[ri] * device_sm_count();
  const int64_t tiles = bx * by;
  int seg = f.nz;
  double best = 1e300;
  for (int64_t segs = 1; segs <= std::min<int64_t>(f.nz, 64); ++segs) {
    const int sl = (int)((f.nz + segs - 1) / segs);
    const int64_t ctas = tiles * ((f.nz + sl - 1) / sl);
    const double cost = (double)((ctas + resident - 1) / resident) * (sl + 2);
    if (cost < best) { best = cost; seg = sl; }
  }
  const int bz = (f.nz + seg - 1) / seg;
  if (bx > 0x7fffffffLL || bz > 65535) return cudaErrorInvalidConfiguration;
  const dim3 grid((unsigned)bx, (unsigned)by, (unsigned)bz);
  if (slot)
    relax3_k<T, V, true><<<grid, 256, smem, st>>>(src, dst, rho, f.nx, f.ny, f.nz, f.ld, f.lp,
                                                  seg, k, slot);
  else
    relax3_k<T, V, false><<<grid, 256, smem, st>>>(src, dst, rho, f.nx, f.ny, f.nz, f.ld, f.lp,
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

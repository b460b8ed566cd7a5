// Fused relaxation sweeps for sm_103a: periodic ghost fill folded into the
// loads, 5-point Laplacian, weighted Jacobi update and the max-norm of the
// input-state residual in one pass (ProtoX Sec. IV, the Sigma-OL merged loop of
// the OL rules Laplace, Jacobi = (1, w, -lambda) x I and
// ||.||_inf = Max o pw|x| o (0, 1/a^2, -1) x I).
//
// Per cell, in the storage type T (FP64 or FP32):
//   s  = (W + E) + (S + N) - 4 C        (unscaled taps, one rounding for the -4C)
//   r  = s / h^2 - rho                  (residual of the input state, fused FMA)
//   C' = C + (omega h^2 / 4) r          (weighted Jacobi, Eq. "jacobi")
// which is the paper's C + w s - lambda rho with w = omega/4, lambda = omega h^2/4.
// On B300 one FP64 FMA issues at 1/64 of the FP32 rate, so the FP64 sweep is
// held to 6 FP64 operations per cell (3 adds, 3 FMAs); |r| and the running max
// run on the integer pipe as bit patterns.
//
// Two kernels:
//  * relax1_stream: one sweep per launch. A warp owns an x-strip of 32*V cells
//    (V = 16 bytes / element) and marches down a segment of rows keeping rows
//    j-1, j, j+1 in registers with loads issued two rows ahead; x neighbours
//    come from warp shuffles, the strip edges from two scalar loads. DRAM
//    traffic is the algorithmic 2 reads + 1 write per cell. V = 1 is the
//    general path (any pitch, alignment, ghost layout, tiny grids).
//  * relaxT_tile: TB sweeps per launch (temporal blocking). A CTA stages a
//    (TY + 2 TB) x (TX + 2 HX) tile of phi and rho in shared memory with
//    cp.async (periodic wrap applied to the global coordinates), runs TB
//    Jacobi sweeps between two shared buffers, each sweep valid on a region
//    one cell smaller per side, and stores only its TX x TY interior, so DRAM
//    sees one read of phi and rho and one write per TB sweeps.
#include "px_internal.cuh"

#include <algorithm>
#include <cstdlib>
#include <cstring>

namespace px {

namespace {

template <typename T, int V> struct VecOf;
template <> struct VecOf<float, 4> { using type = float4; };
template <> struct VecOf<double, 2> { using type = double2; };
template <> struct VecOf<float, 1> { using type = float; };
template <> struct VecOf<double, 1> { using type = double; };

template <typename T, int V>
__device__ __forceinline__ void ldv(T (&v)[V], const T* p) {
  using VT = typename VecOf<T, V>::type;
  VT t = *reinterpret_cast<const VT*>(p);
  static_assert(sizeof(VT) == sizeof(T) * V, "vector size");
  *reinterpret_cast<VT*>(v) = t;
}
template <typename T, int V>
__device__ __forceinline__ void ldv_stream(T (&v)[V], const T* p) {
  using VT = typename VecOf<T, V>::type;
  VT t = __ldcs(reinterpret_cast<const VT*>(p));
  *reinterpret_cast<VT*>(v) = t;
}
template <typename T, int V>
__device__ __forceinline__ void stv(T* p, const T (&v)[V]) {
  using VT = typename VecOf<T, V>::type;
  *reinterpret_cast<VT*>(p) = *reinterpret_cast<const VT*>(v);
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Store v at interior cell (x, j) and, for the ghosted layout, at every ghost
// cell that is a periodic image of it (rows -1 / ny, columns -1 / nx).
template <typename T>
__device__ __forceinline__ void store_images(T* O, int x, int j, int nx, int ny,
                                             int64_t ld, T v) {
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

// One ring entry of the streaming kernel: the thread's V cells of a row plus
// the strip-edge neighbours (left: lane 0, right: the strip's last valid lane).
template <typename T, int V> struct RowReg {
  T v[V];
  T el, er;
};

template <typename T, int V, bool kRep>
__global__ void __launch_bounds__(256)
relax1_stream(const T* __restrict__ phi, T* __restrict__ out, const T* __restrict__ rho,
              int nx, int ny, int64_t ld, int ghost, int ry, int nstrips, int nseg,
              Coef<T> k, double* __restrict__ slot) {
  using MB = typename MaxBits<T>::type;
  constexpr int SW = kWarp * V;
  const int lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const int ntasks = nstrips * nseg;
  MB mx = 0;

  for (int task = gw; task < ntasks; task += nw) {
    const int strip = task % nstrips, seg = task / nstrips;
    const int xs = strip * SW;
    const int x = xs + lane * V;
    const bool valid = x < nx;
    const int xc = valid ? x : xs;  // in-bounds address for idle lanes
    const int xend = min(xs + SW, nx);
    const bool need_l = lane == 0;
    const bool need_r = valid && (x + V >= xend);
    const int xl = wrap1(xs - 1, nx);
    const int xr = wrap1(x + V, nx);
    const int j0 = seg * ry, j1 = min(j0 + ry, ny);

    auto load_row = [&](int j, RowReg<T, V>& rr) {
      const int jw = wrap1(j, ny);
      const T* rp = phi + (int64_t)jw * ld;
      if (PX_IN_RANGE(1, jw, 0, ny) && PX_IN_RANGE(2, xc, 0, nx - V + 1)) ldv<T, V>(rr.v, rp + xc);
      if (need_l && PX_IN_RANGE(3, xl, 0, nx)) rr.el = rp[xl];
      if (need_r && PX_IN_RANGE(4, xr, 0, nx)) rr.er = rp[xr];
    };
    RowReg<T, V> up, cur, dn, pf;
    T rh0[V], rh1[V];
    load_row(j0 - 1, up);
    load_row(j0, cur);
    load_row(j0 + 1, dn);  // j0 + 1 <= j1 always (segments are non-empty)
    if (j0 + 2 <= j1) load_row(j0 + 2, pf);
    ldv_stream<T, V>(rh0, rho + (int64_t)j0 * ld + xc);
    if (j0 + 1 < j1) ldv_stream<T, V>(rh1, rho + (int64_t)(j0 + 1) * ld + xc);

    for (int j = j0; j < j1; ++j) {
      RowReg<T, V> nxt;
      T rh2[V];
      if (j + 3 <= j1) load_row(j + 3, nxt);
      if (j + 2 < j1) ldv_stream<T, V>(rh2, rho + (int64_t)(j + 2) * ld + xc);

      T left0 = __shfl_up_sync(0xffffffffu, cur.v[V - 1], 1);
      T rightV = __shfl_down_sync(0xffffffffu, cur.v[0], 1);
      if (need_l) left0 = cur.el;
      if (need_r) rightV = cur.er;
      T o[V];
#pragma unroll
      for (int i = 0; i < V; ++i) {
        const T w = (i == 0) ? left0 : cur.v[i - 1];
        const T e = (i == V - 1) ? rightV : cur.v[i + 1];
        const T q = (w + e) + (up.v[i] + dn.v[i]);
        const T s = fma((T)-4, cur.v[i], q);
        const T r = fma(s, k.ih2, -rh0[i]);
        o[i] = fma(k.c, r, cur.v[i]);
        if (kRep && valid) mx = umax(mx, absbits(r));
      }
      if (valid && PX_IN_RANGE(5, j, 0, ny) && PX_IN_RANGE(6, x, 0, nx - V + 1)) {
        T* op = out + (int64_t)j * ld + x;
        if constexpr (V == 1) {
          op[0] = o[0];
          if (ghost) store_images<T>(out, x, j, nx, ny, ld, o[0]);
        } else {
          stv<T, V>(op, o);
        }
      }
      up = cur;
      cur = dn;
      dn = pf;
      pf = nxt;
#pragma unroll
      for (int i = 0; i < V; ++i) { rh0[i] = rh1[i]; rh1[i] = rh2[i]; }
    }
  }

  if constexpr (kRep) {
    __shared__ MB wmax[8];
    mx = warp_max(mx);
    const int warp = threadIdx.x >> 5;
    if (lane == 0) wmax[warp] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      MB m = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = umax(m, wmax[w]);
      atomic_max_bits(slot, to_f64_bits(m));
    }
  }
}

constexpr int kTileRows = 72;  // shared-memory tile height R = TY + 2 TB
constexpr int kTileThreads = 256;

template <typename T, int TB>
struct TileGeom {
  static constexpr int V = 16 / (int)sizeof(T);
  static constexpr int PX = kWarp * V;                   // tile width in cells
  static constexpr int HX = ((TB + V - 1) / V) * V;      // x halo, multiple of V
  static constexpr int TX = PX - 2 * HX;                 // owned width
  static constexpr int R = kTileRows;
  static constexpr int TY = R - 2 * TB;                  // owned height
  static constexpr size_t smem = sizeof(T) * (size_t)PX * (2 * R + (R - 2));
};

template <typename T, int TB>
__global__ void __launch_bounds__(kTileThreads, 2)
relaxT_tile(const T* __restrict__ phi, T* __restrict__ out, const T* __restrict__ rho,
            int nx, int ny, int64_t ld, int tiles_x, Coef<T> k, Reports rep) {
  using G = TileGeom<T, TB>;
  using MB = typename MaxBits<T>::type;
  constexpr int V = G::V, PX = G::PX, HX = G::HX, TX = G::TX, R = G::R, TY = G::TY;
  constexpr int NW = kTileThreads / kWarp;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* A = reinterpret_cast<T*>(smem_raw);
  T* B = A + R * PX;
  T* RH = B + R * PX;  // row r (1..R-2) at RH + (r - 1) * PX
  __shared__ MB sres[TB][NW];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
  const int gx0 = tx * TX - HX, gy0 = ty * TY - TB;

  if (tid < TB * NW) (&sres[0][0])[tid] = 0;

  {
    const int gx = wrapn(gx0 + lane * V, nx);
    for (int r = warp; r < R; r += NW) {
      const int64_t row = (int64_t)wrapn(gy0 + r, ny) * ld + gx;
      cp_async16(A + r * PX + lane * V, phi + row);
      if (r >= 1 && r <= R - 2) cp_async16(RH + (r - 1) * PX + lane * V, rho + row);
    }
    cp_async_wait_all();
    __syncthreads();
  }

  // Rows 1..R-2 split over the warps.
  const int rb = 1 + ((R - 2) * warp) / NW, re = 1 + ((R - 2) * (warp + 1)) / NW;
  const int cx = lane * V;                       // first tile column of this lane
  const bool own_x = cx >= HX && cx < HX + TX && (tx * TX + cx - HX) < nx;
  const int gxo = tx * TX + cx - HX;

#pragma unroll
  for (int t = 0; t < TB; ++t) {
    const T* S = (t & 1) ? B : A;
    T* D = (t & 1) ? A : B;
    const bool last = t == TB - 1;
    const bool rep_t = rep.due(t);
    int r0 = max(rb, t + 1), r1 = min(re, R - 1 - t);
    if (last) { r0 = max(r0, TB); r1 = min(r1, TB + TY); }
    MB mx = 0;
    if (r0 < r1) {
      T up[V], cur[V];
      ldv<T, V>(up, S + (r0 - 1) * PX + cx);
      ldv<T, V>(cur, S + r0 * PX + cx);
      for (int r = r0; r < r1; ++r) {
        T dn[V], rh[V], o[V];
        ldv<T, V>(dn, S + (r + 1) * PX + cx);
        ldv<T, V>(rh, RH + (r - 1) * PX + cx);
        const T left0 = __shfl_up_sync(0xffffffffu, cur[V - 1], 1);
        const T rightV = __shfl_down_sync(0xffffffffu, cur[0], 1);
        const int gy = ty * TY + r - TB;
        const bool own = own_x && r >= TB && r < TB + TY && gy < ny;
#pragma unroll
        for (int i = 0; i < V; ++i) {
          const T w = (i == 0) ? left0 : cur[i - 1];
          const T e = (i == V - 1) ? rightV : cur[i + 1];
          const T q = (w + e) + (up[i] + dn[i]);
          const T s = fma((T)-4, cur[i], q);
          const T rr = fma(s, k.ih2, -rh[i]);
          o[i] = fma(k.c, rr, cur[i]);
          if (rep_t && own) mx = umax(mx, absbits(rr));
        }
        if (!last) {
          stv<T, V>(D + r * PX + cx, o);
        } else if (own) {
          stv<T, V>(out + (int64_t)gy * ld + gxo, o);
        }
#pragma unroll
        for (int i = 0; i < V; ++i) { up[i] = cur[i]; cur[i] = dn[i]; }
      }
    }
    if (rep_t) {
      mx = warp_max(mx);
      if (lane == 0) sres[t][warp] = mx;
    }
    __syncthreads();
  }

  if (tid < TB && rep.due(tid)) {
    MB m = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) m = umax(m, sres[tid][w]);
    atomic_max_bits(rep.slot(tid), to_f64_bits(m));
  }
}

int g_sms[64];

template <typename T, int V, bool kRep>
cudaError_t launch_stream_t(const FieldDesc& f, const T* src, T* dst, const T* rho,
                            Coef<T> k, double* slot, cudaStream_t st) {
  constexpr int SW = kWarp * V;
  const int nstrips = (f.nx + SW - 1) / SW;
  // Rows per warp task: 32 on large grids; fewer on small grids so that there
  // are about four warp tasks per resident warp slot of the device.
  const int64_t target = (int64_t)device_sm_count() * 32 * 4;
  const int ry = (int)std::max<int64_t>(1, std::min<int64_t>(32, (int64_t)f.ny * nstrips / target));
  const int nseg = (f.ny + ry - 1) / ry;
  const int64_t ntasks = (int64_t)nstrips * nseg;
  static int blocks_by_dev[64] = {};
  int& blocks_per_sm = blocks_by_dev[dev_index()];
  if (blocks_per_sm == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &blocks_per_sm, relax1_stream<T, V, kRep>, 256, 0);
    if (e != cudaSuccess) return e;
    if (blocks_per_sm < 1) blocks_per_sm = 1;
  }
  const int64_t resident = (int64_t)blocks_per_sm * device_sm_count();
  const int64_t want = (ntasks + 7) / 8;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(want, resident));
  relax1_stream<T, V, kRep><<<blocks, 256, 0, st>>>(
      src + f.off, dst + f.off, rho + f.off, f.nx, f.ny, f.ld, f.ghost, ry, nstrips,
      nseg, k, slot);
  return cudaGetLastError();
}

template <typename T, int TB>
cudaError_t launch_tile_t(const FieldDesc& f, const T* src, T* dst, const T* rho,
                          Coef<T> k, Reports rep, cudaStream_t st) {
  using G = TileGeom<T, TB>;
  static bool attr_by_dev[64] = {};
  bool& attr = attr_by_dev[dev_index()];
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(relaxT_tile<T, TB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)G::smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int tiles_x = (f.nx + G::TX - 1) / G::TX;
  const int tiles_y = (f.ny + G::TY - 1) / G::TY;
  const int64_t blocks = (int64_t)tiles_x * tiles_y;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  relaxT_tile<T, TB><<<(unsigned)blocks, kTileThreads, G::smem, st>>>(
      src, dst, rho, f.nx, f.ny, f.ld, tiles_x, k, rep);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// relaxW_f32: wavefront temporal blocking for FP32 storage, TB sweeps per launch.
//
// A CTA owns a strip of 256 cells (32 lanes x two float4 groups, columns
// 4*lane and 128 + 4*lane) and a segment of H output rows. It streams down the
// segment: stage t (warp t - 1) turns level t - 1 (the state after t - 1
// sweeps) into level t one row per step, two rows behind stage t - 1, keeping
// rows r - 1 and r of its input level in registers and reading row r + 1 from a
// 4-row shared-memory ring. A loader warp keeps level 0 (phi) and rho rows
// arriving kWPrefetch steps ahead with cp.async, so DRAM reads overlap the
// sweeps; the last stage stores straight from registers. One barrier per step.
// Each sweep is valid on a region one cell narrower per side, so the strip
// owns its central 256 - 2*HX columns; in y the segment loads TB extra rows
// above and below. Redundant work is (256 / (256 - 2 HX)) x (1 + TB / H).
constexpr int kWStrip = 256;

template <int TB>
struct WGeom {
  static constexpr int P = 6;                               // rows loaded ahead
  static constexpr int HX = ((TB + 3) / 4) * 4;             // x halo, multiple of 4
  static constexpr int OW = kWStrip - 2 * HX;               // owned width
  static constexpr int R0 = 16;                             // level-0 ring rows (>= P + 4)
  static constexpr int RR = (2 * TB + P + 1) <= 16 ? 16 : 32;  // rho ring rows (>= 2 TB + P + 1)
  static constexpr int RL = 4;                              // rows per level ring
  static constexpr int kThreads = (TB + 1) * kWarp;         // TB stages + loader
  static constexpr size_t smem = sizeof(float) * kWStrip * (size_t)(R0 + RR + RL * (TB - 1));
  static_assert(R0 >= P + 4 && RR >= 2 * TB + P + 1, "ring sizes");
};

__device__ __forceinline__ void lds4(float* v, const float* p) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void sts4(float* p, const float* v) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

template <int TB>
__global__ void __launch_bounds__(WGeom<TB>::kThreads)
relaxW_f32(const float* __restrict__ phi, float* __restrict__ out, const float* __restrict__ rho,
           int nx, int ny, int64_t ld, int H, int nstrips, Coef<float> k, Reports rep) {
  using G = WGeom<TB>;
  extern __shared__ __align__(16) float wsm[];
  float* L0 = wsm;                        // level 0, R0 rows
  float* RH = L0 + G::R0 * kWStrip;       // rho, RR rows
  float* LV = RH + G::RR * kWStrip;       // levels 1..TB-1, RL rows each
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int strip = blockIdx.x % nstrips, seg = blockIdx.x / nstrips;
  const int y0 = seg * H;
  const int base = y0 - TB;               // global row of load index 0
  const int nload = H + 2 * TB;
  const int gx0 = strip * G::OW - G::HX;  // global column of strip column 0 (unwrapped)
  const int steps = H + 3 * TB;
  const int c0 = lane * 4, c1 = 128 + lane * 4;

  if (warp == TB) {
    // Loader: load index i (global row base + i) of phi and rho into ring slots.
    const int gxa = wrapn(gx0 + c0, nx), gxb = wrapn(gx0 + c1, nx);
    int grow = wrapn(base, ny);           // global row of the next load index
    int i = 0;
    auto issue = [&]() {
      if (i < nload) {
        const int64_t row = (int64_t)grow * ld;
        float* d0 = L0 + (i & (G::R0 - 1)) * kWStrip;
        float* d1 = RH + (i & (G::RR - 1)) * kWStrip;
        cp_async16(d0 + c0, phi + row + gxa);
        cp_async16(d0 + c1, phi + row + gxb);
        cp_async16(d1 + c0, rho + row + gxa);
        cp_async16(d1 + c1, rho + row + gxb);
        grow = (grow + 1 == ny) ? 0 : grow + 1;
      }
      ++i;
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
#pragma unroll 1
    for (int q = 0; q < G::P; ++q) issue();
#pragma unroll 1
    for (int st = 0; st < steps; ++st) {
      issue();
      // row st is complete; rows st+1 .. st+P may still be in flight
      asm volatile("cp.async.wait_group %0;\n" ::"n"(G::P) : "memory");
      __syncthreads();
    }
    return;
  }

  const int t = warp + 1;  // stage: computes level t from level t - 1
  const float* src = (t == 1) ? L0 : LV + (t - 2) * G::RL * kWStrip;
  const int smask = (t == 1) ? G::R0 - 1 : G::RL - 1;
  float* dstL = LV + (t - 1) * G::RL * kWStrip;  // used when t < TB
  const bool rep_t = rep.due(t - 1);
  const bool own0 = c0 >= G::HX && c0 < kWStrip - G::HX && gx0 + c0 < nx;
  const bool own1 = c1 >= G::HX && c1 < kWStrip - G::HX && gx0 + c1 < nx;
  const int own_hi = min(TB + H, TB + ny - y0);  // owned rows: TB <= ridx < own_hi
  float* const orow0 = out + gx0;                 // + gy * ld + column
  const int first = t, count = H + 2 * TB - 2 * t;
  uint32_t mx = 0;

#pragma unroll 1
  for (int st = 0; st < 3 * t; ++st) __syncthreads();

  float A[8], B[8], C[8];
  lds4(A, src + ((first - 1) & smask) * kWStrip + c0);
  lds4(A + 4, src + ((first - 1) & smask) * kWStrip + c1);
  lds4(B, src + (first & smask) * kWStrip + c0);
  lds4(B + 4, src + (first & smask) * kWStrip + c1);
  int ridx = first;

  // One row of level t: up, cu hold rows ridx-1, ridx of level t-1; dn receives ridx+1.
  auto row = [&](const float* up, const float* cu, float* dn) {
    const float* sdn = src + ((ridx + 1) & smask) * kWStrip;
    const float* srh = RH + (ridx & (G::RR - 1)) * kWStrip;
    lds4(dn, sdn + c0);
    lds4(dn + 4, sdn + c1);
    float rh[8];
    lds4(rh, srh + c0);
    lds4(rh + 4, srh + c1);
    // x neighbours across the lanes; columns -1 and 256 are never owned
    const float l0 = __shfl_sync(0xffffffffu, cu[3], (lane + 31) & 31);
    const float l1 = __shfl_sync(0xffffffffu, lane == 31 ? cu[3] : cu[7], (lane + 31) & 31);
    const float r0 = __shfl_sync(0xffffffffu, lane == 0 ? cu[4] : cu[0], (lane + 1) & 31);
    const float r1 = __shfl_sync(0xffffffffu, cu[4], (lane + 1) & 31);
    float o[8], rr[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float w = (i == 0) ? l0 : (i == 4) ? l1 : cu[i - 1];
      const float e = (i == 3) ? r0 : (i == 7) ? r1 : cu[i + 1];
      const float q = (w + e) + (up[i] + dn[i]);
      const float sv = fmaf(-4.0f, cu[i], q);
      rr[i] = fmaf(sv, k.ih2, -rh[i]);
      o[i] = fmaf(k.c, rr[i], cu[i]);
    }
    if (rep_t) {
      const bool own_row = ridx >= TB && ridx < own_hi;
      const uint32_t m0 = (own_row && own0) ? 0x7fffffffu : 0u;
      const uint32_t m1 = (own_row && own1) ? 0x7fffffffu : 0u;
      mx = __vimax3_u32(mx, __float_as_uint(rr[0]) & m0, __float_as_uint(rr[1]) & m0);
      mx = __vimax3_u32(mx, __float_as_uint(rr[2]) & m0, __float_as_uint(rr[3]) & m0);
      mx = __vimax3_u32(mx, __float_as_uint(rr[4]) & m1, __float_as_uint(rr[5]) & m1);
      mx = __vimax3_u32(mx, __float_as_uint(rr[6]) & m1, __float_as_uint(rr[7]) & m1);
    }
    if (t < TB) {
      float* d = dstL + (ridx & (G::RL - 1)) * kWStrip;
      sts4(d + c0, o);
      sts4(d + c1, o + 4);
    } else {
      const int gy = base + ridx;
      if (gy < ny) {
        float* orow = orow0 + (int64_t)gy * ld;
        if (own0) sts4(orow + c0, o);
        if (own1) sts4(orow + c1, o + 4);
      }
    }
    ++ridx;
    __syncthreads();
  };

  int n = count;
#pragma unroll 1
  while (n >= 3) {
    row(A, B, C);
    row(B, C, A);
    row(C, A, B);
    n -= 3;
  }
  if (n >= 1) row(A, B, C);
  if (n >= 2) row(B, C, A);

#pragma unroll 1
  for (int st = 3 * t + count; st < steps; ++st) __syncthreads();

  if (rep_t) {
    mx = warp_max(mx);
    if (lane == 0) atomic_max_bits(rep.slot(t - 1), to_f64_bits(mx));
  }
}

// ---------------------------------------------------------------------------
// relaxW2_f32: the wavefront kernel with two rows per step per stage. Stage t
// computes level-t rows r, r+1 with r = 2s - 3t at step s (one pair behind
// stage t-1 by two steps), from level t-1 rows r-1 .. r+2: rows r-1, r are
// kept from the previous step and r+1, r+2 come from a 4-row shared ring (a
// stage reads its first window during its last idle step, while those rows'
// slots are not being rewritten). The loader brings row pairs kW2Prefetch
// steps ahead; the rho ring holds exactly the 3 TB + 2 P + 2 live rows.
// Half the barriers of relaxW_f32 and twice the independent work per warp.
constexpr int kW2Prefetch = 3;  // row pairs loaded ahead

template <int TB>
struct W2Geom {
  static constexpr int P = kW2Prefetch;
  static constexpr int HX = ((TB + 3) / 4) * 4;
  static constexpr int OW = kWStrip - 2 * HX;
  static constexpr int R0 = 16;                  // >= 2P + 4 (power of two: mask)
  static constexpr int RR = 3 * TB + 2 * P + 2;  // rho rows live at once (slot counters)
  static constexpr int RL = 4;                   // rows per level ring (power of two: mask)
  static constexpr int kThreads = (TB + 1) * kWarp;
  static constexpr size_t smem = sizeof(float) * kWStrip * (size_t)(R0 + RR + RL * (TB - 1));
  static_assert(R0 >= 2 * P + 4 && RR >= 3 * TB + 2 * P + 2, "ring sizes");
};

template <int TB>
__global__ void __launch_bounds__(W2Geom<TB>::kThreads)
relaxW2_f32(const float* __restrict__ phi, float* __restrict__ out, const float* __restrict__ rho,
            int nx, int ny, int64_t ld, int H, int nstrips, Coef<float> k, Reports rep) {
  using G = W2Geom<TB>;
  extern __shared__ __align__(16) float wsm[];
  float* L0 = wsm;
  float* RH = L0 + G::R0 * kWStrip;
  float* LV = RH + G::RR * kWStrip;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int strip = blockIdx.x % nstrips, seg = blockIdx.x / nstrips;
  const int y0 = seg * H;
  const int base = y0 - TB;
  const int npairs = (H + 2 * TB) / 2;    // H is even
  const int gx0 = strip * G::OW - G::HX;
  const int steps = H / 2 + 2 * TB;
  const int c0 = lane * 4, c1 = 128 + lane * 4;

  if (warp == TB) {
    const int gxa = wrapn(gx0 + c0, nx), gxb = wrapn(gx0 + c1, nx);
    int grow = wrapn(base, ny);
    int i = 0;   // next load index (row)
    int ri = 0;  // its rho ring slot, i mod RR
    auto issue_pair = [&]() {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (i < 2 * npairs) {
          const int64_t row = (int64_t)grow * ld;
          float* d0 = L0 + (i & (G::R0 - 1)) * kWStrip;
          float* d1 = RH + ri * kWStrip;
          cp_async16(d0 + c0, phi + row + gxa);
          cp_async16(d0 + c1, phi + row + gxb);
          cp_async16(d1 + c0, rho + row + gxa);
          cp_async16(d1 + c1, rho + row + gxb);
          grow = (grow + 1 == ny) ? 0 : grow + 1;
        }
        ++i;
        ri = (ri + 1 == G::RR) ? 0 : ri + 1;
      }
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
#pragma unroll 1
    for (int q = 0; q < G::P; ++q) issue_pair();
#pragma unroll 1
    for (int st = 0; st < steps; ++st) {
      issue_pair();
      asm volatile("cp.async.wait_group %0;\n" ::"n"(G::P) : "memory");  // pair st complete
      __syncthreads();
    }
    return;
  }

  const int t = warp + 1;
  const float* src = (t == 1) ? L0 : LV + (t - 2) * G::RL * kWStrip;
  const int smask = (t == 1) ? G::R0 - 1 : G::RL - 1;
  float* dstL = LV + (t - 1) * G::RL * kWStrip;
  const bool rep_t = rep.due(t - 1);
  const bool own0 = c0 >= G::HX && c0 < kWStrip - G::HX && gx0 + c0 < nx;
  const bool own1 = c1 >= G::HX && c1 < kWStrip - G::HX && gx0 + c1 < nx;
  const int own_hi = min(TB + H, TB + ny - y0);
  float* const orow0 = out + gx0;
  const int first = t;                          // first row (load index) of level t
  const int npair_t = (H + 2 * TB - 2 * t) / 2;  // pairs of level t
  uint32_t mx = 0;

  // Idle steps 0 .. 2t-1; the first window (level t-1 rows t-1, t, written by
  // stage t-1 at step 2t-2) is read during step 2t-1.
#pragma unroll 1
  for (int st = 0; st < 2 * t - 1; ++st) __syncthreads();
  float X[16], Y[16];  // row pairs: [0..7] = lower row, [8..15] = upper row
  {
    const float* ra = src + ((first - 1) & smask) * kWStrip;
    const float* rb = src + (first & smask) * kWStrip;
    lds4(X, ra + c0); lds4(X + 4, ra + c1);
    lds4(X + 8, rb + c0); lds4(X + 12, rb + c1);
  }
  __syncthreads();
  int r = first;
  int rs = first % G::RR;  // rho ring slot of row r

  // rows r, r+1 of level t from input rows up = r-1, cu = r (in P), r+1, r+2 (into Q)
  auto pair = [&](const float* Pp, float* Q) {
    const float* s1 = src + ((r + 1) & smask) * kWStrip;
    const float* s2 = src + ((r + 2) & smask) * kWStrip;
    lds4(Q, s1 + c0); lds4(Q + 4, s1 + c1);
    lds4(Q + 8, s2 + c0); lds4(Q + 12, s2 + c1);
    float rh[16];
    const int rs1 = (rs + 1 == G::RR) ? 0 : rs + 1;
    const float* h0 = RH + rs * kWStrip;
    const float* h1 = RH + rs1 * kWStrip;
    lds4(rh, h0 + c0); lds4(rh + 4, h0 + c1);
    lds4(rh + 8, h1 + c0); lds4(rh + 12, h1 + c1);
    float o[16], rr[16];
#pragma unroll
    for (int row = 0; row < 2; ++row) {
      const float* up = row == 0 ? Pp : Pp + 8;
      const float* cu = row == 0 ? Pp + 8 : Q;
      const float* dn = row == 0 ? Q : Q + 8;
      const float l0 = __shfl_sync(0xffffffffu, cu[3], (lane + 31) & 31);
      const float l1 = __shfl_sync(0xffffffffu, lane == 31 ? cu[3] : cu[7], (lane + 31) & 31);
      const float r0 = __shfl_sync(0xffffffffu, lane == 0 ? cu[4] : cu[0], (lane + 1) & 31);
      const float r1 = __shfl_sync(0xffffffffu, cu[4], (lane + 1) & 31);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float w = (i == 0) ? l0 : (i == 4) ? l1 : cu[i - 1];
        const float e = (i == 3) ? r0 : (i == 7) ? r1 : cu[i + 1];
        const float q = (w + e) + (up[i] + dn[i]);
        const float sv = fmaf(-4.0f, cu[i], q);
        rr[row * 8 + i] = fmaf(sv, k.ih2, -rh[row * 8 + i]);
        o[row * 8 + i] = fmaf(k.c, rr[row * 8 + i], cu[i]);
      }
    }
    if (rep_t) {
#pragma unroll
      for (int row = 0; row < 2; ++row) {
        const bool own_row = (r + row) >= TB && (r + row) < own_hi;
        const uint32_t m0 = (own_row && own0) ? 0x7fffffffu : 0u;
        const uint32_t m1 = (own_row && own1) ? 0x7fffffffu : 0u;
        const float* v = rr + row * 8;
        mx = __vimax3_u32(mx, __float_as_uint(v[0]) & m0, __float_as_uint(v[1]) & m0);
        mx = __vimax3_u32(mx, __float_as_uint(v[2]) & m0, __float_as_uint(v[3]) & m0);
        mx = __vimax3_u32(mx, __float_as_uint(v[4]) & m1, __float_as_uint(v[5]) & m1);
        mx = __vimax3_u32(mx, __float_as_uint(v[6]) & m1, __float_as_uint(v[7]) & m1);
      }
    }
    if (t < TB) {
      float* d0 = dstL + (r & (G::RL - 1)) * kWStrip;
      float* d1 = dstL + ((r + 1) & (G::RL - 1)) * kWStrip;
      sts4(d0 + c0, o); sts4(d0 + c1, o + 4);
      sts4(d1 + c0, o + 8); sts4(d1 + c1, o + 12);
    } else {
#pragma unroll
      for (int row = 0; row < 2; ++row) {
        const int gy = base + r + row;
        if (gy < ny) {
          float* orow = orow0 + (int64_t)gy * ld;
          if (own0) sts4(orow + c0, o + row * 8);
          if (own1) sts4(orow + c1, o + row * 8 + 4);
        }
      }
    }
    r += 2;
    rs = (rs1 + 1 == G::RR) ? 0 : rs1 + 1;
    __syncthreads();
  };

  int n = npair_t;
#pragma unroll 1
  while (n >= 2) {
    pair(X, Y);
    pair(Y, X);
    n -= 2;
  }
  if (n == 1) pair(X, Y);

#pragma unroll 1
  for (int st = 2 * t + npair_t; st < steps; ++st) __syncthreads();

  if (rep_t) {
    mx = warp_max(mx);
    if (lane == 0) atomic_max_bits(rep.slot(t - 1), to_f64_bits(mx));
  }
}

template <int TB>
cudaError_t launch_wave2_t(const FieldDesc& f, const float* src, float* dst, const float* rho,
                           Coef<float> k, Reports rep, cudaStream_t st) {
  using G = W2Geom<TB>;
  static int occ_by_dev[64] = {};
  int& occ = occ_by_dev[dev_index()];
  if (occ == 0) {
    cudaError_t e = cudaFuncSetAttribute(relaxW2_f32<TB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)G::smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, relaxW2_f32<TB>, G::kThreads, G::smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
  }
  const int nstrips = (f.nx + G::OW - 1) / G::OW;
  const int64_t resident = (int64_t)occ * device_sm_count();
  static const int cand[] = {8, 16, 32, 64, 96, 128, 192, 256, 384, 512, 768, 1024};
  int H = 8;
  double best = 1e300;
  for (int h : cand) {
    const int64_t ctas = (int64_t)nstrips * ((f.ny + h - 1) / h);
    const double cost = (double)((ctas + resident - 1) / resident) * (h / 2 + 2 * TB);
    if (cost <= best) { best = cost; H = h; }
    if (h >= f.ny) break;
  }
  const int64_t blocks = (int64_t)nstrips * ((f.ny + H - 1) / H);
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  relaxW2_f32<TB><<<(unsigned)blocks, G::kThreads, G::smem, st>>>(src, dst, rho, f.nx, f.ny, f.ld,
                                                                   H, nstrips, k, rep);
  return cudaGetLastError();
}

// Whether the automatic choice takes the packed-pair (f32x2) form of the
// register wavefront's Jacobi stages.
constexpr bool kRegPackedDefault = false;

// FP32 kernel family for depth >= 2, from the context option
// PX_OPT_FP32_FAMILY carried in the field descriptor: 1 the one-row
// wavefront, 2 the two-row wavefront, 3 the register wavefront at every size,
// 4 the same with packed-pair arithmetic, 0 (the default) the fastest measured (200 sweeps, a report every sweep):
// the register wavefront at depths 3..8 on fields of 2^23 cells or more
// (depth 8: 2406 vs 1424 GLUP/s on the two-row wavefront at 16384^2, 1431 vs
// 912 at 3072^2); below, where the two-row wavefront wins at depth 8 (997 vs
// 909 at 2048^2), the one-row wavefront for depths 6 and 7 and the two-row
// one for the others; depth 2 always the two-row one.

// ---------------------------------------------------------------------------
// relaxR2_f32: register wavefront, TB stages per launch, no shared tiles and
// no CTA barriers. A stage is a Jacobi sweep (TB = 3 or 4) or, with kRB, half
// a red-black sweep (TB = 2, 4, 6, 8: red, black, red, ...; a stage updates
// the cells of its colour and copies the others).
//
// One warp owns a strip of 128 cells (4 per lane, periodic columns x0 - 4 ..
// x0 + 123) and a range of output rows, and runs every stage itself. Step s
// brings level-0 rows r0 = 2s and r0 + 1 into registers; stage t (t = 1..TB,
// in order) then computes level-t rows r0 - t and r0 - t + 1 from level t-1
// rows r0 - t - 1 .. r0 - t + 2, the newest two of which stage t-1 produced
// in this step. Each level keeps a four-row window in registers (slot = row
// mod 4) and the step loop is unrolled by two, so the window rotation is
// register renaming; the per-step work that is not arithmetic (ring slots,
// cp.async, waits, addresses, predicates) is shared by two rows. x neighbours
// come from shuffles. Rows and columns outside the valid cone (one cell and
// one row smaller per stage) are computed and discarded: the strip owns its
// central 128 - 8 HL columns (HL = ceil(TB / 4) halo lanes per side: lanes
// 1..30 up to 4 stages, 2..29 up to 8) and the range's own rows.
//
// phi and rho rows stream through per-warp shared-memory rings filled by
// cp.async kR2Ahead row pairs ahead; each lane copies and reads back only its
// own 16 bytes, so the thread's own cp.async.wait_group is the only wait.
//
// Residual. The state t-1 residual of a row is exact once level t-1 is exact
// on the row and its two neighbours: from row index t on at the top, and at
// the bottom always (stage t reads no row beyond the newest loaded one).
// Exact values of rows and wrapped columns outside the owned ones are
// residuals of real cells, so including them leaves the max unchanged; only
// the HL edge lanes per side, whose columns lose exactness stage by stage,
// are dropped, once, before the warp reduction.
//
// Load balance. SMs run this kernel at different speeds (how many warps share
// the SM, where its GPC sits), so equal static shares leave fast warps idle.
// Each warp starts with one static range of output rows of one strip and
// publishes it as one 64-bit word (strip, end, cur) in `sched`; it claims its
// rows kRClaim at a time with atomicAdd on cur. A warp whose range is done
// samples 32 words, picks the one with the most unclaimed rows and, with a
// bounded atomicCAS loop, lowers that range's end to its midpoint and takes
// the upper half as its own new range (a fresh wavefront: 2 TB extra rows).
// The owner sees the lower end at its next claim. Nothing waits on another
// warp: every loop is bounded, and a failed steal ends the warp. Without
// `sched` the static ranges are used as they are.
constexpr int kRStrip = 128;
// Halo lanes per side: each stage's valid region is one column narrower per
// side, so TB stages need TB halo columns (4 per lane).
template <int TB> __host__ __device__ constexpr int r_halo_lanes() { return (TB + 3) / 4; }
template <int TB> __host__ __device__ constexpr int r_owned() { return kRStrip - 8 * r_halo_lanes<TB>(); }
constexpr int kRPhiRing = 8, kRRhoRing = 16;    // ring rows (powers of two)
// Warps per CTA: 8 (two CTAs per SM up to 128 registers a thread), or 12
// where a depth needs more registers: one CTA per SM then, three warps per
// scheduler at up to 168 registers (each scheduler has 16K). Measured at
// 16384^2, depth 8: 2570 GLUP/s with 12 warps, 2406 with 8 (183 registers).
template <int TB, bool kRB> __host__ __device__ constexpr int r_warps() {
  return (kRB ? TB >= 8 : TB >= 5) ? 12 : 8;
}
constexpr int kRWarpFloats = (kRPhiRing + kRRhoRing) * kRStrip;
// Report pattern: kRepRun reads the per-stage flags, kRepNone reports nothing
// (known at compile time: fewer live registers than the flags).
constexpr int kRepRun = 0, kRepNone = 1;
template <int TB, bool kRB> constexpr size_t r_smem() {
  return (size_t)r_warps<TB, kRB>() * kRWarpFloats * sizeof(float);
}

__device__ __forceinline__ void cp16(float* sdst, const float* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// max(m, |a|, |b|) with NaN propagation (any NaN input gives NaN).
__device__ __forceinline__ float max3_nan_abs(float m, float a, float b) {
  float r;
  asm("max.NaN.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(m), "f"(fabsf(a)), "f"(fabsf(b)));
  return r;
}

constexpr int kR2Ahead = 3;     // row pairs in flight ahead of the step
constexpr int kRClaim = 16;     // output rows per claim (even)
constexpr int kRStealMin = 64;  // steal only ranges with this many rows unclaimed
static_assert(2 * kR2Ahead + 2 <= kRPhiRing && 2 * kR2Ahead + 2 + 4 <= kRRhoRing,
              "two-row prefetch depth exceeds the rings");
static_assert(kRClaim % 2 == 0, "claims keep the row-pair parity");

// Range word: bits 0..21 cur (next unclaimed row), 22..43 end, 44..63 strip.
constexpr int kRRowBits = 22, kRStripBits = 20;
__device__ __forceinline__ unsigned long long range_pack(int s, int e, int c) {
  return ((unsigned long long)s << 44) | ((unsigned long long)e << 22) | (unsigned long long)c;
}
__device__ __forceinline__ int range_cur(unsigned long long w) { return (int)(w & 0x3fffffu); }
__device__ __forceinline__ int range_end(unsigned long long w) { return (int)((w >> 22) & 0x3fffffu); }
__device__ __forceinline__ int range_strip(unsigned long long w) { return (int)(w >> 44); }

template <int TB>
struct R2State {
  float win[TB][4][4];  // level l (input of stage l+1): slot = row mod 4
  float mx[TB];         // running max |residual| of state t (NaN-sticky)
  int rl;               // global row of the next row to load
};

// One task's bounds: output rows y0 .. lim-1 are claimed; level-0 load
// indices up to lmax may be loaded (rows up to the known end + TB).
struct R2Task {
  int y0, lim, lmax;
};

// Bilinear interpolation of the coarse correction onto fine rows 2J, 2J + 1
// (row pair a, b) at this lane's columns gx .. gx + 3 (gx a multiple of 4),
// added to the loaded values: the expressions and order of mg_prolong_k.
__device__ __forceinline__ void prolong_add(float (&ra)[4], float (&rb)[4], const Prolong& pl,
                                            int J, int gx) {
  const int I0 = gx >> 1, I1 = I0 + 1;
  const int Il = I0 == 0 ? pl.nxc - 1 : I0 - 1, Ir = I1 + 1 == pl.nxc ? 0 : I1 + 1;
  const int Ju = J == 0 ? pl.nyc - 1 : J - 1, Jd = J + 1 == pl.nyc ? 0 : J + 1;
  float u[4] = {0.f, 0.f, 0.f, 0.f}, m[4] = {0.f, 0.f, 0.f, 0.f}, d[4] = {0.f, 0.f, 0.f, 0.f};
  if (PX_IN_RANGE(35, J, 0, pl.nyc) && PX_IN_RANGE(36, I1, 0, pl.nxc)) {
    const float* Eu = pl.e + (int64_t)Ju * pl.ldc;
    const float* E0 = pl.e + (int64_t)J * pl.ldc;
    const float* Ed = pl.e + (int64_t)Jd * pl.ldc;
    u[0] = Eu[Il]; u[1] = Eu[I0]; u[2] = Eu[I1]; u[3] = Eu[Ir];
    m[0] = E0[Il]; m[1] = E0[I0]; m[2] = E0[I1]; m[3] = E0[Ir];
    d[0] = Ed[Il]; d[1] = Ed[I0]; d[2] = Ed[I1]; d[3] = Ed[Ir];
  }
  const float q = 0.1875f, o = 0.0625f;
  const float c0 = 0.5625f * m[1], c1 = 0.5625f * m[2];
  // columns gx, gx + 1 belong to coarse cell I0 (x neighbours Il, I1); gx + 2,
  // gx + 3 to I1 (x neighbours I0, Ir); row a to J (y neighbour Ju), b (Jd)
  ra[0] += fma(o, u[0], fma(q, m[0] + u[1], c0));
  ra[1] += fma(o, u[2], fma(q, m[2] + u[1], c0));
  ra[2] += fma(o, u[1], fma(q, m[1] + u[2], c1));
  ra[3] += fma(o, u[3], fma(q, m[3] + u[2], c1));
  rb[0] += fma(o, d[0], fma(q, m[0] + d[1], c0));
  rb[1] += fma(o, d[2], fma(q, m[2] + d[1], c0));
  rb[2] += fma(o, d[1], fma(q, m[1] + d[2], c1));
  rb[3] += fma(o, d[3], fma(q, m[3] + d[2], c1));
}

template <int TB, int P, bool kEdge, bool kRB, bool kPack, int kRep, bool kProl = false>
__device__ __forceinline__ void rstep2(R2State<TB>& S, int r0, const float* __restrict__ phi,
                                       const float* __restrict__ rho, float* __restrict__ out,
                                       float* ring, int nx, int ny, int64_t ld, int gx, bool own,
                                       const R2Task& T, Coef<float> k, const bool (&due)[TB],
                                       const Prolong& pl) {
  constexpr int W = 128;                      // strip floats per ring row
  float* const pr = ring;                     // phi ring, this lane's columns
  float* const rr_ = ring + kRPhiRing * W;    // rho ring
  const int la = r0 + 2 * kR2Ahead;           // first row of the pair to load
  if (la <= T.lmax) {
    const int64_t g0 = (int64_t)S.rl * ld + gx;
    S.rl = S.rl + 1 == ny ? 0 : S.rl + 1;
    const int64_t g1 = (int64_t)S.rl * ld + gx;
    S.rl = S.rl + 1 == ny ? 0 : S.rl + 1;
    if (PX_IN_RANGE(11, g0, 0, (int64_t)(ny - 1) * ld + nx - 3) &&
        PX_IN_RANGE(12, g1, 0, (int64_t)(ny - 1) * ld + nx - 3)) {
      cp16(pr + (la & (kRPhiRing - 1)) * W, phi + g0);
      cp16(pr + ((la + 1) & (kRPhiRing - 1)) * W, phi + g1);
      cp16(rr_ + (la & (kRRhoRing - 1)) * W, rho + g0);
      cp16(rr_ + ((la + 1) & (kRRhoRing - 1)) * W, rho + g1);
    }
  }
  cp_commit();
  cp_wait<kR2Ahead>();
  lds4(S.win[0][2 * P], pr + (r0 & (kRPhiRing - 1)) * W);
  lds4(S.win[0][2 * P + 1], pr + ((r0 + 1) & (kRPhiRing - 1)) * W);
  // input row r0 is global row y0 - TB + r0, even (red-black ranges start on
  // even rows and TB is even), so the pair is coarse row (y0 - TB + r0) / 2
  if constexpr (kProl) prolong_add(S.win[0][2 * P], S.win[0][2 * P + 1], pl,
                                   wrapn(T.y0 - TB + r0, ny) >> 1, gx);
#pragma unroll
  for (int t = 1; t <= TB; ++t) {
    // level t-1 rows r0-t-1 .. r0-t+2; r0 mod 4 = 2P
    const float* a = S.win[t - 1][(2 * P - t - 1 + 8) & 3];
    const float* b = S.win[t - 1][(2 * P - t + 8) & 3];
    const float* c = S.win[t - 1][(2 * P - t + 1 + 8) & 3];
    const float* d = S.win[t - 1][(2 * P - t + 2 + 8) & 3];
    float rh0[4], rh1[4];
    lds4(rh0, rr_ + ((r0 - t) & (kRRhoRing - 1)) * W);
    lds4(rh1, rr_ + ((r0 - t + 1) & (kRRhoRing - 1)) * W);
    const float bl = __shfl_up_sync(0xffffffffu, b[3], 1);
    const float br = __shfl_down_sync(0xffffffffu, b[0], 1);
    const float cl = __shfl_up_sync(0xffffffffu, c[3], 1);
    const float cr = __shfl_down_sync(0xffffffffu, c[0], 1);
    float o0[4], o1[4], q0[4], q1[4];
    if constexpr (kPack && !kRB) {
      // The same operations in the same order on packed pairs of cells
      // (add/fma.rn.f32x2: each half rounds like the scalar instruction, so
      // the results are bitwise those of the scalar form below). The
      // horizontal sums stay scalar, which lets them land in aligned pairs
      // without moves; rho is negated exactly by a product with -1.
      const float h0[4] = {bl + b[1], b[0] + b[2], b[1] + b[3], b[2] + br};
      const float h1[4] = {cl + c[1], c[0] + c[2], c[1] + c[3], c[2] + cr};
      const float2 m4 = make_float2(-4.0f, -4.0f), n1 = make_float2(-1.0f, -1.0f);
      const float2 ih2 = make_float2(k.ih2, k.ih2), kc = make_float2(k.c, k.c);
#pragma unroll
      for (int x = 0; x < 4; x += 2) {
        const float2 av = make_float2(a[x], a[x + 1]), bv = make_float2(b[x], b[x + 1]);
        const float2 cv = make_float2(c[x], c[x + 1]), dv = make_float2(d[x], d[x + 1]);
        const float2 S0 = __fadd2_rn(make_float2(h0[x], h0[x + 1]), __fadd2_rn(av, cv));
        const float2 S1 = __fadd2_rn(make_float2(h1[x], h1[x + 1]), __fadd2_rn(bv, dv));
        const float2 s0 = __ffma2_rn(m4, bv, S0), s1 = __ffma2_rn(m4, cv, S1);
        const float2 Q0 = __ffma2_rn(s0, ih2, __fmul2_rn(make_float2(rh0[x], rh0[x + 1]), n1));
        const float2 Q1 = __ffma2_rn(s1, ih2, __fmul2_rn(make_float2(rh1[x], rh1[x + 1]), n1));
        const float2 O0 = __ffma2_rn(kc, Q0, bv), O1 = __ffma2_rn(kc, Q1, cv);
        q0[x] = Q0.x; q0[x + 1] = Q0.y; q1[x] = Q1.x; q1[x + 1] = Q1.y;
        o0[x] = O0.x; o0[x + 1] = O0.y; o1[x] = O1.x; o1[x + 1] = O1.y;
      }
    } else if constexpr (!kRB && (TB < 8 || kRep != kRepRun)) {
      // Tap sums per cell (scalar: every cell an independent chain), then the
      // residual and the update on packed pairs of neighbouring cells of a
      // row, which already sit in aligned register pairs. With the signs
      // flipped, q' = fma(s, -1/h^2, rho) = -q exactly (round to nearest is
      // symmetric) and fma(-c, q', C) = fma(c, q, C), so the states are bitwise
      // those of the scalar form and |q'| = |q| for the residual. Measured at
      // 16384^2 with a report every sweep: depth 4 1844 against 1789 GLUP/s,
      // depth 6 2405 against 2339; at depth 8 its extra live registers spill
      // (2478 against 2570), so depth 8 takes it only with the report pattern
      // fixed at compile time (no per-stage flags live).
      const float2 nih2 = make_float2(-k.ih2, -k.ih2), nc = make_float2(-k.c, -k.c);
#pragma unroll
      for (int x = 0; x < 4; x += 2) {
        float s0[2], s1[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int xx = x + u;
          const float w0 = xx == 0 ? bl : b[xx - 1], e0 = xx == 3 ? br : b[xx + 1];
          const float w1 = xx == 0 ? cl : c[xx - 1], e1 = xx == 3 ? cr : c[xx + 1];
          s0[u] = fmaf(-4.0f, b[xx], (w0 + e0) + (a[xx] + c[xx]));
          s1[u] = fmaf(-4.0f, c[xx], (w1 + e1) + (b[xx] + d[xx]));
        }
        const float2 Q0 = __ffma2_rn(make_float2(s0[0], s0[1]), nih2, make_float2(rh0[x], rh0[x + 1]));
        const float2 Q1 = __ffma2_rn(make_float2(s1[0], s1[1]), nih2, make_float2(rh1[x], rh1[x + 1]));
        const float2 O0 = __ffma2_rn(nc, Q0, make_float2(b[x], b[x + 1]));
        const float2 O1 = __ffma2_rn(nc, Q1, make_float2(c[x], c[x + 1]));
        q0[x] = Q0.x; q0[x + 1] = Q0.y; q1[x] = Q1.x; q1[x + 1] = Q1.y;
        o0[x] = O0.x; o0[x + 1] = O0.y; o1[x] = O1.x; o1[x + 1] = O1.y;
      }
    } else {
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const float w0 = x == 0 ? bl : b[x - 1], e0 = x == 3 ? br : b[x + 1];
      const float w1 = x == 0 ? cl : c[x - 1], e1 = x == 3 ? cr : c[x + 1];
      const float s0 = fmaf(-4.0f, b[x], (w0 + e0) + (a[x] + c[x]));
      const float s1 = fmaf(-4.0f, c[x], (w1 + e1) + (b[x] + d[x]));
      q0[x] = fmaf(s0, k.ih2, -rh0[x]);
      q1[x] = fmaf(s1, k.ih2, -rh1[x]);
      if constexpr (kRB) {
        // red-black stages: row r0 - t has the parity of its stage's colour
        // flipped at every stage, so the updated cells are the odd columns of
        // the first row and the even ones of the second at every stage
        o0[x] = (x & 1) ? fmaf(k.c, q0[x], b[x]) : b[x];
        o1[x] = (x & 1) ? c[x] : fmaf(k.c, q1[x], c[x]);
      } else {
        o0[x] = fmaf(k.c, q0[x], b[x]);
        o1[x] = fmaf(k.c, q1[x], c[x]);
      }
    }
    }
    // Residual of state t-1 at rows r0-t, r0-t+1: exact once the row index
    // is >= t (level t-1 is exact from index t-1 on, and at the bottom every
    // computed row is exact because stage t reads rows up to r0 + 1 only).
    // Exact values of rows outside the task are residuals of real cells, so
    // including them leaves the max unchanged.
    const bool rep_t = kRep == kRepNone ? false : due[t - 1];
    if (rep_t) {
      if (!kEdge || r0 >= 2 * t) {
        S.mx[t - 1] = max3_nan_abs(S.mx[t - 1], q0[0], q0[1]);
        S.mx[t - 1] = max3_nan_abs(S.mx[t - 1], q0[2], q0[3]);
      }
      if (!kEdge || r0 + 1 >= 2 * t) {
        S.mx[t - 1] = max3_nan_abs(S.mx[t - 1], q1[0], q1[1]);
        S.mx[t - 1] = max3_nan_abs(S.mx[t - 1], q1[2], q1[3]);
      }
    }
    if (t < TB) {
      float* d0 = S.win[t][(2 * P - t + 8) & 3];      // level-t row r0 - t
      float* d1 = S.win[t][(2 * P - t + 1 + 8) & 3];  // level-t row r0 - t + 1
#pragma unroll
      for (int x = 0; x < 4; ++x) { d0[x] = o0[x]; d1[x] = o1[x]; }
    } else if (own) {
      // level-TB row index j is global row y0 + j - TB
      const int yo = T.y0 + r0 - 2 * TB;
      if (yo >= T.y0 && yo < T.lim && PX_IN_RANGE(13, yo, 0, ny) && PX_IN_RANGE(14, gx, 0, nx - 3))
        *reinterpret_cast<float4*>(out + (int64_t)yo * ld + gx) = make_float4(o0[0], o0[1], o0[2], o0[3]);
      if (yo + 1 >= T.y0 && yo + 1 < T.lim && PX_IN_RANGE(15, yo + 1, 0, ny))
        *reinterpret_cast<float4*>(out + (int64_t)(yo + 1) * ld + gx) =
            make_float4(o1[0], o1[1], o1[2], o1[3]);
    }
  }
}

// Claims the next kRClaim output rows of the warp's own range; false when the
// range is exhausted. Updates the claimed bound and the known end.
template <int TB>
__device__ __forceinline__ bool r2_claim(unsigned long long* word, R2Task& T) {
  unsigned long long old = 0;
  if ((threadIdx.x & 31) == 0) old = atomicAdd(word, (unsigned long long)kRClaim);
  old = __shfl_sync(0xffffffffu, old, 0);
  const int c = range_cur(old), e = range_end(old);
  if (c >= e) return false;
  T.lim = min(c + kRClaim, e);
  T.lmax = e - T.y0 + 2 * TB;
  return true;
}

// Steals the upper half of the unclaimed rows of some other warp's range.
__device__ bool r2_steal(unsigned long long* sched, int me, int nw, int nstrips, int ny, int& s,
                         int& y0, int& e) {
  const int lane = threadIdx.x & 31;
  const int stride = (nw + 31) / 32;
  for (int attempt = 0; attempt < 4; ++attempt) {
    const int v = (int)(((int64_t)me + 1 + (int64_t)lane * stride + 7 * attempt) % nw);
    const unsigned long long wv = *reinterpret_cast<volatile unsigned long long*>(sched + v);
    int best = range_end(wv) - range_cur(wv), bl = lane;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const int r2 = __shfl_xor_sync(0xffffffffu, best, o), l2 = __shfl_xor_sync(0xffffffffu, bl, o);
      if (r2 > best || (r2 == best && l2 < bl)) { best = r2; bl = l2; }
    }
    if (best < kRStealMin) continue;
    const int vb = __shfl_sync(0xffffffffu, v, bl);
    int ok = 0, ns = 0, nb = 0, ne = 0;
    if (lane == 0) {
      unsigned long long old = *reinterpret_cast<volatile unsigned long long*>(sched + vb);
      for (int tries = 0; tries < 8; ++tries) {
        const int c = range_cur(old), en = range_end(old), st = range_strip(old);
        // a range from another geometry (never expected) is left alone
        if (en - c < kRStealMin || st >= nstrips || en > ny) break;
        const int mid = c + (((en - c) / 2) & ~1);  // even offset keeps the pair parity
        const unsigned long long got = atomicCAS(sched + vb, old, range_pack(st, mid, c));
        if (got == old) { ok = 1; ns = st; nb = mid; ne = en; break; }
        old = got;
      }
      if (ok) atomicExch(sched + me, range_pack(ns, ne, nb));
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (ok) {
      s = __shfl_sync(0xffffffffu, ns, 0);
      y0 = __shfl_sync(0xffffffffu, nb, 0);
      e = __shfl_sync(0xffffffffu, ne, 0);
      return true;
    }
  }
  return false;
}

template <int TB, bool kRB, bool kPack, int kRep, bool kProl = false>
__global__ void __launch_bounds__(r_warps<TB, kRB>() * 32)
relaxR2_f32(const float* __restrict__ phi, float* __restrict__ out, const float* __restrict__ rho,
            int nx, int ny, int64_t ld, int H, int nstrips, int nseg, Coef<float> k, Reports rep,
            unsigned long long* sched, Prolong pl) {
  static_assert(!kProl || kRB, "the interpolation is folded into red-black launches only");
  static_assert(TB + 2 * kR2Ahead + 2 <= kRRhoRing, "rho rows in use exceed the ring");
  static_assert(!kRB || TB % 2 == 0, "red-black launches hold whole sweeps");
  extern __shared__ __align__(16) float rsm[];
  const int lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  float* const ring = rsm + (threadIdx.x >> 5) * kRWarpFloats + lane * 4;
  // report of stage t: Jacobi, sweep s0 + t; red-black, the red stage t = 2 i
  // of sweep s0 + i (its input state is the sweep's)
  bool due[TB];
#pragma unroll
  for (int t = 0; t < TB; ++t) due[t] = kRB ? (t % 2 == 0 && rep.due(t / 2)) : rep.due(t);
  R2State<TB> S;
#pragma unroll
  for (int t = 0; t < TB; ++t) S.mx[t] = 0.f;
  const int ntasks = nstrips * nseg;
  int task = gw, s = 0, y0 = 0, e = 0;
  bool have = task < ntasks;
  if (have) { s = task % nstrips; y0 = (task / nstrips) * H; e = min(y0 + H, ny); }
  // with sched, every warp publishes its range (empty if none) before anything else
  if (sched && lane == 0) atomicExch(sched + gw, have ? range_pack(s, e, y0) : 0ull);
  for (int guard = 0; guard < (1 << 24); ++guard) {
    if (!have) {
      if (sched) {
        have = r2_steal(sched, gw, nw, nstrips, ny, s, y0, e);
      } else if ((task += nw) < ntasks) {  // static grid stride
        s = task % nstrips; y0 = (task / nstrips) * H; e = min(y0 + H, ny); have = true;
      }
      if (!have) break;
    }
    constexpr int HL = r_halo_lanes<TB>();
    const int col = s * r_owned<TB>() - 4 * HL + lane * 4;
    const int gx = wrapn(col, nx);
    const bool own = lane >= HL && lane < 32 - HL && col < nx;
    R2Task T;
    T.y0 = y0;
    T.lim = sched ? y0 : e;  // with sched, rows are claimed as the wavefront reaches them
    T.lmax = e - y0 + 2 * TB;
#pragma unroll
    for (int t = 0; t < TB; ++t)
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int x = 0; x < 4; ++x) S.win[t][a][x] = 0.f;
    int rl = wrapn(y0 - TB, ny);
#pragma unroll
    for (int q = 0; q < 2 * kR2Ahead; q += 2) {
      if (q <= T.lmax) {
        const int64_t g0 = (int64_t)rl * ld + gx;
        rl = rl + 1 == ny ? 0 : rl + 1;
        const int64_t g1 = (int64_t)rl * ld + gx;
        rl = rl + 1 == ny ? 0 : rl + 1;
        cp16(ring + (q & (kRPhiRing - 1)) * 128, phi + g0);
        cp16(ring + ((q + 1) & (kRPhiRing - 1)) * 128, phi + g1);
        cp16(ring + kRPhiRing * 128 + (q & (kRRhoRing - 1)) * 128, rho + g0);
        cp16(ring + kRPhiRing * 128 + ((q + 1) & (kRRhoRing - 1)) * 128, rho + g1);
      }
      cp_commit();
    }
    S.rl = rl;
    unsigned long long* const word = sched ? sched + gw : nullptr;
    // a step at r0 outputs rows y0 + r0 - 2 TB (+1); claim before passing lim
    auto ready = [&](int r0) -> bool {
      const int yo = y0 + r0 - 2 * TB;
      if (yo < T.lim) return true;
      return word != nullptr && r2_claim<TB>(word, T);
    };
    constexpr int kPro = 2 * TB;  // r0 < 2 TB: residual rows not yet all exact
    int r0 = 0;
#pragma unroll 1
    for (; r0 < kPro; r0 += 4) {
      if (!ready(r0)) goto task_done;
      rstep2<TB, 0, true, kRB, kPack, kRep, kProl>(S, r0, phi, rho, out, ring, nx, ny, ld, gx, own, T, k, due, pl);
      if (!ready(r0 + 2)) goto task_done;
      rstep2<TB, 1, true, kRB, kPack, kRep, kProl>(S, r0 + 2, phi, rho, out, ring, nx, ny, ld, gx, own, T, k, due, pl);
    }
#pragma unroll 1
    for (;; r0 += 4) {
      if (!ready(r0)) break;
      rstep2<TB, 0, false, kRB, kPack, kRep, kProl>(S, r0, phi, rho, out, ring, nx, ny, ld, gx, own, T, k, due, pl);
      if (!ready(r0 + 2)) break;
      rstep2<TB, 1, false, kRB, kPack, kRep, kProl>(S, r0 + 2, phi, rho, out, ring, nx, ny, ld, gx, own, T, k, due, pl);
    }
  task_done:
    cp_wait<0>();  // the next task's prologue reuses the ring slots
    have = false;
  }
  const bool edge_lane = lane < r_halo_lanes<TB>() || lane >= 32 - r_halo_lanes<TB>();
#pragma unroll
  for (int t = 0; t < TB; ++t) {
    if (due[t]) {
      const uint32_t m = warp_max(edge_lane ? 0u : __float_as_uint(S.mx[t]));
      if (lane == 0) atomic_max_bits(rep.slot(kRB ? t / 2 : t), to_f64_bits(m));
    }
  }
}

template <int TB, bool kRB, bool kPack, int kRep, bool kProl = false>
cudaError_t reg2_occupancy(int& occ) {
  static int occ_by_dev[64] = {};
  int& o = occ_by_dev[dev_index()];
  if (o == 0) {
    cudaError_t e = cudaFuncSetAttribute(relaxR2_f32<TB, kRB, kPack, kRep, kProl>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)r_smem<TB, kRB>());
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, relaxR2_f32<TB, kRB, kPack, kRep, kProl>,
                                                      r_warps<TB, kRB>() * 32, r_smem<TB, kRB>());
    if (e != cudaSuccess) return e;
    if (o < 1) return cudaErrorInvalidConfiguration;
  }
  occ = o;
  return cudaSuccess;
}

template <int TB, bool kRB = false, bool kPack = false>
cudaError_t launch_reg2_t(const FieldDesc& f, const float* src, float* dst, const float* rho,
                          Coef<float> k, Reports rep, unsigned long long* sched, int sched_cap,
                          cudaStream_t st, const Prolong* pl = nullptr) {
  // Jacobi depth 8 without reports: no per-stage flags live, which leaves the
  // packed residual and update room without spills (2828 against 2673 GLUP/s
  // at 16384^2). With every stage reported the compile-time pattern measured
  // no faster than the flags (2559 packed, 2550 scalar, against 2571), so a
  // reporting launch keeps them.
  int kind = kRepRun;
  if (!kRB && !kPack && TB == 8) {
    bool any = false;
    for (int t = 0; t < TB; ++t) any = any || rep.due(t);
    kind = any ? kRepRun : kRepNone;
  }
  const bool prol = kRB && pl != nullptr;
  int occ = 0;
  cudaError_t e0 = kind == kRepNone ? reg2_occupancy<TB, kRB, kPack, kRepNone>(occ)
                   : prol           ? reg2_occupancy<TB, kRB, kPack, kRepRun, kRB>(occ)
                                    : reg2_occupancy<TB, kRB, kPack, kRepRun>(occ);
  if (e0 != cudaSuccess) return e0;
  const int nstrips = (f.nx + r_owned<TB>() - 1) / r_owned<TB>();
  const int64_t resident = (int64_t)occ * device_sm_count();
  const int64_t warps = resident * r_warps<TB, kRB>();
  // Dynamic balance needs one range per warp at most and rows that fit the
  // range word; otherwise ranges are static (grid stride over tasks).
  const bool dyn = sched != nullptr && warps <= sched_cap && nstrips <= warps &&
                   nstrips < (1 << kRStripBits) && (int64_t)f.ny + kRClaim < (1 << kRRowBits);
  // One range per resident warp, at least 32 rows (the ramp costs 2 TB rows).
  const int64_t segs = std::max<int64_t>(1, warps / nstrips);
  int64_t H = std::max<int64_t>(32, (f.ny + segs - 1) / segs);
  if (!dyn) H = std::min<int64_t>(1024, H);
  // red-black: every range starts on an even row (claims and steals keep the
  // parity), which fixes each stage's updated columns at compile time
  if (kRB) H += H & 1;
  const int nseg = (int)((f.ny + H - 1) / H);
  const int64_t tasks = (int64_t)nstrips * nseg;
  const int blocks = (int)std::max<int64_t>(
      1, std::min<int64_t>((tasks + r_warps<TB, kRB>() - 1) / r_warps<TB, kRB>(), resident));
  const dim3 grid(blocks), cta(r_warps<TB, kRB>() * 32);
  const size_t smem = r_smem<TB, kRB>();
  unsigned long long* const sc = dyn ? sched : nullptr;
  const Prolong p = pl ? *pl : Prolong{nullptr, 0, 0, 0};
  if (kind == kRepNone)
    relaxR2_f32<TB, kRB, kPack, kRepNone><<<grid, cta, smem, st>>>(
        src, dst, rho, f.nx, f.ny, f.ld, (int)H, nstrips, nseg, k, rep, sc, p);
  else if (prol)
    relaxR2_f32<TB, kRB, kPack, kRepRun, kRB><<<grid, cta, smem, st>>>(
        src, dst, rho, f.nx, f.ny, f.ld, (int)H, nstrips, nseg, k, rep, sc, p);
  else
    relaxR2_f32<TB, kRB, kPack, kRepRun><<<grid, cta, smem, st>>>(
        src, dst, rho, f.nx, f.ny, f.ld, (int)H, nstrips, nseg, k, rep, sc, p);
  return cudaGetLastError();
}


template <int TB>
cudaError_t launch_wave_t(const FieldDesc& f, const float* src, float* dst, const float* rho,
                          Coef<float> k, Reports rep, cudaStream_t st) {
  using G = WGeom<TB>;
  static int occ_by_dev[64] = {};
  int& occ = occ_by_dev[dev_index()];
  if (occ == 0) {
    cudaError_t e = cudaFuncSetAttribute(relaxW_f32<TB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)G::smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, relaxW_f32<TB>, G::kThreads, G::smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
  }
  const int nstrips = (f.nx + G::OW - 1) / G::OW;
  const int64_t resident = (int64_t)occ * device_sm_count();
  // Segment height: minimise (waves of CTAs) x (steps per CTA).
  static const int cand[] = {8, 16, 32, 64, 96, 128, 192, 256, 384, 512, 768, 1024};
  int H = 8;
  double best = 1e300;
  for (int h : cand) {
    const int64_t ctas = (int64_t)nstrips * ((f.ny + h - 1) / h);
    const double cost = (double)((ctas + resident - 1) / resident) * (h + 3 * TB);
    if (cost <= best) { best = cost; H = h; }
    if (h >= f.ny) break;
  }
  const int64_t blocks = (int64_t)nstrips * ((f.ny + H - 1) / H);
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  relaxW_f32<TB><<<(unsigned)blocks, G::kThreads, G::smem, st>>>(src, dst, rho, f.nx, f.ny, f.ld,
                                                                  H, nstrips, k, rep);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_relax_t(const FieldDesc& f, const T* src, T* dst, const T* rho,
                           double omega, int tb, bool vec, Reports rep,
                           unsigned long long* sched, int sched_cap, cudaStream_t st) {
  Coef<T> k;
  k.c = (T)(omega * f.h * f.h / 4.0);
  k.ih2 = (T)(1.0 / (f.h * f.h));
  if (tb == 1) {
    const bool r = rep.due(0);
    double* slot = r ? rep.slot(0) : nullptr;
    constexpr int VV = 16 / (int)sizeof(T);
    if (vec) {
      return r ? launch_stream_t<T, VV, true>(f, src, dst, rho, k, slot, st)
               : launch_stream_t<T, VV, false>(f, src, dst, rho, k, slot, st);
    }
    return r ? launch_stream_t<T, 1, true>(f, src, dst, rho, k, slot, st)
             : launch_stream_t<T, 1, false>(f, src, dst, rho, k, slot, st);
  }
  if constexpr (sizeof(T) == 4) {
    const int fam = f.family;
    // the register wavefront needs many warps' worth of rows: from 2^23 cells
    if (fam == 3 || fam == 4 || (fam == 0 && tb >= 3 && (int64_t)f.nx * f.ny >= ((int64_t)1 << 23))) {
      if (fam == 4 || (fam == 0 && kRegPackedDefault)) {
        switch (tb) {
          case 2: return launch_reg2_t<2, false, true>(f, src, dst, rho, k, rep, sched, sched_cap, st);
          case 3: return launch_reg2_t<3, false, true>(f, src, dst, rho, k, rep, sched, sched_cap, st);
          case 4: return launch_reg2_t<4, false, true>(f, src, dst, rho, k, rep, sched, sched_cap, st);
          case 5: return launch_reg2_t<5, false, true>(f, src, dst, rho, k, rep, sched, sched_cap, st);
          case 6: return launch_reg2_t<6, false, true>(f, src, dst, rho, k, rep, sched, sched_cap, st);
          case 7: return launch_reg2_t<7, false, true>(f, src, dst, rho, k, rep, sched, sched_cap, st);
          case 8: return launch_reg2_t<8, false, true>(f, src, dst, rho, k, rep, sched, sched_cap, st);
          default: return cudaErrorInvalidValue;
        }
      }
      switch (tb) {
        case 2: return launch_reg2_t<2>(f, src, dst, rho, k, rep, sched, sched_cap, st);
        case 3: return launch_reg2_t<3>(f, src, dst, rho, k, rep, sched, sched_cap, st);
        case 4: return launch_reg2_t<4>(f, src, dst, rho, k, rep, sched, sched_cap, st);
        case 5: return launch_reg2_t<5>(f, src, dst, rho, k, rep, sched, sched_cap, st);
        case 6: return launch_reg2_t<6>(f, src, dst, rho, k, rep, sched, sched_cap, st);
        case 7: return launch_reg2_t<7>(f, src, dst, rho, k, rep, sched, sched_cap, st);
        case 8: return launch_reg2_t<8>(f, src, dst, rho, k, rep, sched, sched_cap, st);
        default: return cudaErrorInvalidValue;
      }
    }
    if (fam == 2 || (fam == 0 && tb != 6 && tb != 7)) {
      switch (tb) {
        case 2: return launch_wave2_t<2>(f, src, dst, rho, k, rep, st);
        case 3: return launch_wave2_t<3>(f, src, dst, rho, k, rep, st);
        case 4: return launch_wave2_t<4>(f, src, dst, rho, k, rep, st);
        case 5: return launch_wave2_t<5>(f, src, dst, rho, k, rep, st);
        case 6: return launch_wave2_t<6>(f, src, dst, rho, k, rep, st);
        case 7: return launch_wave2_t<7>(f, src, dst, rho, k, rep, st);
        case 8: return launch_wave2_t<8>(f, src, dst, rho, k, rep, st);
        default: return cudaErrorInvalidValue;
      }
    }
    switch (tb) {
      case 2: return launch_wave_t<2>(f, src, dst, rho, k, rep, st);
      case 3: return launch_wave_t<3>(f, src, dst, rho, k, rep, st);
      case 4: return launch_wave_t<4>(f, src, dst, rho, k, rep, st);
      case 5: return launch_wave_t<5>(f, src, dst, rho, k, rep, st);
      case 6: return launch_wave_t<6>(f, src, dst, rho, k, rep, st);
      case 7: return launch_wave_t<7>(f, src, dst, rho, k, rep, st);
      case 8: return launch_wave_t<8>(f, src, dst, rho, k, rep, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (tb) {
    case 2: return launch_tile_t<T, 2>(f, src, dst, rho, k, rep, st);
    case 3: return launch_tile_t<T, 3>(f, src, dst, rho, k, rep, st);
    case 4: return launch_tile_t<T, 4>(f, src, dst, rho, k, rep, st);
    case 5: return launch_tile_t<T, 5>(f, src, dst, rho, k, rep, st);
    case 6: return launch_tile_t<T, 6>(f, src, dst, rho, k, rep, st);
    case 7: return launch_tile_t<T, 7>(f, src, dst, rho, k, rep, st);
    case 8: return launch_tile_t<T, 8>(f, src, dst, rho, k, rep, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

int dev_index() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  return dev < 0 ? 0 : (dev > 63 ? 63 : dev);
}

int device_sm_count() {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 148;
  if (g_sms[dev] == 0) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    g_sms[dev] = n > 0 ? n : 148;
  }
  return g_sms[dev];
}

cudaError_t launch_rbsor_reg(const FieldDesc& f, const float* src, float* dst, const float* rho,
                             double omega, int sweeps, double* resid, int s0, int every,
                             unsigned long long* sched, int sched_cap, cudaStream_t st,
                             const Prolong* pl) {
  Reports rep;
  rep.resid = (resid && every > 0) ? resid : nullptr;
  rep.s0 = s0;
  rep.every = every > 0 ? every : 1;
  Coef<float> k;
  k.c = (float)(omega * f.h * f.h / 4.0);
  k.ih2 = (float)(1.0 / (f.h * f.h));
  switch (sweeps) {
    case 1: return launch_reg2_t<2, true>(f, src, dst, rho, k, rep, sched, sched_cap, st, pl);
    case 2: return launch_reg2_t<4, true>(f, src, dst, rho, k, rep, sched, sched_cap, st, pl);
    case 3: return launch_reg2_t<6, true>(f, src, dst, rho, k, rep, sched, sched_cap, st, pl);
    case 4: return launch_reg2_t<8, true>(f, src, dst, rho, k, rep, sched, sched_cap, st, pl);
    default: return cudaErrorInvalidValue;
  }
}

bool vector_ok(const FieldDesc& f, const void* a, const void* b, const void* c) {
  if (f.ghost) return false;
  const int V = f.dtype == 0 ? 2 : 4;
  if (f.nx % V != 0 || f.ld % V != 0) return false;
  auto al = [](const void* p) { return ((uintptr_t)p & 15u) == 0; };
  return al(a) && al(b) && al(c);
}

cudaError_t launch_relax(const FieldDesc& f, const void* src, void* dst, const void* rho,
                         double omega, int tb, bool vec, double* resid, int s0,
                         int every, unsigned long long* sched, int sched_cap, cudaStream_t st) {
  Reports rep;
  rep.resid = (resid && every > 0) ? resid : nullptr;
  rep.s0 = s0;
  rep.every = every > 0 ? every : 1;
  if (!vec) tb = 1;
  if (f.dtype == 0)
    return launch_relax_t<double>(f, (const double*)src, (double*)dst, (const double*)rho,
                                  omega, tb, vec, rep, sched, sched_cap, st);
  return launch_relax_t<float>(f, (const float*)src, (float*)dst, (const float*)rho, omega,
                               tb, vec, rep, sched, sched_cap, st);
}

}  // namespace px

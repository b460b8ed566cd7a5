// 2D Euler finite-volume step (the paper's second workload: Sec. IV, the
// Euler result of Fig. "Euler"; Sec. V), fused: one kernel per Runge-Kutta
// stage does what an operator library runs as separate passes over memory
// (primitive variables, limited slopes, face states, Rusanov fluxes, flux
// divergence, the stage update and, in the second stage, the maximum wave
// speed of the new state for the next step's time step).
//
// Scheme (the paper gives none; the textbook second-order one): cell averages
// U = (rho, rho u, rho v, E) of an ideal gas, p = (gamma - 1)(E - rho |u|^2 / 2);
// minmod-limited piecewise-linear reconstruction of (rho, u, v, p); Rusanov
// flux F = (F(W_L) + F(W_R)) / 2 - a (U_R - U_L) / 2 with
// a = max(|u_n| + c) over the two face states; SSP-RK2
//   U1 = U + dt L(U),   U' = (U + (U1 + dt L(U1))) / 2,
// dt = cfl / max((|u| + c) / dx + (|v| + c) / dy) over the cells of U.
//
// Layout: four component planes (rho, rho u, rho v, E), each ny rows of nx
// cells with row pitch ld, planes cs elements apart; periodic in x and y.
//
// Tiling: a CTA of 256 threads computes a TX x TY = 32 x 16 tile. It loads the
// tile and a two-cell periodic halo, converts it to primitives in shared
// memory, computes each of the (TX + 1) TY x-face and TX (TY + 1) y-face fluxes
// once into shared memory, then updates its cells from the flux differences.
// Grid-stride over tiles, one resident wave of CTAs.
#include "px_internal.cuh"

#include <cuda.h>

#include <algorithm>
#include <cfloat>
#include <cstring>

namespace px {
namespace {

constexpr int kETX = 32, kETY = 16, kEHalo = 2;
constexpr int kEWX = kETX + 2 * kEHalo, kEWY = kETY + 2 * kEHalo;  // 36 x 20
constexpr int kEThreads = 256;

constexpr int kEWP = kEWX + 1;  // row pitch 37: the x-face threads of a warp (4 rows x 8
                                // segments 4 cells apart) hit 32 different banks
// Raw rows of the next tile: the halo's first column sits at kRawOff so that
// the row starts on a 16-byte boundary of the field when the tile is copied
// as one tensor-memory-accelerator box (x0 is a multiple of 32).
template <typename T> struct RawGeom {
  static constexpr int kOff = sizeof(T) == 4 ? 2 : 0;  // x0 - 2 - kOff is 16-byte aligned
  static constexpr int kW = kEWX + 2 * kOff;          // 40 (FP32) or 36 (FP64) columns
};

template <typename T>
struct ESmem {
  T raw[4][kEWY][RawGeom<T>::kW];  // conserved values of the next tile + halo
  T w[4][kEWY][kEWP];        // primitives rho, u, v, p of the tile and its halo
  T fx[4][kETY][kETX + 1];   // x-face fluxes: fx[.][j][k] at face k - 1/2 of row j
  T fy[4][kETY + 1][kETX];   // y-face fluxes: fy[.][j][i] at face j - 1/2 of column i
  uint64_t wmax[kEThreads / 32];  // per-warp wave-speed maxima (stage 2)
  uint64_t bar;                   // completion barrier of the box copy
};
// raw must start on a 128-byte boundary for the box copy; the kernel declares
// no static shared variables, so it sits at the dynamic block's start.
static_assert(sizeof(ESmem<float>::raw) % 128 == 0 && sizeof(ESmem<double>::raw) % 128 == 0,
              "raw is followed by the other arrays");

// Reciprocal and sound speed sqrt(g p / rho) (g p passed as gp), the latter
// as c = gp rsqrt(gp rho): no division and no square root. FP32 takes the
// hardware approximations (relative error about 2^-22, far below the storage's
// own rounding of the fluxes); FP64 the IEEE reciprocal and the library's
// rsqrt (1 ulp), which costs the FP64 pipe about half of an IEEE division and
// square root. The smallest normal number is added to gp rho (in the FMA that
// forms the product, so at no cost): at p = 0 the product form would otherwise
// be 0 * inf, and it gives c = 0 as sqrt(0 / rho) does; for gp rho well above
// that number the rounded sum is the rounded product (one ulp apart only when
// the exact product lies within the added number of a rounding midpoint), and a
// negative or NaN pressure still gives NaN.
template <typename T> __device__ __forceinline__ T recip(T v);
template <> __device__ __forceinline__ float recip<float>(float v) { return __fdividef(1.0f, v); }
template <> __device__ __forceinline__ double recip<double>(double v) { return 1.0 / v; }
template <typename T> __device__ __forceinline__ T sound(T gp, T rho);
template <> __device__ __forceinline__ float sound<float>(float gp, float rho) {
  return gp * rsqrtf(fmaf(gp, rho, FLT_MIN));
}
template <> __device__ __forceinline__ double sound<double>(double gp, double rho) {
  return gp * rsqrt(fma(gp, rho, DBL_MIN));
}

template <typename T>
__device__ __forceinline__ T minmod(T a, T b) {
  return a * b <= T(0) ? T(0) : (fabs(a) < fabs(b) ? a : b);
}

template <typename T>
struct EParams {
  const T* u0;     // state at the start of the step
  const T* u1;     // stage-1 state (stage 2 only)
  T* out;
  int nx, ny;
  int64_t ld, cs;
  T gamma, gm1, igm1;  // gamma, gamma - 1, 1 / (gamma - 1)
  T idx, idy;          // 1 / dx, 1 / dy
  double dx, dy;
  double cfl, dt_fixed;
  double* wave_cur;    // max wave speed of u0 (dt source when dt_fixed == 0)
  double* wave_next;   // stage 1 zeroes it, stage 2 folds the new state's max into it
  double* dt_out;      // this step's dt (stage 1 writes it) or null
  int tiles_x, ntiles;
  int use_tma;         // tmap describes the stage's source planes
  CUtensorMap tmap;    // (x, y, plane) boxes of kW x 20 x 4
};

// Rusanov flux through one face from the cells b | c that straddle it and
// their limited slopes sb, sc along the face normal. Component order rho, u,
// v, p; kXFace selects the normal velocity (u for x faces, v for y faces).
template <typename T, bool kXFace>
__device__ __forceinline__ void face_flux(const T (&b)[4], const T (&sb)[4], const T (&c)[4],
                                          const T (&sc)[4], T gamma, T igm1, T (&f)[4]) {
  T L[4], R[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    L[q] = b[q] + T(0.5) * sb[q];
    R[q] = c[q] - T(0.5) * sc[q];
  }
  const T unL = kXFace ? L[1] : L[2], unR = kXFace ? R[1] : R[2];
  const T EL = L[3] * igm1 + T(0.5) * L[0] * (L[1] * L[1] + L[2] * L[2]);
  const T ER = R[3] * igm1 + T(0.5) * R[0] * (R[1] * R[1] + R[2] * R[2]);
  const T cL = sound(gamma * L[3], L[0]), cR = sound(gamma * R[3], R[0]);
  const T am = fmax(fabs(unL) + cL, fabs(unR) + cR);
  const T mL = L[0] * unL, mR = R[0] * unR;  // mass fluxes
  const T FL1 = mL * L[1] + (kXFace ? L[3] : T(0)), FR1 = mR * R[1] + (kXFace ? R[3] : T(0));
  const T FL2 = mL * L[2] + (kXFace ? T(0) : L[3]), FR2 = mR * R[2] + (kXFace ? T(0) : R[3]);
  const T FL3 = unL * (EL + L[3]), FR3 = unR * (ER + R[3]);
  f[0] = T(0.5) * (mL + mR) - T(0.5) * am * (R[0] - L[0]);
  f[1] = T(0.5) * (FL1 + FR1) - T(0.5) * am * (R[0] * R[1] - L[0] * L[1]);
  f[2] = T(0.5) * (FL2 + FR2) - T(0.5) * am * (R[0] * R[2] - L[0] * L[2]);
  f[3] = T(0.5) * (FL3 + FR3) - T(0.5) * am * (ER - EL);
}

// Fluxes of a run of consecutive faces along one line of the shared tile:
// faces f0 .. f0 + nf - 1 (nf = 4 or 5), face f lying between the cells at
// line positions f + 1 and f + 2 (position p of the line is element
// base + p * step). The cell window slides along the line, so each cell is
// read once and its slope computed once for the run; the loop is unrolled
// (the window's shift is register renaming, the offsets immediates) and the
// fifth face is predicated. Flux of face f goes to out + f * ostep.
template <typename T, bool kXFace, int kStep, int kPlane, int kOStep, int kOPlane>
__device__ __forceinline__ void face_run(const T* base, int f0, int nf, T* out, T gamma, T igm1) {
  const T* b0 = base + f0 * kStep;
  T* o0 = out + f0 * kOStep;
  T w0[4], w1[4], w2[4], s1[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    w0[m] = b0[m * kPlane];
    w1[m] = b0[m * kPlane + kStep];
    w2[m] = b0[m * kPlane + 2 * kStep];
    s1[m] = minmod(w1[m] - w0[m], w2[m] - w1[m]);
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    if (k < nf) {
      T w3[4], s2[4], fl[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        w3[m] = b0[m * kPlane + (k + 3) * kStep];
        s2[m] = minmod(w2[m] - w1[m], w3[m] - w2[m]);
      }
      face_flux<T, kXFace>(w1, s1, w2, s2, gamma, igm1, fl);
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        o0[m * kOPlane + k * kOStep] = fl[m];
        w1[m] = w2[m];
        w2[m] = w3[m];
        s1[m] = s2[m];
      }
    }
  }
}

template <typename T>
__device__ __forceinline__ double wave_speed(T r, T mx, T my, T e, T gamma, T gm1, T idx, T idy) {
  const T ir = recip(r);
  const T u = mx * ir, v = my * ir;
  const T p = gm1 * (e - T(0.5) * r * (u * u + v * v));
  const T c = sound(gamma * p, r);
  return (double)((fabs(u) + c) * idx + (fabs(v) + c) * idy);
}

template <int kBytes>
__device__ __forceinline__ void cp_async_elem(void* sdst, const void* gsrc) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(gsrc), "n"(kBytes)
               : "memory");
}

// Issue the copies of one tile and its two-cell periodic halo (four planes)
// into S.raw. A tile whose halo lies inside the field is one box of the
// tensor memory accelerator (kW x 20 x 4 planes), issued by thread 0 on the
// CTA's barrier `bar` (expect-tx bytes); returns true. Otherwise every cell
// is a cp.async of its own (the periodic images), one commit group; false.
template <typename T>
__device__ __forceinline__ bool prefetch_tile(ESmem<T>& S, const T* src, int tile, int tiles_x,
                                              int nx, int ny, int64_t ld, int64_t cs,
                                              bool near_x, bool near_y, const CUtensorMap* tmap,
                                              bool use_tma, uint32_t bar) {
  using RG = RawGeom<T>;
  const int ty = tile / tiles_x, tx = tile - ty * tiles_x;
  const int x0 = tx * kETX, y0 = ty * kETY;
  const int xs = x0 - kEHalo - RG::kOff, ys = y0 - kEHalo;
  if (use_tma && xs >= 0 && xs + RG::kW <= nx && ys >= 0 && ys + kEWY <= ny) {
    if (threadIdx.x == 0) {
      // the buffer's earlier (generic) reads are ordered before the async copy
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                   ::"r"(bar), "r"((uint32_t)(4 * kEWY * RG::kW * sizeof(T))) : "memory");
      asm volatile(
          "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
          "[%0], [%1, {%2, %3, %4}], [%5];"
          ::"r"((uint32_t)__cvta_generic_to_shared(&S.raw[0][0][0])),
            "l"(reinterpret_cast<uint64_t>(tmap)), "r"(xs), "r"(ys), "r"(0), "r"(bar)
          : "memory");
    }
    return true;
  }
  for (int q = threadIdx.x; q < kEWX * kEWY; q += kEThreads) {
    const int ly = q / kEWX, lx = q - ly * kEWX;
    const int gx = near_x ? wrap1(x0 + lx - kEHalo, nx) : wrapn(x0 + lx - kEHalo, nx);
    const int gy = near_y ? wrap1(y0 + ly - kEHalo, ny) : wrapn(y0 + ly - kEHalo, ny);
    const int64_t o = (int64_t)gy * ld + gx;
    if (!PX_IN_RANGE(21, gx, 0, nx) || !PX_IN_RANGE(22, gy, 0, ny)) continue;
#pragma unroll
    for (int m = 0; m < 4; ++m)
      cp_async_elem<sizeof(T)>(&S.raw[m][ly][lx + RG::kOff], src + m * cs + o);
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  return false;
}

// Bounded wait for a tile box's bytes (phase `parity` of `bar`); false if the
// limit ran out (the results are then meaningless and the next step's wave
// speed is set to NaN, which makes its dt and state NaN).
__device__ __forceinline__ bool wait_box(uint32_t bar, uint32_t parity) {
  for (uint32_t it = 0; it < (1u << 26); ++it) {
    uint32_t done;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 "selp.u32 %0, 1, 0, p;\n}" : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ uint64_t dbits(double v) {
  return (uint64_t)__double_as_longlong(v) & 0x7fffffffffffffffull;
}

template <typename T, int kStage>
__global__ void __launch_bounds__(kEThreads)
euler_stage_k(const __grid_constant__ EParams<T> P) {
  // no static shared variables: S.raw, the box copy's destination, must start
  // on a 128-byte boundary, and the tensor map on a 64-byte one; if either
  // does not, every tile takes the per-cell copies
  extern __shared__ __align__(128) unsigned char esm_raw[];
  ESmem<T>& S = *reinterpret_cast<ESmem<T>*>(esm_raw);
  const int tid = threadIdx.x;
  const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&S.bar);
  const bool use_tma = P.use_tma &&
                       ((uint32_t)__cvta_generic_to_shared(&S.raw[0][0][0]) & 127u) == 0 &&
                       (reinterpret_cast<uintptr_t>(&P.tmap) & 63u) == 0;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  uint32_t box_parity = 0;
  bool box_pending = false, box_fault = false;
  // this step's dt
  double dtd = P.dt_fixed;
  if (!(dtd > 0.0)) dtd = P.cfl / *P.wave_cur;
  const T dt = (T)dtd;
  if (kStage == 1 && blockIdx.x == 0 && tid == 0) {
    if (P.dt_out) *P.dt_out = dtd;
    if (P.wave_next) *P.wave_next = 0.0;
  }
  const T* src = kStage == 1 ? P.u0 : P.u1;
  const bool near_x = P.nx >= kEWX, near_y = P.ny >= kEWY;
  uint64_t wm = 0;

  if ((int)blockIdx.x < P.ntiles)
    box_pending = prefetch_tile(S, src, blockIdx.x, P.tiles_x, P.nx, P.ny, P.ld, P.cs, near_x,
                                near_y, &P.tmap, use_tma, bar);
  for (int tile = blockIdx.x; tile < P.ntiles; tile += gridDim.x) {
    const int ty = tile / P.tiles_x, tx = tile - ty * P.tiles_x;
    const int x0 = tx * kETX, y0 = ty * kETY;
    // this tile's copies have landed (each thread waits for its own, the
    // barrier for everyone's); the previous tile's fluxes are consumed
    if (box_pending) {
      if (!wait_box(bar, box_parity)) box_fault = true;
      box_parity ^= 1u;
    } else {
      asm volatile("cp.async.wait_all;\n" ::: "memory");
    }
    __syncthreads();
    // ---- primitives of the tile + halo
    for (int q = tid; q < kEWX * kEWY; q += kEThreads) {
      const int ly = q / kEWX, lx = q - ly * kEWX + RawGeom<T>::kOff;
      const T r = S.raw[0][ly][lx], mx = S.raw[1][ly][lx], my = S.raw[2][ly][lx],
              e = S.raw[3][ly][lx];
      const T ir = recip(r);
      const T u = mx * ir, v = my * ir;
      const int wx = lx - RawGeom<T>::kOff;
      S.w[0][ly][wx] = r;
      S.w[1][ly][wx] = u;
      S.w[2][ly][wx] = v;
      S.w[3][ly][wx] = P.gm1 * (e - T(0.5) * r * (u * u + v * v));
    }
    __syncthreads();
    // the raw buffer is free: start the next tile's copies under this tile's fluxes
    if (tile + (int)gridDim.x < P.ntiles)
      box_pending = prefetch_tile(S, src, tile + (int)gridDim.x, P.tiles_x, P.nx, P.ny, P.ld,
                                  P.cs, near_x, near_y, &P.tmap, use_tma, bar);
    // ---- face fluxes. Warps 0-3: x faces, one run of 4 faces (5 for the last
    // segment of a row) per thread, rows 4w + lane / 8, segment lane % 8.
    // Warps 4-7: y faces, column lane, segment w - 4 of 4 faces (5 last).
    {
      const int warp = tid >> 5, lane = tid & 31;
      if (warp < 4) {
        const int j = 4 * warp + (lane >> 3), sg = lane & 7;
        face_run<T, true, 1, kEWY * kEWP, 1, kETY * (kETX + 1)>(
            &S.w[0][j + kEHalo][0], 4 * sg, sg == 7 ? 5 : 4, &S.fx[0][j][0], P.gamma, P.igm1);
      } else {
        const int i = lane, sg = warp - 4;
        face_run<T, false, kEWP, kEWY * kEWP, kETX, (kETY + 1) * kETX>(
            &S.w[0][0][i + kEHalo], 4 * sg, sg == 3 ? 5 : 4, &S.fy[0][0][i], P.gamma, P.igm1);
      }
    }
    __syncthreads();
    // ---- update the tile's cells
    for (int q = tid; q < kETX * kETY; q += kEThreads) {
      const int j = q / kETX, i = q - j * kETX;
      const int gx = x0 + i, gy = y0 + j;
      if (gx >= P.nx || gy >= P.ny) continue;
      if (!PX_IN_RANGE(23, gx, 0, P.nx) || !PX_IN_RANGE(24, gy, 0, P.ny)) continue;
      const int64_t o = (int64_t)gy * P.ld + gx;
      T nv[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const T Lm = -(S.fx[m][j][i + 1] - S.fx[m][j][i]) * P.idx -
                     (S.fy[m][j + 1][i] - S.fy[m][j][i]) * P.idy;
        const T um = __ldg(src + m * P.cs + o);
        if (kStage == 1) {
          nv[m] = um + dt * Lm;
        } else {
          nv[m] = T(0.5) * (__ldg(P.u0 + m * P.cs + o) + (um + dt * Lm));
        }
        P.out[m * P.cs + o] = nv[m];
      }
      if (kStage == 2 && P.wave_next)
        wm = umax(wm, dbits(wave_speed(nv[0], nv[1], nv[2], nv[3], P.gamma, P.gm1, P.idx, P.idy)));
    }
  }
  if (box_fault && P.wave_next) atomic_max_bits(P.wave_next, 0x7ff8000000000000ull);  // NaN
  if (kStage == 2 && P.wave_next) {
    wm = warp_max(wm);
    if ((tid & 31) == 0) S.wmax[tid >> 5] = wm;
    __syncthreads();
    if (tid == 0) {
      uint64_t m = 0;
#pragma unroll
      for (int w = 0; w < kEThreads / 32; ++w) m = umax(m, S.wmax[w]);
      atomic_max_bits(P.wave_next, m);
    }
  }
}

// Max wave speed of a state (the first step's dt source).
template <typename T>
__global__ void __launch_bounds__(kEThreads)
euler_wave_k(const T* __restrict__ u, int nx, int ny, int64_t ld, int64_t cs, T gamma, T gm1,
             T idx, T idy, double* slot) {
  __shared__ uint64_t sm[kEThreads / 32];
  uint64_t m = 0;
  const int64_t n = (int64_t)nx * ny;
  for (int64_t q = blockIdx.x * (int64_t)kEThreads + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * kEThreads) {
    const int64_t y = q / nx, x = q - y * nx;
    const int64_t o = y * ld + x;
    m = umax(m, dbits(wave_speed(u[o], u[cs + o], u[2 * cs + o], u[3 * cs + o], gamma, gm1, idx, idy)));
  }
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t t = 0;
    for (int w = 0; w < kEThreads / 32; ++w) t = umax(t, sm[w]);
    atomic_max_bits(slot, t);
  }
}

// Conserved variables from primitives (rho, u, v, p), same layout.
template <typename T>
__global__ void euler_conserved_k(const T* __restrict__ w, T* __restrict__ u, int nx, int ny,
                                  int64_t ld, int64_t cs, T igm1) {
  const int64_t n = (int64_t)nx * ny;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t y = q / nx, x = q - y * nx;
    const int64_t o = y * ld + x;
    const T r = w[o], vx = w[cs + o], vy = w[2 * cs + o], p = w[3 * cs + o];
    u[o] = r;
    u[cs + o] = r * vx;
    u[2 * cs + o] = r * vy;
    u[3 * cs + o] = p * igm1 + T(0.5) * r * (vx * vx + vy * vy);
  }
}

template <typename T>
cudaError_t euler_setup_t() {
  static bool done_by_dev[64] = {};
  bool& done = done_by_dev[dev_index()];
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(euler_stage_k<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(ESmem<T>));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(euler_stage_k<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(ESmem<T>));
  if (e == cudaSuccess) done = true;
  return e;
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
// cuTensorMapEncodeTiled through the runtime's driver entry point; null if
// unavailable (the per-cell copies are used then).
EncodeTiledFn euler_encoder() {
  static EncodeTiledFn fn = nullptr;
  static bool resolved = false;
  if (!resolved) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess && q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(f);
    cudaGetLastError();
    resolved = true;
  }
  return fn;
}

// Tensor map of the four planes of a state for tile boxes (kW x 20 x 4); false
// if the layout does not allow one (pitches not multiples of 16 bytes, a field
// narrower than the box, a misaligned base) or the driver cannot encode it.
template <typename T>
bool euler_tensor_map(CUtensorMap* m, const EulerDesc& g, const T* base) {
  std::memset(m, 0, sizeof *m);
  const EncodeTiledFn enc = euler_encoder();
  const int64_t es = sizeof(T);
  if (!enc || ((uintptr_t)base & 15u) || (g.ld * es) % 16 || (g.cs * es) % 16 ||
      g.nx < RawGeom<T>::kW || g.ny < kEWY)
    return false;
  const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, 4};
  const cuuint64_t strides[2] = {(cuuint64_t)(g.ld * es), (cuuint64_t)(g.cs * es)};
  const cuuint32_t box[3] = {(cuuint32_t)RawGeom<T>::kW, (cuuint32_t)kEWY, 4};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(m, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
             3, const_cast<T*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename T>
cudaError_t euler_step_t(const EulerDesc& g, const T* u0, T* out, T* s1, double gamma, double cfl,
                         double dt_fixed, double* wave_cur, double* wave_next, double* dt_out,
                         cudaStream_t st) {
  cudaError_t e = euler_setup_t<T>();
  if (e != cudaSuccess) return e;
  static int occ_by_dev[64] = {};
  int& occ = occ_by_dev[dev_index()];
  if (occ == 0) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, euler_stage_k<T, 2>, kEThreads,
                                                      sizeof(ESmem<T>));
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
  }
  EParams<T> P;
  P.u0 = u0;
  P.u1 = s1;
  P.nx = g.nx;
  P.ny = g.ny;
  P.ld = g.ld;
  P.cs = g.cs;
  P.gamma = (T)gamma;
  P.gm1 = (T)(gamma - 1.0);
  P.igm1 = (T)(1.0 / (gamma - 1.0));
  P.idx = (T)(1.0 / g.dx);
  P.idy = (T)(1.0 / g.dy);
  P.dx = g.dx;
  P.dy = g.dy;
  P.cfl = cfl;
  P.dt_fixed = dt_fixed;
  P.wave_cur = wave_cur;
  P.wave_next = wave_next;
  P.dt_out = dt_out;
  P.tiles_x = (g.nx + kETX - 1) / kETX;
  const int64_t tiles = (int64_t)P.tiles_x * ((g.ny + kETY - 1) / kETY);
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  P.ntiles = (int)tiles;
  const int grid = (int)std::min<int64_t>(tiles, (int64_t)occ * device_sm_count());
  // stage 1: u0 -> s1
  P.out = s1;
  P.use_tma = euler_tensor_map<T>(&P.tmap, g, u0) ? 1 : 0;
  euler_stage_k<T, 1><<<grid, kEThreads, sizeof(ESmem<T>), st>>>(P);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // stage 2: (u0, s1) -> out, max wave speed of out -> wave_next
  P.out = out;
  P.dt_out = nullptr;
  P.use_tma = euler_tensor_map<T>(&P.tmap, g, s1) ? 1 : 0;
  euler_stage_k<T, 2><<<grid, kEThreads, sizeof(ESmem<T>), st>>>(P);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_euler_wave(const EulerDesc& g, const void* u, double gamma, double* slot,
                              cudaStream_t st) {
  const int64_t n = (int64_t)g.nx * g.ny;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + kEThreads - 1) / kEThreads,
                                                                 (int64_t)device_sm_count() * 8));
  if (g.dtype == 0)
    euler_wave_k<double><<<blocks, kEThreads, 0, st>>>((const double*)u, g.nx, g.ny, g.ld, g.cs,
                                                       gamma, gamma - 1.0, 1.0 / g.dx, 1.0 / g.dy, slot);
  else
    euler_wave_k<float><<<blocks, kEThreads, 0, st>>>((const float*)u, g.nx, g.ny, g.ld, g.cs,
                                                      (float)gamma, (float)(gamma - 1.0),
                                                      (float)(1.0 / g.dx), (float)(1.0 / g.dy), slot);
  return cudaGetLastError();
}

cudaError_t launch_euler_step(const EulerDesc& g, const void* u0, void* out, void* s1, double gamma,
                              double cfl, double dt_fixed, double* wave_cur, double* wave_next,
                              double* dt_out, cudaStream_t st) {
  if (g.dtype == 0)
    return euler_step_t<double>(g, (const double*)u0, (double*)out, (double*)s1, gamma, cfl,
                                dt_fixed, wave_cur, wave_next, dt_out, st);
  return euler_step_t<float>(g, (const float*)u0, (float*)out, (float*)s1, gamma, cfl, dt_fixed,
                             wave_cur, wave_next, dt_out, st);
}

cudaError_t launch_euler_conserved(const EulerDesc& g, const void* w, void* u, double gamma,
                                   cudaStream_t st) {
  const int64_t n = (int64_t)g.nx * g.ny;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256,
                                                                 (int64_t)device_sm_count() * 8));
  if (g.dtype == 0)
    euler_conserved_k<double><<<blocks, 256, 0, st>>>((const double*)w, (double*)u, g.nx, g.ny,
                                                      g.ld, g.cs, 1.0 / (gamma - 1.0));
  else
    euler_conserved_k<float><<<blocks, 256, 0, st>>>((const float*)w, (float*)u, g.nx, g.ny, g.ld,
                                                     g.cs, (float)(1.0 / (gamma - 1.0)));
  return cudaGetLastError();
}

}  // namespace px

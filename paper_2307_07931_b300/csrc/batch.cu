// Batched relaxation of many independent periodic Poisson instances of uneven
// sizes in ONE persistent launch (replayed from a CUDA graph).
//
// Each instance runs nsweeps fused sweeps (the Sec. IV merged loop: Laplace,
// weighted Jacobi of Eq. "jacobi", residual max-norm of each reported input
// state). Instances are independent, so the batch shards with no exchange.
// Two execution modes, chosen per size class by the autotuner:
//  * WHOLE: one CTA holds the instance (both ping-pong copies) in shared
//    memory and runs every sweep there; rho is read through the read-only
//    cache. No global traffic per sweep.
//  * BANDED: a thread-block cluster of csize CTAs shares the instance; CTA r
//    sweeps rows [r*band, (r+1)*band) from global memory (the instance stays
//    L2-resident) with warps streaming 32*V-wide strips, and the cluster's
//    hardware barrier separates sweeps. The caller's phi and a plan-owned
//    scratch field ping-pong; an odd sweep count ends with a copy back.
// A sweep that reports no residual needs only the update, which reads
//   phi' = (1 - omega) C + (omega / 4) q - c rho,  q = (W + E) + (S + N):
// three additions and two FMAs once -c rho is stored (BANDED FP64 instances
// keep it in a plan-owned field, written by each CTA for its own rows), one
// FP64 operation fewer than the residual form; FP64 sweeps are bound by the
// FP64 pipe. Reported sweeps take the residual form.
//  * BANDED_T: BANDED with temporal blocking. Each CTA covers its rows in
//    tiles of kTY x kTX cells; a tile and a halo of tb cells per side (the
//    periodic images, read from the other CTAs' rows of the previous block)
//    are loaded into shared memory with rho, swept tb times there (the valid
//    region shrinking by one cell per side and sweep) and its own cells
//    written back: one cluster barrier and one pass over the instance per tb
//    sweeps. The per-cell arithmetic is that of band_sweep, so the states are
//    bitwise those of BANDED.
// The host assigns BANDED instances to clusters and WHOLE instances to CTAs
// (longest first, to the least loaded, with costs from the tuned rates), so
// every CTA of a cluster executes the same sequence of cluster barriers and
// no CTA ever waits on a flag: there is no spin-wait in this kernel.
#include "px_internal.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

namespace cg = cooperative_groups;

namespace px {

constexpr int kBatchThreads = 512;
constexpr int kMaxCluster = 8;
constexpr size_t kWholeSmem = 200 * 1024;  // shared bytes for WHOLE instances

namespace {

template <typename T> struct V2;
template <> struct V2<float> { using type = float4; static constexpr int n = 4; };
template <> struct V2<double> { using type = double2; static constexpr int n = 2; };

template <typename T, int V>
__device__ __forceinline__ void ldvec(T (&v)[V], const T* p) {
  *reinterpret_cast<typename V2<T>::type*>(v) = *reinterpret_cast<const typename V2<T>::type*>(p);
}

template <typename MB>
__device__ __forceinline__ void block_report(MB mx, double* slot, MB* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  mx = warp_max(mx);
  if (lane == 0) red[warp] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    MB m = 0;
    for (int w = 0; w < kBatchThreads / 32; ++w) m = umax(m, red[w]);
    atomic_max_bits(slot, to_f64_bits(m));
  }
  __syncthreads();
}

// One sweep of rows [ra, rb) of an instance from src into dst, by the warps of
// this CTA: tasks are (strip of 32*V columns) x (ry rows); a warp keeps rows
// j-1, j, j+1 in registers, x neighbours come from shuffles and the strip-edge
// scalars from memory. Requires nx % V == 0, ld % V == 0, 16-byte alignment.
template <typename T, bool kRep, bool kScaled = false>
__device__ __forceinline__ typename MaxBits<T>::type
band_sweep(const T* __restrict__ src, T* __restrict__ dst, const T* __restrict__ rho, int nx,
           int ny, int64_t ld, int ra, int rb, int ry, T c, T ih2, T a1 = 0, T w4 = 0) {
  constexpr int V = V2<T>::n;
  constexpr int SW = 32 * V;
  using MB = typename MaxBits<T>::type;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = kBatchThreads / 32;
  const int nstrips = (nx + SW - 1) / SW;
  const int nseg = (rb - ra + ry - 1) / ry;
  MB mx = 0;
  for (int task = warp; task < nstrips * nseg; task += nw) {
    const int strip = task % nstrips, seg = task / nstrips;
    const int xs = strip * SW, x = xs + lane * V;
    const bool valid = x < nx;
    const int xc = valid ? x : xs;
    const int xend = min(xs + SW, nx);
    const bool need_l = lane == 0, need_r = valid && (x + V >= xend);
    const int xl = wrap1(xs - 1, nx), xr = wrap1(x + V, nx);
    const int j0 = ra + seg * ry, j1 = min(j0 + ry, rb);
    T up[V], cu[V], dn[V];
    T cel = 0, cer = 0;
    ldvec<T, V>(up, src + (int64_t)wrap1(j0 - 1, ny) * ld + xc);
    {
      const T* rp = src + (int64_t)j0 * ld;
      ldvec<T, V>(cu, rp + xc);
      if (need_l) cel = rp[xl];
      if (need_r) cer = rp[xr];
    }
    for (int j = j0; j < j1; ++j) {
      const T* np = src + (int64_t)wrap1(j + 1, ny) * ld;
      ldvec<T, V>(dn, np + xc);
      T nel = 0, ner = 0;
      if (need_l) nel = np[xl];
      if (need_r) ner = np[xr];
      T rh[V];
      ldvec<T, V>(rh, rho + (int64_t)j * ld + xc);
      T l0 = __shfl_up_sync(0xffffffffu, cu[V - 1], 1);
      T rV = __shfl_down_sync(0xffffffffu, cu[0], 1);
      if (need_l) l0 = cel;
      if (need_r) rV = cer;
      T o[V];
#pragma unroll
      for (int i = 0; i < V; ++i) {
        const T w = i == 0 ? l0 : cu[i - 1];
        const T e = i == V - 1 ? rV : cu[i + 1];
        const T q = (w + e) + (up[i] + dn[i]);
        if constexpr (kScaled && !kRep) {
          o[i] = fma(w4, q, fma(a1, cu[i], rh[i]));  // rh holds -c rho
        } else {
          const T s = fma((T)-4, cu[i], q);
          const T r = fma(s, ih2, -rh[i]);
          o[i] = fma(c, r, cu[i]);
          if (kRep && valid) mx = umax(mx, absbits(r));
        }
      }
      if (valid)
        *reinterpret_cast<typename V2<T>::type*>(dst + (int64_t)j * ld + x) =
            *reinterpret_cast<typename V2<T>::type*>(o);
#pragma unroll
      for (int i = 0; i < V; ++i) { up[i] = cu[i]; cu[i] = dn[i]; }
      cel = nel;
      cer = ner;
    }
  }
  return mx;
}

template <typename T>
__device__ void run_banded(const BInst& I, const BParams& p, cg::cluster_group& cl, int rank,
                           typename MaxBits<T>::type* red) {
  using MB = typename MaxBits<T>::type;
  const int band = (I.ny + p.csize - 1) / p.csize;
  const int ra = min(I.ny, rank * band), rb = min(I.ny, ra + band);
  const T c = (T)I.c, ih2 = (T)I.ih2;
  const T* rho = (const T*)I.rho;
  T* a = (T*)I.phi;
  T* b = (T*)I.scratch;
  T* rs = (T*)I.rhos;
  if (rs) {
    // -c rho of this CTA's own rows (the only rows its sweeps read)
    for (int j = ra + (threadIdx.x >> 5); j < rb; j += kBatchThreads / 32)
      for (int i = threadIdx.x & 31; i < I.nx; i += 32)
        rs[(int64_t)j * I.ld + i] = -c * rho[(int64_t)j * I.ld + i];
    __syncthreads();
  }
  const T a1 = (T)I.a1, w4 = (T)I.w4;
  for (int s = 0; s < p.nsweeps; ++s) {
    const bool rep = I.resid != nullptr && p.every > 0 && (s % p.every) == 0;
    if (rep) {
      MB mx = ra < rb ? band_sweep<T, true>(a, b, rho, I.nx, I.ny, I.ld, ra, rb, I.ry, c, ih2) : 0;
      block_report<MB>(mx, I.resid + s / p.every, red);
    } else if (ra < rb) {
      if (rs) band_sweep<T, false, true>(a, b, rs, I.nx, I.ny, I.ld, ra, rb, I.ry, c, ih2, a1, w4);
      else band_sweep<T, false>(a, b, rho, I.nx, I.ny, I.ld, ra, rb, I.ry, c, ih2);
    }
    __threadfence();
    cl.sync();
    T* t = a; a = b; b = t;
  }
  if (p.nsweeps & 1) {
    // the result is in scratch: copy this CTA's rows back into phi
    T* dst = (T*)I.phi;
    for (int j = ra + (threadIdx.x >> 5); j < rb; j += kBatchThreads / 32)
      for (int i = threadIdx.x & 31; i < I.nx; i += 32) dst[(int64_t)j * I.ld + i] = a[(int64_t)j * I.ld + i];
    __threadfence();
    cl.sync();
  }
}

constexpr int kTY = 64, kTX = 128;  // BANDED_T output tile
// Row pitch of a BANDED_T tile with its halo: a multiple of 4 floats (16-byte
// rows for the float4 accesses; a warp reads consecutive cells of one row).
__host__ __device__ constexpr int tpitch(int tb) { return kTX + 2 * tb; }

// FP32 only (FP64 instances are bound by the FP64 pipe, where the halo's
// recomputation would cost more than the saved traffic). tb is 4 or 8, so the
// owned cells start on 16-byte boundaries of the tile rows. A thread handles
// four consecutive cells (float4 loads of the cells, the rows above and below
// and rho; two scalar loads for the outer neighbours). A sweep's rows are
// rounded outward to whole float4 groups: the extra cells lie outside the
// region that later sweeps read, so their (meaningless) values are never used,
// and every access stays inside the tile arrays.
__device__ void run_banded_tiled(const BInst& I, const BParams& p, cg::cluster_group& cl, int rank,
                                 unsigned char* smem, uint32_t* red) {
  constexpr int kMaxTB = 8;
  const int tb = I.tb, nx = I.nx, ny = I.ny;
  const int64_t ld = I.ld;
  const int band = (ny + p.csize - 1) / p.csize;
  const int ra = min(ny, rank * band), rb = min(ny, ra + band);
  const float c = (float)I.c, ih2 = (float)I.ih2;
  const float* rho = (const float*)I.rho;
  const int HP = kTY + 2 * tb, WP = tpitch(tb);
  float* A = reinterpret_cast<float*>(smem);
  float* B = A + HP * WP;
  float* R = B + HP * WP;
  const int tiles_y = (rb - ra + kTY - 1) / kTY, tiles_x = (nx + kTX - 1) / kTX;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = kBatchThreads / 32;
  const bool near_x = nx >= tb, near_y = ny >= tb;
  float* src = (float*)I.phi;
  float* dst = (float*)I.scratch;
  for (int s0 = 0; s0 < p.nsweeps; s0 += tb) {
    const int nb = min(tb, p.nsweeps - s0);
    uint32_t mx[kMaxTB];
#pragma unroll
    for (int t = 0; t < kMaxTB; ++t) mx[t] = 0;
    for (int tile = 0; tile < tiles_y * tiles_x && ra < rb; ++tile) {
      const int ty = tile / tiles_x, tx = tile - ty * tiles_x;
      const int y0 = ra + ty * kTY, x0 = tx * kTX;
      const int oy = min(kTY, rb - y0), ox = min(kTX, nx - x0);  // owned rows / columns
      const int LW = ox + 2 * tb;                                 // loaded columns (multiple of 4)
      const bool inner_x = x0 - tb >= 0 && x0 + ox + tb <= nx;
      // load phi and rho of the tile and its halo (periodic images)
      for (int ly = warp; ly < oy + 2 * tb; ly += nw) {
        const int gy = near_y ? wrap1(y0 + ly - tb, ny) : wrapn(y0 + ly - tb, ny);
        const int64_t gro = (int64_t)gy * ld;
        if (inner_x) {
          const float4* sp = reinterpret_cast<const float4*>(src + gro + x0 - tb);
          const float4* rp = reinterpret_cast<const float4*>(rho + gro + x0 - tb);
          for (int v = lane; v < LW / 4; v += 32) {
            reinterpret_cast<float4*>(A + ly * WP)[v] = sp[v];
            reinterpret_cast<float4*>(R + ly * WP)[v] = __ldg(rp + v);
          }
        } else {
          for (int lx = lane; lx < LW; lx += 32) {
            const int gx = near_x ? wrap1(x0 + lx - tb, nx) : wrapn(x0 + lx - tb, nx);
            A[ly * WP + lx] = src[gro + gx];
            R[ly * WP + lx] = __ldg(rho + gro + gx);
          }
        }
      }
      __syncthreads();
      for (int t = 0; t < nb; ++t) {
        // sweep t computes the cells at distance >= t + 1 from the loaded edge
        // (columns rounded outward to float4 groups)
        const int y1 = t + 1, y2 = 2 * tb + oy - t - 1;
        const int v1 = (t + 1) >> 2, v2 = (2 * tb + ox - t - 1 + 3) >> 2;
        const bool rep = I.resid != nullptr && p.every > 0 && ((s0 + t) % p.every) == 0;
        for (int ly = y1 + warp; ly < y2; ly += nw) {
          const bool orow = ly >= tb && ly < tb + oy;
          const float* row = A + ly * WP;
          for (int v = v1 + lane; v < v2; v += 32) {
            const int x = 4 * v;
            const float4 C = *reinterpret_cast<const float4*>(row + x);
            const float4 U = *reinterpret_cast<const float4*>(row - WP + x);
            const float4 D = *reinterpret_cast<const float4*>(row + WP + x);
            const float4 Rh = *reinterpret_cast<const float4*>(R + ly * WP + x);
            const float l = row[x - 1], r4 = row[x + 4];
            const float cc[4] = {C.x, C.y, C.z, C.w}, uu[4] = {U.x, U.y, U.z, U.w};
            const float dd[4] = {D.x, D.y, D.z, D.w}, rr[4] = {Rh.x, Rh.y, Rh.z, Rh.w};
            float o[4];
            const bool own = rep && orow && x >= tb && x < tb + ox;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const float w = i == 0 ? l : cc[i - 1], e = i == 3 ? r4 : cc[i + 1];
              const float q = (w + e) + (uu[i] + dd[i]);
              const float sv = fmaf(-4.0f, cc[i], q);
              const float rs = fmaf(sv, ih2, -rr[i]);
              o[i] = fmaf(c, rs, cc[i]);
              // the residual of the sweep's input state, over the owned cells
              if (own) mx[t] = umax(mx[t], absbits(rs));
            }
            *reinterpret_cast<float4*>(B + ly * WP + x) = make_float4(o[0], o[1], o[2], o[3]);
          }
        }
        __syncthreads();
        float* tmp = A; A = B; B = tmp;
      }
      for (int ly = warp; ly < oy; ly += nw) {
        float4* drow = reinterpret_cast<float4*>(dst + (int64_t)(y0 + ly) * ld + x0);
        const float4* srow = reinterpret_cast<const float4*>(A + (tb + ly) * WP + tb);
        for (int v = lane; v < ox / 4; v += 32) drow[v] = srow[v];
      }
      __syncthreads();
    }
    for (int t = 0; t < nb; ++t)
      if (I.resid != nullptr && p.every > 0 && ((s0 + t) % p.every) == 0)
        block_report<uint32_t>(mx[t], I.resid + (s0 + t) / p.every, red);
    __threadfence();
    cl.sync();
    float* tmp = src; src = dst; dst = tmp;
  }
  if (((p.nsweeps + tb - 1) / tb) & 1) {
    // the result is in scratch: copy this CTA's rows back into phi
    float* out = (float*)I.phi;
    for (int j = ra + (threadIdx.x >> 5); j < rb; j += kBatchThreads / 32)
      for (int i = threadIdx.x & 31; i < nx; i += 32) out[(int64_t)j * ld + i] = src[(int64_t)j * ld + i];
    __threadfence();
    cl.sync();
  }
}

template <typename T>
__device__ void run_whole(const BInst& I, const BParams& p, unsigned char* smem,
                          typename MaxBits<T>::type* red) {
  using MB = typename MaxBits<T>::type;
  const int nx = I.nx, ny = I.ny;
  T* A = reinterpret_cast<T*>(smem);
  T* B = A + (int64_t)nx * ny;
  const T* phi = (const T*)I.phi;
  const T* rho = (const T*)I.rho;
  const T c = (T)I.c, ih2 = (T)I.ih2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = kBatchThreads / 32;
  for (int j = warp; j < ny; j += nw)
    for (int i = lane; i < nx; i += 32) A[j * nx + i] = phi[(int64_t)j * I.ld + i];
  __syncthreads();
  for (int s = 0; s < p.nsweeps; ++s) {
    const bool rep = I.resid != nullptr && p.every > 0 && (s % p.every) == 0;
    MB mx = 0;
    for (int j = warp; j < ny; j += nw) {
      const T* up = A + wrap1(j - 1, ny) * nx;
      const T* cu = A + j * nx;
      const T* dn = A + wrap1(j + 1, ny) * nx;
      const T* rr = rho + (int64_t)j * I.ld;
      for (int i = lane; i < nx; i += 32) {
        const T C = cu[i];
        const T q = (cu[wrap1(i - 1, nx)] + cu[wrap1(i + 1, nx)]) + (up[i] + dn[i]);
        const T sv = fma((T)-4, C, q);
        const T r = fma(sv, ih2, -__ldg(rr + i));
        B[j * nx + i] = fma(c, r, C);
        if (rep) mx = umax(mx, absbits(r));
      }
    }
    if (rep) block_report<MB>(mx, I.resid + s / p.every, red);  // includes barriers
    else __syncthreads();
    T* t = A; A = B; B = t;
  }
  T* out = (T*)I.phi;
  for (int j = warp; j < ny; j += nw)
    for (int i = lane; i < nx; i += 32) out[(int64_t)j * I.ld + i] = A[j * nx + i];
  __syncthreads();
}

// At most 64 registers a thread (two CTAs of 512 threads per SM), so that the
// two launches of a mixed-precision plan can share every SM.
__global__ void __launch_bounds__(kBatchThreads, 2) batch_k(BParams p) {
  extern __shared__ __align__(16) unsigned char bsm[];
  __shared__ uint64_t red64[kBatchThreads / 32];
  __shared__ uint32_t red32[kBatchThreads / 32];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int cid = blockIdx.x / p.csize;
  for (int u = p.cl_off[cid]; u < p.cl_off[cid + 1]; ++u) {
    const BInst& I = p.inst[p.cl_items[u]];
    if (I.mode == MODE_BANDED_T && I.dtype == 1) {
      run_banded_tiled(I, p, cl, rank, bsm, red32);
    } else if (I.dtype == 0) {
      run_banded<double>(I, p, cl, rank, red64);
    } else {
      run_banded<float>(I, p, cl, rank, red32);
    }
  }
  for (int u = p.cta_off[blockIdx.x]; u < p.cta_off[blockIdx.x + 1]; ++u) {
    const BInst& I = p.inst[p.cta_items[u]];
    if (I.dtype == 0) run_whole<double>(I, p, bsm, red64);
    else run_whole<float>(I, p, bsm, red32);
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side: plan (classes, tuning, schedule), graph, run.

size_t whole_bytes(int nx, int ny, int dtype) {
  return 2 * (size_t)nx * (size_t)ny * (dtype == 0 ? 8 : 4);
}

cudaError_t batch_attr() {
  static bool attr_by_dev[64] = {};
  bool& attr = attr_by_dev[dev_index()];
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(batch_k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kWholeSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  return cudaSuccess;
}

cudaError_t batch_max_clusters(int* n, size_t smem, int csize) {
  cudaError_t e0 = batch_attr();
  if (e0 != cudaSuccess) return e0;
  const int kCluster = csize;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kCluster * 256, 1, 1);
  cfg.blockDim = dim3(kBatchThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kCluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaOccupancyMaxActiveClusters(n, batch_k, &cfg);
}

cudaError_t batch_launch(const BParams& p, int nclusters, size_t smem, cudaStream_t st) {
  const int kCluster = p.csize;
  if (kCluster < 1 || kCluster > kMaxCluster) return cudaErrorInvalidValue;
  if (smem > kWholeSmem) return cudaErrorInvalidValue;
  cudaError_t e0 = batch_attr();
  if (e0 != cudaSuccess) return e0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kCluster * nclusters, 1, 1);
  cfg.blockDim = dim3(kBatchThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kCluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, batch_k, p);
}

bool batch_coresident(size_t smem) {
  if (batch_attr() != cudaSuccess) { cudaGetLastError(); return false; }
  int k = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, batch_k, kBatchThreads, smem) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return k >= 2;
}

int batch_max_cluster_size() { return kMaxCluster; }
size_t batch_whole_smem() { return kWholeSmem; }
size_t banded_t_smem(int dtype, int tb) {
  return (size_t)3 * (kTY + 2 * tb) * tpitch(tb) * (dtype == 0 ? 8 : 4);
}
bool banded_t_ok(int dtype, int tb) { return dtype == 1 && (tb == 4 || tb == 8); }

}  // namespace px

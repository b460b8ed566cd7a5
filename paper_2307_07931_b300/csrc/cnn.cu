// Learned initial guess: a 6-layer periodic 3x3 CNN (widths 1-32-32-32-32-32-1,
// GELU after every layer but the last), BF16 weights and activations with FP32
// accumulation, trained and run by the kernels in this file.
//
// Layout: BF16 activations of 32 channels stored chunk-planar: per image, four
// planes of 8 channels (16 bytes per pixel), element (b, chunk, y, x, c) at
// (((b * 4 + chunk) * H + y) * W + x) * 8 + c. A row of 64 pixels of one
// plane is 1 KB contiguous, which is exactly one core-matrix row block of the
// tensor-core operand, so a tap tile is one rectangular box for the tensor
// memory accelerator. The network input x and output y are single-channel
// FP32 images. Convolutions
// are periodic cross-correlations: z[p][o] = b[o] + sum_{dy,dx,c} W[o][c][dy][dx]
// x[p + (dy - 1, dx - 1)][c].
//
// The 32 -> 32 layers are implicit GEMMs on the 5th-generation tensor cores
// (tcgen05.mma, BF16 in, FP32 accumulate in tensor memory): M = pixels, N = 32
// output channels, K = 9 taps x 32 channels, one 4 x 64 output tile per step
// of a persistent, warp-specialised kernel (producer warps stage each tap's
// shifted tile with cp.async, periodic wrap in the loads; one thread issues
// the MMAs; epilogue warps drain the accumulators). Epilogues are fused:
// bias + GELU (forward, storing the pre-activation for the backward pass) or
// the product with GELU'(z) of the previous layer (input gradient, which is
// the same convolution with the weights flipped in both taps and transposed).
// The weight gradient is a GEMM over pixels on tcgen05 as well (M = 4 taps x
// 32 channels, N = 32, K = pixels), accumulated in tensor memory per CTA and
// reduced in a fixed order. The 1 -> 32 and 32 -> 1 layers have 288
// multiply-adds per pixel and run on the CUDA cores.
#include "px_internal.cuh"

#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <vector>

namespace px {
namespace cnn {

constexpr int C = 32;            // channels of the hidden layers
constexpr int K9 = 9 * C;        // GEMM K of a 32 -> 32 layer
constexpr int TR = 4, TW = 64;   // output tile: rows x columns (one row per warp)
static_assert(TW == 64, "load_tap_cm_p splits pixel indices with shifts");
constexpr int kConvThreads = 128;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp16(void* s, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait_group() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}



// GELU(z) = z Phi(z) and GELU'(z) = Phi(z) + z phi(z), with the normal
// distribution Phi(z) = (1 + erf(z / sqrt 2)) / 2 and density phi(z) =
// exp(-z^2 / 2) / sqrt(2 pi). erf from Abramowitz and Stegun, Handbook of
// Mathematical Functions, formula 7.1.26: for x >= 0,
//   erf(x) = 1 - t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) exp(-x^2),
//   t = 1 / (1 + p x),  |error| <= 1.5e-7,
// so with x = |z| / sqrt 2 one exponential exp(-z^2 / 2) serves both erf and
// phi. The upper tail Q = 1 - erf(x) gives Phi(z) = 1 - Q / 2 for z >= 0 and
// Q / 2 for z < 0; the coefficients below are a_i / 2, so the polynomial
// gives Q / 2 directly. The reciprocal (of 1 + p x >= 1) and the exponential
// (2^y with y = -z^2 log2(e) / 2) are the hardware approximations with
// subnormal results flushed to zero (relative errors near 2^-22; a flushed
// exp(-z^2 / 2) < 2^-126 contributes below 1e-37); the activations are
// stored in BF16 (2^-9).
__device__ __forceinline__ float rcp_ftz(float v) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ float exp2_ftz(float v) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}
// The formula is evaluated on pairs of values with the packed FP32
// instructions (add/mul/fma.rn.f32x2 round each half like the scalar
// instruction, so each half takes the scalar sequence of roundings: t, the
// polynomial in Horner form, E, h = (q t) E, then 1 - h): one issue slot per
// two values for the polynomial and the products. The reciprocal, the
// exponential and the sign select stay per value.
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
struct NormalCdf2 {
  float2 Phi, E;
};
__device__ __forceinline__ NormalCdf2 normal_cdf2(float2 z) {
  const float2 t = make_float2(rcp_ftz(fmaf(0.3275911f * 0.70710678118654752f, fabsf(z.x), 1.0f)),
                               rcp_ftz(fmaf(0.3275911f * 0.70710678118654752f, fabsf(z.y), 1.0f)));
  float2 q = __ffma2_rn(f2(0.5f * 1.061405429f), t, f2(0.5f * -1.453152027f));
  q = __ffma2_rn(q, t, f2(0.5f * 1.421413741f));
  q = __ffma2_rn(q, t, f2(0.5f * -0.284496736f));
  q = __ffma2_rn(q, t, f2(0.5f * 0.254829592f));
  const float2 y = __fmul2_rn(__fmul2_rn(z, f2(-0.5f * 1.4426950408889634f)), z);
  const float2 E = make_float2(exp2_ftz(y.x), exp2_ftz(y.y));
  const float2 h = __fmul2_rn(__fmul2_rn(q, t), E);          // Q / 2
  const float2 u = __ffma2_rn(h, f2(-1.0f), f2(1.0f));       // 1 - h, one rounding
  return {make_float2(z.x >= 0.0f ? u.x : h.x, z.y >= 0.0f ? u.y : h.y), E};
}
__device__ __forceinline__ float2 gelu_f2(float2 z) { return __fmul2_rn(z, normal_cdf2(z).Phi); }
__device__ __forceinline__ float2 gelu_grad_f2(float2 z) {
  const NormalCdf2 c = normal_cdf2(z);
  return __ffma2_rn(__fmul2_rn(z, f2(0.39894228040143268f)), c.E, c.Phi);
}


// Element offset of channel chunk `chunk` (8 channels) of pixel (b, y, x).
__host__ __device__ __forceinline__ int64_t act_off(int b, int y, int x, int chunk, int H, int W) {
  return ((((int64_t)b * 4 + chunk) * H + y) * W + x) * 8;
}

// The 32 channels of one pixel: four 16-byte loads, `plane` elements apart.
__device__ __forceinline__ void load_px32(float (&f)[C], const __nv_bfloat16* p, int64_t plane) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    uint4 u = *reinterpret_cast<const uint4*>(p + k * plane);
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float2 t = __bfloat1622float2(h[e]);
      f[k * 8 + 2 * e] = t.x;
      f[k * 8 + 2 * e + 1] = t.y;
    }
  }
}

// Index of element (n, k) of an N = 32 x K = 288 K-major operand in the
// tensor cores' no-swizzle core-matrix order: [k / 8][n][k % 8].
__host__ __device__ __forceinline__ int cm_index(int n, int k) { return (k / 8) * (C * 8) + n * 8 + (k % 8); }

// Periodic column index for |x - wrapped| < W (a conditional add or subtract)
// or any x (a full modulo), chosen once per launch from the dilation.
__device__ __forceinline__ int wrap_col(int x, int W, bool near) { return near ? wrap1(x, W) : wrapn(x, W); }
__device__ __forceinline__ int tap_dy(int tap, int d) { return (tap / 3 - 1) * d; }
__device__ __forceinline__ int tap_dx(int tap, int d) { return (tap % 3 - 1) * d; }

// ---------------------------------------------------------------------------
// 32 -> 32 periodic convolution (dilation d) on the 5th-generation tensor
// cores: tcgen05.mma (kind::f16, BF16 operands, FP32 accumulators in tensor
// memory). A 4 x 64 output tile is two M = 128 pixel halves, the left and the
// right 4 x 32 pixels, each with a 128-lane x 32-column FP32 accumulator in
// TMEM (lane 32 i + p: row i, pixel p of the half). Operands live in shared
// memory in the no-swizzle K-major core-matrix layout (a core matrix is 8 rows
// x 16 bytes, contiguous). A staged tile of R rows is [half][chunk][row][32
// px][8 ch]: a half-row of one 8-channel chunk is 512 contiguous bytes (the
// box rows of the tensor memory accelerator: 32 pixels x 16 B, so no 32-byte
// sector is fetched for 16 useful bytes), row r of a half at r * 512 B, chunk
// c at c * R * 512 B, half h at h * 4 R * 512 B. The half's 128 pixels are
// then 16 core matrices 128 B apart whatever the row: the MMA reads A at
// (tile + h * 4 R * 512 + 2 cc * R * 512 + (first row) * 512, LBO R * 512,
// SBO 128) and B at (weights + (4 tap + 2 cc) * 512, LBO 512, SBO 128); the
// weights [32 n][288 k] are pre-packed as [k / 8][n][k % 8] (18 KB).
constexpr int kUmmaM = 128;                               // pixels per MMA = TMEM lanes
constexpr int kHW = TW / 2;                               // 32: pixels of a half-row
constexpr uint32_t kHRow = kHW * 16;                      // 512 B: one half-row of one chunk
constexpr uint32_t kCmChunk = TR * kHRow;                 // 2048 B: next chunk of a half tile
constexpr uint32_t kCmHalf = 4 * kCmChunk;                // 8 KB: one half of a tap tile
constexpr size_t kCmTile = (size_t)2 * kCmHalf;           // 16 KB: one tap tile
constexpr uint32_t kCmWChunk = C * 16;                    // 512 B: next 8-k chunk of the weights
constexpr size_t kWBytes = (size_t)(K9 / 8) * kCmWChunk;  // 18 KB
constexpr uint32_t kSpinLimit = 1u << 24;  // polls per wait (a healthy wait takes microseconds)
__device__ unsigned g_conv_fault;  // set by a conv CTA whose bounded wait ran out
// instruction descriptor: FP32 accumulate, BF16 A and B, both K-major, N = 32, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(C >> 3) << 17) |
                            ((uint32_t)(kUmmaM >> 4) << 24);
static_assert(TR * TW == 2 * kUmmaM, "two M = 128 halves per tile");

// shared-memory matrix descriptor, no swizzle (start, leading = K-direction
// and stride = M/N-direction byte offsets between core matrices)
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
__device__ __forceinline__ void umma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t acc) {
  asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
               "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
               ::"r"(tmem), "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc) : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t (&v)[32], uint32_t taddr) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
               "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
               "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                 "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                 "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]),
                 "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
                 "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
                 "=r"(v[30]), "=r"(v[31])
               : "r"(taddr) : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Warp-specialised persistent form of the same convolution (the one launched).
// A CTA of 9 warps loops over 4 x 64 tiles:
//   warps 4..7  producers: stage each tap's tile (cp.async, core-matrix
//               layout) into a 4-stage ring; a thread waits for its own
//               copies one step later, fences them to the async proxy and
//               arrives on the stage's `full` barrier (128 arrivals);
//   warp 8      lane 0 issues the 4 MMAs of a tap once `full` flips and
//               commits them to the stage's `empty` barrier; after the 9th
//               tap it commits the tile to `tfull` of its accumulator set;
//               the warp also owns the tensor memory (2 sets x 64 columns);
//   warps 0..3  epilogue: wait `tfull`, read their 32 TMEM lanes per half,
//               apply bias + GELU or the GELU' product, store, and release the
//               set on `tempty` (128 arrivals).
// The epilogue of tile i overlaps the staging and MMAs of tile i + 1.
// Barrier uses are counted per object and waited on with the use's parity;
// every waiter of use u waits before use u + 1 can complete, so a parity
// never refers to a stale phase. Every wait is bounded and gives up when the
// shared abort flag is set; on an abort the CTA raises *fault, lets its MMAs
// drain (bounded) and frees its tensor memory.
constexpr int kWsStages = 4;
// Unit-offset layers (dilation 1, or a dilated layer whose input is stored
// relabelled, below): one stage is the (TR + 2)-row patch of one column
// offset dx in the same [half][chunk][row][32 px][8 ch] layout; it serves the
// three taps of that dx, whose A operands start one half-row (512 B) apart.
// Three stages per tile instead of nine tap tiles.
constexpr int kURows = TR + 2;
constexpr uint32_t kUChunk = kURows * kHRow;           // 3 KB
constexpr uint32_t kUHalf = 4 * kUChunk;               // 12 KB
constexpr size_t kUTile = (size_t)2 * kUHalf;          // 24 KB
constexpr int kUStages = 3;
constexpr size_t kRingBytes = kUStages * kUTile > kWsStages * kCmTile ? kUStages * kUTile
                                                                      : kWsStages * kCmTile;
// A producer declares a step with per-pixel copies complete one step later
// (after the next step's copies are issued: its own copies then wait only
// for the older group), and a step of boxes only at once. One step ahead
// measured fastest for the copies: with more copies in flight the tap tiles
// contend in L2 (whole forward at 16 x 256^2: 0.93 ms at one step ahead,
// 1.03 ms at three, with per-pixel copies throughout).
constexpr int kWsEpiWarps = 4, kWsProdWarps = 4;
constexpr int kWsConvThreads = (kWsEpiWarps + kWsProdWarps + 1) * 32;  // 288
constexpr uint32_t kWsTmemCols = 128;                                 // 2 sets x (2 x 32)
constexpr int kWsBars = 2 * kWsStages + 4 + 1;  // full, empty, tfull[2], tempty[2], weights
// ring | weights | barriers, abort flag, TMEM slot (128 B) | bias (128 B): 90 KB, two CTAs per SM
static_assert(kWsBars * 8 + 8 <= 128, "barrier block");
constexpr size_t kWsSmem = kRingBytes + kWBytes + 256;

// Handshake wait: up to `limit` polls of the barrier's phase, giving up early
// once another thread of the CTA has set the abort flag; on running out it
// sets the flag itself. Each poll may suspend the thread for up to
// kPollSuspendNs until the phase completes (try_wait's suspend-time hint), so
// waiting warps sleep instead of taking issue slots from the working ones;
// a wait lasts at most limit x kPollSuspendNs.
constexpr uint32_t kPollSuspendNs = 1000;
__device__ __forceinline__ bool mbar_wait_ab(uint32_t bar, uint32_t parity, volatile int* abort_,
                                             uint32_t limit) {
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
                 "selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done) : "r"(bar), "r"(parity), "r"(kPollSuspendNs) : "memory");
    if (done) return true;
    if ((it & 63) == 63 && *abort_) return false;
  }
  *abort_ = 1;
  return false;
}
// Drain wait: up to kSpinLimit polls, ignoring the abort flag. Used only for
// the completion of MMAs already issued, which needs no other thread, so it
// ends well inside the limit; tensor memory is freed only after it.
__device__ __forceinline__ bool mbar_wait_drain(uint32_t bar, uint32_t parity) {
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 "selp.u32 %0, 1, 0, p;\n}" : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               ::"r"(bar) : "memory");
}

// Tensor memory accelerator: one 4D box of the chunk-planar activations,
// dims (W x 8 elements: a row of one chunk, H, 4 chunks, B), box (256, R, 4,
// 1) = 32 pixels x R rows x 4 chunks, lands in shared memory as
// [chunk][row][32 px][8 ch], one half of the operand layout; x is the first
// pixel times 8 (a multiple of 16 bytes). Completion is counted in bytes on
// the stage's `full` barrier.
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load_half(uint32_t dst, const CUtensorMap* map, int px, int y,
                                              int b, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4, %5}], [%6];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(px * 8), "r"(y), "r"(0), "r"(b),
        "r"(bar)
      : "memory");
}

// Stage one tap's [R * 64 px][32 ch] input tile in the core-matrix layout
// (chunk c of 8 channels at c * R * 1024 B, pixel p at p * 16 B), threads pid
// of np. Consecutive threads copy consecutive pixels of one channel plane
// (a warp: 512 contiguous global bytes). The periodic wrap is a conditional
// add or subtract when the tap offset is smaller than the image, a full
// modulo otherwise.
// The same for one half of a conv operand tile: the R x 32 pixels from
// (y0 + oy, x0 + ox) into [chunk][row][32 px][8 ch] (chunk stride R * 512 B).
template <int R>
__device__ __forceinline__ void load_half_cm_p(unsigned char* dst, const __nv_bfloat16* act, int b,
                                               int y0, int x0, int oy, int ox, int H, int W,
                                               int pid, int np) {
  const bool near = oy > -H && oy < H && ox > -W && ox < W;
  for (int q = pid; q < R * kHW * 4; q += np) {
    const int chunk = q / (R * kHW), pix = q - chunk * (R * kHW);
    const int r = pix >> 5, c = pix & (kHW - 1);
    const int gy = near ? wrap1(y0 + r + oy, H) : wrapn(y0 + r + oy, H);
    const int gx = near ? wrap1(x0 + c + ox, W) : wrapn(x0 + c + ox, W);
    cp16(dst + chunk * (R * kHRow) + pix * 16, act + act_off(b, gy, gx, chunk, H, W));
  }
}

template <int R>
__device__ __forceinline__ void load_tap_cm_p(unsigned char* dst, const __nv_bfloat16* act, int b,
                                              int y0, int x0, int oy, int ox, int H, int W,
                                              int pid, int np) {
  const bool near = oy > -H && oy < H && ox > -W && ox < W;
  for (int q = pid; q < R * TW * 4; q += np) {
    const int chunk = q / (R * TW), pix = q - chunk * (R * TW);
    const int r = pix >> 6, c = pix & (TW - 1);
    const int gy = near ? wrap1(y0 + r + oy, H) : wrapn(y0 + r + oy, H);
    const int gx = near ? wrap1(x0 + c + ox, W) : wrapn(x0 + c + ox, W);
    cp16(dst + chunk * (R * TW * 16) + pix * 16, act + act_off(b, gy, gx, chunk, H, W));
  }
}

// Position of the output pixel computed at input position (y, x): the
// coordinates times (ry, rx), modulo the image (identity when both are 1).
// 0 <= v, r < n: the product fits 32 unsigned bits for n <= 65535, where the
// 32-bit remainder (a few instructions) replaces the 64-bit one (a library
// routine per call).
__device__ __forceinline__ int relabel(int v, int r, int n) {
  if (r == 1) return v;
  if (n <= 65535) return (int)(((unsigned)v * (unsigned)r) % (unsigned)n);
  return (int)(((int64_t)v * r) % n);
}

template <int kMode>
__device__ __forceinline__ void conv_epilogue_half(const uint32_t (&v)[32], int pix, int b, int y0,
                                                   int x0, int H, int W, int ry, int rx,
                                                   const float* sbias,  // shared memory
                                                   const __nv_bfloat16* __restrict__ zprev,
                                                   __nv_bfloat16* __restrict__ zout,
                                                   __nv_bfloat16* __restrict__ aout) {
  // accumulator lane pix & 127 of half pix >> 7: row (pix >> 5) & 3, pixel pix & 31
  const int y = y0 + ((pix >> 5) & 3), x = x0 + (pix >> 7) * kHW + (pix & (kHW - 1));
  // pb: the output's position; zprev shares the input's positions
  const int64_t pb = act_off(b, relabel(y, ry, H), relabel(x, rx, W), 0, H, W),
                plane = (int64_t)H * W * 8;
  if (kMode == 0) {
    // one 8-channel chunk at a time, its two 16-byte stores right after its
    // values: few values live between the accumulator read and the stores
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      __nv_bfloat162 zz[4], aa[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int o = 8 * k + 2 * e;
        const float2 bb = *reinterpret_cast<const float2*>(sbias + o);  // same address: broadcast
        const float2 vz = __fadd2_rn(make_float2(__uint_as_float(v[o]), __uint_as_float(v[o + 1])), bb);
        zz[e] = __float22bfloat162_rn(vz);
        aa[e] = __float22bfloat162_rn(gelu_f2(vz));
      }
      if (zout) *reinterpret_cast<uint4*>(zout + pb + k * plane) = *reinterpret_cast<const uint4*>(zz);
      *reinterpret_cast<uint4*>(aout + pb + k * plane) = *reinterpret_cast<const uint4*>(aa);
    }
  } else {
    // the input gradient: all four chunks of z in flight first (chunk-wise
    // loads next to their uses measured 20 % slower)
    float zf[C];
    load_px32(zf, zprev + act_off(b, y, x, 0, H, W), plane);
    __nv_bfloat162 aa[C / 2];
#pragma unroll
    for (int o = 0; o < C; o += 2)
      aa[o / 2] = __float22bfloat162_rn(
          __fmul2_rn(make_float2(__uint_as_float(v[o]), __uint_as_float(v[o + 1])),
                     gelu_grad_f2(make_float2(zf[o], zf[o + 1]))));
#pragma unroll
    for (int k = 0; k < 4; ++k)
      *reinterpret_cast<uint4*>(aout + pb + k * plane) = reinterpret_cast<const uint4*>(aa)[k];
  }
}

// kUnit: the unit-offset staging (three dx patches per tile; `dil` is then
// ignored); otherwise nine tap tiles at offsets of `dil`. (ry, rx): output
// position = input position times (ry, rx) modulo the image.
template <int kMode, bool kUnit>
__global__ void __launch_bounds__(kWsConvThreads, 2)
conv32_ws(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ wk,
          const float* __restrict__ bias, const __nv_bfloat16* __restrict__ zprev,
          __nv_bfloat16* __restrict__ zout, __nv_bfloat16* __restrict__ aout, int H, int W,
          int tiles_x, int tiles_y, int ntiles, int dil, int ry, int rx,
          unsigned* __restrict__ fault, uint32_t wait_limit,
          const __grid_constant__ CUtensorMap tmap_in, int use_tma) {
  constexpr int kSteps = kUnit ? 3 : 9;               // stages per tile
  constexpr int kStages = kUnit ? kUStages : kWsStages;
  constexpr uint32_t kStage = kUnit ? (uint32_t)kUTile : (uint32_t)kCmTile;
  // no static shared variables: the core matrices must start on 128-byte boundaries
  extern __shared__ __align__(128) unsigned char wsu[];
  unsigned char* ring = wsu;
  unsigned char* wsm = wsu + kRingBytes;
  uint64_t* bar = reinterpret_cast<uint64_t*>(wsm + kWBytes);
  const uint32_t full0 = smem_u32(bar), empty0 = smem_u32(bar + kWsStages);
  const uint32_t tfull0 = smem_u32(bar + 2 * kWsStages), tempty0 = smem_u32(bar + 2 * kWsStages + 2);
  const uint32_t wfull = smem_u32(bar + 2 * kWsStages + 4);
  volatile int* abort_ = reinterpret_cast<volatile int*>(bar + kWsBars);
  volatile uint32_t* tslot = reinterpret_cast<volatile uint32_t*>(abort_ + 1);
  float* const sbias = reinterpret_cast<float*>(wsm + kWBytes + 128);
  if (threadIdx.x < C) sbias[threadIdx.x] = bias ? bias[threadIdx.x] : 0.0f;  // read after the barrier below
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int my_tiles = (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;

  if (threadIdx.x == 0) {
    for (int k = 0; k < kWsStages; ++k) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(full0 + 8 * k), "r"(kWsProdWarps * 32) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(empty0 + 8 * k) : "memory");
    }
    for (int a = 0; a < 2; ++a) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tfull0 + 8 * a) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tempty0 + 8 * a), "r"(kWsEpiWarps * 32) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(wfull), "r"(kWsProdWarps * 32) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *abort_ = (smem_u32(wsu) & 127u) != 0;  // misaligned operands: no MMA, raise the fault
  }
  if (warp == 8) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32((const void*)tslot)), "r"(kWsTmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  uint32_t last_bar = 0, last_par = 0;  // MMA thread: its last commit

  if (warp >= kWsEpiWarps && warp < kWsEpiWarps + kWsProdWarps) {
    // ---- producers
    const int pid = threadIdx.x - kWsEpiWarps * 32, np = kWsProdWarps * 32;
    for (int q = pid; q < (int)(kWBytes / 16); q += np) cp16(wsm + q * 16, wk + q * 8);
    cp_commit();
    cp_wait_group<0>();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive(wfull);
    bool go = *abort_ == 0;
    int g = 0;
    int pend = -1;  // step whose copies this thread has issued but not declared
    const bool pnear = kUnit || (dil < H && dil < W);
    for (int i = 0; i < my_tiles && go; ++i) {
      const int tile = (int)blockIdx.x + i * (int)gridDim.x;
      const int tx = tile % tiles_x, ty = (tile / tiles_x) % tiles_y, b = tile / (tiles_x * tiles_y);
      for (int step = 0; step < kSteps; ++step, ++g) {
        const int st = g % kStages, u = g / kStages;
        if (u >= 1 && !mbar_wait_ab(empty0 + 8 * st, (u - 1) & 1, abort_, wait_limit)) { go = false; break; }
        // unit: the patch of rows y0 - 1 .. y0 + TR at column offset step - 1;
        // otherwise tap `step`'s tile at offset (dy, dx) d
        const int oy = kUnit ? -1 : tap_dy(step, dil), ox = kUnit ? step - 1 : tap_dx(step, dil);
        constexpr int kR = kUnit ? kURows : TR;
        constexpr uint32_t kHalfB = kStage / 2;
        // the starts lie within one period of the image when the offsets do
        // (always for unit offsets): a conditional add instead of a remainder
        const int ys = pnear ? wrap1(ty * TR + oy, H) : wrapn(ty * TR + oy, H);
        const int xs0 = pnear ? wrap1(tx * TW + ox, W) : wrapn(tx * TW + ox, W);
        const int xs1 = pnear ? wrap1(tx * TW + kHW + ox, W) : wrapn(tx * TW + kHW + ox, W);
        // a half that lies inside the image is one box, issued by one thread;
        // one that wraps around the periodic edge takes per-pixel copies
        const bool box0 = use_tma && ys + kR <= H && xs0 + kHW <= W;
        const bool box1 = use_tma && ys + kR <= H && xs1 + kHW <= W;
        unsigned char* const dst = ring + st * kStage;
        if ((box0 || box1) && pid == 0) {
          mbar_expect_tx(full0 + 8 * st, (box0 ? kHalfB : 0u) + (box1 ? kHalfB : 0u));
          if (box0) tma_load_half(smem_u32(dst), &tmap_in, xs0, ys, b, full0 + 8 * st);
          if (box1) tma_load_half(smem_u32(dst + kHalfB), &tmap_in, xs1, ys, b, full0 + 8 * st);
        }
        if (!box0) load_half_cm_p<kR>(dst, in, b, ty * TR, tx * TW, oy, ox, H, W, pid, np);
        if (!box1) load_half_cm_p<kR>(dst + kHalfB, in, b, ty * TR, tx * TW + kHW, oy, ox, H, W, pid, np);
        cp_commit();
        // A step with copies is declared one step later, once they have
        // landed (the thread's older copy groups: all but the newest); a step
        // of boxes only is declared at once, its boxes completing the phase
        // by their byte count.
        if (pend >= 0) {
          cp_wait_group<1>();
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          mbar_arrive(full0 + 8 * (pend % kStages));
          pend = -1;
        }
        if (box0 && box1) mbar_arrive(full0 + 8 * st);
        else pend = g;
      }
    }
    cp_wait_group<0>();
    if (go && pend >= 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(full0 + 8 * (pend % kStages));
    }
  } else if (warp == kWsEpiWarps + kWsProdWarps) {
    // ---- MMA issue
    if (lane == 0) {
      bool go = mbar_wait_ab(wfull, 0, abort_, wait_limit);
      const uint32_t tbase = smem_u32(ring), wbase = smem_u32(wsm);
      int g = 0;
      for (int i = 0; i < my_tiles && go; ++i) {
        const int a = i & 1;
        if (i >= 2 && !mbar_wait_ab(tempty0 + 8 * a, ((i >> 1) - 1) & 1, abort_, wait_limit)) { go = false; break; }
        for (int step = 0; step < kSteps; ++step, ++g) {
          const int st = g % kStages;
          if (!mbar_wait_ab(full0 + 8 * st, (g / kStages) & 1, abort_, wait_limit)) { go = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t abase = tbase + st * kStage;
          if constexpr (kUnit) {
            // taps (dy, step) for dy = 0..2: output rows 0..3 read patch rows
            // dy .. dy + 3
#pragma unroll
            for (int dy = 0; dy < 3; ++dy) {
              const int tap = dy * 3 + step;
#pragma unroll
              for (int cc = 0; cc < 2; ++cc) {
                const uint64_t bd = umma_desc(wbase + (uint32_t)(tap * 4 + cc * 2) * kCmWChunk, kCmWChunk, 128);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                  const uint64_t ad = umma_desc(abase + h * kUHalf + cc * 2 * kUChunk + dy * kHRow, kUChunk, 128);
                  umma_bf16(tmem + a * 2 * C + h * C, ad, bd, (step > 0 || dy > 0 || cc > 0) ? 1u : 0u);
                }
              }
            }
          } else {
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
              const uint64_t bd = umma_desc(wbase + (uint32_t)(step * 4 + cc * 2) * kCmWChunk, kCmWChunk, 128);
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const uint64_t ad = umma_desc(abase + h * kCmHalf + cc * 2 * kCmChunk, kCmChunk, 128);
                umma_bf16(tmem + a * 2 * C + h * C, ad, bd, (step > 0 || cc > 0) ? 1u : 0u);
              }
            }
          }
          umma_commit(empty0 + 8 * st);
          last_bar = empty0 + 8 * st;
          last_par = (g / kStages) & 1;
        }
        if (!go) break;
        umma_commit(tfull0 + 8 * a);
        last_bar = tfull0 + 8 * a;  // the last commit: a drain waits for this one
        last_par = (i >> 1) & 1;
      }
      if (!go) *abort_ = 1;
    }
    __syncwarp();
  } else {
    // ---- epilogue
    for (int i = 0; i < my_tiles; ++i) {
      const int a = i & 1;
      if (!mbar_wait_ab(tfull0 + 8 * a, (i >> 1) & 1, abort_, wait_limit)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int tile = (int)blockIdx.x + i * (int)gridDim.x;
      const int tx = tile % tiles_x, ty = (tile / tiles_x) % tiles_y, b = tile / (tiles_x * tiles_y);
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        uint32_t v[32];
        tmem_ld32(v, tmem + a * 2 * C + h * C + ((uint32_t)(warp * 32) << 16));
        conv_epilogue_half<kMode>(v, h * kUmmaM + warp * 32 + lane, b, ty * TR, tx * TW, H, W,
                                  ry, rx, sbias, zprev, zout, aout);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(tempty0 + 8 * a);
    }
  }

  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == kWsEpiWarps + kWsProdWarps) {
    if (*abort_) {
      if (lane == 0) {
        atomicOr(fault, 1u);
        // MMAs already issued finish on their own: wait (bounded) for the last commit
        if (last_bar) mbar_wait_drain(last_bar, last_par);
      }
      __syncwarp();
    }
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kWsTmemCols)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// Weight gradient of a 32 -> 32 layer on tcgen05 (the one launched):
//   D[(tap, c)][o] = sum_p in[p + off(tap)][c] * dz[p][o],  db[o] = sum_p dz[p][o].
// The contraction runs over pixels. The staged tiles ([chunk][pixel][8 ch])
// are then MN-major operands: a core matrix is 8 pixels (K) x 8 channels
// (16 B), K-neighbours 128 B apart (leading byte offset) and channel groups
// 2048 B apart (stride byte offset). A CTA keeps 12 tiles of 16 KB in shared
// memory, in this order: the 9 tap tiles of `in`, a tile of ones, the dz tile
// and one spare (2 x 64-pixel tiles of 8 KB: 96 KB, two CTAs per SM, so one
// CTA's MMAs overlap the other's staging). Three M = 128 blocks cover
// (taps 0-3), (taps 4-7) and (tap 8, ones, two unused row groups): the ones
// rows give db. N = 32 output channels; 8 MMAs of K = 16 pixels per block
// and tile. The CTA loops over
// its tiles accumulating in TMEM (3 x 32 columns), waits for each tile's MMAs
// before restaging, and finally writes its partial
// (part[o * 288 + tap * 32 + c], part[9216 + o]) for the fixed-order reduction.
constexpr int kWgTiles = 12;
constexpr int kWgRows = 2;                              // tile: 2 x 64 pixels (K = 128)
constexpr uint32_t kWgChunk = kWgRows * TW * 16;        // 2048 B: next 8-channel group
constexpr size_t kWgTile = (size_t)4 * kWgChunk;        // 8 KB
constexpr size_t kWgUmmaSmem = kWgTiles * kWgTile + 64; // 96 KB: two CTAs per SM
constexpr uint32_t kWgTmemCols = 128;
constexpr uint32_t kIdescMN = kIdesc | (1u << 15) | (1u << 16);  // A and B MN-major

__global__ void __launch_bounds__(kConvThreads, 2)
wgrad32_umma(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ dz,
             float* __restrict__ part, int H, int W, int tiles_x, int tiles_y, int ntiles,
             int dil, unsigned* __restrict__ fault, uint32_t wait_limit) {
  // no static shared variables: the core matrices must start on 128-byte boundaries
  extern __shared__ __align__(128) unsigned char wgu[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(wgu + kWgTiles * kWgTile);
  volatile int* s_ok = reinterpret_cast<volatile int*>(bar + 1);
  volatile uint32_t* tslot = reinterpret_cast<volatile uint32_t*>(bar + 2);
  volatile int* abort_ = reinterpret_cast<volatile int*>(bar + 3);  // stays 0: one waiter only
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int my_tiles = (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  {
    uint4* ones = reinterpret_cast<uint4*>(wgu + 9 * kWgTile);  // BF16 1.0 = 0x3f80
    for (int q = threadIdx.x; q < (int)(kWgTile / 16); q += blockDim.x)
      ones[q] = make_uint4(0x3f803f80u, 0x3f803f80u, 0x3f803f80u, 0x3f803f80u);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32((const void*)tslot)), "r"(kWgTmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *s_ok = (smem_u32(wgu) & 127u) == 0;
    *abort_ = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t base = smem_u32(wgu);

#pragma unroll 1
  for (int i = 0; i < my_tiles; ++i) {
    const int tile = (int)blockIdx.x + i * (int)gridDim.x;
    const int tx = tile % tiles_x, ty = (tile / tiles_x) % tiles_y, b = tile / (tiles_x * tiles_y);
    if (*s_ok) {
      for (int tap = 0; tap < 9; ++tap)
        load_tap_cm_p<kWgRows>(wgu + tap * kWgTile, in, b, ty * kWgRows, tx * TW, tap_dy(tap, dil),
                               tap_dx(tap, dil), H, W, threadIdx.x, blockDim.x);
      load_tap_cm_p<kWgRows>(wgu + 10 * kWgTile, dz, b, ty * kWgRows, tx * TW, 0, 0, H, W,
                             threadIdx.x, blockDim.x);
    }
    cp_commit();
    cp_wait_group<0>();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // tiles -> tensor core
    __syncthreads();
    if (threadIdx.x == 0 && *s_ok) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
      for (int blk = 0; blk < 3; ++blk) {
#pragma unroll 4
        for (int ks = 0; ks < (kWgRows * TW) / 16; ++ks) {
          const uint64_t ad = umma_desc(base + blk * 4 * (uint32_t)kWgTile + ks * 256, 128, kWgChunk);
          const uint64_t bd = umma_desc(base + 10 * (uint32_t)kWgTile + ks * 256, 128, kWgChunk);
          asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                       "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                       ::"r"(tmem + blk * C), "l"(ad), "l"(bd), "r"(kIdescMN),
                         "r"((i > 0 || ks > 0) ? 1u : 0u) : "memory");
        }
      }
      umma_commit(smem_u32(bar));
      // the tiles are restaged only after these MMAs have read them; a wait
      // that runs out still drains them before the CTA goes on
      if (!mbar_wait_ab(smem_u32(bar), i & 1, abort_, wait_limit)) {
        mbar_wait_drain(smem_u32(bar), i & 1);
        *s_ok = 0;
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }

  float* out = part + (size_t)blockIdx.x * (C * K9 + C);
  const bool ok = *s_ok != 0;
#pragma unroll 1
  for (int blk = 0; blk < 3; ++blk) {
    const int tap = 4 * blk + warp;  // row group of this warp: tap 0..8, 9 = the ones rows
    uint32_t v[32];
    if (ok && my_tiles > 0) tmem_ld32(v, tmem + blk * C + ((uint32_t)(warp * 32) << 16));
    else
#pragma unroll
      for (int o = 0; o < C; ++o) v[o] = 0u;
    if (tap < 9) {
#pragma unroll
      for (int o = 0; o < C; ++o) out[o * K9 + tap * C + lane] = __uint_as_float(v[o]);
    } else if (tap == 9 && lane == 0) {
#pragma unroll
      for (int o = 0; o < C; ++o) out[C * K9 + o] = __uint_as_float(v[o]);
    }
  }
  if (!ok && threadIdx.x == 0) atomicOr(fault, 1u);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kWgTmemCols)
                 : "memory");
}


// Weight gradient of a unit-offset 32 -> 32 layer (dilation 1, or a dilated
// layer over relabelled activations, whose input and dz share positions):
// the same sums as wgrad32_umma from one staged patch per half. A 2 x 64-pixel
// tile (K = 128 pixels) stages, per 32-pixel half, the rows y0 - 1 .. y0 + 2
// at columns x0 + 32 h - 1 .. x0 + 32 h + 32 (one halo pixel per side), as
// [chunk][row][34 px][8 ch] with 544-byte rows: one box of the tensor memory
// accelerator (32-bit elements, so that a 34-pixel row is one box row) where
// the half and its halo lie inside the image, per-pixel copies where they
// wrap. The dz tile is staged as before ([half][chunk][row][32 px][8 ch]).
// In this MN-major A operand (M = channels, K = pixels) a core matrix is
// 8 pixels x 16 bytes, contiguous, and the next 8 pixels follow 128 bytes on,
// so the column offset dx = 0..2 of a tap is a start address 16 dx bytes on:
// the three column offsets share the patch. M = (chunk c, dy) for dy = 0..3,
// core matrices at (4c + dy) x 544 B: one descriptor (stride byte offset 544)
// covers the three taps (dy, dx) of a column offset; the fourth dy reads one
// row past the patch (inside the buffer) and its rows of D are dropped. A
// fourth block multiplies a tile of ones: db. D of block dx, TMEM lane
// 32 w + l: channel 8 w + l % 8, tap (l / 8, dx).
constexpr int kWuRows = 2;                          // output rows per tile (K = 128 pixels)
constexpr int kWuPRows = kWuRows + 2;               // patch rows
constexpr int kWuHW = kHW + 2;                      // 34: a half-row and its two halo pixels
constexpr uint32_t kWuHRow = kWuHW * 16;            // 544 B
constexpr uint32_t kWuPChunk = kWuPRows * kWuHRow;  // 2176 B
constexpr uint32_t kWuPHalf = 4 * kWuPChunk;        // 8704 B (a multiple of 128)
constexpr uint32_t kWuPatch = 2 * kWuPHalf;         // 17408 B
constexpr uint32_t kWuZChunk = kWuRows * kHRow;     // 1 KB
constexpr uint32_t kWuZHalf = 4 * kWuZChunk;        // 4 KB
constexpr uint32_t kWuZ = kWuPatch;                 // dz tile offset (after the patch)
constexpr uint32_t kWuOnes = kWuZ + 2 * kWuZHalf;   // ones tile offset (4 KB)
constexpr uint32_t kWuBars = kWuOnes + 4096;        // barriers and flags (64 B)
constexpr size_t kWuSmem = kWuBars + 64;            // 29.1 KB
constexpr int kWuCtasPerSm = 4;                     // 4 x 128 TMEM columns per SM
static_assert(kWuPHalf % 128 == 0 && kWuZ % 128 == 0 && kWuOnes % 128 == 0,
              "box destinations and core matrices on 128-byte boundaries");
// the second half's dropped fourth dy reads at most up to here
static_assert(kWuPHalf + 15 * kWuHRow + 2 * 16 + kWuHRow + 16 * 16 <= kWuBars,
              "the dropped fourth dy stays inside the buffer");

// Per-pixel copies of one halo-padded patch half (rows y0 - 1 .., columns
// x0 - 1 ..), periodic wrap, into [chunk][row][34 px][8 ch].
__device__ __forceinline__ void load_patch_half(unsigned char* dst, const __nv_bfloat16* act,
                                                int b, int y0, int x0, int H, int W, int pid,
                                                int np) {
  constexpr int kN = kWuPRows * kWuHW * 4;
  for (int q = pid; q < kN; q += np) {
    const int chunk = q / (kWuPRows * kWuHW), pix = q - chunk * (kWuPRows * kWuHW);
    const int r = pix / kWuHW, c = pix - r * kWuHW;
    const int gy = wrap1(y0 + r - 1, H), gx = wrap1(x0 + c - 1, W);
    cp16(dst + chunk * kWuPChunk + pix * 16, act + act_off(b, gy, gx, chunk, H, W));
  }
}

// One halo-padded patch half as a box: 32-bit elements, x = first pixel x 4.
__device__ __forceinline__ void tma_load_patch_half(uint32_t dst, const CUtensorMap* map, int px,
                                                    int y, int b, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4, %5}], [%6];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(px * 4), "r"(y), "r"(0), "r"(b),
        "r"(bar)
      : "memory");
}

__global__ void __launch_bounds__(kConvThreads, kWuCtasPerSm)
wgrad32_unit(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ dz,
             float* __restrict__ part, int H, int W, int tiles_x, int tiles_y, int ntiles,
             unsigned* __restrict__ fault, uint32_t wait_limit,
             const __grid_constant__ CUtensorMap tmap_in, const __grid_constant__ CUtensorMap tmap_dz,
             int use_tma) {
  // no static shared variables: the core matrices must start on 128-byte boundaries
  extern __shared__ __align__(128) unsigned char wuu[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(wuu + kWuBars);  // [0] boxes, [1] MMAs
  volatile int* s_ok = reinterpret_cast<volatile int*>(bar + 2);
  volatile uint32_t* tslot = reinterpret_cast<volatile uint32_t*>(bar + 3);
  volatile int* abort_ = reinterpret_cast<volatile int*>(bar + 4);  // stays 0: one waiter only
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
  const int my_tiles = (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  {
    uint4* ones = reinterpret_cast<uint4*>(wuu + kWuOnes);  // BF16 1.0 = 0x3f80
    for (int q = tid; q < 4096 / 16; q += blockDim.x)
      ones[q] = make_uint4(0x3f803f80u, 0x3f803f80u, 0x3f803f80u, 0x3f803f80u);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32((const void*)tslot)), "r"(kWgTmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar + 1)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *s_ok = (smem_u32(wuu) & 127u) == 0;
    *abort_ = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t base = smem_u32(wuu);
  uint32_t box_par = 0, mma_par = 0;

#pragma unroll 1
  for (int i = 0; i < my_tiles; ++i) {
    const int tile = (int)blockIdx.x + i * (int)gridDim.x;
    const int tx = tile % tiles_x, ty = (tile / tiles_x) % tiles_y, b = tile / (tiles_x * tiles_y);
    const int y0 = ty * kWuRows, x0 = tx * TW;
    const bool ok = *s_ok != 0;
    // which halves come as boxes: bit h for the patch, bit 2 + h for dz
    uint32_t boxes = 0;
    if (use_tma && ok) {
      const bool rows_in = y0 >= 1 && y0 - 1 + kWuPRows <= H;
      for (int h = 0; h < 2; ++h) {
        const int xs = x0 + kHW * h - 1;
        if (rows_in && xs >= 0 && xs + kWuHW <= W) boxes |= 1u << h;
      }
      boxes |= 3u << 2;  // the dz tile never wraps (y0 + 2 <= H, x0 + 64 <= W)
    }
    if (tid == 0 && boxes) {
      const uint32_t bytes = (uint32_t)__popc(boxes & 3u) * kWuPHalf +
                             (uint32_t)__popc(boxes >> 2) * kWuZHalf;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                   ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
      for (int h = 0; h < 2; ++h)
        if (boxes & (1u << h))
          tma_load_patch_half(base + h * kWuPHalf, &tmap_in, x0 + kHW * h - 1, y0 - 1, b,
                              smem_u32(bar));
      for (int h = 0; h < 2; ++h)
        tma_load_half(base + kWuZ + h * kWuZHalf, &tmap_dz, x0 + kHW * h, y0, b, smem_u32(bar));
    }
    if (ok) {
      for (int h = 0; h < 2; ++h)
        if (!(boxes & (1u << h)))
          load_patch_half(wuu + h * kWuPHalf, in, b, y0, x0 + kHW * h, H, W, tid, blockDim.x);
      for (int h = 0; h < 2; ++h)
        if (!(boxes & (1u << (2 + h))))
          load_half_cm_p<kWuRows>(wuu + kWuZ + h * kWuZHalf, dz, b, y0, x0 + kHW * h, 0, 0, H, W,
                                  tid, blockDim.x);
    }
    cp_commit();
    cp_wait_group<0>();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // copies -> tensor core
    __syncthreads();
    if (tid == 0 && ok) {
      bool good = true;
      if (boxes) {
        good = mbar_wait_ab(smem_u32(bar), box_par, abort_, wait_limit);
        box_par ^= 1u;
      }
      if (good) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
        for (int blk = 0; blk < 4; ++blk) {
#pragma unroll
          for (int ks = 0; ks < (kWuRows * TW) / 16; ++ks) {
            // output row ro, pixels px0 .. px0 + 15: half px0 / 32 of the tile;
            // in the patch, output pixel p of a half sits at column p + 1, so
            // column offset dx - 1 reads from column p + dx
            const int ro = ks >> 2, px0 = (ks & 3) * 16;
            const uint32_t half = px0 / kHW;
            const uint64_t ad = blk < 3
                ? umma_desc(base + half * kWuPHalf + ro * kWuHRow + ((px0 % kHW) + blk) * 16, 128, kWuHRow)
                : umma_desc(base + kWuOnes, 128, 256);
            const uint32_t koff = ro * kHRow + (px0 % kHW) * 16;
            const uint64_t bd = umma_desc(base + kWuZ + half * kWuZHalf + koff, 128, kWuZChunk);
            asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                         "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                         ::"r"(tmem + blk * C), "l"(ad), "l"(bd), "r"(kIdescMN),
                           "r"((i > 0 || ks > 0) ? 1u : 0u) : "memory");
          }
        }
        umma_commit(smem_u32(bar + 1));
        // the buffers are restaged only after these MMAs have read them; a
        // wait that runs out still drains them before the CTA goes on
        if (!mbar_wait_ab(smem_u32(bar + 1), mma_par, abort_, wait_limit)) {
          mbar_wait_drain(smem_u32(bar + 1), mma_par);
          good = false;
        }
        mma_par ^= 1u;
      } else if (boxes) {
        mbar_wait_drain(smem_u32(bar), box_par ^ 1u);  // boxes still landing: let them finish
      }
      if (!good) *s_ok = 0;
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }

  float* out = part + (size_t)blockIdx.x * (C * K9 + C);
  const bool ok = *s_ok != 0;
#pragma unroll 1
  for (int blk = 0; blk < 4; ++blk) {
    uint32_t v[32];
    if (ok && my_tiles > 0) tmem_ld32(v, tmem + blk * C + ((uint32_t)(warp * 32) << 16));
    else
#pragma unroll
      for (int o = 0; o < C; ++o) v[o] = 0u;
    const int dy = lane >> 3, c = warp * 8 + (lane & 7);
    if (blk < 3 && dy < 3) {
      const int tap = dy * 3 + blk;
#pragma unroll
      for (int o = 0; o < C; ++o) out[o * K9 + tap * C + c] = __uint_as_float(v[o]);
    } else if (blk == 3 && tid == 0) {
#pragma unroll
      for (int o = 0; o < C; ++o) out[C * K9 + o] = __uint_as_float(v[o]);
    }
  }
  if (!ok && tid == 0) atomicOr(fault, 1u);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kWgTmemCols)
                 : "memory");
}

// First layer (1 -> 32) forward: z = b + sum_tap W1[o][tap] x[p + tap]; a = gelu(z).
// Row-structured loops shared by the three single-channel layers: a CTA takes
// whole image rows (one division per row), its 4 W threads slots cover
// (pixel x = slot / 4, channel group slot % 4), the three wrapped tap rows
// are found once per row and the columns wrap with a conditional add when
// the dilation is below the width.

// (ny, nx): the outputs are stored relabelled: output position (yy, xx) holds
// the natural pixel (yy ny mod H, xx nx mod W) (1, 1: natural order).
__global__ void conv_first(const float* __restrict__ x, const float* __restrict__ w1,
                           const float* __restrict__ b1, __nv_bfloat16* __restrict__ zout,
                           __nv_bfloat16* __restrict__ aout, int B, int H, int W, int dil,
                           int ny, int nx) {
  const int cg = threadIdx.x & 3;  // blockDim is a multiple of 4: fixed per thread
  float wr[8][9], br[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    br[j] = __ldg(b1 + cg * 8 + j);
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) wr[j][tap] = __ldg(w1 + (cg * 8 + j) * 9 + tap);
  }
  const bool near = dil < W;
  for (int row = blockIdx.x; row < B * H; row += gridDim.x) {
    const int img = row / H, yy = row - img * H, yn = relabel(yy, ny, H);
    const float* xr[3];
#pragma unroll
    for (int ty = 0; ty < 3; ++ty) xr[ty] = x + ((int64_t)img * H + wrapn(yn + (ty - 1) * dil, H)) * W;
    for (int t = threadIdx.x; t < 4 * W; t += blockDim.x) {
      const int xx = t >> 2, xn = relabel(xx, nx, W);
      const int xs[3] = {wrap_col(xn - dil, W, near), xn, wrap_col(xn + dil, W, near)};
      float v[9];
#pragma unroll
      for (int ty = 0; ty < 3; ++ty)
#pragma unroll
        for (int tx = 0; tx < 3; ++tx) v[ty * 3 + tx] = __ldg(xr[ty] + xs[tx]);
      __nv_bfloat162 zz[4], aa[4];
#pragma unroll
      for (int j = 0; j < 8; j += 2) {
        float s0 = br[j], s1 = br[j + 1];
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
          s0 = fmaf(wr[j][tap], v[tap], s0);
          s1 = fmaf(wr[j + 1][tap], v[tap], s1);
        }
        zz[j / 2] = __floats2bfloat162_rn(s0, s1);
        aa[j / 2] = __float22bfloat162_rn(gelu_f2(make_float2(s0, s1)));
      }
      const int64_t po = act_off(img, yy, xx, cg, H, W);
      if (zout) *reinterpret_cast<uint4*>(zout + po) = *reinterpret_cast<const uint4*>(zz);
      *reinterpret_cast<uint4*>(aout + po) = *reinterpret_cast<const uint4*>(aa);
    }
  }
}


// Last layer (32 -> 1) forward: y = b6 + sum_{tap,c} W6[c][tap] a[p + tap][c] (FP32 out).
// Four threads per pixel sum 8 channels each (coalesced 16-byte loads: a warp
// reads 8 whole pixels per tap), then combine their partial sums in a fixed
// order with two shuffles (W is a multiple of 8, so whole warps iterate).
// The kernel is bound by the L1 bandwidth of its 16-byte tap loads (9 per
// thread and pixel). At dilation 1 (kRows = 4) a thread computes four output
// rows of one column: each of the six input rows' three columns is loaded
// once and serves every output row it is a tap of, 4.5 loads per pixel
// instead of 9; each output keeps its own sum in tap order.
template <int kRows>
__global__ void conv_last(const __nv_bfloat16* __restrict__ a, const float* __restrict__ w6,
                          const float* __restrict__ b6, float* __restrict__ y, int B, int H, int W,
                          int dil) {
  const int cg = threadIdx.x & 3;
  float wr[8][9];
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) wr[j][tap] = __ldg(w6 + (cg * 8 + j) * 9 + tap);
  const float bias = __ldg(b6);
  const bool near = dil < W;
  // kRows > 1: dil == 1 and H % kRows == 0 (checked by the launcher)
  for (int rb = blockIdx.x; rb < B * H / kRows; rb += gridDim.x) {
    const int row = rb * kRows;  // first output row of the block
    const int img = row / H, yy = row - img * H;
    constexpr int kIn = kRows == 1 ? 3 : kRows + 2;  // distinct input rows
    const __nv_bfloat16* ar[kIn];
#pragma unroll
    for (int r = 0; r < kIn; ++r)
      ar[r] = a + act_off(img, wrapn(yy + (kRows == 1 ? (r - 1) * dil : r - 1), H), 0, cg, H, W);
    for (int t = threadIdx.x; t < 4 * W; t += blockDim.x) {
      const int xx = t >> 2;
      const int xs[3] = {wrap_col(xx - dil, W, near), xx, wrap_col(xx + dil, W, near)};
      float s[kRows];
#pragma unroll
      for (int j = 0; j < kRows; ++j) s[j] = 0.f;
#pragma unroll
      for (int r = 0; r < kIn; ++r)
#pragma unroll
        for (int tx = 0; tx < 3; ++tx) {
          const uint4 u = __ldg(reinterpret_cast<const uint4*>(ar[r] + (int64_t)xs[tx] * 8));
          const __nv_bfloat162* hv = reinterpret_cast<const __nv_bfloat162*>(&u);
          // input row r is tap row ty = r - j of output row j
#pragma unroll
          for (int j = 0; j < kRows; ++j) {
            const int ty = r - j;
            if (ty < 0 || ty > 2) continue;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float2 f = __bfloat1622float2(hv[e]);
              s[j] = fmaf(wr[2 * e][ty * 3 + tx], f.x, s[j]);
              s[j] = fmaf(wr[2 * e + 1][ty * 3 + tx], f.y, s[j]);
            }
          }
        }
#pragma unroll
      for (int j = 0; j < kRows; ++j) {
        float v = s[j];
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        if (cg == 0) y[(int64_t)(row + j) * W + xx] = bias + v;
      }
    }
  }
}

// Loss: d[p] = y - t; per-block partial sums of d^2; dy = 2 d / n.
__global__ void mse_grad(const float* __restrict__ y, const float* __restrict__ t,
                         float* __restrict__ dy, double* __restrict__ part, int64_t n) {
  double acc = 0.0;
  const float inv = 2.0f / (float)n;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const float d = y[p] - t[p];
    dy[p] = d * inv;
    acc += (double)d * (double)d;
  }
  __shared__ double sh[256];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// Backward of the last layer: dz5[q][c] = gelu'(z5[q][c]) * sum_tap W6[c][tap] dy[q - tap].
// (ny, nx): dz5 is stored relabelled, position (yy, xx) holding the natural
// pixel (yy ny mod H, xx nx mod W); z5 and dy are in natural order.
__global__ void back_last(const float* __restrict__ dy, const float* __restrict__ w6,
                          const __nv_bfloat16* __restrict__ z5, __nv_bfloat16* __restrict__ dz5,
                          int B, int H, int W, int dil, int ny, int nx) {
  // four threads per pixel, 8 channels each (coalesced 16-byte z5 loads and dz5 stores)
  const int cg = threadIdx.x & 3;
  float wr[8][9];
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) wr[j][tap] = __ldg(w6 + (cg * 8 + j) * 9 + tap);
  const bool near = dil < W;
  for (int row = blockIdx.x; row < B * H; row += gridDim.x) {
    const int img = row / H, yy = row - img * H, yn = relabel(yy, ny, H);
    const float* gr[3];  // dy at (q - off(tap)): tap row ty reads row y - (ty - 1) d
#pragma unroll
    for (int ty = 0; ty < 3; ++ty) gr[ty] = dy + ((int64_t)img * H + wrapn(yn - (ty - 1) * dil, H)) * W;
    for (int t = threadIdx.x; t < 4 * W; t += blockDim.x) {
      const int xx = t >> 2, xn = relabel(xx, nx, W);
      const int xs[3] = {wrap_col(xn + dil, W, near), xn, wrap_col(xn - dil, W, near)};
      float g[9];
#pragma unroll
      for (int ty = 0; ty < 3; ++ty)
#pragma unroll
        for (int tx = 0; tx < 3; ++tx) g[ty * 3 + tx] = __ldg(gr[ty] + xs[tx]);
      const int64_t po = act_off(img, yy, xx, cg, H, W);
      const uint4 u = __ldg(reinterpret_cast<const uint4*>(z5 + act_off(img, yn, xn, cg, H, W)));
      const __nv_bfloat162* hz = reinterpret_cast<const __nv_bfloat162*>(&u);
      __nv_bfloat162 o[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float2 z = __bfloat1622float2(hz[e]);
        float s0 = 0.f, s1 = 0.f;
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
          s0 = fmaf(wr[2 * e][tap], g[tap], s0);
          s1 = fmaf(wr[2 * e + 1][tap], g[tap], s1);
        }
        o[e] = __float22bfloat162_rn(__fmul2_rn(make_float2(s0, s1), gelu_grad_f2(z)));
      }
      *reinterpret_cast<uint4*>(dz5 + po) = *reinterpret_cast<const uint4*>(o);
    }
  }
}

// Weight gradient of a single-channel side (first and last layers):
//   mode 0 (first): dW1[o][tap] = sum_p g32[p][o] * s1[p + off(tap)],  db1[o] = sum_p g32[p][o]
//   mode 1 (last):  dW6[c][tap] = sum_p s1[p] * g32[p + off(tap)][c],  db6    = sum_p s1[p]
// Mode 1 is computed as sum_q g32[q][c] * s1[q - off(tap)]: both modes are
// then "32-channel image times a shifted single-channel image", with the
// shift sign flipped. A CTA of 256 threads owns a range of image rows; kQ
// threads share a pixel, thread t taking channels (32 / kQ) (t % kQ) .. and
// pixel slot t / kQ (striding along each row), with 9 x 32 / kQ independent
// accumulators. kQ = 8 (36 accumulators, three CTAs per SM) measured faster
// for the last layer (220 against 372 us at batch 64), kQ = 4 (72, two CTAs,
// half the loads of the shifted image per pixel) for the first (201 against
// 222 us). The wrapped neighbour rows are found once per row. The CTA reduces
// its threads in a fixed order (shuffles within a warp, then warps in index
// order) and writes one partial per CTA, so the result is deterministic.
constexpr int kWsThreads = 256;
template <int kMode> constexpr int ws_q() { return kMode == 0 ? 4 : 8; }
template <int kMode> constexpr int ws_ctas_per_sm() { return kMode == 0 ? 2 : 3; }
// CTAs launched per SM: one resident wave for kQ = 8, two waves for kQ = 4
// (measured at batch 64; the row ranges are then shorter)
template <int kMode> constexpr int ws_split_per_sm() { return kMode == 0 ? 4 : 3; }
template <int kMode>
__global__ void __launch_bounds__(kWsThreads, ws_ctas_per_sm<kMode>())
wgrad_single(const __nv_bfloat16* __restrict__ g32, const float* __restrict__ s1,
             float* __restrict__ part, int B, int H, int W, int rows_per_cta, int dil) {
  constexpr int kQ = ws_q<kMode>();   // threads per pixel
  constexpr int kN = C / kQ;          // channels per thread: 8 or 4
  constexpr int kSlots = kWsThreads / kQ;
  constexpr int kJ = kN * 9 + kN;     // a thread's products and sums
  __shared__ float red[kWsThreads / 32][kQ][kJ];
  const int cq = threadIdx.x & (kQ - 1), slot = threadIdx.x / kQ;
  const int c0 = cq * kN, chunk = c0 / 8, sub = c0 % 8;  // channels c0 .. c0 + kN - 1
  const int sd = kMode == 0 ? dil : -dil;  // shift of s1 relative to g32
  const bool near = dil < W;
  const int rows = B * H;
  const int r0 = blockIdx.x * rows_per_cta, r1 = min(rows, r0 + rows_per_cta);
  float acc[kN][9], accb[kN];
#pragma unroll
  for (int k = 0; k < kN; ++k) {
    accb[k] = 0.f;
#pragma unroll
    for (int tp = 0; tp < 9; ++tp) acc[k][tp] = 0.f;
  }
  for (int row = r0; row < r1; ++row) {
    const int img = row / H, y = row - img * H;
    const int64_t ibase = (int64_t)img * H * W;
    const float* srow[3];
#pragma unroll
    for (int ty = 0; ty < 3; ++ty) srow[ty] = s1 + ibase + (int64_t)wrapn(y + (ty - 1) * sd, H) * W;
    const __nv_bfloat16* grow = g32 + act_off(img, y, 0, chunk, H, W) + sub;
    for (int x = slot; x < W; x += kSlots) {
      const int xs[3] = {wrap_col(x - sd, W, near), x, wrap_col(x + sd, W, near)};
      float sv[9];
#pragma unroll
      for (int ty = 0; ty < 3; ++ty)
#pragma unroll
        for (int tx = 0; tx < 3; ++tx) sv[ty * 3 + tx] = __ldg(srow[ty] + xs[tx]);
      float g[kN];
      if constexpr (kN == 8) {
        const uint4 u = __ldg(reinterpret_cast<const uint4*>(grow + (int64_t)x * 8));
        const __nv_bfloat162* hv = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float2 f = __bfloat1622float2(hv[e]);
          g[2 * e] = f.x;
          g[2 * e + 1] = f.y;
        }
      } else {
        const uint2 u = __ldg(reinterpret_cast<const uint2*>(grow + (int64_t)x * 8));
        const __nv_bfloat162* hv = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const float2 f = __bfloat1622float2(hv[e]);
          g[2 * e] = f.x;
          g[2 * e + 1] = f.y;
        }
      }
#pragma unroll
      for (int k = 0; k < kN; ++k) {
#pragma unroll
        for (int tp = 0; tp < 9; ++tp) acc[k][tp] = fmaf(g[k], sv[tp], acc[k][tp]);
        if (kMode == 0) accb[k] += g[k];
      }
      if (kMode == 1 && cq == 0) accb[0] += sv[4];
    }
  }
  // lanes l, l ^ kQ, l ^ 2 kQ, ... share a channel group: reduce them
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kN; ++k) {
#pragma unroll
    for (int tp = 0; tp < 9; ++tp) {
      float v = acc[k][tp];
#pragma unroll
      for (int o = kQ; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane < kQ) red[warp][cq][k * 9 + tp] = v;
    }
    float vb = accb[k];
#pragma unroll
    for (int o = kQ; o < 32; o <<= 1) vb += __shfl_xor_sync(0xffffffffu, vb, o);
    if (lane < kQ) red[warp][cq][kN * 9 + k] = vb;
  }
  __syncthreads();
  float* out = part + (size_t)blockIdx.x * (C * 9 + C);
  for (int i = threadIdx.x; i < kQ * kJ; i += blockDim.x) {
    const int q = i / kJ, j = i - q * kJ;
    float v = 0.f;
    for (int w = 0; w < kWsThreads / 32; ++w) v += red[w][q][j];
    if (j < kN * 9) {
      const int k = j / 9, tp = j - k * 9;
      out[(q * kN + k) * 9 + tp] = v;  // channel q kN + k, tap tp
    } else if (kMode == 0) {
      out[C * 9 + q * kN + (j - kN * 9)] = v;
    } else if (q == 0 && j == kN * 9) {
      out[C * 9] = v;  // db6: only group 0 summed s1
    }
  }
}

// Sum partials over CTAs (deterministic): dst[i] = sum_k part[k][i]. A block
// covers 32 outputs with 8 warps; warp w sums partials k = w, w + 8, ... in
// order (coalesced: 32 consecutive outputs per load), then the 8 slices are
// added in warp order.
constexpr int kRedSlices = 8;
__device__ __forceinline__ float reduce_slices(const float* __restrict__ part, int nparts,
                                               int stride, int i, bool in) {
  __shared__ float sl[kRedSlices][32];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  float v = 0.f;
  if (in)
    for (int k = w; k < nparts; k += kRedSlices) v += part[(size_t)k * stride + i];
  sl[w][l] = v;
  __syncthreads();
  float t = 0.f;
  if (w == 0)
    for (int q = 0; q < kRedSlices; ++q) t += sl[q][l];
  return t;
}
__global__ void __launch_bounds__(32 * kRedSlices)
reduce_partials(const float* __restrict__ part, int nparts, int stride, int count,
                float* __restrict__ dst) {
  const int i = blockIdx.x * 32 + (threadIdx.x & 31);
  const float t = reduce_slices(part, nparts, stride, i, i < count);
  if (threadIdx.x < 32 && i < count) dst[i] = t;
}

// Adam on the flat FP32 parameter vector, then refresh the kernel-layout copies.
__global__ void adam_update(float* __restrict__ p, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, int n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// Kernel-layout weights of a 32 -> 32 layer from the FP32 (o, c, dy, dx) tensor:
// fwd[o][tap*32 + c] = W[o][c][tap]; bwd[c][tap*32 + o] = W[o][c][8 - tap].
__global__ void pack_weights(const float* __restrict__ Wt, __nv_bfloat16* __restrict__ fwd,
                             __nv_bfloat16* __restrict__ bwd) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < C * C * 9; i += gridDim.x * blockDim.x) {
    const int o = i / (C * 9), c = (i / 9) % C, tap = i % 9;
    const __nv_bfloat16 w = __float2bfloat16_rn(Wt[i]);
    fwd[cm_index(o, tap * C + c)] = w;
    bwd[cm_index(c, (8 - tap) * C + o)] = w;
  }
}

// Per-image scaling of the network input and of the returned guess.
//   prepare: s = max|rho h^2| (per image), x = rho h^2 / s (FP32), optional
//            t = phi 4 pi^2 h^2 / s (the lowest mode of a unit-square field then
//            has a target of order one);
//   finish:  phi0 = s / (4 pi^2 h^2) (y - mean(y)).
constexpr double kTargetScale = 39.478417604357434;  // 4 pi^2
__global__ void prepare_images(const double* __restrict__ rho, const double* __restrict__ phi,
                               float* __restrict__ x, float* __restrict__ t,
                               double* __restrict__ scale, int H, int W, double h2) {
  const int img = blockIdx.x;
  const int64_t n = (int64_t)H * W, off = (int64_t)img * n;
  uint64_t mx = 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) mx = umax(mx, absbits(rho[off + i] * h2));
  __shared__ uint64_t sm[32];
  mx = warp_max(mx);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = umax(m, sm[w]);
    double s = __longlong_as_double((long long)m);
    if (!(s > 0.0)) s = 1.0;
    scale[img] = s;
    sm[0] = (uint64_t)__double_as_longlong(s);
  }
  __syncthreads();
  const double s = __longlong_as_double((long long)sm[0]);
  const double is = 1.0 / s;
  const double ts = kTargetScale * h2 * is;  // targets: phi * 4 pi^2 h^2 / s
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    x[off + i] = (float)(rho[off + i] * h2 * is);
    if (t) t[off + i] = (float)(phi[off + i] * ts);
  }
}

__global__ void finish_images(const float* __restrict__ y, const double* __restrict__ scale,
                              double* __restrict__ phi0, int H, int W, double h2) {
  const int img = blockIdx.x;
  const int64_t n = (int64_t)H * W, off = (int64_t)img * n;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += (double)y[off + i];
  __shared__ double sh[1024];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  const double mean = sh[0] / (double)n;
  const double s = scale[img] / (kTargetScale * h2);
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) phi0[off + i] = s * ((double)y[off + i] - mean);
}

// Natural-order copy of a relabelled activation tensor: pixel (y, x) of dst
// from position (y my mod H, x mx mod W) of src; one 16-byte chunk per thread.
__global__ void unrelabel(const __nv_bfloat16* __restrict__ src, __nv_bfloat16* __restrict__ dst,
                          int B, int H, int W, int my, int mx) {
  const int64_t n = (int64_t)B * 4 * H * W;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % W);
    const int64_t r = i / W;
    const int y = (int)(r % H);
    const int64_t bc = r / H;  // b * 4 + chunk
    const int64_t q = (bc * H + relabel(y, my, H)) * W + relabel(x, mx, W);
    reinterpret_cast<uint4*>(dst)[i] = reinterpret_cast<const uint4*>(src)[q];
  }
}

}  // namespace cnn
}  // namespace px

namespace px {
namespace cnn {
// [o][tap*32 + c] partials (plus 32 bias sums) summed over CTAs in index order,
// written as W[o][c][tap] and b[o].
__global__ void __launch_bounds__(32 * kRedSlices)
reduce_w32(const float* __restrict__ part, int nparts, float* __restrict__ dw,
           float* __restrict__ db) {
  const int stride = C * K9 + C;
  const int i = blockIdx.x * 32 + (threadIdx.x & 31);
  const float t = reduce_slices(part, nparts, stride, i, i < stride);
  if (threadIdx.x < 32 && i < stride) {
    if (i < C * K9) {
      const int o = i / K9, rem = i - o * K9, tap = rem / C, c = rem - tap * C;
      dw[o * K9 + c * 9 + tap] = t;
    } else {
      db[i - C * K9] = t;
    }
  }
}
}  // namespace cnn
}  // namespace px

// ---------------------------------------------------------------------------
// Host side.
namespace {

using namespace px::cnn;
constexpr int kLayers = 6;
const int kWidth[kLayers + 1] = {1, 32, 32, 32, 32, 32, 1};

struct Offsets {
  size_t w[kLayers], b[kLayers], total;
  Offsets() {
    size_t o = 0;
    for (int l = 0; l < kLayers; ++l) {
      w[l] = o;
      o += (size_t)kWidth[l + 1] * kWidth[l] * 9;
      b[l] = o;
      o += kWidth[l + 1];
    }
    total = o;
  }
};
const Offsets kOff;

int grid_1d(int64_t n, int threads) {
  const int64_t cap = (int64_t)px::device_sm_count() * 16;
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, cap));
}

}  // namespace

struct px_cnn {
  px_ctx* ctx = nullptr;
  int dil[kLayers] = {1, 1, 1, 1, 1, 1};  // per-layer dilation
  float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16* wf[kLayers] = {};
  __nv_bfloat16* wb[kLayers] = {};
  int64_t step = 0;
  int64_t cap_px = 0;
  __nv_bfloat16* z[kLayers] = {};
  __nv_bfloat16* a[kLayers] = {};
  __nv_bfloat16 *g0 = nullptr, *g1 = nullptr;
  float *y = nullptr, *dy = nullptr, *part = nullptr;
  double* lpart = nullptr;
  size_t part_floats = 0;
  float *xb = nullptr, *tb = nullptr;
  double* scales = nullptr;
  double* lpart_host = nullptr;
  int64_t cap_img = 0;
  uint32_t wait_limit = kSpinLimit;  // polls per handshake wait of the tensor-core kernels
  int use_tma = 1;                     // stage in-image tap tiles with the tensor memory accelerator
  int relabel = 1;                     // store activations relabelled for unit-offset dilated layers
  // layout of the last call's hidden tensors: a[l], z[l] stored at natural
  // position times (my[l], mx[l]) modulo (H, W)
  int last_b = 0, last_h = 0, last_w = 0;
  int my[kLayers] = {1, 1, 1, 1, 1, 1}, mx[kLayers] = {1, 1, 1, 1, 1, 1};
};

namespace {

px_status cnn_cuda(px_cnn* n, cudaError_t e, const char* what) {
  cudaGetLastError();
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return px::ctx_fail(n ? n->ctx : nullptr, e == cudaErrorMemoryAllocation ? PX_ENOMEM : PX_ECUDA,
                      m.c_str());
}

void free_work(px_cnn* n) {
  for (int l = 0; l < kLayers; ++l) {
    if (n->z[l]) cudaFree(n->z[l]);
    if (n->a[l]) cudaFree(n->a[l]);
    n->z[l] = n->a[l] = nullptr;
  }
  for (void* p : {(void*)n->g0, (void*)n->g1, (void*)n->y, (void*)n->dy, (void*)n->part,
                  (void*)n->lpart, (void*)n->xb, (void*)n->tb, (void*)n->scales})
    if (p) cudaFree(p);
  n->g0 = n->g1 = nullptr;
  n->y = n->dy = n->part = n->xb = n->tb = nullptr;
  n->lpart = n->scales = nullptr;
  n->cap_px = n->cap_img = 0;
}

// Workspace for B images of H x W: activations and pre-activations of layers
// 1..5, two gradient buffers, output, loss and weight-gradient partials.
px_status ensure_work(px_cnn* n, int64_t px, int64_t imgs) {
  if (n->cap_px >= px && n->cap_img >= imgs) return PX_OK;
  free_work(n);
  const size_t act = (size_t)px * C * sizeof(__nv_bfloat16);
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < 5 && e == cudaSuccess; ++l) {
    e = cudaMalloc(&n->z[l], act);
    if (e == cudaSuccess) e = cudaMalloc(&n->a[l], act);
  }
  if (e == cudaSuccess) e = cudaMalloc(&n->g0, act);
  if (e == cudaSuccess) e = cudaMalloc(&n->g1, act);
  if (e == cudaSuccess) e = cudaMalloc(&n->y, px * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&n->dy, px * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&n->xb, px * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&n->tb, px * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&n->scales, std::max<int64_t>(imgs, 1) * sizeof(double));
  n->part_floats = (size_t)std::max(px::device_sm_count() * 4, 1024) * (C * K9 + C);
  if (e == cudaSuccess) e = cudaMalloc(&n->part, n->part_floats * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&n->lpart, 4096 * sizeof(double));
  if (e != cudaSuccess) {
    free_work(n);
    return cnn_cuda(n, e, "network workspace");
  }
  n->cap_px = px;
  n->cap_img = imgs;
  return PX_OK;
}

px_status repack(px_cnn* n, cudaStream_t st) {
  for (int l = 1; l <= 4; ++l)
    pack_weights<<<36, 256, 0, st>>>(n->params + kOff.w[l], n->wf[l], n->wb[l]);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PX_OK : cnn_cuda(n, e, "pack weights");
}

px_status check_shape(px_cnn* n, int B, int H, int W) {
  if (B < 1 || H < 4 || W < 64 || H % TR || W % TW)
    return px::ctx_fail(n->ctx, PX_EUNSUPPORTED,
                        "network images need B >= 1, H a multiple of 4, W a multiple of 64");
  return PX_OK;
}

// Device address of the conv fault word on the current device (looked up
// once per device, then cached).
unsigned* conv_fault_ptr() {
  static unsigned* by_dev[64] = {};
  unsigned*& p = by_dev[px::dev_index()];
  if (!p) {
    void* q = nullptr;
    if (cudaGetSymbolAddress(&q, g_conv_fault) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    p = static_cast<unsigned*>(q);
  }
  return p;
}

// PX_ETIMEOUT (and the word cleared) if a conv CTA gave up on a bounded wait
// since the last check; synchronises the stream.
px_status check_conv_fault(px_cnn* n, cudaStream_t st) {
  unsigned* p = conv_fault_ptr();
  if (!p) return cnn_cuda(n, cudaErrorInvalidSymbol, "conv fault word");
  unsigned h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, p, sizeof h, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cnn_cuda(n, e, "conv fault readback");
  if (h) {
    cudaMemsetAsync(p, 0, sizeof h, st);
    return px::ctx_fail(n->ctx, PX_ETIMEOUT, "a tensor-core conv CTA timed out waiting for its MMAs");
  }
  return PX_OK;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// dependency on the driver library); null if unavailable.
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled encode_tiled() {
  static EncodeTiled fn = nullptr;
  static bool resolved = false;
  if (!resolved) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess && q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(f);
    cudaGetLastError();
    resolved = true;
  }
  return fn;
}

// Tensor map of B chunk-planar activation images of H x W for boxes of R
// rows x 32 pixels x 32 channels (one half of an operand tile); false (and
// the per-pixel copy path) if the driver cannot encode it.
bool act_tensor_map(CUtensorMap* m, const __nv_bfloat16* act, int B, int H, int W, int R) {
  std::memset(m, 0, sizeof *m);
  const EncodeTiled enc = encode_tiled();
  if (!enc || ((uintptr_t)act & 15u)) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)W * 8, (cuuint64_t)H, 4, (cuuint64_t)B};
  const cuuint64_t strides[3] = {(cuuint64_t)W * 16, (cuuint64_t)W * H * 16,
                                 (cuuint64_t)W * H * 64};
  const cuuint32_t box[4] = {(cuuint32_t)kHW * 8, (cuuint32_t)R, 4, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16*>(act), dims,
             strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The same activations seen as 32-bit elements (two channels each), with a
// box of kWuHW pixels x R rows x 4 chunks: a halo-padded patch half of the
// weight gradient, 544-byte box rows.
bool act_tensor_map_halo(CUtensorMap* m, const __nv_bfloat16* act, int B, int H, int W, int R) {
  std::memset(m, 0, sizeof *m);
  const EncodeTiled enc = encode_tiled();
  if (!enc || ((uintptr_t)act & 15u) || W < kWuHW) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)W * 4, (cuuint64_t)H, 4, (cuuint64_t)B};
  const cuuint64_t strides[3] = {(cuuint64_t)W * 16, (cuuint64_t)W * H * 16,
                                 (cuuint64_t)W * H * 64};
  const cuuint32_t box[4] = {(cuuint32_t)kWuHW * 4, (cuuint32_t)R, 4, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT32, 4, const_cast<__nv_bfloat16*>(act), dims,
             strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

px_status set_conv_attrs() {
  static bool done_by_dev[64] = {};
  bool& done = done_by_dev[px::dev_index()];
  if (done) return PX_OK;
  cudaError_t e = cudaFuncSetAttribute(conv32_ws<0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWsSmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(conv32_ws<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWsSmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(conv32_ws<0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWsSmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(conv32_ws<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWsSmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(wgrad32_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWgUmmaSmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(wgrad32_unit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWuSmem);
  if (e != cudaSuccess) { cudaGetLastError(); return PX_ECUDA; }
  done = true;
  return PX_OK;
}

// Inverse of d modulo m (0 if gcd(d, m) > 1).
int inv_mod(int64_t d, int64_t m) {
  int64_t r0 = m, r1 = ((d % m) + m) % m, t0 = 0, t1 = 1;
  while (r1 != 0) {
    const int64_t q = r0 / r1, r2 = r0 - q * r1, t2 = t0 - q * t1;
    r0 = r1; r1 = r2; t0 = t1; t1 = t2;
  }
  if (r0 != 1) return m == 1 ? 1 : 0;
  return (int)(((t0 % m) + m) % m);
}

// Relabelling of a dilated layer. With d invertible modulo H and W (d odd and
// the sides powers of two, for instance), storing the layer's input with
// natural pixel p at position p d^-1 makes the taps p + (dy, dx) d land at
// positions q + (dy, dx): the layer is a unit-offset convolution over
// positions, whose output at position q is the natural pixel q d. Each
// producer stores its outputs in the positions its consumer wants.
//   rel[l]        layer l (1..4) runs over its input's relabelled positions
//   unit[l]       layer l stages unit-offset patches (relabelled or d = 1)
//   my/mx[l]      a[l], z[l] (l = 0..4) and dZ[l+1] are stored at natural * m
//   ny/nx[l]      the inverse: natural = position * n
struct Plan {
  bool rel[kLayers] = {}, unit[kLayers] = {};
  int my[kLayers], mx[kLayers], ny[kLayers], nx[kLayers];
};
Plan plan_of(const px_cnn* n, int H, int W) {
  Plan p;
  for (int l = 0; l < kLayers; ++l) p.my[l] = p.mx[l] = p.ny[l] = p.nx[l] = 1;
  for (int l = 1; l <= 4; ++l) {
    p.rel[l] = n->relabel && n->dil[l] > 1 && inv_mod(n->dil[l], H) && inv_mod(n->dil[l], W);
    p.unit[l] = p.rel[l] || n->dil[l] == 1;
  }
  for (int l = 0; l < 4; ++l)
    if (p.rel[l + 1]) {
      p.my[l] = inv_mod(n->dil[l + 1], H);
      p.mx[l] = inv_mod(n->dil[l + 1], W);
      p.ny[l] = n->dil[l + 1] % H;
      p.nx[l] = n->dil[l + 1] % W;
    }
  return p;
}

// Multiplier (a * b) mod m of two relabellings.
int mul_mod(int a, int b, int m) { return (int)(((int64_t)a * b) % m); }

// Launches the 32 -> 32 tensor-core convolution in its staging form.
template <int kMode>
void launch_conv32(bool unit, int grid, cudaStream_t st, const __nv_bfloat16* in,
                   const __nv_bfloat16* wk, const float* bias, const __nv_bfloat16* zprev,
                   __nv_bfloat16* zout, __nv_bfloat16* aout, int H, int W, int tiles_x,
                   int tiles_y, int ntiles, int dil, int ry, int rx, unsigned* fault,
                   uint32_t wait_limit, const CUtensorMap& tm, int use) {
  if (unit)
    conv32_ws<kMode, true><<<grid, kWsConvThreads, kWsSmem, st>>>(
        in, wk, bias, zprev, zout, aout, H, W, tiles_x, tiles_y, ntiles, 1, ry, rx, fault,
        wait_limit, tm, use);
  else
    conv32_ws<kMode, false><<<grid, kWsConvThreads, kWsSmem, st>>>(
        in, wk, bias, zprev, zout, aout, H, W, tiles_x, tiles_y, ntiles, dil, ry, rx, fault,
        wait_limit, tm, use);
}

// Forward pass into n->a / n->z (z only when training) and output y.
px_status forward(px_cnn* n, const float* x, float* y, int B, int H, int W, bool train,
                  cudaStream_t st) {
  const int tiles_x = W / TW, tiles_y = H / TR;
  const int tiles = B * tiles_x * tiles_y;
  const int rows_grid = std::min(B * H, 8 * px::device_sm_count());  // whole rows per CTA
  const Plan P = plan_of(n, H, W);
  n->last_b = B;
  n->last_h = H;
  n->last_w = W;
  for (int l = 0; l < kLayers; ++l) { n->my[l] = P.my[l]; n->mx[l] = P.mx[l]; }
  conv_first<<<rows_grid, 256, 0, st>>>(x, n->params + kOff.w[0], n->params + kOff.b[0],
                                        train ? n->z[0] : nullptr, n->a[0], B, H, W, n->dil[0],
                                        P.ny[0], P.nx[0]);
  unsigned* fault = conv_fault_ptr();
  if (!fault) return cnn_cuda(n, cudaErrorInvalidSymbol, "conv fault word");
  const int cgrid = std::min(tiles, 2 * px::device_sm_count());  // persistent: 2 CTAs per SM
  for (int l = 1; l <= 4; ++l) {
    alignas(64) CUtensorMap tm;
    const int use = n->use_tma && act_tensor_map(&tm, n->a[l - 1], B, H, W, P.unit[l] ? kURows : TR);
    // output position = natural (input position times d if relabelled) times m[l]
    const int ny = P.rel[l] ? P.ny[l - 1] : 1, nx = P.rel[l] ? P.nx[l - 1] : 1;
    launch_conv32<0>(P.unit[l], cgrid, st, n->a[l - 1], n->wf[l], n->params + kOff.b[l], nullptr,
                     train ? n->z[l] : nullptr, n->a[l], H, W, tiles_x, tiles_y, tiles, n->dil[l],
                     mul_mod(ny, P.my[l], H), mul_mod(nx, P.mx[l], W), fault, n->wait_limit, tm,
                     use);
  }
  if (n->dil[5] == 1 && H % 4 == 0)
    conv_last<4><<<std::min(B * H / 4, 8 * px::device_sm_count()), 256, 0, st>>>(
        n->a[4], n->params + kOff.w[5], n->params + kOff.b[5], y, B, H, W, 1);
  else
    conv_last<1><<<rows_grid, 256, 0, st>>>(n->a[4], n->params + kOff.w[5],
                                            n->params + kOff.b[5], y, B, H, W, n->dil[5]);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PX_OK : cnn_cuda(n, e, "network forward");
}

// Forward + backward: gradients into n->grads, loss partials into n->lpart.
px_status grads(px_cnn* n, const float* x, const float* t, int B, int H, int W, int* nloss,
                cudaStream_t st) {
  px_status s = forward(n, x, n->y, B, H, W, true, st);
  if (s != PX_OK) return s;
  const int64_t px = (int64_t)B * H * W;
  const int tiles_x = W / TW, tiles_y = H / TR;
  const int tiles = B * tiles_x * tiles_y;
  const int lblocks = std::min<int64_t>(4096, grid_1d(px, 256));
  mse_grad<<<lblocks, 256, 0, st>>>(n->y, t, n->dy, n->lpart, px);
  *nloss = lblocks;
  // last layer
  // single-channel weight gradients: whole image rows per CTA
  const int rows = B * H;
  auto single_split = [&](int per_sm, int* rpc_out) {
    const int64_t want = std::min<int64_t>((int64_t)px::device_sm_count() * per_sm,
                                           (int64_t)(n->part_floats / (C * 9 + C)));
    const int r = (int)((rows + want - 1) / want);
    *rpc_out = r;
    return (rows + r - 1) / r;
  };
  int rpc = 0, rpc0 = 0;
  const int nsc_cap = single_split(ws_split_per_sm<1>(), &rpc);
  const int nsc0 = single_split(ws_split_per_sm<0>(), &rpc0);
  wgrad_single<1><<<nsc_cap, kWsThreads, 0, st>>>(n->a[4], n->dy,
                                                  n->part, B, H, W, rpc, n->dil[5]);
  reduce_partials<<<(C * 9 + C + 31) / 32, 32 * kRedSlices, 0, st>>>(n->part, nsc_cap, C * 9 + C, C * 9 + 1, n->grads + kOff.w[5]);
  const Plan P = plan_of(n, H, W);
  // dZ of layer 4 goes in the positions of layer 4's input a[3]
  back_last<<<std::min(B * H, 8 * px::device_sm_count()), 256, 0, st>>>(
      n->dy, n->params + kOff.w[5], n->z[4], n->g0, B, H, W, n->dil[5], P.ny[3], P.nx[3]);
  __nv_bfloat16* gcur = n->g0;
  __nv_bfloat16* gnext = n->g1;
  // weight gradients: 2 x 64-pixel tiles, two CTAs per SM
  const int wg_tiles = B * tiles_x * (H / kWgRows);
  const int wg_ctas = std::min(wg_tiles, 2 * px::device_sm_count());
  for (int l = 4; l >= 1; --l) {
    // a[l - 1] and dZ[l] share their positions: unit offsets when relabelled
    int nparts = wg_ctas;
    if (P.unit[l]) {
      alignas(64) CUtensorMap tmi, tmz;
      const int use = n->use_tma && act_tensor_map_halo(&tmi, n->a[l - 1], B, H, W, kWuPRows) &&
                      act_tensor_map(&tmz, gcur, B, H, W, kWuRows);
      nparts = std::min(wg_tiles, kWuCtasPerSm * px::device_sm_count());
      wgrad32_unit<<<nparts, kConvThreads, kWuSmem, st>>>(
          n->a[l - 1], gcur, n->part, H, W, tiles_x, H / kWuRows, wg_tiles, conv_fault_ptr(),
          n->wait_limit, tmi, tmz, use);
    } else {
      wgrad32_umma<<<wg_ctas, kConvThreads, kWgUmmaSmem, st>>>(
          n->a[l - 1], gcur, n->part, H, W, tiles_x, H / kWgRows, wg_tiles, n->dil[l],
          conv_fault_ptr(), n->wait_limit);
    }
    // reorder [o][tap*32 + c] + bias into W[o][c][tap] + b
    reduce_w32<<<(C * K9 + C + 31) / 32, 32 * kRedSlices, 0, st>>>(n->part, nparts, n->grads + kOff.w[l], n->grads + kOff.b[l]);
    alignas(64) CUtensorMap tm;
    const int use = n->use_tma && act_tensor_map(&tm, gcur, B, H, W, P.unit[l] ? kURows : TR);
    // dZ[l - 1] goes in the positions of a[l - 2] (natural order for l = 1)
    const int ny = P.rel[l] ? P.ny[l - 1] : 1, nx = P.rel[l] ? P.nx[l - 1] : 1;
    const int my = l >= 2 ? P.my[l - 2] : 1, mx = l >= 2 ? P.mx[l - 2] : 1;
    launch_conv32<1>(P.unit[l], std::min(tiles, 2 * px::device_sm_count()), st, gcur, n->wb[l],
                     nullptr, n->z[l - 1], nullptr, gnext, H, W, tiles_x, tiles_y, tiles,
                     n->dil[l], mul_mod(ny, my, H), mul_mod(nx, mx, W), conv_fault_ptr(),
                     n->wait_limit, tm, use);
    std::swap(gcur, gnext);
  }
  wgrad_single<0><<<nsc0, kWsThreads, 0, st>>>(gcur, x, n->part, B, H, W, rpc0, n->dil[0]);
  reduce_partials<<<(C * 9 + C + 31) / 32, 32 * kRedSlices, 0, st>>>(n->part, nsc0, C * 9 + C, C * 9 + C, n->grads + kOff.w[0]);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PX_OK : cnn_cuda(n, e, "network backward");
}

px_status read_loss(px_cnn* n, int nloss, int64_t px, double* loss, cudaStream_t st) {
  const px_status fs = check_conv_fault(n, st);
  if (fs != PX_OK) return fs;
  std::vector<double> h(nloss);
  cudaError_t e = cudaMemcpyAsync(h.data(), n->lpart, nloss * sizeof(double),
                                  cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cnn_cuda(n, e, "loss readback");
  double s = 0.0;
  for (double v : h) s += v;
  *loss = s / (double)px;
  return PX_OK;
}

struct DevScope {
  int prev = -1, dev;
  explicit DevScope(int d) : dev(d) {
    cudaGetDevice(&prev);
    if (prev != d) cudaSetDevice(d);
  }
  ~DevScope() { if (prev >= 0 && prev != dev) cudaSetDevice(prev); }
};

}  // namespace


extern "C" {

size_t px_cnn_param_count(void) { return kOff.total; }

px_status px_cnn_create(px_ctx* c, uint64_t seed, const int32_t* dilations, px_cnn** out) {
  if (!c || !out) return PX_EINVAL;
  c->err.clear();
  *out = nullptr;
  if (dilations)
    for (int l = 0; l < kLayers; ++l)
      if (dilations[l] < 1 || dilations[l] > 4096)
        return px::ctx_fail(c, PX_EINVAL, "dilations must be in 1..4096");
  DevScope ds(c->device);
  if (set_conv_attrs() != PX_OK) return px::ctx_fail(c, PX_ECUDA, "conv kernel attributes");
  px_cnn* n = new (std::nothrow) px_cnn();
  if (!n) return px::ctx_fail(c, PX_ENOMEM, "host allocation failed");
  n->ctx = c;
  if (dilations)
    for (int l = 0; l < kLayers; ++l) n->dil[l] = dilations[l];
  const size_t P = kOff.total;
  cudaError_t e = cudaMalloc(&n->params, P * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&n->grads, P * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&n->m, P * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&n->v, P * sizeof(float));
  for (int l = 1; l <= 4 && e == cudaSuccess; ++l) {
    e = cudaMalloc(&n->wf[l], C * K9 * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc(&n->wb[l], C * K9 * sizeof(__nv_bfloat16));
  }
  if (e == cudaSuccess) e = cudaMemset(n->m, 0, P * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(n->v, 0, P * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(n->grads, 0, P * sizeof(float));
  // He-normal initialisation (std sqrt(2 / (9 Cin))), zero biases; seeded.
  std::vector<float> h(P, 0.0f);
  std::mt19937_64 rng(seed);
  for (int l = 0; l < kLayers; ++l) {
    std::normal_distribution<double> nd(0.0, std::sqrt(2.0 / (9.0 * kWidth[l])));
    for (size_t i = 0; i < (size_t)kWidth[l + 1] * kWidth[l] * 9; ++i) h[kOff.w[l] + i] = (float)nd(rng);
  }
  if (e == cudaSuccess) e = cudaMemcpy(n->params, h.data(), P * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    px_status s = cnn_cuda(n, e, "network parameters");
    px_cnn_destroy(n);
    return s;
  }
  px_status s = repack(n, 0);
  if (s == PX_OK && cudaDeviceSynchronize() != cudaSuccess) s = cnn_cuda(n, cudaGetLastError(), "pack");
  if (s != PX_OK) { px_cnn_destroy(n); return s; }
  *out = n;
  return PX_OK;
}

px_status px_cnn_destroy(px_cnn* n) {
  if (!n) return PX_OK;
  DevScope ds(n->ctx->device);
  cudaDeviceSynchronize();
  free_work(n);
  for (int l = 0; l < kLayers; ++l) {
    if (n->wf[l]) cudaFree(n->wf[l]);
    if (n->wb[l]) cudaFree(n->wb[l]);
  }
  for (void* p : {(void*)n->params, (void*)n->grads, (void*)n->m, (void*)n->v})
    if (p) cudaFree(p);
  delete n;
  return PX_OK;
}

px_status px_cnn_get_params(px_cnn* n, float* host, size_t count) {
  if (!n || !host || count != kOff.total) return PX_EINVAL;
  DevScope ds(n->ctx->device);
  cudaError_t e = cudaMemcpy(host, n->params, count * sizeof(float), cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? PX_OK : cnn_cuda(n, e, "get params");
}

px_status px_cnn_set_params(px_cnn* n, const float* host, size_t count) {
  if (!n || !host || count != kOff.total) return PX_EINVAL;
  DevScope ds(n->ctx->device);
  cudaError_t e = cudaMemcpy(n->params, host, count * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cnn_cuda(n, e, "set params");
  px_status s = repack(n, 0);
  if (s != PX_OK) return s;
  e = cudaDeviceSynchronize();
  return e == cudaSuccess ? PX_OK : cnn_cuda(n, e, "set params");
}

size_t px_cnn_state_count(void) { return 3 * kOff.total; }

// Stored hidden tensors of the last forward pass (for inspection and
// tests): which = 0 the activation a_l = gelu(z_l), 1 the pre-activation z_l
// (kept only by px_cnn_grads / px_cnn_train_step), of hidden layer l = 1..5;
// NHWC BF16 bit patterns, B * H * W * 32 values for the last call's shape.
px_status px_cnn_get_hidden(px_cnn* n, int layer, int which, uint16_t* host, size_t count,
                            void* stream) {
  if (!n || !host || layer < 1 || layer > 5 || which < 0 || which > 1) return PX_EINVAL;
  if (n->cap_px == 0 || count > (size_t)n->cap_px * C) return PX_EINVAL;
  DevScope ds(n->ctx->device);
  const __nv_bfloat16* src = which == 0 ? n->a[layer - 1] : n->z[layer - 1];
  cudaStream_t st = (cudaStream_t)stream;
  const int l = layer - 1, B = n->last_b, H = n->last_h, W = n->last_w;
  if (n->my[l] != 1 || n->mx[l] != 1) {
    // stored relabelled: gather natural order into the gradient scratch
    unrelabel<<<grid_1d((int64_t)B * 4 * H * W, 256), 256, 0, st>>>(src, n->g1, B, H, W, n->my[l],
                                                                     n->mx[l]);
    src = n->g1;
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(host, src, count * sizeof(uint16_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? PX_OK : cnn_cuda(n, e, "hidden readback");
}

// How the tensor-core convolutions stage their tap tiles: 1 (the default)
// with the tensor memory accelerator for tiles inside the image and
// per-pixel copies for tiles that wrap around the periodic edge, 0 with
// per-pixel copies only. Both stage the same bytes: results are bitwise equal.
px_status px_cnn_set_staging(px_cnn* n, int mode) {
  if (!n || mode < 0 || mode > 1) return PX_EINVAL;
  n->use_tma = mode;
  return PX_OK;
}

// Whether dilated layers run over relabelled activations (1, the default:
// each activation is stored in the positions that make its consumer's taps
// unit offsets, where the dilation is invertible modulo the image sides) or
// over natural-order activations with nine offset tap tiles (0).
px_status px_cnn_set_relabel(px_cnn* n, int on) {
  if (!n || on < 0 || on > 1) return PX_EINVAL;
  n->relabel = on;
  return PX_OK;
}

// Polls per handshake wait of the tensor-core kernels (0 restores the
// default). A wait that runs out makes its CTA stop, drain the MMAs it has
// issued, free its tensor memory and raise the fault word, which the next
// loss readback reports as PX_ETIMEOUT.
px_status px_cnn_set_wait_limit(px_cnn* n, uint32_t polls) {
  if (!n) return PX_EINVAL;
  n->wait_limit = polls == 0 ? kSpinLimit : polls;
  return PX_OK;
}

// Training state for checkpoints: FP32 parameters, Adam first and second
// moments (each px_cnn_param_count() floats, in that order) and the step.
px_status px_cnn_get_state(px_cnn* n, float* host, size_t count, int64_t* step) {
  if (!n || !host || !step || count != 3 * kOff.total) return PX_EINVAL;
  DevScope ds(n->ctx->device);
  const size_t P = kOff.total;
  cudaError_t e = cudaMemcpy(host, n->params, P * sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(host + P, n->m, P * sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(host + 2 * P, n->v, P * sizeof(float), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cnn_cuda(n, e, "get state");
  *step = n->step;
  return PX_OK;
}

px_status px_cnn_set_state(px_cnn* n, const float* host, size_t count, int64_t step) {
  if (!n || !host || count != 3 * kOff.total || step < 0) return PX_EINVAL;
  DevScope ds(n->ctx->device);
  const size_t P = kOff.total;
  cudaError_t e = cudaMemcpy(n->params, host, P * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(n->m, host + P, P * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(n->v, host + 2 * P, P * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cnn_cuda(n, e, "set state");
  n->step = step;
  px_status s = repack(n, 0);
  if (s != PX_OK) return s;
  e = cudaDeviceSynchronize();
  return e == cudaSuccess ? PX_OK : cnn_cuda(n, e, "set state");
}

px_status px_cnn_forward(px_cnn* n, const float* x, float* y, int B, int H, int W, void* stream) {
  PX_NVTX_RANGE("px_cnn_forward");
  if (!n || !x || !y) return PX_EINVAL;
  n->ctx->err.clear();
  px_status s = check_shape(n, B, H, W);
  if (s != PX_OK) return s;
  DevScope ds(n->ctx->device);
  s = ensure_work(n, (int64_t)B * H * W, B);
  if (s != PX_OK) return s;
  return forward(n, x, y, B, H, W, false, (cudaStream_t)stream);
}

px_status px_cnn_grads(px_cnn* n, const float* x, const float* t, int B, int H, int W,
                       float* grads_host, double* loss_host, void* stream) {
  PX_NVTX_RANGE("px_cnn_grads");
  if (!n || !x || !t) return PX_EINVAL;
  n->ctx->err.clear();
  px_status s = check_shape(n, B, H, W);
  if (s != PX_OK) return s;
  DevScope ds(n->ctx->device);
  s = ensure_work(n, (int64_t)B * H * W, B);
  if (s != PX_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  int nl = 0;
  s = grads(n, x, t, B, H, W, &nl, st);
  if (s != PX_OK) return s;
  if (loss_host) {
    s = read_loss(n, nl, (int64_t)B * H * W, loss_host, st);
    if (s != PX_OK) return s;
  }
  if (grads_host) {
    cudaError_t e = cudaMemcpyAsync(grads_host, n->grads, kOff.total * sizeof(float),
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cnn_cuda(n, e, "grads readback");
  }
  return PX_OK;
}

px_status px_cnn_train_step(px_cnn* n, const float* x, const float* t, int B, int H, int W,
                            float lr, double* loss_host, void* stream) {
  PX_NVTX_RANGE("px_cnn_train_step");
  if (!n || !x || !t || !(lr >= 0.0f)) return PX_EINVAL;
  n->ctx->err.clear();
  px_status s = check_shape(n, B, H, W);
  if (s != PX_OK) return s;
  DevScope ds(n->ctx->device);
  s = ensure_work(n, (int64_t)B * H * W, B);
  if (s != PX_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  int nl = 0;
  s = grads(n, x, t, B, H, W, &nl, st);
  if (s != PX_OK) return s;
  n->step++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - (float)std::pow(0.9, (double)n->step);
  const float c2 = 1.0f - (float)std::pow(0.999, (double)n->step);
  adam_update<<<64, 256, 0, st>>>(n->params, n->grads, n->m, n->v, (int)kOff.total, lr, b1, b2,
                                  1e-8f, c1, c2);
  s = repack(n, st);
  if (s != PX_OK) return s;
  if (loss_host) return read_loss(n, nl, (int64_t)B * H * W, loss_host, st);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PX_OK : cnn_cuda(n, e, "train step");
}

px_status px_cnn_prepare(px_cnn* n, const double* rho, const double* phi, float* x, float* t,
                         int B, int H, int W, double h, double* scales_host, void* stream) {
  PX_NVTX_RANGE("px_cnn_prepare");
  if (!n || !rho || !x || (phi && !t) || !(h > 0)) return PX_EINVAL;
  n->ctx->err.clear();
  DevScope ds(n->ctx->device);
  px_status s = ensure_work(n, (int64_t)B * H * W, B);
  if (s != PX_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  prepare_images<<<B, 512, 0, st>>>(rho, phi, x, phi ? t : nullptr, n->scales, H, W, h * h);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && scales_host) {
    e = cudaMemcpyAsync(scales_host, n->scales, B * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  return e == cudaSuccess ? PX_OK : cnn_cuda(n, e, "prepare images");
}

px_status px_cnn_guess(px_cnn* n, const double* rho, double* phi0, int B, int H, int W, double h,
                       void* stream) {
  PX_NVTX_RANGE("px_cnn_guess");
  if (!n || !rho || !phi0 || !(h > 0)) return PX_EINVAL;
  n->ctx->err.clear();
  px_status s = check_shape(n, B, H, W);
  if (s != PX_OK) return s;
  DevScope ds(n->ctx->device);
  s = ensure_work(n, (int64_t)B * H * W, B);
  if (s != PX_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  prepare_images<<<B, 512, 0, st>>>(rho, nullptr, n->xb, nullptr, n->scales, H, W, h * h);
  s = forward(n, n->xb, n->y, B, H, W, false, st);
  if (s != PX_OK) return s;
  finish_images<<<B, 1024, 0, st>>>(n->y, n->scales, phi0, H, W, h * h);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PX_OK : cnn_cuda(n, e, "guess");
}

}  // extern "C"

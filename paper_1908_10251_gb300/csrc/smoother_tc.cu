// Fused forward pass of the learned post-smoother on the 5th-generation tensor
// cores (tcgen05, sm_103a): one CTA computes N(r) on a 14 x 6 output tile of 8
// pairs, keeping every activation on chip; two CTAs share an SM.
//
//   layer 1 (1 -> 16, CUDA cores, float32): z1 on the 18 x 10 halo tile,
//            a1+ = relu(z1), a1- = relu(-z1) stored as bf16 in shared memory in
//            the canonical K-major layout of the tensor-core operand;
//   layer 2 (16 -> 16, tcgen05.mma kind::f16, bf16 x bf16 -> f32 in TMEM):
//            for each of the 8 rows of the 16 x 8 tile of h, both branches,
//            an implicit GEMM over the 9 taps: M = 128 rows = 16 pixels x 8
//            pairs, N = 16 output channels, K = 16 input channels per tap; the
//            tap shift is a shift of the operand's start address;
//   epilogue: tcgen05.ld of the accumulators, h = (relu(z2+) - relu(z2-)) / 2
//            (float32, shared memory, reusing the a1 space, as [row][col][channel
//            quad][pair][4] so that the 16-byte reads of layer 3 by consecutive
//            pairs hit consecutive banks);
//   layer 3 (16 -> 1, CUDA cores, float32): d on the 14 x 6 tile.
// One elected thread issues the MMAs and commits them to an mbarrier; the
// wait is bounded and reports through an error counter instead of hanging.
#include "common.cuh"
#include "smoother.cuh"

#include <cuda_bf16.h>
#include <stdint.h>

#include <cstring>

namespace pasm {
namespace {

// Output tile 14 x 6 pixels: 105 KB of shared memory and 256 TMEM columns, so two CTAs share an SM
// and one CTA's MMAs, loads and CUDA-core layers overlap the other's.
constexpr int TW = 14, TR = 6;           // output tile (pixels)
constexpr int HW = TW + 2, HR = TR + 2;  // h tile: 16 x 8 (one 128-row MMA block per row)
constexpr int AW = TW + 4, AR = TR + 4;  // a1 tile: 18 x 10
constexpr int RW = TW + 6, RR = TR + 6;  // r tile: 20 x 12
constexpr int PB = 8;                    // pairs per CTA
constexpr int kThreads = 512;            // 16 warps: four per TMEM lane quarter
constexpr int kCtasPerSm = 2;
constexpr int kWarpsPerQuarter = kThreads / 128;

constexpr int kPlane = AR * AW * PB * 16;          // bytes of one channel half of one branch
constexpr int kA1Bytes = 4 * kPlane;               // 2 branches x 2 halves
constexpr int kHBytes = HR * HW * PB * 16 * 4;     // float32 h (aliases the a1 space)
constexpr int kRBytes = RR * RW * PB * 4;
constexpr int kW2Bytes = 9 * 512;                  // bf16, canonical K-major, per tap 2x2 core matrices
constexpr int kSmem = kA1Bytes + kRBytes + kW2Bytes + 16;
static_assert(kHBytes <= kA1Bytes, "h must fit in the a1 space");
static_assert(HW * PB == 128, "one MMA block per h row");
constexpr uint32_t kTmemCols = HR * 2 * 16;        // h rows x 2 branches x 16 columns
static_assert(kTmemCols == 256 && kSmem * kCtasPerSm <= 227 * 1024, "two CTAs per SM");
constexpr int kWaitLimit = 1 << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, no swizzle, K-major canonical layout:
// element (row, k) at (row % 8) * 16 + (row / 8) * SBO + (k / 8) * LBO + (k % 8) * 2 bytes.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Layers 1 and 3 (CUDA cores) read their weights from the kernel's parameter
// space: every FMA takes its weight as a constant-bank operand, no load.
__global__ void __launch_bounds__(kThreads, kCtasPerSm) k_nn_tc(int nx, int ny, int ldk, int k, int tiles_x,
                                                       const NNOuterWeights w13, const uint8_t* __restrict__ w2g,
                                                       const float* __restrict__ R, float* __restrict__ D,
                                                       int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* a1 = smem;                                           // [branch][half][AR][AW][PB][8] bf16
  float* hs = reinterpret_cast<float*>(smem);                   // [HR][HW][4][PB][4] f32 (after the MMAs)
  float* rs = reinterpret_cast<float*>(smem + kA1Bytes);        // [RR][RW][PB]
  uint8_t* w2 = smem + kA1Bytes + kRBytes;                      // 9 x [2 n-groups][2 k-chunks][8][8] bf16
  uint64_t* mbar = reinterpret_cast<uint64_t*>(w2 + kW2Bytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
  const int x0 = tx * TW, y0 = ty * TR, c0 = blockIdx.y * PB;

  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // W2, already bf16 in the canonical layout (nn_tc_layer2_layout), by 16-byte asynchronous copies
  for (int t = tid; t < kW2Bytes / 16; t += kThreads)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(w2 + 16 * t)), "l"(w2g + 16 * t));
  // residual tile with a 3-pixel halo (zero outside the grid and for padded pairs).  A block of 8
  // real pairs is one 32-byte segment per pixel: two 16-byte asynchronous copies (cp.async, all in
  // flight at once), zero-filled outside the grid; a block with padded pairs loads element-wise.
  if (c0 + PB <= k) {
    for (int t = tid; t < RR * RW * 2; t += kThreads) {
      const int hlf = t & 1, col = (t >> 1) % RW, row = (t >> 1) / RW;
      const int x = x0 - 3 + col, y = y0 - 3 + row;
      const bool in = x >= 0 && x < nx && y >= 0 && y < ny;
      const float* src = in ? R + ((int64_t)y * nx + x) * ldk + c0 + 4 * hlf : R;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(rs + (row * RW + col) * PB + 4 * hlf)),
                   "l"(src), "r"(in ? 16 : 0));
    }
  } else {
    for (int t = tid; t < RR * RW * PB; t += kThreads) {
      const int q = t % PB, col = (t / PB) % RW, row = t / (PB * RW);
      const int x = x0 - 3 + col, y = y0 - 3 + row, c = c0 + q;
      float v = 0.f;
      if (x >= 0 && x < nx && y >= 0 && y < ny && c < k) v = R[((int64_t)y * nx + x) * ldk + c];
      rs[t] = v;
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  // layer 1 on the 18 x 10 tile: a1+- as bf16, zero outside the grid
  for (int t = tid; t < AR * AW * PB; t += kThreads) {
    const int q = t % PB, col = (t / PB) % AW, row = t / (PB * AW);
    const int x = x0 - 2 + col, y = y0 - 2 + row;
    float z[16];
#pragma unroll
    for (int o = 0; o < 16; ++o) z[o] = 0.f;
    if (x >= 0 && x < nx && y >= 0 && y < ny) {
#pragma unroll
      for (int tap = 0; tap < 9; ++tap) {
        const float v = rs[((row + tap / 3) * RW + (col + tap % 3)) * PB + q];
#pragma unroll
        for (int o = 0; o < 16; ++o) z[o] = fmaf(w13.w1[tap * 16 + o], v, z[o]);
      }
    }
    const int pix = (row * AW + col) * PB + q;  // 16-byte row index inside a plane
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      __align__(16) __nv_bfloat162 vp[4], vm[4];  // two channels per conversion
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        const float za = z[half * 8 + 2 * o], zb = z[half * 8 + 2 * o + 1];
        vp[o] = __floats2bfloat162_rn(fmaxf(za, 0.f), fmaxf(zb, 0.f));
        vm[o] = __floats2bfloat162_rn(fmaxf(-za, 0.f), fmaxf(-zb, 0.f));
      }
      *reinterpret_cast<uint4*>(a1 + (0 * 2 + half) * kPlane + pix * 16) = *reinterpret_cast<uint4*>(vp);
      *reinterpret_cast<uint4*>(a1 + (1 * 2 + half) * kPlane + pix * 16) = *reinterpret_cast<uint4*>(vm);
    }
  }
  // make the generic-proxy stores visible to the tensor cores
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;
  // layer 2: 16 h rows x 2 branches x 9 taps, issued by one thread
  if (tid == 0) {
    // kind::f16, D f32, A and B bf16, both K-major, N = 16, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(16 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    // The descriptors are formed once: the start-address field holds (address >> 4) in 14 bits, and
    // every operand here lies below 2^18 bytes, so shifting an operand by `off` bytes adds off >> 4.
    const uint64_t a0 = smem_desc(smem_u32(a1), kPlane, PB * 16);
    const uint64_t b0 = smem_desc(smem_u32(w2), 128, 256);
    for (int i = 0; i < HR; ++i)
      for (int b = 0; b < 2; ++b) {
        const uint32_t dcol = tmem + (uint32_t)((i * 2 + b) * 16);
        const uint64_t ai = a0 + (uint64_t)((b * 2 * kPlane + i * AW * PB * 16) >> 4);
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
          const int dy = tap / 3, dx = tap % 3;  // a1 row i + dy, col j + dx for h pixel (i, j)
          mma_bf16(dcol, ai + (uint64_t)(((dy * AW + dx) * PB * 16) >> 4), b0 + (uint64_t)(tap * 512 >> 4), idesc,
                   tap > 0 ? 1u : 0u);
        }
      }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar)));
  }
  uint32_t done = 0;
  for (int it = 0; it < kWaitLimit && !done; ++it) {
    asm volatile(
        "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], 0;\nselp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(mbar)));
  }
  if (!done && tid == 0) atomicAdd(err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (done) {
    // epilogue: TMEM lane m = 32 * (warp % 4) + lane = (h pixel j, pair q) with m = j * PB + q;
    // the warps of a lane quarter take every kWarpsPerQuarter-th h row
    const int quarter = warp & 3, rowgrp = warp >> 2;
    const int m = quarter * 32 + lane;
    const int j = m / PB, q = m % PB;
    for (int i = rowgrp; i < HR; i += kWarpsPerQuarter) {
      float vp[16], vm[16];
      const uint32_t lanebase = tmem + ((uint32_t)(quarter * 32) << 16);
      tmem_ld16(lanebase + (uint32_t)((i * 2 + 0) * 16), vp);
      tmem_ld16(lanebase + (uint32_t)((i * 2 + 1) * 16), vm);
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      const int x = x0 - 1 + j, y = y0 - 1 + i;
      const bool in = x >= 0 && x < nx && y >= 0 && y < ny;
      float* dst = hs + (i * HW + j) * 16 * PB + q * 4;
#pragma unroll
      for (int o = 0; o < 16; o += 4) {
        float4 h4;
        h4.x = in ? 0.5f * (fmaxf(vp[o], 0.f) - fmaxf(vm[o], 0.f)) : 0.f;
        h4.y = in ? 0.5f * (fmaxf(vp[o + 1], 0.f) - fmaxf(vm[o + 1], 0.f)) : 0.f;
        h4.z = in ? 0.5f * (fmaxf(vp[o + 2], 0.f) - fmaxf(vm[o + 2], 0.f)) : 0.f;
        h4.w = in ? 0.5f * (fmaxf(vp[o + 3], 0.f) - fmaxf(vm[o + 3], 0.f)) : 0.f;
        *reinterpret_cast<float4*>(dst + (o / 4) * PB * 4) = h4;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  if (!done) return;
  // layer 3 on the 14 x 6 tile
  for (int t = tid; t < TR * TW * PB; t += kThreads) {
    const int q = t % PB, col = (t / PB) % TW, row = t / (PB * TW);
    const int x = x0 + col, y = y0 + row, c = c0 + q;
    if (x >= nx || y >= ny) continue;
    float acc = 0.f;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const float4* hp =
          reinterpret_cast<const float4*>(hs + ((row + tap / 3) * HW + (col + tap % 3)) * 16 * PB + q * 4);
#pragma unroll
      for (int c4 = 0; c4 < 4; ++c4) {
        const float4 hv = hp[c4 * PB];
        acc = fmaf(w13.w3[tap * 16 + 4 * c4 + 0], hv.x, acc);
        acc = fmaf(w13.w3[tap * 16 + 4 * c4 + 1], hv.y, acc);
        acc = fmaf(w13.w3[tap * 16 + 4 * c4 + 2], hv.z, acc);
        acc = fmaf(w13.w3[tap * 16 + 4 * c4 + 3], hv.w, acc);
      }
    }
    D[((int64_t)y * nx + x) * ldk + c] = c < k ? acc : 0.f;
  }
}

}  // namespace

// Layer 2's weights W2[tap][ci][co] (2304 floats) as bf16 (round to nearest even) in the kernel's
// canonical K-major operand layout: row n = output channel, k = input channel, per tap two 8 x 8
// core matrices along n (256 B apart) and two along k (128 B apart).
void nn_tc_layer2_layout(const float* W2, uint16_t* out) {
  for (int t = 0; t < 2304; ++t) {
    const int tap = t / 256, ci = (t / 16) % 16, co = t % 16;
    const int off = tap * 512 + (co % 8) * 16 + (co / 8) * 256 + (ci / 8) * 128 + (ci % 8) * 2;
    uint32_t u;
    std::memcpy(&u, W2 + t, sizeof(u));
    uint16_t b;
    if ((u & 0x7F800000u) == 0x7F800000u && (u & 0x7FFFFFu)) b = (uint16_t)((u >> 16) | 0x40u);  // NaN
    else b = (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
    out[off / 2] = b;
  }
}

cudaError_t nn_tc_prepare() {
  return cudaFuncSetAttribute(k_nn_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
}

bool nn_tc_supported(int ldk) { return ldk % PB == 0; }

void nn_forward_tc(const Launch& L, const NNGrid& g, const NNOuterWeights& w13, const void* w2, const float* R,
                   float* D, int* err) {
  const int tiles_x = (g.nx + TW - 1) / TW, tiles_y = (g.ny + TR - 1) / TR;
  dim3 grid(tiles_x * tiles_y, g.ldk / PB);
  const double pix = (double)g.nx * g.ny * g.ldk;
  L.begin(KC_NN, pix * 8.0, pix * 2.0 * (2 * 9 * 16 + 2 * 9 * 256 + 9 * 16));
  k_nn_tc<<<grid, kThreads, kSmem, L.s>>>(g.nx, g.ny, g.ldk, g.k, tiles_x, w13, (const uint8_t*)w2, R, D, err);
  L.bump();
}

}  // namespace pasm

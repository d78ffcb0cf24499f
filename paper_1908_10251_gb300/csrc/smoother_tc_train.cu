// Training kernels of the learned post-smoother's 16 -> 16 layer on the
// 5th-generation tensor cores (tcgen05, sm_103a): bf16 operands, float32
// accumulation in TMEM, one elected thread issuing the MMAs.
//
//   k_tc_conv16  out = W (*) tf(in) for 16 input and 16 output channels
//                (3 x 3 taps, zero padding): the training forward of layer 2
//                (tf = relu or relu of the negation, giving z2+ and z2-) and
//                its input gradient (tf = identity, W = the flipped and
//                channel-transposed kernel, giving dL/da1+-).  Implicit GEMM as
//                in the fused inference kernel: per output row of a 16 x 8
//                tile, M = 128 rows (16 pixels x 8 pairs), N = 16, K = 16 per
//                tap, 9 taps accumulated in TMEM; the tap shift is a shift of
//                the A operand's start address.
//   k_tc_wgrad16 per-CTA partial weight gradient of layer 2 for both branches,
//                gW[tap][ci][co] = sum over (pixel, pair) of
//                a+-[pixel + tap][pair][ci] * g+-[pixel][pair][co]:
//                D[ci][co] += A[ci][k] B[co][k] with K = (pixel, pair) of the
//                tile, 8 pairs of one pixel per 16-byte K chunk, so that the
//                tap shift is again a start-address shift (one pixel = 256 B).
//                M = 128 with rows 0..15 the real ci; rows 16..127 read the
//                next pixels' data (in bounds, results unused).
//
// Activations and gradients are float32 [pixel][pair][16 channels] in global
// memory (the CUDA-core kernels' layout); they are rounded to bf16 (nearest
// even) when staged in shared memory.  Every mbarrier wait is bounded; a wait
// that gives up increments an error counter, the kernel skips what depends on
// it and frees its TMEM.
#include "common.cuh"
#include "smoother.cuh"

#include <cuda_bf16.h>
#include <stdint.h>

namespace pasm {
namespace {

constexpr int PB = 8;                    // pairs per CTA
constexpr int TW = 16, TR = 8;           // output tile of the convolution: 16 x 8 pixels
constexpr int IW = TW + 2, IR = TR + 2;  // input tile with its halo: 18 x 10
constexpr int kThreads = 256;
constexpr int kWaitLimit = 1 << 22;

// conv: A operand [half][IR][IW][PB][8 channels] bf16; weights 9 x 512 B
constexpr int kConvPlane = IR * IW * PB * 16;     // bytes of one channel half
constexpr int kConvHalf = kConvPlane + 64;        // distance of the two halves (bank offset)
constexpr int kConvA = kConvHalf + kConvPlane;
constexpr int kConvW = 9 * 512;
constexpr int kConvSmem = kConvA + kConvW + 16;
constexpr uint32_t kConvTmem = TR * 16;           // 128 columns

// wgrad: per pixel [c/8][c%8][PB] bf16 = 256 B; a on the 18 x 10 halo tile, g on the
// same indexing (only the 16 x 8 interior is used), each with 8 pixels of slack for the
// padding rows of the M = 128 operand (groups 2..15 of 8 rows at 128 B steps)
constexpr int kPix = IR * IW;
constexpr int kSlackPix = 8;
constexpr int kWgArr = (kPix + kSlackPix) * 256;
constexpr int kWgSmem = 2 * kWgArr + 16;
constexpr uint32_t kWgTmem = 256;                 // 9 taps x 16 columns, rounded up
constexpr int kWgradCtas = 2 * 152;               // persistent: two CTAs per SM

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// kind::f16, D f32, A and B bf16, both K-major, N = 16, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(16 >> 3) << 17) |
                            ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar)));
}

// bounded wait for the mbarrier phase `parity`; true when it completed
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity) {
  uint32_t done = 0;
  for (int it = 0; it < kWaitLimit && !done; ++it) {
    asm volatile(
        "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(parity));
  }
  return done != 0;
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

template <int MODE>
__device__ __forceinline__ float tf(float v) {
  if (MODE == 1) return fmaxf(v, 0.f);
  if (MODE == 2) return fmaxf(-v, 0.f);
  return v;
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(cols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

// out[p][c][co] = sum_{tap, ci} W[tap][ci][co] tf(in[p + tap][c][ci]); w2g = W in the canonical bf16
// operand layout (nn_tc_w2_layout); pairs c >= k and pixels outside the grid read as 0.
template <int MODE>
__global__ void __launch_bounds__(kThreads) k_tc_conv16(int nx, int ny, int ldk, int k, int tiles_x,
                                                        const uint8_t* __restrict__ w2g, const float* __restrict__ in,
                                                        float* __restrict__ out, int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* A = smem;
  uint8_t* W = smem + kConvA;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(W + kConvW);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
  const int x0 = tx * TW, y0 = ty * TR, c0 = blockIdx.y * PB;

  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
  if (warp == 0) tmem_alloc(tmem_slot, kConvTmem);
  for (int t = tid; t < kConvW / 16; t += kThreads)
    *reinterpret_cast<uint4*>(W + 16 * t) = __ldg(reinterpret_cast<const uint4*>(w2g) + t);
  // input tile: thread item = (pixel, pair, channel half): 8 floats (32 contiguous bytes; two
  // consecutive threads read the two halves of one (pixel, pair)) -> 8 bf16, one 16-byte row of
  // the half's plane.  The planes are kConvPlane + 64 bytes apart, so the two halves that one
  // group of 8 threads stores fall on different banks.
  for (int t = tid; t < IR * IW * PB * 2; t += kThreads) {
    const int half = t & 1, pp = t >> 1;
    const int q = pp % PB, pix = pp / PB;
    const int col = pix % IW, row = pix / IW;
    const int x = x0 - 1 + col, y = y0 - 1 + row, c = c0 + q;
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
    if (x >= 0 && x < nx && y >= 0 && y < ny && c < k) {
      const float4* src = reinterpret_cast<const float4*>(in + (((int64_t)y * nx + x) * ldk + c) * 16 + half * 8);
      a = __ldg(src);
      b = __ldg(src + 1);
    }
    __align__(16) __nv_bfloat162 v[4];
    v[0] = __floats2bfloat162_rn(tf<MODE>(a.x), tf<MODE>(a.y));
    v[1] = __floats2bfloat162_rn(tf<MODE>(a.z), tf<MODE>(a.w));
    v[2] = __floats2bfloat162_rn(tf<MODE>(b.x), tf<MODE>(b.y));
    v[3] = __floats2bfloat162_rn(tf<MODE>(b.z), tf<MODE>(b.w));
    *reinterpret_cast<uint4*>(A + half * kConvHalf + pp * 16) = *reinterpret_cast<uint4*>(v);
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;
  if (tid == 0) {
    const uint64_t a0 = smem_desc(smem_u32(A), kConvHalf, PB * 16);
    const uint64_t b0 = smem_desc(smem_u32(W), 128, 256);
    for (int i = 0; i < TR; ++i) {
      const uint64_t ai = a0 + (uint64_t)((i * IW * PB * 16) >> 4);
#pragma unroll
      for (int tap = 0; tap < 9; ++tap) {
        const int dy = tap / 3, dx = tap % 3;
        mma_bf16(tmem + (uint32_t)(i * 16), ai + (uint64_t)(((dy * IW + dx) * PB * 16) >> 4),
                 b0 + (uint64_t)(tap * 512 >> 4), tap > 0 ? 1u : 0u);
      }
    }
    mma_commit(mbar);
  }
  const bool done = mbar_wait(mbar, 0);
  if (!done && tid == 0) atomicAdd(err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (done) {
    // TMEM lane m = pixel j * 8 + pair q of an output row; warp w reads lane quarter w % 4,
    // rows i = w / 4, w / 4 + 2, ...
    const int quarter = warp & 3;
    const int m = quarter * 32 + lane;
    const int j = m / PB, q = m % PB;
    for (int i = warp >> 2; i < TR; i += kThreads / 128) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(i * 16), v);
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      const int x = x0 + j, y = y0 + i, c = c0 + q;
      if (x < nx && y < ny && c < ldk) {
        float4* dst = reinterpret_cast<float4*>(out + (((int64_t)y * nx + x) * ldk + c) * 16);
        const bool real = c < k;
#pragma unroll
        for (int o = 0; o < 4; ++o)
          dst[o] = real ? make_float4(v[4 * o], v[4 * o + 1], v[4 * o + 2], v[4 * o + 3])
                        : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kConvTmem));
}

// Stage one (pixel, channel) row of 8 pairs of a [pixel][pair][16] float32 tensor as 8 bf16
// values at dst (pixel-major, [c/8][c%8][pair]); MODE as tf; 0 outside the grid or past k.
template <int MODE>
__device__ __forceinline__ void stage_row(const float* __restrict__ src, int nx, int ny, int ldk, int k, int x,
                                          int y, int c0, int ch, uint8_t* dst) {
  float v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = 0.f;
  if (x >= 0 && x < nx && y >= 0 && y < ny) {
    const float* p = src + (((int64_t)y * nx + x) * ldk + c0) * 16 + ch;
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (c0 + q < k) v[q] = tf<MODE>(__ldg(p + q * 16));
  }
  __align__(16) __nv_bfloat162 b[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) b[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
  *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<uint4*>(b);
}

// Partial weight gradient of layer 2, both branches, by a persistent CTA that walks the
// (16 x 8 pixel, 8 pair) tiles blockIdx.x, blockIdx.x + gridDim.x, ... and accumulates in TMEM:
// partial[cta][tap][ci][co] = sum over its tiles of a+[p+tap][ci] gp[p][co] + a-[p+tap][ci] gm[p][co],
// a+- = bf16(relu(+-z1)), g+- = bf16(gp / gm).  The tile order per CTA is fixed, so the sums
// are deterministic for a given grid.
__global__ void __launch_bounds__(kThreads) k_tc_wgrad16(int nx, int ny, int ldk, int k, int tiles_x,
                                                         int tiles_xy, int n_tiles, const float* __restrict__ z1,
                                                         const float* __restrict__ gp, const float* __restrict__ gm,
                                                         float* __restrict__ partial, int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* Aa = smem;              // a on the halo tile
  uint8_t* Bg = smem + kWgArr;     // g on the same pixel indexing
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + 2 * kWgArr);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
  if (warp == 0) tmem_alloc(tmem_slot, kWgTmem);
  // the slack pixels past the tile are read only by the unused rows: zero them once
  for (int t = tid; t < kSlackPix * 256 / 16; t += kThreads) {
    reinterpret_cast<uint4*>(Aa + kPix * 256)[t] = make_uint4(0, 0, 0, 0);
    reinterpret_cast<uint4*>(Bg + kPix * 256)[t] = make_uint4(0, 0, 0, 0);
  }
  bool ok = true;
  uint32_t commits = 0;
  for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
    const int txy = tile % tiles_xy, cb = tile / tiles_xy;
    const int x0 = (txy % tiles_x) * TW, y0 = (txy / tiles_x) * TR, c0 = cb * PB;
    for (int br = 0; br < 2 && ok; ++br) {
      // stage a (halo tile) and g (interior) of this branch
      for (int t = tid; t < kPix * 16; t += kThreads) {
        const int ch = t & 15, pix = t >> 4;
        const int col = pix % IW, row = pix / IW;
        const int x = x0 - 1 + col, y = y0 - 1 + row;
        uint8_t* da = Aa + pix * 256 + (ch >> 3) * 128 + (ch & 7) * 16;
        if (br == 0) stage_row<1>(z1, nx, ny, ldk, k, x, y, c0, ch, da);
        else stage_row<2>(z1, nx, ny, ldk, k, x, y, c0, ch, da);
        uint8_t* dg = Bg + pix * 256 + (ch >> 3) * 128 + (ch & 7) * 16;
        const bool interior = col >= 1 && col <= TW && row >= 1 && row <= TR;
        if (interior) stage_row<0>(br == 0 ? gp : gm, nx, ny, ldk, k, x, y, c0, ch, dg);
        else *reinterpret_cast<uint4*>(dg) = make_uint4(0, 0, 0, 0);
      }
      asm volatile("fence.proxy.async.shared::cta;");
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (tid == 0) {
        const uint32_t tmem = *tmem_slot;
        // K chunk = one pixel's 8 pairs (16 B per row); an MMA (K = 16) takes two adjacent pixels
        const uint64_t a0 = smem_desc(smem_u32(Aa), 256, 128);
        const uint64_t g0 = smem_desc(smem_u32(Bg), 256, 128);
        for (int i = 0; i < TR; ++i)
          for (int jj = 0; jj < TW; jj += 2) {
            const int P = (i + 1) * IW + (jj + 1);   // g pixel of this K step
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) {
              const int dy = tap / 3 - 1, dx = tap % 3 - 1;
              const int Pa = P + dy * IW + dx;
              mma_bf16(tmem + (uint32_t)(tap * 16), a0 + (uint64_t)((Pa * 256) >> 4),
                       g0 + (uint64_t)((P * 256) >> 4), (commits > 0 || i > 0 || jj > 0) ? 1u : 0u);
            }
          }
        mma_commit(mbar);
      }
      ok = mbar_wait(mbar, commits & 1u);
      ++commits;
      if (!ok && tid == 0) atomicAdd(err, 1);
      asm volatile("tcgen05.fence::after_thread_sync;");
      __syncthreads();   // the next staging overwrites the operands
    }
  }
  const uint32_t tmem = *tmem_slot;
  if (warp == 0) {
    // rows 0..15 of the accumulators (TMEM lanes 0..15) hold gW[tap][ci = lane][co]; a CTA
    // without tiles or with a failed wait contributes zeros
    const bool have = ok && commits > 0;
#pragma unroll 1
    for (int tap = 0; tap < 9; ++tap) {
      float v[16];
      if (have) {
        tmem_ld16(tmem + (uint32_t)(tap * 16), v);
        asm volatile("tcgen05.wait::ld.sync.aligned;");
      } else {
#pragma unroll
        for (int o = 0; o < 16; ++o) v[o] = 0.f;
      }
      if (lane < 16) {
        float4* dst = reinterpret_cast<float4*>(partial + (size_t)blockIdx.x * 2304 + (tap * 16 + lane) * 16);
#pragma unroll
        for (int o = 0; o < 4; ++o) dst[o] = make_float4(v[4 * o], v[4 * o + 1], v[4 * o + 2], v[4 * o + 3]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kWgTmem));
}

// Layer 2's kernel W[tap][ci][co] (float32, device) in the canonical bf16 operand layout of the
// B matrix (row n = output channel, k = input channel, per tap two 8 x 8 core matrices along n,
// 256 B apart, and two along k, 128 B apart); flip: the kernel of the input gradient,
// Wt[tap][co][ci] = W[8 - tap][ci][co] (output and input channels exchanged).
__global__ void k_tc_w2_layout(const float* __restrict__ W, int flip, uint16_t* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2304) return;
  const int tap = t / 256, ci = (t / 16) % 16, co = t % 16;   // W index t = [tap][ci][co]
  int otap = tap, n = co, kk = ci;
  if (flip) { otap = 8 - tap; n = ci; kk = co; }
  const int off = otap * 512 + (n % 8) * 16 + (n / 8) * 256 + (kk / 8) * 128 + (kk % 8) * 2;
  const __nv_bfloat16 b = __float2bfloat16_rn(W[t]);
  out[off / 2] = *reinterpret_cast<const uint16_t*>(&b);
}

}  // namespace

cudaError_t nn_tc_train_prepare() {
  cudaError_t e = cudaFuncSetAttribute(k_tc_conv16<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kConvSmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tc_conv16<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kConvSmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tc_conv16<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kConvSmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tc_wgrad16, cudaFuncAttributeMaxDynamicSharedMemorySize, kWgSmem);
  return e;
}

int nn_tc_wgrad_ctas(const NNGrid& g) {
  const int n_tiles = ((g.nx + TW - 1) / TW) * ((g.ny + TR - 1) / TR) * (g.ldk / PB);
  return n_tiles < kWgradCtas ? n_tiles : kWgradCtas;
}

void nn_tc_w2_layout(const Launch& L, const float* W2, bool flip, uint16_t* out) {
  L.begin(KC_NN, 2304 * 6.0, 0);
  k_tc_w2_layout<<<(2304 + 255) / 256, 256, 0, L.s>>>(W2, flip ? 1 : 0, out);
  L.bump();
}

void nn_tc_conv16(const Launch& L, const NNGrid& g, int mode, const uint16_t* w2, const float* in, float* out,
                  int* err) {
  const int tiles_x = (g.nx + TW - 1) / TW, tiles_y = (g.ny + TR - 1) / TR;
  dim3 grid(tiles_x * tiles_y, g.ldk / PB);
  const double pp = (double)g.nx * g.ny * g.ldk;
  L.begin(KC_NN, pp * 16 * 4.0 * 2, pp * 2.0 * 9 * 256);
  const uint8_t* w = reinterpret_cast<const uint8_t*>(w2);
  if (mode == 1) k_tc_conv16<1><<<grid, kThreads, kConvSmem, L.s>>>(g.nx, g.ny, g.ldk, g.k, tiles_x, w, in, out, err);
  else if (mode == 2) k_tc_conv16<2><<<grid, kThreads, kConvSmem, L.s>>>(g.nx, g.ny, g.ldk, g.k, tiles_x, w, in, out, err);
  else k_tc_conv16<0><<<grid, kThreads, kConvSmem, L.s>>>(g.nx, g.ny, g.ldk, g.k, tiles_x, w, in, out, err);
  L.bump();
}

void nn_tc_wgrad16(const Launch& L, const NNGrid& g, const float* z1, const float* gp, const float* gm,
                   float* partial, int* err) {
  const int tiles_x = (g.nx + TW - 1) / TW, tiles_y = (g.ny + TR - 1) / TR;
  const int n_tiles = tiles_x * tiles_y * (g.ldk / PB);
  const double pp = (double)g.nx * g.ny * g.ldk;
  L.begin(KC_NN, pp * 16 * 4.0 * 3, pp * 2.0 * 2 * 9 * 256);
  k_tc_wgrad16<<<nn_tc_wgrad_ctas(g), kThreads, kWgSmem, L.s>>>(g.nx, g.ny, g.ldk, g.k, tiles_x, tiles_x * tiles_y,
                                                                 n_tiles, z1, gp, gm, partial, err);
  L.bump();
}

}  // namespace pasm

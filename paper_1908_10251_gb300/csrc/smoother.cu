// Learned multigrid post-smoother: forward, backward and Adam kernels (float32).
//
// The network (not in the paper; the workload specification asks for it):
// three bias-free 3x3 convolutions 1 -> 16 -> 16 -> 1 with ReLU after the
// first two, made odd: N(r) = (Nt(r) - Nt(-r)) / 2, so N(s r) = s N(r) for all
// real s.  The two branches share the first convolution z1 = W1 * r:
//   a1+ = relu(z1), a1- = relu(-z1), z2+- = W2 * a1+-,
//   h = (relu(z2+) - relu(z2-)) / 2,   N(r) = W3 * h  (W3 is linear).
// Images are the interior nodes of an nx x ny grid (x fastest), one image per
// pair; activations are stored [pixel][pair][channel] so that a warp reads
// consecutive pairs of one pixel (coalesced 64-byte channel vectors).
// Weight layout: W1[3][3][1][16] | W2[3][3][16][16] | W3[3][3][16][1],
// index [dy+1][dx+1][cin][cout] multiplying input pixel (y+dy, x+dx).
#include "common.cuh"
#include "smoother.cuh"

#include <algorithm>

namespace pasm {

static constexpr int kNNBlock = 128;

enum InMode { IN_ID = 0, IN_RELU = 1, IN_NEGRELU = 2 };

template <int MODE>
__device__ __forceinline__ float in_tf(float v) {
  if (MODE == IN_RELU) return fmaxf(v, 0.f);
  if (MODE == IN_NEGRELU) return fmaxf(-v, 0.f);
  return v;
}

// out[p][c][o] = sum_{dy,dx,i} W[dy][dx][i][o] * tf(in[p+(dy,dx)][c][i]), zero outside.
template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(kNNBlock) k_conv(int nx, int ny, int ldk, int kact, const float* __restrict__ W,
                                                   const float* __restrict__ in, float* __restrict__ out) {
  __shared__ float w[9 * CIN * COUT];
  for (int t = threadIdx.x; t < 9 * CIN * COUT; t += blockDim.x) w[t] = W[t];
  __syncthreads();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)nx * ny * ldk;
  if (idx >= total) return;
  const int c = (int)(idx % ldk);
  const int64_t p = idx / ldk;
  const int x = (int)(p % nx), y = (int)(p / nx);
  float acc[COUT];
#pragma unroll
  for (int o = 0; o < COUT; ++o) acc[o] = 0.f;
  if (c < kact) {
    for (int dy = -1; dy <= 1; ++dy) {
      const int yy = y + dy;
      if (yy < 0 || yy >= ny) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        const int xx = x + dx;
        if (xx < 0 || xx >= nx) continue;
        const float* src = in + (((int64_t)yy * nx + xx) * ldk + c) * CIN;
        const float* wk = w + ((dy + 1) * 3 + (dx + 1)) * CIN * COUT;
#pragma unroll
        for (int i = 0; i < CIN; ++i) {
          const float v = in_tf<MODE>(src[i]);
#pragma unroll
          for (int o = 0; o < COUT; ++o) acc[o] = fmaf(wk[i * COUT + o], v, acc[o]);
        }
      }
    }
  }
  float* dst = out + idx * COUT;
#pragma unroll
  for (int o = 0; o < COUT; ++o) dst[o] = acc[o];
}

// h = (relu(z2p) - relu(z2m)) / 2
__global__ void k_combine(int64_t count, const float* __restrict__ zp, const float* __restrict__ zm,
                          float* __restrict__ h) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    h[i] = 0.5f * (fmaxf(zp[i], 0.f) - fmaxf(zm[i], 0.f));
}

// Backward through the combination: gzp = gh/2 [zp>0], gzm = -gh/2 [zm>0].
__global__ void k_combine_back(int64_t count, const float* __restrict__ gh, const float* __restrict__ zp,
                               const float* __restrict__ zm, float* __restrict__ gzp, float* __restrict__ gzm) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    gzp[i] = zp[i] > 0.f ? 0.5f * gh[i] : 0.f;
    gzm[i] = zm[i] > 0.f ? -0.5f * gh[i] : 0.f;
  }
}

// gz1 = ga+ [z1>0] - ga- [z1<0]
__global__ void k_first_back(int64_t count, const float* __restrict__ gap, const float* __restrict__ gam,
                             const float* __restrict__ z1, float* __restrict__ gz1) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const float z = z1[i];
    gz1[i] = (z > 0.f ? gap[i] : 0.f) - (z < 0.f ? gam[i] : 0.f);
  }
}

// Flipped and channel-transposed kernel: Wt[dy][dx][o][i] = W[2-dy][2-dx][i][o]
// (the input gradient of a convolution is the convolution of the output
// gradient with this kernel).
__global__ void k_flip(int cin, int cout, const float* __restrict__ W, float* __restrict__ Wt) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 9 * cin * cout) return;
  const int o = t % cout, i = (t / cout) % cin, k = t / (cin * cout);
  const int dy = k / 3, dx = k % 3;
  Wt[(((2 - dy) * 3 + (2 - dx)) * cout + o) * cin + i] = W[t];
}

// Weight gradient partials: gW[dy][dx][i][o] = sum_{p,c} tf(x[p+d][c][i]) g[p][c][o].
// Block b sums over its slice of (p, c); thread t owns (dy, dx, i) = t and all o.
template <int CIN, int COUT, int MODE>
__global__ void k_wgrad(int nx, int ny, int ldk, int kact, const float* __restrict__ x, const float* __restrict__ g,
                        float* __restrict__ partial, int64_t per_block) {
  const int t = threadIdx.x;  // 9 * CIN threads
  const int kk = t / CIN, i = t % CIN;
  const int dy = kk / 3 - 1, dx = kk % 3 - 1;
  float acc[COUT];
#pragma unroll
  for (int o = 0; o < COUT; ++o) acc[o] = 0.f;
  const int64_t total = (int64_t)nx * ny * ldk;
  const int64_t b0 = blockIdx.x * per_block, b1 = min(total, b0 + per_block);
  for (int64_t idx = b0; idx < b1; ++idx) {
    const int c = (int)(idx % ldk);
    if (c >= kact) continue;
    const int64_t p = idx / ldk;
    const int xx = (int)(p % nx) + dx, yy = (int)(p / nx) + dy;
    if (xx < 0 || xx >= nx || yy < 0 || yy >= ny) continue;
    const float v = in_tf<MODE>(x[(((int64_t)yy * nx + xx) * ldk + c) * CIN + i]);
    const float* gp = g + idx * COUT;
#pragma unroll
    for (int o = 0; o < COUT; ++o) acc[o] = fmaf(v, gp[o], acc[o]);
  }
  float* dst = partial + (size_t)blockIdx.x * 9 * CIN * COUT + (size_t)t * COUT;
#pragma unroll
  for (int o = 0; o < COUT; ++o) dst[o] = acc[o];
}

// out[w] (+)= sum_b partial[b][w]  (fixed order)
__global__ void k_wsum(int nw, int nblk, const float* __restrict__ partial, float* __restrict__ out, int accumulate) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nw) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partial[(size_t)b * nw + t];
  out[t] = accumulate ? out[t] + (float)s : (float)s;
}

// Column sums of squares of two n x ldk blocks (float64 accumulation) into
// partial[blk][2][ldk].
__global__ void k_colnorms2(int n, int ldk, const float* __restrict__ a, const float* __restrict__ b,
                            double* __restrict__ partial, int rows_per_block) {
  const int c = threadIdx.x % ldk;
  const int r0 = threadIdx.x / ldk, rstep = blockDim.x / ldk;
  double sa = 0.0, sb = 0.0;
  const int row_beg = blockIdx.x * rows_per_block, row_end = min(n, row_beg + rows_per_block);
  for (int r = row_beg + r0; r < row_end; r += rstep) {
    const float va = a[(size_t)r * ldk + c], vb = b[(size_t)r * ldk + c];
    sa += (double)va * va;
    sb += (double)vb * vb;
  }
  __shared__ double red[2][512];
  red[0][threadIdx.x] = sa;
  red[1][threadIdx.x] = sb;
  __syncthreads();
  if (threadIdx.x < ldk) {
    double ta = 0.0, tb = 0.0;
    for (int q = 0; q < rstep; ++q) { ta += red[0][q * ldk + c]; tb += red[1][q * ldk + c]; }
    partial[((size_t)blockIdx.x * 2 + 0) * ldk + c] = ta;
    partial[((size_t)blockIdx.x * 2 + 1) * ldk + c] = tb;
  }
}

__global__ void k_colsum_d(const double* __restrict__ partial, int nblk, int width, double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= width) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partial[(size_t)b * width + t];
  out[t] = s;
}

// Loss gradient seed: Es[p][c] = -2 E[p][c] / (k |r_c|^2)  (0 for padded pairs)
__global__ void k_loss_seed(int64_t total, int ldk, int k, const float* __restrict__ E,
                            const double* __restrict__ norms, float* __restrict__ Es) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % ldk);
    Es[i] = c < k ? (float)(-2.0 * E[i] / ((double)k * norms[c])) : 0.f;
  }
}

// L = mean_c |E_c|^2 / |R_c|^2
__global__ void k_loss_value(int k, int ldk, const double* __restrict__ norms, double* __restrict__ loss) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int c = 0; c < k; ++c) s += norms[ldk + c] / norms[c];
  *loss = s / k;
}

// Adam (Kingma & Ba 2015), t from 1.
__global__ void k_adam(int nw, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nw) return;
  const float gi = g[t];
  const float mi = b1 * m[t] + (1.f - b1) * gi;
  const float vi = b2 * v[t] + (1.f - b2) * gi * gi;
  m[t] = mi;
  v[t] = vi;
  w[t] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Post-smoothing with the learned step and a per-pair fallback:
//   pairs whose residual norm did not grow take e + d, the others a Jacobi step.
__global__ void k_nn_select(int64_t total, int ldk, const float* __restrict__ E, const float* __restrict__ D,
                            const float* __restrict__ R, const float* __restrict__ dinv, float omega,
                            const double* __restrict__ norms, float* __restrict__ out, int* __restrict__ accepted) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % ldk);
    const bool ok = norms[ldk + c] <= norms[c];
    const int64_t row = i / ldk;
    out[i] = ok ? E[i] + D[i] : fmaf(omega * dinv[row], R[i], E[i]);
    if (row == 0 && accepted) accepted[c] += ok ? 1 : 0;
  }
}

__global__ void k_add(int64_t total, const float* __restrict__ a, const float* __restrict__ b, float* __restrict__ o) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    o[i] = a[i] + b[i];
}

static int grid_for(int64_t total, int block = kNNBlock) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((total + block - 1) / block, 1 << 30));
}
static int grid_stride(int64_t total) { return (int)std::min<int64_t>((total + 255) / 256, 152 * 16); }

// ------------------------------------------------------------------------------------------------
void nn_forward(const Launch& L, const NNGrid& g, const NNBuf& b, const float* W, const float* R, float* Dout) {
  const int64_t pix = (int64_t)g.nx * g.ny * g.ldk;
  L.begin(KC_NN, (double)pix * 4.0 * 2, (double)pix * 2.0 * 9 * 16);
  k_conv<1, 16, IN_ID><<<grid_for(pix), kNNBlock, 0, L.s>>>(g.nx, g.ny, g.ldk, g.k, W, R, b.z1);
  L.bump();
  L.begin(KC_NN, (double)pix * 4.0 * 32, (double)pix * 2.0 * 9 * 256);
  k_conv<16, 16, IN_RELU><<<grid_for(pix), kNNBlock, 0, L.s>>>(g.nx, g.ny, g.ldk, g.k, W + 144, b.z1, b.z2p);
  L.bump();
  L.begin(KC_NN, (double)pix * 4.0 * 32, (double)pix * 2.0 * 9 * 256);
  k_conv<16, 16, IN_NEGRELU><<<grid_for(pix), kNNBlock, 0, L.s>>>(g.nx, g.ny, g.ldk, g.k, W + 144, b.z1, b.z2m);
  L.bump();
  L.begin(KC_NN, (double)pix * 16 * 4.0 * 3, (double)pix * 16 * 3);
  k_combine<<<grid_stride(pix * 16), 256, 0, L.s>>>(pix * 16, b.z2p, b.z2m, b.h);
  L.bump();
  L.begin(KC_NN, (double)pix * 4.0 * 17, (double)pix * 2.0 * 9 * 16);
  k_conv<16, 1, IN_ID><<<grid_for(pix), kNNBlock, 0, L.s>>>(g.nx, g.ny, g.ldk, g.k, W + 144 + 2304, b.h, Dout);
  L.bump();
}

// weight gradient of one convolution into gw (accumulate or overwrite)
template <int CIN, int COUT, int MODE>
static void wgrad(const Launch& L, const NNGrid& g, const NNBuf& b, const float* x, const float* gout, float* gw,
                  bool accumulate) {
  const int64_t total = (int64_t)g.nx * g.ny * g.ldk;
  const int nblk = (int)std::min<int64_t>(NNBuf::kWgradBlocks, std::max<int64_t>(1, (total + 255) / 256));
  const int64_t per = (total + nblk - 1) / nblk;
  L.begin(KC_NN, (double)total * 4.0 * (9 * CIN + COUT), (double)total * 2.0 * 9 * CIN * COUT);
  k_wgrad<CIN, COUT, MODE><<<nblk, 9 * CIN, 0, L.s>>>(g.nx, g.ny, g.ldk, g.k, x, gout, b.wpart, per);
  L.bump();
  const int nw = 9 * CIN * COUT;
  L.begin(KC_NN, (double)nblk * nw * 4.0, (double)nblk * nw);
  k_wsum<<<(nw + 127) / 128, 128, 0, L.s>>>(nw, nblk, b.wpart, gw, accumulate ? 1 : 0);
  L.bump();
}

void nn_backward(const Launch& L, const NNGrid& g, const NNBuf& b, const float* W, const float* R, const float* gD,
                 float* gW) {
  const int64_t pix = (int64_t)g.nx * g.ny * g.ldk;
  // flipped kernels for the input gradients
  L.begin(KC_NN, 0, 0);
  k_flip<<<(2304 + 127) / 128, 128, 0, L.s>>>(16, 16, W + 144, b.wflip2);
  L.bump();
  L.begin(KC_NN, 0, 0);
  k_flip<<<(144 + 127) / 128, 128, 0, L.s>>>(16, 1, W + 144 + 2304, b.wflip3);
  L.bump();
  // layer 3: N = W3 * h
  wgrad<16, 1, IN_ID>(L, g, b, b.h, gD, gW + 144 + 2304, false);
  L.begin(KC_NN, 0, (double)pix * 2.0 * 9 * 16);
  k_conv<1, 16, IN_ID><<<grid_for(pix), kNNBlock, 0, L.s>>>(g.nx, g.ny, g.ldk, g.k, b.wflip3, gD, b.gh);
  L.bump();
  // combination
  L.begin(KC_NN, 0, 0);
  k_combine_back<<<grid_stride(pix * 16), 256, 0, L.s>>>(pix * 16, b.gh, b.z2p, b.z2m, b.gzp, b.gzm);
  L.bump();
  // layer 2 (both branches share W2)
  wgrad<16, 16, IN_RELU>(L, g, b, b.z1, b.gzp, gW + 144, false);
  wgrad<16, 16, IN_NEGRELU>(L, g, b, b.z1, b.gzm, gW + 144, true);
  L.begin(KC_NN, 0, (double)pix * 2.0 * 9 * 256);
  k_conv<16, 16, IN_ID><<<grid_for(pix), kNNBlock, 0, L.s>>>(g.nx, g.ny, g.ldk, g.k, b.wflip2, b.gzp, b.gap);
  L.bump();
  L.begin(KC_NN, 0, (double)pix * 2.0 * 9 * 256);
  k_conv<16, 16, IN_ID><<<grid_for(pix), kNNBlock, 0, L.s>>>(g.nx, g.ny, g.ldk, g.k, b.wflip2, b.gzm, b.gam);
  L.bump();
  // layer 1
  L.begin(KC_NN, 0, 0);
  k_first_back<<<grid_stride(pix * 16), 256, 0, L.s>>>(pix * 16, b.gap, b.gam, b.z1, b.gz1);
  L.bump();
  wgrad<1, 16, IN_ID>(L, g, b, R, b.gz1, gW, false);
}

void nn_forward_train_tc(const Launch& L, const NNGrid& g, const NNBuf& b, const float* W, uint16_t* w2f,
                         const float* R, float* Dout, int* err) {
  const int64_t pix = (int64_t)g.nx * g.ny * g.ldk;
  nn_tc_w2_layout(L, W + 144, false, w2f);
  L.begin(KC_NN, (double)pix * 4.0 * 2, (double)pix * 2.0 * 9 * 16);
  k_conv<1, 16, IN_ID><<<grid_for(pix), kNNBlock, 0, L.s>>>(g.nx, g.ny, g.ldk, g.k, W, R, b.z1);
  L.bump();
  nn_tc_conv16(L, g, 1, w2f, b.z1, b.z2p, err);
  nn_tc_conv16(L, g, 2, w2f, b.z1, b.z2m, err);
  L.begin(KC_NN, (double)pix * 16 * 4.0 * 3, (double)pix * 16 * 3);
  k_combine<<<grid_stride(pix * 16), 256, 0, L.s>>>(pix * 16, b.z2p, b.z2m, b.h);
  L.bump();
  L.begin(KC_NN, (double)pix * 4.0 * 17, (double)pix * 2.0 * 9 * 16);
  k_conv<16, 1, IN_ID><<<grid_for(pix), kNNBlock, 0, L.s>>>(g.nx, g.ny, g.ldk, g.k, W + 144 + 2304, b.h, Dout);
  L.bump();
}

void nn_backward_tc(const Launch& L, const NNGrid& g, const NNBuf& b, const float* W, uint16_t* w2t, const float* R,
                    const float* gD, float* gW, int* err) {
  const int64_t pix = (int64_t)g.nx * g.ny * g.ldk;
  nn_tc_w2_layout(L, W + 144, true, w2t);
  L.begin(KC_NN, 0, 0);
  k_flip<<<(144 + 127) / 128, 128, 0, L.s>>>(16, 1, W + 144 + 2304, b.wflip3);
  L.bump();
  // layer 3 (CUDA cores, float32)
  wgrad<16, 1, IN_ID>(L, g, b, b.h, gD, gW + 144 + 2304, false);
  L.begin(KC_NN, 0, (double)pix * 2.0 * 9 * 16);
  k_conv<1, 16, IN_ID><<<grid_for(pix), kNNBlock, 0, L.s>>>(g.nx, g.ny, g.ldk, g.k, b.wflip3, gD, b.gh);
  L.bump();
  L.begin(KC_NN, 0, 0);
  k_combine_back<<<grid_stride(pix * 16), 256, 0, L.s>>>(pix * 16, b.gh, b.z2p, b.z2m, b.gzp, b.gzm);
  L.bump();
  // layer 2 on the tensor cores: weight gradient of both branches, then the input gradients
  const int nblk = nn_tc_wgrad_ctas(g);
  nn_tc_wgrad16(L, g, b.z1, b.gzp, b.gzm, b.wpart, err);
  L.begin(KC_NN, (double)nblk * 2304 * 4.0, (double)nblk * 2304);
  k_wsum<<<(2304 + 127) / 128, 128, 0, L.s>>>(2304, nblk, b.wpart, gW + 144, 0);
  L.bump();
  nn_tc_conv16(L, g, 0, w2t, b.gzp, b.gap, err);
  nn_tc_conv16(L, g, 0, w2t, b.gzm, b.gam, err);
  // layer 1 (CUDA cores, float32)
  L.begin(KC_NN, 0, 0);
  k_first_back<<<grid_stride(pix * 16), 256, 0, L.s>>>(pix * 16, b.gap, b.gam, b.z1, b.gz1);
  L.bump();
  wgrad<1, 16, IN_ID>(L, g, b, R, b.gz1, gW, false);
}

void nn_column_norms(const Launch& L, int n, int ldk, const float* a, const float* bb, double* partial,
                     double* norms) {
  const int rpb = 64;
  const int nblk = (n + rpb - 1) / rpb;
  const int threads = std::min(512, std::max(ldk, (512 / ldk) * ldk));
  L.begin(KC_NN, (double)n * ldk * 8.0, (double)n * ldk * 4.0);
  k_colnorms2<<<nblk, threads, 0, L.s>>>(n, ldk, a, bb, partial, rpb);
  L.bump();
  L.begin(KC_NN, 0, 0);
  k_colsum_d<<<(2 * ldk + 127) / 128, 128, 0, L.s>>>(partial, nblk, 2 * ldk, norms);
  L.bump();
}

void nn_loss_seed(const Launch& L, int64_t total, int ldk, int k, const float* E, const double* norms, float* Es,
                  double* loss) {
  L.begin(KC_NN, (double)total * 8.0, (double)total);
  k_loss_seed<<<grid_stride(total), 256, 0, L.s>>>(total, ldk, k, E, norms, Es);
  L.bump();
  L.begin(KC_NN, 0, 0);
  k_loss_value<<<1, 32, 0, L.s>>>(k, ldk, norms, loss);
  L.bump();
}

void nn_adam(const Launch& L, int nw, float* w, const float* g, float* m, float* v, float lr, int t) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  L.begin(KC_NN, nw * 20.0, nw * 10.0);
  k_adam<<<(nw + 127) / 128, 128, 0, L.s>>>(nw, w, g, m, v, lr, b1, b2, 1e-8f, c1, c2);
  L.bump();
}

void nn_add(const Launch& L, int64_t total, const float* a, const float* b, float* o) {
  L.begin(KC_NN, total * 12.0, (double)total);
  k_add<<<grid_stride(total), 256, 0, L.s>>>(total, a, b, o);
  L.bump();
}

void nn_select(const Launch& L, int n, int ldk, const float* E, const float* D, const float* R, const float* dinv,
               float omega, const double* norms, float* out, int* accepted) {
  const int64_t total = (int64_t)n * ldk;
  L.begin(KC_NN, total * 16.0, total * 2.0);
  k_nn_select<<<grid_stride(total), 256, 0, L.s>>>(total, ldk, E, D, R, dinv, omega, norms, out, accepted);
  L.bump();
}

}  // namespace pasm

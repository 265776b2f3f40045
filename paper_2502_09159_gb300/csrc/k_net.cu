// Kernels of the learned initial guess: 3x3 convolutions on NHWC FP32 tensors (forward,
// input gradient, weight and bias gradients), mean squared error, Adam, per-channel
// statistics.
//
// The convolution is an implicit GEMM: out[p][o] = sum_kk A[p][kk] W[o][kk] with
// p = (b, y, x) a pixel, kk = (ky, kx, c) and A the zero-padded im2col of the input,
// gathered into shared memory tile by tile (never materialised).  The weight gradient is
// the transposed product dW[o][kk] = sum_p G[p][o] A[p][kk], split over pixel ranges whose
// partial tiles are then summed in a fixed order, so training is deterministic.
#include <cuda_runtime.h>

#include "net_internal.h"

namespace stmg {

namespace {
constexpr int CT = 256;   // threads of the GEMM-like kernels
constexpr int BM = 128;   // pixels per forward tile
constexpr int BK = 16;    // reduction slice
constexpr int WT = 64;    // weight-gradient tile (o and kk)
}

// ---------------------------------------------------------------------------------
// forward convolution (also the input gradient, with transposed flipped weights)
// ---------------------------------------------------------------------------------
// Thread (tx, ty) of the 16 x 16 grid computes pixels m0 + 8 ty + i (i < 8) and output
// channels n0 + tx + 16 j (j < TN).  Tiles are double-buffered: the next slice is loaded
// into registers while the current one is multiplied from shared memory.
template <int TN>
__global__ void __launch_bounds__(CT) k_conv3x3(const float* __restrict__ in, const int* __restrict__ index,
                                                const float* __restrict__ Wm, const float* __restrict__ bias,
                                                const float* __restrict__ mask, float* __restrict__ out, int B,
                                                int H, int W, int Cin, int Cout, int relu, int accumulate) {
  constexpr int BN = 16 * TN;
  __shared__ __align__(16) float As[2][BK][BM + 4];
  __shared__ float Bs[2][BK][BN + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const long long HW = (long long)H * W;
  const long long M = (long long)B * HW;
  const int K = 9 * Cin;
  const long long m0 = (long long)blockIdx.x * BM;
  const int n0 = blockIdx.y * BN;

  // this thread loads im2col column ak of pixels (tid >> 4) + 16 q
  const int ak = tid & 15;
  long long pix[8];
  int py[8], px[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const long long m = m0 + (tid >> 4) + 16 * q;
    if (m < M) {
      const long long b = m / HW;
      const long long rem = m - b * HW;
      const int y = (int)(rem / W), x = (int)(rem - (long long)y * W);
      const long long s = index ? (long long)index[b] : b;
      pix[q] = (s * HW + rem) * Cin;
      py[q] = y;
      px[q] = x;
    } else {
      pix[q] = 0;
      py[q] = -4;                 // every tap falls outside
      px[q] = -4;
    }
  }
  float ra[8], rb[TN];
  auto load = [&](int k0) {
    const int kk = k0 + ak;
    const bool kv = kk < K;
    const int tap = kv ? kk / Cin : 0;
    const int c = kk - tap * Cin;
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    const long long off = ((long long)dy * W + dx) * Cin + c;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int iy = py[q] + dy, ix = px[q] + dx;
      ra[q] = (kv && iy >= 0 && iy < H && ix >= 0 && ix < W) ? in[pix[q] + off] : 0.f;
    }
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int e = tid + CT * j;
      const int bk = e & 15, bn = e >> 4;
      const int o = n0 + bn, k = k0 + bk;
      rb[j] = (o < Cout && k < K) ? Wm[(long long)o * K + k] : 0.f;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 8; ++q) As[buf][ak][(tid >> 4) + 16 * q] = ra[q];
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int e = tid + CT * j;
      Bs[buf][e & 15][e >> 4] = rb[j];
    }
  };

  float acc[8][TN];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;

  const int nk = (K + BK - 1) / BK;
  load(0);
  store(0);
  __syncthreads();
  for (int t = 0; t < nk; ++t) {
    const int buf = t & 1;
    if (t + 1 < nk) load((t + 1) * BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 8]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 8 + 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      float bv[TN];
#pragma unroll
      for (int j = 0; j < TN; ++j) bv[j] = Bs[buf][kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], bv[j], acc[i][j]);
    }
    if (t + 1 < nk) store(buf ^ 1);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const long long m = m0 + ty * 8 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int o = n0 + tx + 16 * j;
      if (o >= Cout) continue;
      float v = acc[i][j] + (bias ? bias[o] : 0.f);
      if (relu) v = fmaxf(v, 0.f);
      if (mask && !(mask[m * Cout + o] > 0.f)) v = 0.f;
      if (accumulate) v += out[m * Cout + o];
      out[m * Cout + o] = v;
    }
  }
}

cudaError_t launch_conv3x3(const float* in, const int* index, const float* Wm, const float* bias, const float* mask,
                           float* out, int B, int H, int W, int Cin, int Cout, int relu, int accumulate,
                           cudaStream_t st) {
  const long long M = (long long)B * H * W;
  const unsigned gx = (unsigned)((M + BM - 1) / BM);
  if (Cout <= 32) {
    k_conv3x3<2><<<dim3(gx, 1), CT, 0, st>>>(in, index, Wm, bias, mask, out, B, H, W, Cin, Cout, relu, accumulate);
  } else if (Cout <= 64) {
    k_conv3x3<4><<<dim3(gx, 1), CT, 0, st>>>(in, index, Wm, bias, mask, out, B, H, W, Cin, Cout, relu, accumulate);
  } else if (Cout <= 80) {
    k_conv3x3<5><<<dim3(gx, 1), CT, 0, st>>>(in, index, Wm, bias, mask, out, B, H, W, Cin, Cout, relu, accumulate);
  } else {
    k_conv3x3<4><<<dim3(gx, (unsigned)((Cout + 63) / 64)), CT, 0, st>>>(in, index, Wm, bias, mask, out, B, H, W,
                                                                         Cin, Cout, relu, accumulate);
  }
  return cudaGetLastError();
}

// Wt[c][tap][o] = W[o][8 - tap][c]: the input gradient is the forward convolution of the
// output gradient with the spatially flipped, channel-transposed weights.
__global__ void k_flip_transpose(const float* __restrict__ Wm, float* __restrict__ Wt, int Cin, int Cout) {
  const int tot = Cout * 9 * Cin;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += gridDim.x * blockDim.x) {
    const int o = e % Cout;
    const int t = (e / Cout) % 9;
    const int c = e / (9 * Cout);
    Wt[e] = Wm[((long long)o * 9 + (8 - t)) * Cin + c];
  }
}

cudaError_t launch_flip_transpose(const float* Wm, float* Wt, int Cin, int Cout, cudaStream_t st) {
  const int tot = Cout * 9 * Cin;
  k_flip_transpose<<<(tot + 255) / 256, 256, 0, st>>>(Wm, Wt, Cin, Cout);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// weight gradient: part[s][o][kk] = sum over pixel range s of G[p][o] A[p][kk]
// ---------------------------------------------------------------------------------
// Thread (tx, ty) computes o = o0 + 4 ty + i and kk = k0 + 4 tx + j (i, j < 4).
__global__ void __launch_bounds__(CT) k_conv3x3_wgrad(const float* __restrict__ in, const int* __restrict__ index,
                                                      const float* __restrict__ G, float* __restrict__ part, int B,
                                                      int H, int W, int Cin, int Cout, long long per_split) {
  __shared__ __align__(16) float Gs[BK][WT + 4];
  __shared__ __align__(16) float As[BK][WT + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const long long HW = (long long)H * W;
  const long long M = (long long)B * HW;
  const int K = 9 * Cin;
  const int o0 = blockIdx.x * WT, k0 = blockIdx.y * WT;
  const long long p_lo = (long long)blockIdx.z * per_split;
  const long long p_hi = p_lo + per_split < M ? p_lo + per_split : M;
  // this thread's im2col column (fixed) and G column
  const int akl = tid & 63;
  const int kk = k0 + akl;
  const bool kv = kk < K;
  const int tap = kv ? kk / Cin : 0;
  const int c = kk - tap * Cin;
  const int dy = tap / 3 - 1, dx = tap % 3 - 1;
  const int gol = tid & 63;
  const bool ov = o0 + gol < Cout;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (long long p0 = p_lo; p0 < p_hi; p0 += BK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int pl = (tid >> 6) + 4 * q;
      const long long p = p0 + pl;
      float gv = 0.f, av = 0.f;
      if (p < p_hi) {
        if (ov) gv = G[p * Cout + o0 + gol];
        if (kv) {
          const long long b = p / HW;
          const long long rem = p - b * HW;
          const int y = (int)(rem / W), x = (int)(rem - (long long)y * W);
          const int iy = y + dy, ix = x + dx;
          if (iy >= 0 && iy < H && ix >= 0 && ix < W) {
            const long long s = index ? (long long)index[b] : b;
            av = in[(s * HW + (long long)iy * W + ix) * Cin + c];
          }
        }
      }
      Gs[pl][gol] = gv;
      As[pl][akl] = av;
    }
    __syncthreads();
#pragma unroll
    for (int pl = 0; pl < BK; ++pl) {
      const float4 g4 = *reinterpret_cast<const float4*>(&Gs[pl][ty * 4]);
      const float4 a4 = *reinterpret_cast<const float4*>(&As[pl][tx * 4]);
      const float g[4] = {g4.x, g4.y, g4.z, g4.w}, a[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(g[i], a[j], acc[i][j]);
    }
    __syncthreads();
  }
  float* P = part + (long long)blockIdx.z * Cout * K;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int o = o0 + ty * 4 + i;
    if (o >= Cout) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = k0 + tx * 4 + j;
      if (k < K) P[(long long)o * K + k] = acc[i][j];
    }
  }
}

// out[j] = sum_r part[r][j] in increasing r (FP64 accumulation)
__global__ void k_sum_rows(int nrows, long long ncols, const float* __restrict__ part, float* __restrict__ out) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < ncols;
       j += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int r = 0; r < nrows; ++r) s += (double)part[r * ncols + j];
    out[j] = (float)s;
  }
}

// part[blk][o] = sum over the block's pixels of G[p][o]
__global__ void k_bias_grad(const float* __restrict__ G, long long M, int Cout, long long per_blk,
                            float* __restrict__ part) {
  const long long lo = (long long)blockIdx.x * per_blk;
  const long long hi = lo + per_blk < M ? lo + per_blk : M;
  for (int o = threadIdx.x; o < Cout; o += blockDim.x) {
    double s = 0.0;
    for (long long p = lo; p < hi; ++p) s += (double)G[p * Cout + o];
    part[(long long)blockIdx.x * Cout + o] = (float)s;
  }
}

cudaError_t launch_conv3x3_grads(const float* in, const int* index, const float* G, float* dW, float* db, int B,
                                 int H, int W, int Cin, int Cout, float* part, long long part_cap, cudaStream_t st) {
  const long long M = (long long)B * H * W;
  const int K = 9 * Cin;
  const int tiles_o = (Cout + WT - 1) / WT, tiles_k = (K + WT - 1) / WT;
  long long splits = (2 * 152 + tiles_o * tiles_k - 1) / (tiles_o * tiles_k);
  if (splits > 64) splits = 64;
  while (splits > 1 && splits * Cout * K > part_cap) --splits;
  if (splits * Cout * K > part_cap) return cudaErrorInvalidValue;
  long long per = (M + splits - 1) / splits;
  per = (per + BK - 1) / BK * BK;
  splits = (M + per - 1) / per;
  k_conv3x3_wgrad<<<dim3(tiles_o, tiles_k, (unsigned)splits), CT, 0, st>>>(in, index, G, part, B, H, W, Cin, Cout,
                                                                          per);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long nW = (long long)Cout * K;
  k_sum_rows<<<(unsigned)((nW + 255) / 256), 256, 0, st>>>((int)splits, nW, part, dW);
  e = cudaGetLastError();
  if (e != cudaSuccess || !db) return e;
  // bias: pixel blocks of 512, partial sums reduced in order
  long long nb = (M + 511) / 512;
  if (nb * Cout > part_cap) nb = part_cap / Cout;
  if (nb < 1) return cudaErrorInvalidValue;
  const long long per_b = (M + nb - 1) / nb;
  nb = (M + per_b - 1) / per_b;
  const int th = Cout < 32 ? 32 : (Cout > 256 ? 256 : (Cout + 31) / 32 * 32);
  k_bias_grad<<<(unsigned)nb, th, 0, st>>>(G, M, Cout, per_b, part);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sum_rows<<<(Cout + 255) / 256, 256, 0, st>>>((int)nb, Cout, part, db);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// loss, optimiser, statistics
// ---------------------------------------------------------------------------------
constexpr int MSE_BLOCKS = 304;

// grad = 2 (pred - target) / N; part[blk] = block sum of (pred - target)^2
__global__ void __launch_bounds__(256) k_mse(const float* __restrict__ pred, const float* __restrict__ target,
                                             const int* __restrict__ index, long long per_sample, int batch,
                                             float* __restrict__ grad, double* __restrict__ part) {
  __shared__ double red[256];
  const long long N = per_sample * batch;
  const double scale = 2.0 / (double)N;
  double s = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
    const long long b = e / per_sample;
    const long long rem = e - b * per_sample;
    const long long sb = index ? (long long)index[b] : b;
    const double d = (double)pred[e] - (double)target[sb * per_sample + rem];
    if (grad) grad[e] = (float)(scale * d);
    s += d * d;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_mse_finish(const double* __restrict__ part, int n, double inv_N, double* __restrict__ loss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[i];
    *loss = s * inv_N;
  }
}

cudaError_t launch_mse(const float* pred, const float* target, const int* index, long long per_sample, int batch,
                       float* grad, double* part, double* loss, cudaStream_t st) {
  k_mse<<<MSE_BLOCKS, 256, 0, st>>>(pred, target, index, per_sample, batch, grad, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !loss) return e;
  k_mse_finish<<<1, 32, 0, st>>>(part, MSE_BLOCKS, 1.0 / ((double)per_sample * batch), loss);
  return cudaGetLastError();
}

int mse_partials() { return MSE_BLOCKS; }

__global__ void k_adam(long long n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

cudaError_t launch_adam(long long n, float* p, const float* g, float* m, float* v, float lr, float b1, float b2,
                        float eps, float c1, float c2, cudaStream_t st) {
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_adam<<<(unsigned)(blocks < 1 ? 1 : blocks), 256, 0, st>>>(n, p, g, m, v, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

// one block per group of 32 channels; warp w sums rows w, w + 32, ...; fixed-order combine
__global__ void __launch_bounds__(1024) k_channel_rms(long long rows, int C, const float* __restrict__ data,
                                                      float* __restrict__ rms, float* __restrict__ inv) {
  __shared__ double red[32][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + lane;
  double s = 0.0;
  if (c < C)
    for (long long r = w; r < rows; r += 32) {
      const double v = (double)data[r * C + c];
      s += v * v;
    }
  red[w][lane] = s;
  __syncthreads();
  if (w == 0 && c < C) {
    double t = 0.0;
    for (int i = 0; i < 32; ++i) t += red[i][lane];
    const double q = rows > 0 ? sqrt(t / (double)rows) : 0.0;
    if (rms) rms[c] = (float)q;
    if (inv) inv[c] = q > 0.0 ? (float)(1.0 / q) : 0.f;
  }
}

cudaError_t launch_channel_rms(long long rows, int C, const float* data, float* rms, float* inv, cudaStream_t st) {
  k_channel_rms<<<(C + 31) / 32, 1024, 0, st>>>(rows, C, data, rms, inv);
  return cudaGetLastError();
}

// rms = sqrt(mean data^2) over the whole tensor: one block, fixed-order tree
__global__ void __launch_bounds__(1024) k_tensor_rms(long long n, const float* __restrict__ data,
                                                     float* __restrict__ rms, float* __restrict__ inv) {
  __shared__ double red[1024];
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = (double)data[i];
    s += v * v;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int off = 512; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double q = n > 0 ? sqrt(red[0] / (double)n) : 0.0;
    if (rms) rms[0] = (float)q;
    if (inv) inv[0] = q > 0.0 ? (float)(1.0 / q) : 0.f;
  }
}

cudaError_t launch_tensor_rms(long long n, const float* data, float* rms, float* inv, cudaStream_t st) {
  k_tensor_rms<<<1, 1024, 0, st>>>(n, data, rms, inv);
  return cudaGetLastError();
}

__global__ void k_scale_channels(long long n, int C, float* __restrict__ d, const float* __restrict__ s) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    d[i] *= s[i % C];
}

cudaError_t launch_scale_channels(long long rows, int C, float* d, const float* s, cudaStream_t st) {
  const long long n = rows * C;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_scale_channels<<<(unsigned)(blocks < 1 ? 1 : blocks), 256, 0, st>>>(n, C, d, s);
  return cudaGetLastError();
}

}  // namespace stmg

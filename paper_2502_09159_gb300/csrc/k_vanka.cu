// Additive Vanka smoother (Eq. vanka0, vanka): x += omega D_w sum_T R_T^T A_T R_T res,
// A_T = [R_T S R_T^T]^{-1} stored per patch.
//
// Streaming the stored inverses is the dominant HBM traffic of the whole V-cycle
// (B^2 values per patch against B values of vectors), so the kernel is built around
// that stream:
//   * one thread per patch row; a block holds `ppb` patches (ppb * B threads),
//   * the patch residual R_T res is gathered once into shared memory (zero-padded to
//     Bc, boundary dofs read as 0) and read back as warp-wide broadcasts,
//   * the inverse is stored "column-chunk interleaved": for chunk c of VW consecutive
//     columns, rows j = 0..B-1 are contiguous VW-vectors, so a warp reads 32 adjacent
//     16-byte vectors (512 contiguous bytes) per load and every byte is used once,
//   * the finest levels (inverses far larger than L2) are read with evict-first
//     streaming loads so that the coarse levels' inverses stay L2-resident,
//   * the scaled correction omega/valence * (A_T r_T)_j is scatter-added with atomics
//     (patches overlap on shared dofs; additive, so the order is immaterial up to
//     rounding).
#include <cuda_runtime.h>

#include "internal.h"

namespace stmg {

namespace {

template <typename T> struct Vec;
template <> struct Vec<float> { using type = float4; static constexpr int W = 4; };
template <> struct Vec<double> { using type = double2; static constexpr int W = 2; };

__device__ __forceinline__ float4 load_vec(const float4* p, bool stream) {
  return stream ? __ldcs(p) : __ldg(p);
}
__device__ __forceinline__ double2 load_vec(const double2* p, bool stream) {
  return stream ? __ldcs(p) : __ldg(p);
}
__device__ __forceinline__ float dotv(const float4& a, const float* r) {
  return a.x * r[0] + a.y * r[1] + a.z * r[2] + a.w * r[3];
}
__device__ __forceinline__ double dotv(const double2& a, const double* r) {
  return a.x * r[0] + a.y * r[1];
}

}  // namespace

template <typename T>
__global__ void __launch_bounds__(1024) k_vanka_sweep(const int* __restrict__ dofs, const T* __restrict__ inv,
                                                      const T* __restrict__ res, const T* __restrict__ wgt,
                                                      T* __restrict__ x, long long n_patches, int B, int Bc,
                                                      int ppb, int streaming) {
  using V = typename Vec<T>::type;
  constexpr int VW = Vec<T>::W;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* rs = reinterpret_cast<T*>(smraw);                // [ppb][Bc]
  const long long p0 = (long long)blockIdx.x * ppb;
  for (int t = threadIdx.x; t < ppb * Bc; t += blockDim.x) {
    const int pl = t / Bc, i = t % Bc;
    const long long p = p0 + pl;
    T v = 0;
    if (p < n_patches && i < B) {
      const int g = dofs[p * B + i];
      if (g >= 0) v = res[g];
    }
    rs[t] = v;
  }
  __syncthreads();
  const int pl = threadIdx.x / B, j = threadIdx.x % B;
  const long long p = p0 + pl;
  if (pl >= ppb || p >= n_patches) return;
  const int nch = Bc / VW;
  const V* A = reinterpret_cast<const V*>(inv + (size_t)p * B * Bc) + j;
  const T* r = rs + pl * Bc;
  T acc0 = 0, acc1 = 0;
  const bool st = streaming != 0;
  int c = 0;
  for (; c + 8 <= nch; c += 8) {
    V a[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = load_vec(A + (size_t)(c + u) * B, st);
#pragma unroll
    for (int u = 0; u < 8; u += 2) {
      acc0 += dotv(a[u], r + (c + u) * VW);
      acc1 += dotv(a[u + 1], r + (c + u + 1) * VW);
    }
  }
  for (; c < nch; ++c) acc0 += dotv(load_vec(A + (size_t)c * B, st), r + c * VW);
  const int g = dofs[p * B + j];
  if (g >= 0) atomicAdd(x + g, wgt[g] * (acc0 + acc1));
}

template <typename T>
cudaError_t launch_vanka_sweep(const int* dofs, const T* inv, const T* res, const T* wgt, T* x,
                               long long n_patches, int B, int Bc, int ppb, int streaming, cudaStream_t st) {
  if (ppb * B > 1024) ppb = 1024 / B;
  if (ppb < 1) return cudaErrorInvalidValue;
  const int threads = ((ppb * B + 31) / 32) * 32;
  const long long blocks = (n_patches + ppb - 1) / ppb;
  const size_t smem = sizeof(T) * (size_t)ppb * Bc;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_vanka_sweep<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_vanka_sweep<T><<<(unsigned)blocks, threads, smem, st>>>(dofs, inv, res, wgt, x, n_patches, B, Bc, ppb,
                                                             streaming);
  return cudaGetLastError();
}

// Copy the inverse of each patch's class (FP64, row-major B x B) into the per-patch
// interleaved layout [patch][chunk][row][VW], rounding to T; padded columns are 0.
template <typename T>
__global__ void k_replicate(const double* __restrict__ cls, const int* __restrict__ cls_of_patch,
                            T* __restrict__ inv, long long n_patches, int B, int Bc) {
  constexpr int VW = Vec<T>::W;
  const long long per = (long long)B * Bc;
  const long long tot = n_patches * per;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long p = e / per;
    const long long o = e % per;
    const int v = (int)(o % VW);
    const long long t = o / VW;
    const int row = (int)(t % B);
    const int chunk = (int)(t / B);
    const int col = chunk * VW + v;
    const double* A = cls + (size_t)cls_of_patch[p] * B * B;
    inv[e] = col < B ? (T)A[(size_t)row * B + col] : T(0);
  }
}

template <typename T>
cudaError_t launch_replicate_inverses(const double* cls, const int* cls_of_patch, T* inv, long long n_patches,
                                      int B, int Bc, cudaStream_t st) {
  const long long tot = n_patches * (long long)B * Bc;
  long long blocks = (tot + 255) / 256;
  if (blocks > 152LL * 64) blocks = 152LL * 64;
  k_replicate<T><<<(unsigned)blocks, 256, 0, st>>>(cls, cls_of_patch, inv, n_patches, B, Bc);
  return cudaGetLastError();
}

template cudaError_t launch_vanka_sweep<double>(const int*, const double*, const double*, const double*, double*,
                                                long long, int, int, int, int, cudaStream_t);
template cudaError_t launch_vanka_sweep<float>(const int*, const float*, const float*, const float*, float*,
                                               long long, int, int, int, int, cudaStream_t);
template cudaError_t launch_replicate_inverses<double>(const double*, const int*, double*, long long, int, int,
                                                       cudaStream_t);
template cudaError_t launch_replicate_inverses<float>(const double*, const int*, float*, long long, int, int,
                                                      cudaStream_t);

}  // namespace stmg

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
//   * the rows of A_T carry the valence weight omega/valence of their dof (folded in at
//     setup), and the correction (A_T r_T)_j is scatter-added with atomics
//     (patches overlap on shared dofs; additive, so the order is immaterial up to
//     rounding).
#include <cuda_runtime.h>

#include <cuda_fp16.h>

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
__device__ __forceinline__ float dotvv(const float4& a, const float4& r) {
  return a.x * r.x + a.y * r.y + a.z * r.z + a.w * r.w;
}
__device__ __forceinline__ double dotvv(const double2& a, const double2& r) {
  return a.x * r.x + a.y * r.y;
}

}  // namespace

template <typename T, int U>
__global__ void __launch_bounds__(1024) k_vanka_sweep(const int* __restrict__ dofs, const T* __restrict__ inv,
                                                      const T* __restrict__ res, T* __restrict__ x,
                                                      long long n_patches, int B, int Bc, int ppb, int streaming) {
  using V = typename Vec<T>::type;
  constexpr int VW = Vec<T>::W;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int nch = Bc / VW;
  const int Bp = (nch + U - 1) / U * U * VW;          // residual padded to whole rounds of U chunks
  T* rs = reinterpret_cast<T*>(smraw);                // [ppb][Bp]
  const long long p0 = (long long)blockIdx.x * ppb;
  for (int t = threadIdx.x; t < ppb * Bp; t += blockDim.x) {
    const int pl = t / Bp, i = t % Bp;
    const long long p = p0 + pl;
    T v = 0;
    if (p < n_patches && i < B) {
      const int g = dofs[p * B + i];
      if (g >= 0) v = res[g];
    }
    rs[t] = v;
  }
  __syncthreads();
  const bool st = streaming != 0;
  // one row per thread; blocks of fewer threads than ppb * B rows (B > 1024) loop.  Rounds
  // of U chunks, the last one predicated, so that every round has U loads in flight.
  for (int t = threadIdx.x; t < ppb * B; t += blockDim.x) {
    const int pl = t / B, j = t % B;
    const long long p = p0 + pl;
    if (p >= n_patches) break;
    const V* A = reinterpret_cast<const V*>(inv + (size_t)p * B * Bc) + j;
    const T* r = rs + pl * Bp;
    T acc0 = 0, acc1 = 0;
    for (int c = 0; c < nch; c += U) {
      V a[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        a[u] = V{};
        if (c + u < nch) a[u] = load_vec(A + (size_t)(c + u) * B, st);
      }
#pragma unroll
      for (int u = 0; u < U; u += 2) {
        acc0 += dotv(a[u], r + (c + u) * VW);
        acc1 += dotv(a[u + 1], r + (c + u + 1) * VW);
      }
    }
    const int g = dofs[p * B + j];
    if (g >= 0) atomicAdd(x + g, acc0 + acc1);   // rows carry omega / valence
  }
}

template <typename T>
cudaError_t launch_vanka_sweep(const int* dofs, const T* inv, const T* res, T* x, long long n_patches, int B,
                               int Bc, int ppb, int unroll, int streaming, cudaStream_t st) {
  constexpr int VW = Vec<T>::W;
  if (ppb * B > 1024) ppb = 1024 / B;
  if (ppb < 1) ppb = 1;
  if (B < 1) return cudaErrorInvalidValue;
  const int U = unroll == 4 ? 4 : 8;
  const int nch = Bc / VW;
  const int threads = ppb * B > 1024 ? 1024 : ((ppb * B + 31) / 32) * 32;
  const long long blocks = (n_patches + ppb - 1) / ppb;
  const size_t smem = sizeof(T) * (size_t)ppb * ((nch + U - 1) / U * U * VW);
  auto kern = U == 4 ? k_vanka_sweep<T, 4> : k_vanka_sweep<T, 8>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<(unsigned)blocks, threads, smem, st>>>(dofs, inv, res, x, n_patches, B, Bc, ppb, streaming);
  return cudaGetLastError();
}

// Copy the inverse of each patch's class (FP64, row-major B x B) into the per-patch
// interleaved layout [patch][chunk][row][VW], each row scaled by the valence weight
// omega / valence of its dof (D_w is diagonal: (D_w A_T r)_j = w_j (A_T r)_j), rounded to
// T; boundary / padding rows and padded columns are 0.
template <typename T>
__global__ void k_replicate(const double* __restrict__ cls, const int* __restrict__ cls_of_patch,
                            const int* __restrict__ dofs, const double* __restrict__ w, T* __restrict__ inv,
                            long long n_patches, int B, int Bc) {
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
    const int g = dofs[p * B + row];
    inv[e] = (col < B && g >= 0) ? (T)(w[g] * A[(size_t)row * B + col]) : T(0);
  }
}

template <typename T>
cudaError_t launch_replicate_inverses(const double* cls, const int* cls_of_patch, const int* dofs, const double* w,
                                      T* inv, long long n_patches, int B, int Bc, cudaStream_t st) {
  const long long tot = n_patches * (long long)B * Bc;
  long long blocks = (tot + 255) / 256;
  if (blocks > 152LL * 64) blocks = 152LL * 64;
  k_replicate<T><<<(unsigned)blocks, 256, 0, st>>>(cls, cls_of_patch, dofs, w, inv, n_patches, B, Bc);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Half-precision inverses for the FP32 V-cycle.  Row j of patch p is stored as FP16 values
// of w_j A_jc / s_pj with the row scale s_pj = max_c |w_j A_jc| kept in FP32, so every
// stored value lies in [-1, 1] (no overflow, relative rounding 2^-11); the layout is the
// interleaved one with 8-column chunks: [patch][chunk][row][8 halves] (16-byte vectors).
// The sweep streams half the bytes of the FP32 inverses and accumulates in FP32.
// ------------------------------------------------------------------------------------
__global__ void k_replicate_half(const double* __restrict__ cls, const int* __restrict__ cls_of_patch,
                                 const int* __restrict__ dofs, const double* __restrict__ w, __half* __restrict__ inv,
                                 float* __restrict__ rscale, long long n_patches, int B, int Bh) {
  const long long tot = n_patches * B;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long p = e / B;
    const int row = (int)(e - p * B);
    const double* A = cls + (size_t)cls_of_patch[p] * B * B + (size_t)row * B;
    const int g = dofs[p * B + row];
    const double wr = g >= 0 ? w[g] : 0.0;
    double m = 0.0;
    for (int c = 0; c < B; ++c) m = fmax(m, fabs(wr * A[c]));
    const double s = m > 0.0 ? m : 1.0;
    rscale[e] = (float)s;
    __half* out = inv + (size_t)p * B * Bh + (size_t)row * 8;
    for (int c = 0; c < Bh; ++c) {
      const double v = c < B ? wr * A[c] / s : 0.0;
      out[(size_t)(c / 8) * B * 8 + (c % 8)] = __double2half(v);
    }
  }
}

cudaError_t launch_replicate_inverses_half(const double* cls, const int* cls_of_patch, const int* dofs, const double* w,
                                           __half* inv, float* rscale, long long n_patches, int B, int Bh,
                                           cudaStream_t st) {
  const long long tot = n_patches * (long long)B;
  long long blocks = (tot + 255) / 256;
  if (blocks > 152LL * 64) blocks = 152LL * 64;
  k_replicate_half<<<(unsigned)(blocks < 1 ? 1 : blocks), 256, 0, st>>>(cls, cls_of_patch, dofs, w, inv, rscale,
                                                                      n_patches, B, Bh);
  return cudaGetLastError();
}

__device__ __forceinline__ float dot8h(const uint4& a, const float* r) {
  const __half2* h = reinterpret_cast<const __half2*>(&a);
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 f = __half22float2(h[i]);
    s = fmaf(f.x, r[2 * i], s);
    s = fmaf(f.y, r[2 * i + 1], s);
  }
  return s;
}

__global__ void __launch_bounds__(1024) k_vanka_sweep_half(const int* __restrict__ dofs, const __half* __restrict__ inv,
                                                           const float* __restrict__ rscale,
                                                           const float* __restrict__ res, float* __restrict__ x,
                                                           long long n_patches, int B, int Bh, int ppb, int streaming) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float* rs = reinterpret_cast<float*>(smraw);        // [ppb][Bh]
  const long long p0 = (long long)blockIdx.x * ppb;
  for (int t = threadIdx.x; t < ppb * Bh; t += blockDim.x) {
    const int pl = t / Bh, i = t % Bh;
    const long long p = p0 + pl;
    float v = 0.f;
    if (p < n_patches && i < B) {
      const int g = dofs[p * B + i];
      if (g >= 0) v = res[g];
    }
    rs[t] = v;
  }
  __syncthreads();
  const int nch = Bh / 8;
  const bool st = streaming != 0;
  for (int t = threadIdx.x; t < ppb * B; t += blockDim.x) {
    const int pl = t / B, j = t % B;
    const long long p = p0 + pl;
    if (p >= n_patches) break;
    const uint4* A = reinterpret_cast<const uint4*>(inv + (size_t)p * B * Bh) + j;
    const float* r = rs + pl * Bh;
    float acc0 = 0.f, acc1 = 0.f;
    int c = 0;
    for (; c + 8 <= nch; c += 8) {
      uint4 a[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] = st ? __ldcs(A + (size_t)(c + u) * B) : __ldg(A + (size_t)(c + u) * B);
#pragma unroll
      for (int u = 0; u < 8; u += 2) {
        acc0 += dot8h(a[u], r + (c + u) * 8);
        acc1 += dot8h(a[u + 1], r + (c + u + 1) * 8);
      }
    }
    for (; c < nch; ++c) acc0 += dot8h(st ? __ldcs(A + (size_t)c * B) : __ldg(A + (size_t)c * B), r + c * 8);
    const int g = dofs[p * B + j];
    if (g >= 0) atomicAdd(x + g, (acc0 + acc1) * rscale[p * B + j]);   // rows carry omega / valence
  }
}

cudaError_t launch_vanka_sweep_half(const int* dofs, const __half* inv, const float* rscale, const float* res, float* x,
                                    long long n_patches, int B, int Bh, int ppb, int streaming, cudaStream_t st) {
  if (ppb * B > 1024) ppb = 1024 / B;
  if (ppb < 1) ppb = 1;
  if (B < 1 || Bh % 8 != 0) return cudaErrorInvalidValue;
  const int threads = ppb * B > 1024 ? 1024 : ((ppb * B + 31) / 32) * 32;
  const long long blocks = (n_patches + ppb - 1) / ppb;
  const size_t smem = sizeof(float) * (size_t)ppb * Bh;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_vanka_sweep_half, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_vanka_sweep_half<<<(unsigned)blocks, threads, smem, st>>>(dofs, inv, rscale, res, x, n_patches, B, Bh, ppb,
                                                              streaming);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Pipelined block sweep.  Same work split as k_vanka_sweep (one thread per patch row, ppb
// patches per block), but the inverse stream never waits on anything else:
//   * the first U column chunks of the thread's row are loaded before the residual gather
//     (the gather's two dependent loads, index then value, overlap the inverse stream);
//   * round c+1's U loads are issued before round c is consumed (double buffer), so a
//     thread keeps up to 2U 16-byte loads in flight through its whole row;
//   * the last round is predicated instead of a serial tail loop (a row of 29 chunks is
//     4 rounds of 8, not 3 rounds and 5 single loads).
// The residual is zero-padded in shared memory to whole rounds.
// ------------------------------------------------------------------------------------
template <typename T, int U>
__global__ void __launch_bounds__(512) k_vanka_sweep_pipe(const int* __restrict__ dofs, const T* __restrict__ inv,
                                                          const T* __restrict__ res, T* __restrict__ x,
                                                          long long n_patches, int B, int Bc, int ppb, int streaming) {
  using V = typename Vec<T>::type;
  constexpr int VW = Vec<T>::W;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int nch = Bc / VW;
  const int nrd = (nch + U - 1) / U;                  // rounds per row
  const int Bp = nrd * U * VW;                        // padded residual length per patch
  T* rs = reinterpret_cast<T*>(smraw);                // [ppb][Bp]
  const long long p0 = (long long)blockIdx.x * ppb;
  const bool st = streaming != 0;
  const int t = threadIdx.x;
  const int pl = t / B, j = t - pl * B;
  const long long p = p0 + pl;
  const bool active = pl < ppb && p < n_patches;
  const V* A = active ? reinterpret_cast<const V*>(inv + (size_t)p * B * Bc) + j : nullptr;
  V cur[U], nxt[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    cur[u] = V{};
    if (active && u < nch) cur[u] = load_vec(A + (size_t)u * B, st);
  }
  int g = -1;
  if (active) g = dofs[p * B + j];
  for (int e = t; e < ppb * Bp; e += blockDim.x) {
    const int q = e / Bp, i = e - q * Bp;
    const long long pq = p0 + q;
    T v = 0;
    if (pq < n_patches && i < B) {
      const int gi = dofs[pq * B + i];
      if (gi >= 0) v = res[gi];
    }
    rs[e] = v;
  }
  __syncthreads();
  if (!active) return;
  const T* r = rs + pl * Bp;
  T acc0 = 0, acc1 = 0;
  for (int rd = 0; rd < nrd; ++rd) {
    const int c0 = rd * U;
    if (rd + 1 < nrd) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int c = c0 + U + u;
        nxt[u] = V{};
        if (c < nch) nxt[u] = load_vec(A + (size_t)c * B, st);
      }
    }
#pragma unroll
    for (int u = 0; u < U; u += 2) {
      acc0 += dotv(cur[u], r + (c0 + u) * VW);
      acc1 += dotv(cur[u + 1], r + (c0 + u + 1) * VW);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) cur[u] = nxt[u];
  }
  if (g >= 0) atomicAdd(x + g, acc0 + acc1);          // rows carry omega / valence
}

template <typename T>
bool pipe_sweep_supported(int B, int ppb) {
  return B >= 1 && ppb >= 1 && ppb * B <= 512;
}

template <typename T>
cudaError_t launch_vanka_sweep_pipe(const int* dofs, const T* inv, const T* res, T* x, long long n_patches, int B,
                                    int Bc, int ppb, int unroll, int streaming, cudaStream_t st) {
  constexpr int VW = Vec<T>::W;
  if (!pipe_sweep_supported<T>(B, ppb)) return cudaErrorInvalidValue;
  const int nch = Bc / VW;
  const int threads = ((ppb * B + 31) / 32) * 32;
  const long long blocks = (n_patches + ppb - 1) / ppb;
  const int U = unroll == 4 ? 4 : 8;
  const size_t smem = sizeof(T) * (size_t)ppb * ((nch + U - 1) / U) * U * VW;
  if (U == 4) {
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(k_vanka_sweep_pipe<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
      if (e != cudaSuccess) return e;
    }
    k_vanka_sweep_pipe<T, 4><<<(unsigned)blocks, threads, smem, st>>>(dofs, inv, res, x, n_patches, B, Bc, ppb,
                                                                     streaming);
  } else {
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(k_vanka_sweep_pipe<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
      if (e != cudaSuccess) return e;
    }
    k_vanka_sweep_pipe<T, 8><<<(unsigned)blocks, threads, smem, st>>>(dofs, inv, res, x, n_patches, B, Bc, ppb,
                                                                     streaming);
  }
  return cudaGetLastError();
}

template cudaError_t launch_vanka_sweep_pipe<double>(const int*, const double*, const double*, double*, long long,
                                                     int, int, int, int, int, cudaStream_t);
template cudaError_t launch_vanka_sweep_pipe<float>(const int*, const float*, const float*, float*, long long, int,
                                                    int, int, int, int, cudaStream_t);
template bool pipe_sweep_supported<double>(int, int);
template bool pipe_sweep_supported<float>(int, int);

template cudaError_t launch_vanka_sweep<double>(const int*, const double*, const double*, double*, long long, int,
                                                int, int, int, int, cudaStream_t);
template cudaError_t launch_vanka_sweep<float>(const int*, const float*, const float*, float*, long long, int, int,
                                               int, int, int, cudaStream_t);
template cudaError_t launch_replicate_inverses<double>(const double*, const int*, const int*, const double*,
                                                       double*, long long, int, int, cudaStream_t);
template cudaError_t launch_replicate_inverses<float>(const double*, const int*, const int*, const double*, float*,
                                                      long long, int, int, cudaStream_t);

// ====================================================================================
// Persistent TMA-pipelined sweep.
//
// One CTA per SM owns a contiguous, balanced range of patches (the per-SM byte counts
// differ by at most one patch), so every SM streams until the end instead of the
// 1.68-wave tail of the one-block-per-8-patches launch.  Warp NCW (lane 0) is the
// producer: it streams each patch's inverse, `cps` column chunks (cps * B * 16 bytes) at a
// time, into a ring of `nstage` shared-memory stages with cp.async.bulk, completion
// signalled on the stage's "full" mbarrier (transaction bytes).  Warps 0..NCW-1 consume:
// thread t owns rows t, t + 32 NCW, ... (RPT of them), reads its row's 16-byte vector of
// every chunk from shared memory (conflict-free, consecutive threads read consecutive
// vectors) against the broadcast residual chunk, then releases the stage on its "empty"
// mbarrier.  The residual R_T res of the next patch is gathered into registers while the
// current patch is consumed (double-buffered in shared memory), so the inverse stream is
// never interrupted by the scattered gather.  Every mbarrier wait is bounded: on expiry the
// thread raises *err and leaves its loop; the producer then waits (bounded) for the copies
// it issued before the CTA exits.
// ====================================================================================
namespace {

constexpr unsigned kWaitLimit = 1u << 22;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for the phase with the given parity; false on expiry
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
  for (unsigned it = 0; it < kWaitLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar,
                                         bool evict_first) {
  if (evict_first) {
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
  } else {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
  }
}
}  // namespace

template <typename T, int RPT>
__global__ void __launch_bounds__(32 * (TMA_NCW + 1), 1)
k_vanka_sweep_tma(const int* __restrict__ dofs, const T* __restrict__ inv, const T* __restrict__ res,
                  T* __restrict__ x, long long n_patches, int B, int Bc, int cps, int nstage, int streaming,
                  int* __restrict__ err) {
  using V = typename Vec<T>::type;
  constexpr int VW = Vec<T>::W;
  constexpr int NC = 32 * TMA_NCW;                      // consumer threads
  extern __shared__ __align__(128) unsigned char smraw[];
  const int nch = Bc / VW;                              // column chunks per patch
  const int nst = (nch + cps - 1) / cps;                // stages per patch
  const size_t stage_bytes = (size_t)cps * B * 16;
  unsigned long long* full = reinterpret_cast<unsigned long long*>(smraw);
  unsigned long long* empty = full + nstage;
  unsigned long long* cbar = empty + nstage;            // consumer-only barrier, one arrival per warp
  T* rbuf = reinterpret_cast<T*>(smraw + 16 * nstage + 16);   // [2][Bc], 16-byte aligned
  unsigned char* stages = smraw + ((16 * nstage + 16 + 2 * Bc * sizeof(T) + 127) / 128) * 128;

  // balanced contiguous patch range of this CTA
  const long long G = gridDim.x, c = blockIdx.x;
  const long long p_begin = c * (n_patches / G) + min(c, n_patches % G);
  const long long p_end = p_begin + n_patches / G + (c < n_patches % G ? 1 : 0);
  const long long np = p_end - p_begin;
  const int tid = threadIdx.x;

  if (tid == 0) {
    for (int s = 0; s < nstage; ++s) { mbar_init(full + s, 1); mbar_init(empty + s, TMA_NCW); }
    mbar_init(cbar, TMA_NCW);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // first patch's residual
  if (tid < NC && np > 0)
    for (int i = tid; i < Bc; i += NC) {
      T v = 0;
      if (i < B) { const int g = dofs[p_begin * B + i]; if (g >= 0) v = res[g]; }
      rbuf[i] = v;
    }
  __syncthreads();
  if (np <= 0) return;
  const long long total = np * nst;                     // stages this CTA streams

  if (tid >= NC) {
    // ---------------- producer ----------------
    if (tid != NC) return;
    const bool ef = streaming != 0;
    long long issued = 0;
    bool ok = true;
    for (long long g = 0; g < total && ok; ++g) {
      const int s = (int)(g % nstage);
      const unsigned par = (unsigned)((g / nstage) & 1) ^ 1u;
      if (!mbar_wait(empty + s, par)) { atomicExch(err, 1); ok = false; break; }
      const long long p = p_begin + g / nst;
      const int st = (int)(g % nst);
      const int c0 = st * cps;
      const int cn = min(cps, nch - c0);
      const unsigned bytes = (unsigned)cn * B * 16;
      mbar_arrive_expect_tx(full + s, bytes);
      const unsigned char* src = reinterpret_cast<const unsigned char*>(inv + (size_t)p * B * Bc) + (size_t)c0 * B * 16;
      bulk_g2s(stages + s * stage_bytes, src, bytes, full + s, ef);
      issued = g + 1;
    }
    // the CTA must not exit while copies it issued are still landing in shared memory
    const long long lo = issued > nstage ? issued - nstage : 0;
    for (long long g = lo; g < issued; ++g)
      if (!mbar_wait(full + (int)(g % nstage), (unsigned)((g / nstage) & 1))) atomicExch(err, 1);
    return;
  }

  // ---------------- consumers ----------------
  // Index loads are software-pipelined so that no thread ever waits on a load whose
  // address it has just computed: the gather indices of patch p+2, the residual values of
  // patch p+1 (indices loaded one patch earlier) and this thread's rows' dofs of patch p+1
  // are issued at the start of patch p; the rows' weights of patch p were issued at the
  // start of patch p-... (one patch earlier), so the scatter never stalls either.
  const int lane = tid & 31;
  int gi_n[8], gi_nn[8];       // gather indices of the next and next-next patch
  int dof_c[RPT], dof_n[RPT];  // this thread's rows' dofs, current and next patch
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int i = tid + q * NC;
    gi_n[q] = (np > 1 && i < B) ? dofs[(p_begin + 1) * B + i] : -1;
  }
#pragma unroll
  for (int rr = 0; rr < RPT; ++rr) {
    const int row = tid + rr * NC;
    dof_c[rr] = row < B ? dofs[p_begin * B + row] : -1;
  }
  long long g = 0;
  bool ok = true;
  for (long long pi = 0; pi < np && ok; ++pi) {
    const long long p = p_begin + pi;
    const T* r = rbuf + (pi & 1) * Bc;
    const bool has_next = pi + 1 < np, has_nn = pi + 2 < np;
    // issue: indices of patch p+2, residual values of patch p+1, row dofs of patch p+1
    T nxt[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int i = tid + q * NC;
      gi_nn[q] = (has_nn && i < B) ? dofs[(p + 2) * B + i] : -1;
      nxt[q] = gi_n[q] >= 0 ? res[gi_n[q]] : T(0);
    }
#pragma unroll
    for (int rr = 0; rr < RPT; ++rr) {
      const int row = tid + rr * NC;
      dof_n[rr] = (has_next && row < B) ? dofs[(p + 1) * B + row] : -1;
    }
    T acc[RPT], acc2[RPT];
#pragma unroll
    for (int rr = 0; rr < RPT; ++rr) { acc[rr] = 0; acc2[rr] = 0; }
    for (int st = 0; st < nst; ++st, ++g) {
      const int s = (int)(g % nstage);
      if (!mbar_wait(full + s, (unsigned)((g / nstage) & 1))) { atomicExch(err, 1); ok = false; break; }
      const int c0 = st * cps;
      const int cn = min(cps, nch - c0);
      const V* A = reinterpret_cast<const V*>(stages + s * stage_bytes);
      const V* rv = reinterpret_cast<const V*>(r + c0 * VW);
      int cc = 0;
      for (; cc + 2 <= cn; cc += 2) {
        const V r0 = rv[cc], r1 = rv[cc + 1];
#pragma unroll
        for (int rr = 0; rr < RPT; ++rr) {
          const int row = tid + rr * NC;
          if (row < B) {
            acc[rr] += dotvv(A[cc * B + row], r0);
            acc2[rr] += dotvv(A[(cc + 1) * B + row], r1);
          }
        }
      }
      if (cc < cn) {
        const V r0 = rv[cc];
#pragma unroll
        for (int rr = 0; rr < RPT; ++rr) {
          const int row = tid + rr * NC;
          if (row < B) acc[rr] += dotvv(A[cc * B + row], r0);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(empty + s);
    }
    if (!ok) break;
#pragma unroll
    for (int rr = 0; rr < RPT; ++rr)
      if (dof_c[rr] >= 0) atomicAdd(x + dof_c[rr], acc[rr] + acc2[rr]);   // rows carry omega / valence
    if (has_next) {
      T* rn = rbuf + ((pi + 1) & 1) * Bc;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int i = tid + q * NC;
        if (i < Bc) rn[i] = nxt[q];
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) gi_n[q] = gi_nn[q];
#pragma unroll
    for (int rr = 0; rr < RPT; ++rr) dof_c[rr] = dof_n[rr];
    // all consumers done with this patch (and the next residual written) before any
    // starts the next one; a bounded mbarrier wait instead of a named barrier, so that a
    // consumer that gave up cannot leave the others blocked
    __syncwarp();
    if (lane == 0) mbar_arrive(cbar);
    if (!mbar_wait(cbar, (unsigned)(pi & 1))) { atomicExch(err, 1); ok = false; }
  }
}

// shared memory of the TMA sweep for (B, Bc, cps, nstage)
template <typename T>
static size_t tma_smem(int B, int Bc, int cps, int nstage) {
  return ((16 * (size_t)nstage + 16 + 2 * Bc * sizeof(T) + 127) / 128) * 128 + (size_t)nstage * cps * B * 16;
}

template <typename T>
bool tma_sweep_supported(int B) {
  return B >= 1 && B <= 4 * 32 * TMA_NCW;
}

template <typename T>
cudaError_t launch_vanka_sweep_tma(const int* dofs, const T* inv, const T* res, T* x, long long n_patches, int B,
                                   int Bc, int n_sm, int streaming, int* err, cudaStream_t st) {
  constexpr int VW = Vec<T>::W;
  const int nch = Bc / VW;
  int cps = (int)(16384 / ((size_t)B * 16));
  cps = cps < 1 ? 1 : (cps > nch ? nch : cps);
  const size_t budget = 200 * 1024;
  int nstage = (int)((budget - 2 * Bc * sizeof(T) - 1024) / ((size_t)cps * B * 16 + 16));
  if (nstage > 2 * (int)((nch + cps - 1) / cps) + 2) nstage = 2 * (int)((nch + cps - 1) / cps) + 2;
  if (nstage > 16) nstage = 16;
  if (nstage < 2) return cudaErrorInvalidValue;
  const size_t smem = tma_smem<T>(B, Bc, cps, nstage);
  long long grid = n_patches < n_sm ? n_patches : n_sm;
  if (grid < 1) grid = 1;
  const int rpt = (B + 32 * TMA_NCW - 1) / (32 * TMA_NCW);
#define STMG_TMA_CASE(R)                                                                                        \
  if (rpt <= R) {                                                                                               \
    cudaError_t e = cudaFuncSetAttribute(k_vanka_sweep_tma<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                         (int)smem);                                                            \
    if (e != cudaSuccess) return e;                                                                             \
    k_vanka_sweep_tma<T, R><<<(unsigned)grid, 32 * (TMA_NCW + 1), smem, st>>>(                                  \
        dofs, inv, res, x, n_patches, B, Bc, cps, nstage, streaming, err);                                      \
    return cudaGetLastError();                                                                                  \
  }
  STMG_TMA_CASE(1) STMG_TMA_CASE(2) STMG_TMA_CASE(4)
#undef STMG_TMA_CASE
  return cudaErrorInvalidValue;
}

template cudaError_t launch_vanka_sweep_tma<double>(const int*, const double*, const double*, double*, long long,
                                                    int, int, int, int, int*, cudaStream_t);
template cudaError_t launch_vanka_sweep_tma<float>(const int*, const float*, const float*, float*, long long, int,
                                                   int, int, int, int*, cudaStream_t);
template bool tma_sweep_supported<double>(int);
template bool tma_sweep_supported<float>(int);

}  // namespace stmg

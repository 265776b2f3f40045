// Vector kernels of the FGMRES driver (FP64) and the coarse-level direct solve.
//
// The Arnoldi step uses classical Gram-Schmidt applied twice (CGS2): the projections
// h = V^T w of all previous basis vectors are computed in one pass over V (multidot:
// per block partial sums for every basis vector, then a deterministic tree over the
// blocks), and w -= V h is one more pass (multiaxpy).  Scalars stay on the device.
#include <cuda_runtime.h>

#include "internal.h"

namespace stmg {

namespace {
constexpr int RED_THREADS = 256;
constexpr int MD_VEC = 8;   // basis vectors handled per multidot pass
}

template <typename Ti, typename To>
__global__ void k_convert(long long n, const Ti* __restrict__ in, To* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (To)in[i];
}

static unsigned grid_for(long long n) {
  long long b = (n + 255) / 256;
  const long long cap = 152LL * 16;
  return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

template <typename Ti, typename To>
cudaError_t launch_convert(long long n, const Ti* in, To* out, cudaStream_t st) {
  k_convert<Ti, To><<<grid_for(n), 256, 0, st>>>(n, in, out);
  return cudaGetLastError();
}
template cudaError_t launch_convert<double, float>(long long, const double*, float*, cudaStream_t);
template cudaError_t launch_convert<float, double>(long long, const float*, double*, cudaStream_t);

__global__ void k_scale(long long n, double a, const double* __restrict__ x, double* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}
cudaError_t launch_scale(long long n, double a, const double* x, double* y, cudaStream_t st) {
  k_scale<<<grid_for(n), 256, 0, st>>>(n, a, x, y);
  return cudaGetLastError();
}

__global__ void k_scale_by_inverse(long long n, const double* __restrict__ s, const double* __restrict__ x,
                                   double* __restrict__ y) {
  const double a = 1.0 / s[0];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}
cudaError_t launch_scale_by_inverse(long long n, const double* s, const double* x, double* y, cudaStream_t st) {
  k_scale_by_inverse<<<grid_for(n), 256, 0, st>>>(n, s, x, y);
  return cudaGetLastError();
}

__global__ void k_sqrt(double* v) { v[0] = sqrt(v[0]); }
cudaError_t launch_sqrt_inplace(double* v, cudaStream_t st) {
  k_sqrt<<<1, 1, 0, st>>>(v);
  return cudaGetLastError();
}

int multidot_blocks(long long n) {
  long long b = (n + RED_THREADS * 8 - 1) / (RED_THREADS * 8);
  if (b > 304) b = 304;
  if (b < 1) b = 1;
  return (int)b;
}

// partial[blk * nvec + i] = sum over this block's rows of V[i][row] * w[row]
__global__ void __launch_bounds__(RED_THREADS) k_multidot(long long n, int nvec, const double* __restrict__ V,
                                                          long long ld, const double* __restrict__ w,
                                                          double* __restrict__ partial) {
  __shared__ double red[RED_THREADS / 32][MD_VEC];
  const long long chunk = (n + gridDim.x - 1) / gridDim.x;
  const long long lo = blockIdx.x * chunk;
  const long long hi = lo + chunk < n ? lo + chunk : n;
  for (int v0 = 0; v0 < nvec; v0 += MD_VEC) {
    const int nv = nvec - v0 < MD_VEC ? nvec - v0 : MD_VEC;
    double acc[MD_VEC];
#pragma unroll
    for (int i = 0; i < MD_VEC; ++i) acc[i] = 0.0;
    for (long long r = lo + threadIdx.x; r < hi; r += blockDim.x) {
      const double wr = w[r];
#pragma unroll
      for (int i = 0; i < MD_VEC; ++i)
        if (i < nv) acc[i] += V[(size_t)(v0 + i) * ld + r] * wr;
    }
#pragma unroll
    for (int i = 0; i < MD_VEC; ++i) {
      double a = acc[i];
      for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][i] = a;
    }
    __syncthreads();
    if (threadIdx.x < nv) {
      double s = 0.0;
      for (int wv = 0; wv < RED_THREADS / 32; ++wv) s += red[wv][threadIdx.x];
      partial[(size_t)blockIdx.x * nvec + v0 + threadIdx.x] = s;
    }
    __syncthreads();
  }
}

cudaError_t launch_multidot(long long n, int nvec, const double* V, long long ld, const double* w, double* partial,
                            int nblocks, cudaStream_t st) {
  k_multidot<<<nblocks, RED_THREADS, 0, st>>>(n, nvec, V, ld, w, partial);
  return cudaGetLastError();
}

// out[i] (+)= sum_blk partial[blk * nvec + i], fixed order (deterministic)
__global__ void k_reduce_partials(int nvec, int nblocks, const double* __restrict__ partial, double* __restrict__ out,
                                  int accumulate) {
  const int i = blockIdx.x;
  __shared__ double red[RED_THREADS];
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partial[(size_t)b * nvec + i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int off = RED_THREADS / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[i] = accumulate ? out[i] + red[0] : red[0];
}

cudaError_t launch_reduce_partials(int nvec, int nblocks, const double* partial, double* out, int accumulate,
                                   cudaStream_t st) {
  k_reduce_partials<<<nvec, RED_THREADS, 0, st>>>(nvec, nblocks, partial, out, accumulate);
  return cudaGetLastError();
}

// y[r] += sign * sum_i coef[i] V[i][r]
__global__ void k_multiaxpy(long long n, int nvec, const double* __restrict__ V, long long ld,
                            const double* __restrict__ coef, double sign, double* __restrict__ y) {
  extern __shared__ double cs[];
  for (int i = threadIdx.x; i < nvec; i += blockDim.x) cs[i] = sign * coef[i];
  __syncthreads();
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < nvec; ++i) s += cs[i] * V[(size_t)i * ld + r];
    y[r] += s;
  }
}

cudaError_t launch_multiaxpy(long long n, int nvec, const double* V, long long ld, const double* coef, double sign,
                             double* y, cudaStream_t st) {
  k_multiaxpy<<<grid_for(n), 256, sizeof(double) * (nvec > 0 ? nvec : 1), st>>>(n, nvec, V, ld, coef, sign, y);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// One Arnoldi step of FGMRES in a single cooperative launch (CGS2):
//   h  = V^T w,  w -= V h,  h2 = V^T w,  w -= V h2,  hcol[0..nv) = h + h2,
//   hcol[nv] = ||w||,  vnext = w / ||w||.
// Every block owns a contiguous range of rows, so the axpys and the next pass's partial
// dot products touch only the block's own rows; grid-wide barriers are needed only after
// partial sums are written (three per step).  Each block sums all blocks' partials itself,
// in block order (deterministic).  The barriers are bounded: a wait that exceeds its
// iteration limit raises *err and the kernel returns (the host reports STMG_ERR_TIMEOUT).
// The launch is cooperative, so all blocks are resident and every barrier completes.
// ------------------------------------------------------------------------------------
namespace {
constexpr int CGS_THREADS = 256;
constexpr int CGS_MAXV = 256;          // basis vectors per step (gmres_max_iter + 1)
constexpr long long BARRIER_SPINS = 1LL << 22;

// sense-free generation barrier over all blocks; returns false if the wait timed out
__device__ bool grid_barrier(unsigned* count, volatile unsigned* gen, unsigned nblocks, int* err,
                             int* sh_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned my = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(count, 1u);
    bool ok = true;
    if (arrived == nblocks - 1) {
      *count = 0;
      __threadfence();
      atomicAdd((unsigned*)gen, 1u);
    } else {
      long long it = 0;
      while (*gen == my) {
        if (++it > BARRIER_SPINS) { atomicExch(err, 2); ok = false; break; }
        __nanosleep(64);
      }
    }
    __threadfence();
    *sh_ok = ok ? 1 : 0;
  }
  __syncthreads();
  return *sh_ok != 0;
}

// partial[blk * nv + i] = sum over rows [lo, hi) of V_i w, eight vectors per sweep over w
__device__ void block_partials(long long lo, long long hi, int nv, const double* __restrict__ V, long long ld,
                               const double* __restrict__ w, double* __restrict__ out, double (*red)[8]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int v0 = 0; v0 < nv; v0 += 8) {
    const int cnt = nv - v0 < 8 ? nv - v0 : 8;
    double acc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = 0.0;
    for (long long r = lo + threadIdx.x; r < hi; r += CGS_THREADS) {
      const double wr = w[r];
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (i < cnt) acc[i] += V[(size_t)(v0 + i) * ld + r] * wr;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      double a = acc[i];
      for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
      if (lane == 0) red[wid][i] = a;
    }
    __syncthreads();
    if (threadIdx.x < cnt) {
      double t = 0.0;
      for (int q = 0; q < CGS_THREADS / 32; ++q) t += red[q][threadIdx.x];
      out[v0 + threadIdx.x] = t;
    }
    __syncthreads();
  }
}
// out[i] = sum_bb part[bb * nv + i], i < nv: one warp per vector, lanes strided over the
// blocks, then a fixed shuffle tree (deterministic)
__device__ void sum_partials(const double* __restrict__ part, unsigned G, int nv, double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = wid; i < nv; i += CGS_THREADS / 32) {
    double s = 0.0;
    for (unsigned bb = lane; bb < G; bb += 32) s += part[(size_t)bb * nv + i];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) out[i] = s;
  }
}
}  // namespace

// part: 3 regions of gridDim.x * CGS_MAXV doubles (first pass, second pass, norm), so that
// no region is overwritten while another block may still read it.
__global__ void __launch_bounds__(CGS_THREADS) k_cgs2(long long n, int nv, const double* __restrict__ V, long long ld,
                                                    double* __restrict__ w, double* __restrict__ part,
                                                    double* __restrict__ hcol, double* __restrict__ vnext,
                                                    unsigned* bar, int* err) {
  __shared__ double h[CGS_MAXV], h2[CGS_MAXV], red[CGS_THREADS / 32][8];
  __shared__ int sh_ok;
  __shared__ double nrm;
  const unsigned G = gridDim.x;
  const long long chunk = (n + G - 1) / G;
  const long long lo = (long long)blockIdx.x * chunk;
  const long long hi = lo + chunk < n ? lo + chunk : n;
  unsigned* count = bar;
  volatile unsigned* gen = bar + 1;
  const size_t region = (size_t)G * CGS_MAXV;
  for (int pass = 0; pass < 2; ++pass) {
    double* pp = part + pass * region;
    block_partials(lo, hi, nv, V, ld, w, pp + (size_t)blockIdx.x * nv, red);
    if (!grid_barrier(count, gen, G, err, &sh_ok)) return;
    double* hh = pass == 0 ? h : h2;
    sum_partials(pp, G, nv, hh);
    __syncthreads();
    for (long long r = lo + threadIdx.x; r < hi; r += CGS_THREADS) {
      double s = 0.0;
      for (int i = 0; i < nv; ++i) s += hh[i] * V[(size_t)i * ld + r];
      w[r] -= s;
    }
    __syncthreads();
  }
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < nv; i += CGS_THREADS) hcol[i] = h[i] + h2[i];
  double* pn = part + 2 * region;
  block_partials(lo, hi, 1, w, 0, w, pn + blockIdx.x, red);
  if (!grid_barrier(count, gen, G, err, &sh_ok)) return;
  sum_partials(pn, G, 1, &nrm);
  __syncthreads();
  if (threadIdx.x == 0) {
    nrm = sqrt(nrm);
    if (blockIdx.x == 0) hcol[nv] = nrm;
  }
  __syncthreads();
  const double inv = 1.0 / nrm;
  for (long long r = lo + threadIdx.x; r < hi; r += CGS_THREADS) vnext[r] = w[r] * inv;
}

int cgs2_scratch(int nblocks) { return 3 * nblocks * CGS_MAXV; }

int cgs2_max_vectors() { return CGS_MAXV; }

cudaError_t launch_cgs2(long long n, int nv, const double* V, long long ld, double* w, double* partial, double* hcol,
                        double* vnext, unsigned* bar, int* err, int nblocks, cudaStream_t st) {
  if (nv < 1 || nv > CGS_MAXV || nblocks < 1) return cudaErrorInvalidValue;
  void* args[] = {&n, &nv, &V, &ld, &w, &partial, &hcol, &vnext, &bar, &err};
  return cudaLaunchCooperativeKernel((const void*)k_cgs2, dim3(nblocks), dim3(CGS_THREADS), args, 0, st);
}

int cgs2_blocks(int n_sm) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cgs2, CGS_THREADS, 0) != cudaSuccess || per_sm < 1)
    return 0;
  int b = n_sm * (per_sm < 2 ? per_sm : 2);
  return b > 304 ? 304 : b;
}

// Coarse direct solve: x = G b, G column-major D x D in FP64; vectors of type T.
template <typename T>
__global__ void k_coarse(int D, const double* __restrict__ Gcm, const T* __restrict__ b, T* __restrict__ x) {
  extern __shared__ double bs[];
  for (int i = threadIdx.x; i < D; i += blockDim.x) bs[i] = (double)b[i];
  __syncthreads();
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < D; row += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < D; ++c) s += Gcm[(size_t)c * D + row] * bs[c];
    x[row] = (T)s;
  }
}

// Large coarse levels (D > 1024): tiles of 256 rows x 64 columns of G, four independent
// FP64 accumulators per row, partial products accumulated in FP64 (acc, zeroed first),
// then rounded to the vector type.  Enough tiles to cover every SM.
template <typename T>
__global__ void __launch_bounds__(256) k_coarse_tiled(int D, const double* __restrict__ Gcm,
                                                      const T* __restrict__ b, double* __restrict__ acc) {
  constexpr int CT = 64;
  __shared__ double bs[CT];
  const int c0 = blockIdx.y * CT;
  const int cn = min(CT, D - c0);
  if (threadIdx.x < CT) bs[threadIdx.x] = threadIdx.x < cn ? (double)b[c0 + threadIdx.x] : 0.0;
  __syncthreads();
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= D) return;
  const double* g = Gcm + (size_t)c0 * D + row;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int c = 0;
  for (; c + 4 <= cn; c += 4) {
    s0 += g[(size_t)c * D] * bs[c];
    s1 += g[(size_t)(c + 1) * D] * bs[c + 1];
    s2 += g[(size_t)(c + 2) * D] * bs[c + 2];
    s3 += g[(size_t)(c + 3) * D] * bs[c + 3];
  }
  for (; c < cn; ++c) s0 += g[(size_t)c * D] * bs[c];
  atomicAdd(acc + row, (s0 + s1) + (s2 + s3));
}

template <typename T>
__global__ void k_coarse_finish(int D, const double* __restrict__ acc, T* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < D) x[i] = (T)acc[i];
}

template <typename T>
cudaError_t launch_coarse_tiled(int D, const double* Gcm, const T* b, T* x, double* acc, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double) * D, st);
  if (e != cudaSuccess) return e;
  const int nr = (D + 255) / 256, nc = (D + 63) / 64;
  k_coarse_tiled<T><<<dim3(nr, nc), 256, 0, st>>>(D, Gcm, b, acc);
  k_coarse_finish<T><<<nr, 256, 0, st>>>(D, acc, x);
  return cudaGetLastError();
}
template cudaError_t launch_coarse_tiled<double>(int, const double*, const double*, double*, double*, cudaStream_t);
template cudaError_t launch_coarse_tiled<float>(int, const double*, const float*, float*, double*, cudaStream_t);

template <typename T>
cudaError_t launch_coarse(int D, const double* Gcm, const T* b, T* x, cudaStream_t st) {
  const int blocks = (D + 255) / 256;
  const size_t smem = sizeof(double) * (size_t)D;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_coarse<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_coarse<T><<<blocks, 256, smem, st>>>(D, Gcm, b, x);
  return cudaGetLastError();
}
template cudaError_t launch_coarse<double>(int, const double*, const double*, double*, cudaStream_t);
template cudaError_t launch_coarse<float>(int, const double*, const float*, float*, cudaStream_t);

}  // namespace stmg

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

// out = (To) in and zero = 0 in one pass (the V-cycle's right-hand side and its zero
// initial iterate on the finest level)
template <typename Ti, typename To>
__global__ void k_convert_zero(long long n, const Ti* __restrict__ in, To* __restrict__ out, To* __restrict__ zero) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    out[i] = (To)in[i];
    zero[i] = To(0);
  }
}

template <typename Ti, typename To>
cudaError_t launch_convert_zero(long long n, const Ti* in, To* out, To* zero, cudaStream_t st) {
  k_convert_zero<Ti, To><<<grid_for(n), 256, 0, st>>>(n, in, out, zero);
  return cudaGetLastError();
}
template cudaError_t launch_convert_zero<double, float>(long long, const double*, float*, float*, cudaStream_t);
template cudaError_t launch_convert_zero<double, double>(long long, const double*, double*, double*, cudaStream_t);

// zero up to ZeroList::MAX float vectors in one launch (the coarser levels' right-hand
// sides that the V-cycle's fused restrictions accumulate into)
__global__ void k_zero_many(ZeroList z) {
  long long total = 0;
  for (int s = 0; s < z.count; ++s) total += z.n[s];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    long long j = i;
    int s = 0;
    while (s + 1 < z.count && j >= z.n[s]) j -= z.n[s++];
    z.p[s][j] = 0.0f;
  }
}
cudaError_t launch_zero_many(const ZeroList& z, cudaStream_t st) {
  long long total = 0;
  for (int s = 0; s < z.count; ++s) total += z.n[s];
  if (total <= 0) return cudaSuccess;
  k_zero_many<<<grid_for(total), 256, 0, st>>>(z);
  return cudaGetLastError();
}

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
// At the sizes of one slab the step is bound by FP64 issue and memory latency, not by
// bandwidth: see the notes on the partial dot products below.
// ------------------------------------------------------------------------------------
namespace {
constexpr int CGS_THREADS = 512;
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

// FP64 instructions are the scarce resource of this step on GB300 (FP64 issues at about
// 1/64 of the FP32 rate), so the partial dot products spend none on absent vectors and
// reduce across lanes by a butterfly reduce-scatter (9 FP64 adds per lane for 8 sums,
// not 40 for eight shuffle trees).
constexpr int ROWS = 4;                // rows per thread per step, their loads issued together

// acc[i] += sum over this thread's rows in [lo, hi) of V_i(r) w(r), i < CNT.  w is read
// through L2 (__ldcg): it is rewritten inside the launch.  V is read-only here.
template <int CNT>
__device__ __forceinline__ void rows_dots(long long lo, long long hi, const double* __restrict__ V, long long ld,
                                          const double* w, double* acc) {
  for (long long r0 = lo + threadIdx.x; r0 < hi; r0 += ROWS * CGS_THREADS) {
    if (r0 + (long long)(ROWS - 1) * CGS_THREADS < hi) {
      double wr[ROWS], vv[CNT][ROWS];
#pragma unroll
      for (int u = 0; u < ROWS; ++u) {
        wr[u] = __ldcg(w + r0 + (long long)u * CGS_THREADS);
#pragma unroll
        for (int i = 0; i < CNT; ++i) vv[i][u] = V[(size_t)i * ld + r0 + (long long)u * CGS_THREADS];
      }
#pragma unroll
      for (int u = 0; u < ROWS; ++u)
#pragma unroll
        for (int i = 0; i < CNT; ++i) acc[i] += vv[i][u] * wr[u];
    } else {
      for (long long r = r0; r < hi; r += CGS_THREADS) {
        const double wr = __ldcg(w + r);
#pragma unroll
        for (int i = 0; i < CNT; ++i) acc[i] += V[(size_t)i * ld + r] * wr;
      }
    }
  }
}

// Butterfly reduce-scatter of eight per-lane values over a warp: returns, in every lane,
// the warp sum of value *vidx (lanes with lane % 4 == 0 hold distinct indices 0..7).
__device__ __forceinline__ double warp_reduce8(const double* acc, int lane, int* vidx) {
  const int u1 = (lane >> 4) & 1, u2 = (lane >> 3) & 1, u3 = (lane >> 2) & 1;
  double b[4], c[2];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double keep = u1 ? acc[4 + k] : acc[k], send = u1 ? acc[k] : acc[4 + k];
    b[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const double keep = u2 ? b[2 + k] : b[k], send = u2 ? b[k] : b[2 + k];
    c[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  const double keep = u3 ? c[1] : c[0], send = u3 ? c[0] : c[1];
  double d = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  d += __shfl_xor_sync(0xffffffffu, d, 2);
  d += __shfl_xor_sync(0xffffffffu, d, 1);
  *vidx = 4 * u1 + 2 * u2 + u3;
  return d;
}

// partial[blk * nv + i] = sum over rows [lo, hi) of V_i w, eight vectors per sweep over w
__device__ void block_partials(long long lo, long long hi, int nv, const double* __restrict__ V, long long ld,
                               const double* w, double* __restrict__ out, double (*red)[8]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int v0 = 0; v0 < nv; v0 += 8) {
    const int cnt = nv - v0 < 8 ? nv - v0 : 8;
    const double* Vg = V + (size_t)v0 * ld;
    double acc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = 0.0;
    switch (cnt) {
      case 1: rows_dots<1>(lo, hi, Vg, ld, w, acc); break;
      case 2: rows_dots<2>(lo, hi, Vg, ld, w, acc); break;
      case 3: rows_dots<3>(lo, hi, Vg, ld, w, acc); break;
      case 4: rows_dots<4>(lo, hi, Vg, ld, w, acc); break;
      case 5: rows_dots<5>(lo, hi, Vg, ld, w, acc); break;
      case 6: rows_dots<6>(lo, hi, Vg, ld, w, acc); break;
      case 7: rows_dots<7>(lo, hi, Vg, ld, w, acc); break;
      default: rows_dots<8>(lo, hi, Vg, ld, w, acc); break;
    }
    int vi;
    const double d = warp_reduce8(acc, lane, &vi);
    if ((lane & 3) == 0) red[wid][vi] = d;
    __syncthreads();
    if (threadIdx.x < cnt) {
      double t = 0.0;
      for (int q = 0; q < CGS_THREADS / 32; ++q) t += red[q][threadIdx.x];
      out[v0 + threadIdx.x] = t;
    }
    __syncthreads();
  }
}

// *out = sum over rows [lo, hi) of w(r)^2 (w read through L2, as above)
__device__ void block_norm_partial(long long lo, long long hi, const double* w, double* __restrict__ out,
                                   double (*red)[8]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double acc = 0.0;
  for (long long r = lo + threadIdx.x; r < hi; r += CGS_THREADS) {
    const double t = __ldcg(w + r);
    acc += t * t;
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if (lane == 0) red[wid][0] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < CGS_THREADS / 32; ++q) t += red[q][0];
    *out = t;
  }
  __syncthreads();
}

// out[i] = sum_bb part[bb * nv + i], i < nv: one warp per vector, lanes strided over the
// blocks with all of a lane's loads issued together (read through L2: other blocks wrote
// them in this launch), then a fixed shuffle tree (deterministic)
constexpr int PLANE = 10;              // partial sums per lane per step
__device__ void sum_partials(const double* part, unsigned G, int nv, double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = wid; i < nv; i += CGS_THREADS / 32) {
    double s = 0.0;
    for (unsigned b0 = lane; b0 < G; b0 += 32u * PLANE) {
      double t[PLANE];
#pragma unroll
      for (int u = 0; u < PLANE; ++u) {
        const unsigned bb = b0 + 32u * u;
        t[u] = bb < G ? __ldcg(part + (size_t)bb * nv + i) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < PLANE; ++u) s += t[u];
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) out[i] = s;
  }
}
}  // namespace

// part: 3 regions of gridDim.x * CGS_MAXV doubles (first pass, second pass, norm), so that
// no region is overwritten while another block may still read it.
__global__ void __launch_bounds__(CGS_THREADS) k_cgs2(long long n, int nv, const double* __restrict__ V, long long ld,
                                                    double* w, double* __restrict__ part,
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
  block_norm_partial(lo, hi, w, pn + blockIdx.x, red);
  if (!grid_barrier(count, gen, G, err, &sh_ok)) return;
  sum_partials(pn, G, 1, &nrm);
  __syncthreads();
  if (threadIdx.x == 0) {
    nrm = sqrt(nrm);
    if (blockIdx.x == 0) hcol[nv] = nrm;
    nrm = 1.0 / nrm;                  // one FP64 division per block, not per thread
  }
  __syncthreads();
  const double inv = nrm;
  for (long long r = lo + threadIdx.x; r < hi; r += CGS_THREADS) vnext[r] = w[r] * inv;
}

// ------------------------------------------------------------------------------------
// The same Arnoldi step with the block's rows of w held in registers from the first load
// to the normalisation (at most CGS_RPT rows per thread), for nv <= CGS_RV basis vectors.
// The update of each pass and the next pass's dot products share one load of V:
//   pass 1: h = V^T w                                   (V read once)
//   pass 2: w -= V h, then h2 = V^T w and ||w||^2       (V read once)
//   pass 3: v_next = (w - V h2) / ||w - V h2||          (V read once)
// with ||w - V h2||^2 = ||w||^2 - ||h2||^2, so two grid barriers instead of three; V is
// read three times instead of four, w once instead of five times, and w is never written
// back (the step's outputs are hcol and vnext).  Each thread owns the rows
// lo + threadIdx.x + u * CGS_THREADS, u < CGS_RPT, the rows the split form gives it.
// Every loop is unrolled over the compile-time vector count, so all U * NV loads of a row
// group are in flight together, and the updates' sums run as two interleaved chains.
// ------------------------------------------------------------------------------------
constexpr int CGS_RPT = 4;             // rows of w per thread held in registers
constexpr int CGS_RV = 16;             // largest basis size of the register form

template <int NV>
__device__ __forceinline__ void block_partials_reg(const double* acc, double* __restrict__ out, double (*red)[8]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int v0 = 0; v0 < NV; v0 += 8) {
    double a8[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a8[i] = v0 + i < NV ? acc[v0 + i] : 0.0;
    int vi;
    const double d = warp_reduce8(a8, lane, &vi);
    if ((lane & 3) == 0) red[wid][vi] = d;
    __syncthreads();
    if (threadIdx.x < NV - v0 && threadIdx.x < 8) {
      double t = 0.0;
      for (int q = 0; q < CGS_THREADS / 32; ++q) t += red[q][threadIdx.x];
      out[v0 + threadIdx.x] = t;
    }
    __syncthreads();
  }
}

template <int NV>
__global__ void __launch_bounds__(CGS_THREADS) k_cgs2r(long long n, const double* __restrict__ V, long long ld,
                                                     const double* __restrict__ w, double* __restrict__ part,
                                                     double* __restrict__ hcol, double* __restrict__ vnext,
                                                     float* __restrict__ vnext32, float* __restrict__ zero32,
                                                     unsigned* bar, int* err) {
  constexpr int U = NV <= 8 ? 4 : (NV <= 11 ? 2 : 1);   // rows whose V values are loaded together
  static_assert(CGS_RPT % U == 0, "row groups must tile the thread's rows");
  __shared__ double h[NV], h2[NV + 1], red[CGS_THREADS / 32][8];
  __shared__ int sh_ok;
  __shared__ double nrm;
  const unsigned G = gridDim.x;
  const long long chunk = (n + G - 1) / G;
  const long long lo = (long long)blockIdx.x * chunk;
  const long long hi = lo + chunk < n ? lo + chunk : n;
  unsigned* count = bar;
  volatile unsigned* gen = bar + 1;
  const size_t region = (size_t)G * CGS_MAXV;
  long long row[CGS_RPT];
  bool in[CGS_RPT];
  double wr[CGS_RPT];
#pragma unroll
  for (int u = 0; u < CGS_RPT; ++u) {
    row[u] = lo + threadIdx.x + (long long)u * CGS_THREADS;
    in[u] = row[u] < hi;
    wr[u] = in[u] ? w[row[u]] : 0.0;
  }
  auto load_group = [&](int u0, double (*vv)[NV]) {
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int i = 0; i < NV; ++i) vv[u][i] = in[u0 + u] ? __ldg(V + (size_t)i * ld + row[u0 + u]) : 0.0;
  };
  // pass 1
  double acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = 0.0;
#pragma unroll
  for (int u0 = 0; u0 < CGS_RPT; u0 += U) {
    double vv[U][NV];
    load_group(u0, vv);
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int i = 0; i < NV; ++i) acc[i] += vv[u][i] * wr[u0 + u];
  }
  block_partials_reg<NV>(acc, part + (size_t)blockIdx.x * NV, red);
  if (!grid_barrier(count, gen, G, err, &sh_ok)) return;
  sum_partials(part, G, NV, h);
  __syncthreads();
  // pass 2 (also ||w||^2 after the update, for the norm of pass 3's result)
  double acc2[NV + 1];
#pragma unroll
  for (int i = 0; i <= NV; ++i) acc2[i] = 0.0;
#pragma unroll
  for (int u0 = 0; u0 < CGS_RPT; u0 += U) {
    double vv[U][NV];
    load_group(u0, vv);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      double s0 = 0.0, s1 = 0.0;        // two chains: half the dependent FP64 latency
#pragma unroll
      for (int i = 0; i < NV; i += 2) {
        s0 += h[i] * vv[u][i];
        if (i + 1 < NV) s1 += h[i + 1] * vv[u][i + 1];
      }
      wr[u0 + u] -= s0 + s1;
#pragma unroll
      for (int i = 0; i < NV; ++i) acc2[i] += vv[u][i] * wr[u0 + u];
      acc2[NV] += wr[u0 + u] * wr[u0 + u];
    }
  }
  block_partials_reg<NV + 1>(acc2, part + region + (size_t)blockIdx.x * (NV + 1), red);
  if (!grid_barrier(count, gen, G, err, &sh_ok)) return;
  sum_partials(part + region, G, NV + 1, h2);
  __syncthreads();
  // the norm of w - V h2 without a third pass over the blocks: the columns of V are
  // orthonormal and h2 = V^T w, so ||w - V h2||^2 = ||w||^2 - ||h2||^2 (h2 is a rounding-
  // level correction after the first pass, so nothing cancels unless w itself vanishes)
  if (threadIdx.x == 0) {
    double hh = 0.0;
    for (int i = 0; i < NV; ++i) hh += h2[i] * h2[i];
    const double n2 = h2[NV] - hh;
    nrm = sqrt(n2 > 0.0 ? n2 : 0.0);
    if (blockIdx.x == 0) hcol[NV] = nrm;
    nrm = 1.0 / nrm;                  // one FP64 division per block, not per thread
  }
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < NV; i += CGS_THREADS) hcol[i] = h[i] + h2[i];
  __syncthreads();
  const double inv = nrm;
  // pass 3: w -= V h2, v_next = w / ||w||
#pragma unroll
  for (int u0 = 0; u0 < CGS_RPT; u0 += U) {
    double vv[U][NV];
    load_group(u0, vv);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      double s0 = 0.0, s1 = 0.0;
#pragma unroll
      for (int i = 0; i < NV; i += 2) {
        s0 += h2[i] * vv[u][i];
        if (i + 1 < NV) s1 += h2[i + 1] * vv[u][i + 1];
      }
      if (in[u0 + u]) {
        const double v = (wr[u0 + u] - (s0 + s1)) * inv;
        vnext[row[u0 + u]] = v;
        if (vnext32) {                  // the next FP32 V-cycle's right-hand side and zero iterate
          vnext32[row[u0 + u]] = (float)v;
          zero32[row[u0 + u]] = 0.0f;
        }
      }
    }
  }
}

template <int... I>
struct CgsTable {
  static inline const void* const fn[sizeof...(I)] = {(const void*)k_cgs2r<I + 1>...};
};
using CgsRegTable = CgsTable<0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15>;

// whether the register form takes nv vectors of n rows on nblocks blocks
bool cgs2_reg_ok(long long n, int nv, int nblocks) {
  const long long chunk = (n + nblocks - 1) / nblocks;
  return nv >= 1 && nv <= CGS_RV && chunk <= (long long)CGS_RPT * CGS_THREADS;
}

int cgs2_scratch(int nblocks) { return 3 * nblocks * CGS_MAXV; }

int cgs2_max_vectors() { return CGS_MAXV; }

cudaError_t launch_cgs2(long long n, int nv, const double* V, long long ld, double* w, double* partial, double* hcol,
                        double* vnext, float* vnext32, float* zero32, bool* wrote32, unsigned* bar, int* err,
                        int nblocks, bool reg, cudaStream_t st) {
  if (nv < 1 || nv > CGS_MAXV || nblocks < 1) return cudaErrorInvalidValue;
  if (wrote32) *wrote32 = false;
  if (reg && cgs2_reg_ok(n, nv, nblocks)) {
    const double* wc = w;
    if (wrote32) *wrote32 = vnext32 != nullptr;
    void* args[] = {&n, &V, &ld, &wc, &partial, &hcol, &vnext, &vnext32, &zero32, &bar, &err};
    return cudaLaunchCooperativeKernel(CgsRegTable::fn[nv - 1], dim3(nblocks), dim3(CGS_THREADS), args, 0, st);
  }
  void* args[] = {&n, &nv, &V, &ld, &w, &partial, &hcol, &vnext, &bar, &err};
  return cudaLaunchCooperativeKernel((const void*)k_cgs2, dim3(nblocks), dim3(CGS_THREADS), args, 0, st);
}

// One 512-thread block per SM: fewer partial sums for every block to reduce than with two
// 256-thread blocks per SM, measured 15-20 % faster per step at 3e5 rows.
int cgs2_blocks(int n_sm) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cgs2, CGS_THREADS, 0) != cudaSuccess || per_sm < 1)
    return 0;
  // the register form must fit one block per SM too
  for (int v = 0; v < CGS_RV; ++v) {
    per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, CgsRegTable::fn[v], CGS_THREADS, 0) != cudaSuccess ||
        per_sm < 1)
      return 0;
  }
  return n_sm > 304 ? 304 : n_sm;
}

// Coarse direct solve: x = G b, G column-major D x D, stored in FP64 (M = double) or, for
// the FP32 V-cycle, as its FP32 rounding (M = float); vectors of type T, products in M.
template <typename T, typename M>
__global__ void k_coarse(int D, const M* __restrict__ Gcm, const T* __restrict__ b, T* __restrict__ x) {
  extern __shared__ double bs[];
  for (int i = threadIdx.x; i < D; i += blockDim.x) bs[i] = (double)b[i];
  __syncthreads();
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < D; row += gridDim.x * blockDim.x) {
    M s = 0;
    for (int c = 0; c < D; ++c) s += Gcm[(size_t)c * D + row] * (M)bs[c];
    x[row] = (T)s;
  }
}

// Large coarse levels (D > 1024): tiles of 256 rows x 32 columns of G (enough tiles to
// cover every SM several times), all 32 loads of a thread issued before the products,
// eight independent accumulators per row, each tile's partial sum accumulated in FP64
// (acc, zeroed first), then rounded to the vector type.
template <typename T, typename M>
__global__ void __launch_bounds__(256) k_coarse_tiled(int D, const M* __restrict__ Gcm,
                                                      const T* __restrict__ b, double* __restrict__ acc) {
  constexpr int CT = 32;
  __shared__ M bs[CT];
  const int c0 = blockIdx.y * CT;
  const int cn = min(CT, D - c0);
  if (threadIdx.x < CT) bs[threadIdx.x] = threadIdx.x < cn ? (M)b[c0 + threadIdx.x] : M(0);
  __syncthreads();
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= D) return;
  const M* g = Gcm + (size_t)c0 * D + row;
  M s[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) s[i] = 0;
  if (cn == CT) {
    M v[CT];
#pragma unroll
    for (int c = 0; c < CT; ++c) v[c] = g[(size_t)c * D];
#pragma unroll
    for (int c = 0; c < CT; ++c) s[c & 7] += v[c] * bs[c];
  } else {
    for (int c = 0; c < cn; ++c) s[0] += g[(size_t)c * D] * bs[c];
  }
  atomicAdd(acc + row, (double)(((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]))));
}

// x = acc, and acc = 0 again for the next solve (acc is zeroed once when it is allocated)
template <typename T>
__global__ void k_coarse_finish(int D, double* __restrict__ acc, T* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < D) {
    x[i] = (T)acc[i];
    acc[i] = 0.0;
  }
}

// acc: D doubles, zero on entry (and on return)
template <typename T, typename M>
cudaError_t launch_coarse_tiled(int D, const M* Gcm, const T* b, T* x, double* acc, cudaStream_t st) {
  const int nr = (D + 255) / 256, nc = (D + 31) / 32;
  k_coarse_tiled<T, M><<<dim3(nr, nc), 256, 0, st>>>(D, Gcm, b, acc);
  k_coarse_finish<T><<<nr, 256, 0, st>>>(D, acc, x);
  return cudaGetLastError();
}
template cudaError_t launch_coarse_tiled<double, double>(int, const double*, const double*, double*, double*,
                                                         cudaStream_t);
template cudaError_t launch_coarse_tiled<float, double>(int, const double*, const float*, float*, double*,
                                                        cudaStream_t);
template cudaError_t launch_coarse_tiled<float, float>(int, const float*, const float*, float*, double*, cudaStream_t);

template <typename T, typename M>
cudaError_t launch_coarse(int D, const M* Gcm, const T* b, T* x, cudaStream_t st) {
  const int blocks = (D + 255) / 256;
  const size_t smem = sizeof(double) * (size_t)D;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_coarse<T, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_coarse<T, M><<<blocks, 256, smem, st>>>(D, Gcm, b, x);
  return cudaGetLastError();
}
template cudaError_t launch_coarse<double, double>(int, const double*, const double*, double*, cudaStream_t);
template cudaError_t launch_coarse<float, double>(int, const double*, const float*, float*, cudaStream_t);
template cudaError_t launch_coarse<float, float>(int, const float*, const float*, float*, cudaStream_t);

}  // namespace stmg

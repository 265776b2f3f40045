// Persistent multigrid kernel: the part of one V-cycle (Alg. 1 with the subroutines of
// App. B) that lies below the finest level, in a single launch.
//
// On the coarser levels every operation is a few microseconds of latency (a launch, a
// dependent load chain, a tail) for a fraction of a microsecond of bandwidth, and one
// V-cycle has about twenty of them.  Here one grid of persistent blocks (at most as many
// as are resident at once) runs them all as phases separated by grid-wide barriers:
//   down   per level: sweep on b (zero iterate), residual, restriction (next b, next x = 0)
//   coarse FP64 product with the bordered inverse (column tiles, FP64 accumulator)
//   up     per level: prolongation, residual, sweep
// with nu1 / nu2 smoothing steps.  Each phase loops its blocks of work over the grid
// ("virtual blocks"); the bodies are the ones of the standalone kernels (mg_device.cuh),
// reading what earlier phases wrote through L2.  The residual's velocity rows are
// scatter-added, so their zero fill rides along with the phase before it.
//
// Levels covered: 2D, Q2/P1 in space (r = 1), k + 1 <= 4, cell or vertex-star patches with
// B <= 256 (the default hierarchies below their p-coarsening); the finest level keeps one
// kernel per operation.  Every barrier wait is bounded: on expiry the block raises the
// device error flag and returns, and the host reports STMG_ERR_TIMEOUT.
#include <cuda_runtime.h>

#include "internal.h"
#include "mg_device.cuh"

namespace stmg {

namespace {

constexpr int PT = 256;                       // threads per block
constexpr long long PBAR_SPINS = 1LL << 22;   // about 0.3 s of waiting before giving up

// generation barrier over all blocks of the grid; false if the wait timed out
__device__ bool pbarrier(unsigned* count, volatile unsigned* gen, int* err, int* sh_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned my = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(count, 1u);
    bool ok = true;
    if (arrived == gridDim.x - 1) {
      *count = 0;
      __threadfence();
      atomicAdd((unsigned*)gen, 1u);
    } else {
      long long it = 0;
      while (*gen == my) {
        if (++it > PBAR_SPINS) { atomicExch(err, 3); ok = false; break; }
        __nanosleep(32);
      }
    }
    __threadfence();
    *sh_ok = ok ? 1 : 0;
  }
  __syncthreads();
  return *sh_ok != 0;
}

template <typename T> struct VecOf;
template <> struct VecOf<float> { using type = float4; static constexpr int W = 4; };
template <> struct VecOf<double> { using type = double2; static constexpr int W = 2; };

__device__ __forceinline__ float vdot(const float4& a, const float* r) {
  return a.x * r[0] + a.y * r[1] + a.z * r[2] + a.w * r[3];
}
__device__ __forceinline__ double vdot(const double2& a, const double* r) { return a.x * r[0] + a.y * r[1]; }

// Work items of the thread-indexed phases: warps interleaved over the blocks, so that the
// few warps of a small level run on as many SMs as they can instead of a block's worth of
// them queueing on one SM (their instruction chains, not bandwidth, bound those levels).
__device__ __forceinline__ long long item_first() {
  return ((long long)(threadIdx.x >> 5) * gridDim.x + blockIdx.x) * 32 + (threadIdx.x & 31);
}
__device__ __forceinline__ long long item_stride() { return (long long)gridDim.x * PT; }

template <typename T>
__device__ void zero_fill(T* p, long long n) {
  for (long long i = item_first(); i < n; i += item_stride()) p[i] = T(0);
}

// the level's operator tables into shared memory (the entries a Q2 level uses), so that the
// operator's coefficients are shared-memory operands rather than global loads
template <typename T>
__device__ void stage_apply_tables(const ApplyRegParams<T>& g, ApplyRegParams<T>* s) {
  const int t = threadIdx.x;
  if (t < 9) { s->M1[t] = g.M1[t]; s->K1[t] = g.K1[t]; }
  if (t < 2 * MAXNP * MAXNP) {
    const int d = t / (MAXNP * MAXNP), e = t % (MAXNP * MAXNP);
    s->FX[d][e] = g.FX[d][e];
    s->FY[d][e] = g.FY[d][e];
  }
  if (t < MAXKT * MAXKT) s->Kt[t] = g.Kt[t];
  if (t < MAXKT) { s->beta[t] = g.beta[t]; s->bscale[t] = g.bscale[t]; }
  if (t == 0) {
    s->n = g.n; s->G = g.G; s->kt = g.kt; s->npm = g.npm;
    s->n_nodes = g.n_nodes; s->n_vel = g.n_vel; s->n_pres = g.n_pres; s->hd = g.hd;
  }
  __syncthreads();
}

template <typename T>
__device__ void stage_transfer_tables(const TransferParams<T>& g, TransferParams<T>* s) {
  const int* src = reinterpret_cast<const int*>(&g);
  int* dst = reinterpret_cast<int*>(s);
  for (int i = threadIdx.x; i < (int)(sizeof(TransferParams<T>) / sizeof(int)); i += PT) dst[i] = src[i];
  __syncthreads();
}

// x += W res over all patches (Eq. vanka; rows carry omega / valence): ppb patches per
// virtual block, one row per thread, the patch residual gathered into rs first
template <typename T>
__device__ __noinline__ void phase_sweep(const MGLevelDesc<T>& L, const T* res, T* rs) {
  using V = typename VecOf<T>::type;
  constexpr int VW = VecOf<T>::W;
  const int B = L.B, Bc = L.Bc, ppb = L.ppb, nch = Bc / VW;
  const long long np = L.n_patches, nvb = (np + ppb - 1) / ppb;
  const int t = threadIdx.x, pl = t / B, j = t - pl * B;
  for (long long vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
    const long long p0 = vb * ppb;
    for (int e = t; e < ppb * Bc; e += PT) {
      const int q = e / Bc, i = e - q * Bc;
      const long long p = p0 + q;
      T v = 0;
      if (p < np && i < B) {
        const int g = __ldg(L.dofs + p * B + i);
        if (g >= 0) v = __ldcg(res + g);
      }
      rs[e] = v;
    }
    __syncthreads();
    const long long p = p0 + pl;
    if (pl < ppb && p < np) {
      const V* A = reinterpret_cast<const V*>(L.inv + (size_t)p * B * Bc) + j;
      const T* r = rs + pl * Bc;
      T acc0 = 0, acc1 = 0;
      int c = 0;
      for (; c + 4 <= nch; c += 4) {
        const V a0 = __ldg(A + (size_t)c * B), a1 = __ldg(A + (size_t)(c + 1) * B);
        const V a2 = __ldg(A + (size_t)(c + 2) * B), a3 = __ldg(A + (size_t)(c + 3) * B);
        acc0 += vdot(a0, r + c * VW) + vdot(a2, r + (c + 2) * VW);
        acc1 += vdot(a1, r + (c + 1) * VW) + vdot(a3, r + (c + 3) * VW);
      }
      for (; c < nch; ++c) acc0 += vdot(__ldg(A + (size_t)c * B), r + c * VW);
      const int g = __ldg(L.dofs + p * B + j);
      if (g >= 0) atomicAdd(L.x + g, acc0 + acc1);
    }
    __syncthreads();
  }
}

// r = b - S x on a Q2/P1 level (register-resident operator, velocity rows of r zero on entry)
template <typename T>
__device__ __noinline__ void phase_residual(const MGLevelDesc<T>& L, ApplyRegParams<T>* sp) {
  stage_apply_tables(L.rp, sp);
  const ApplyRegParams<T>& P = *sp;
  const long long tot = (long long)L.rp.n * L.rp.n * L.kt * 2;      // (cell, temporal dof, component)
  for (long long t = item_first(); t < tot; t += item_stride()) {
    switch (L.kt) {
      case 1: apply2d_reg_thread<T, 3, 1, true>(P, L.x, L.b, L.r, RESIDUAL, t); break;
      case 2: apply2d_reg_thread<T, 3, 2, true>(P, L.x, L.b, L.r, RESIDUAL, t); break;
      case 3: apply2d_reg_thread<T, 3, 3, true>(P, L.x, L.b, L.r, RESIDUAL, t); break;
      default: apply2d_reg_thread<T, 3, 4, true>(P, L.x, L.b, L.r, RESIDUAL, t); break;
    }
  }
}

// b_c = P^T src (and x_c = 0)
template <typename T>
__device__ __noinline__ void phase_restrict(const MGLevelDesc<T>& L, const T* src, const MGLevelDesc<T>& C, T* tsh,
                                            TransferParams<T>* sp) {
  stage_transfer_tables(L.tp, sp);
  const TransferParams<T>& P = *sp;
  const long long nvb = restrict_g_blocks(P);
  for (long long vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
    if (L.ht) restrict_g_block<T, 3, 3, 1, true>(P, src, C.b, C.x, vb, tsh);
    else restrict_g_block<T, 3, 3, 0, true>(P, src, C.b, C.x, vb, tsh);
  }
}

// x += P x_c
template <typename T>
__device__ __noinline__ void phase_prolongate(const MGLevelDesc<T>& L, const MGLevelDesc<T>& C,
                                              TransferParams<T>* sp) {
  stage_transfer_tables(L.tp, sp);
  const TransferParams<T>& P = *sp;
  const long long tot = prolongate_g_items(P);
  for (long long t = item_first(); t < tot; t += item_stride()) {
    if (L.ht) prolongate_g_thread<T, 3, 3, 1, true>(P, C.x, L.x, t);
    else prolongate_g_thread<T, 3, 3, 0, true>(P, C.x, L.x, t);
  }
}

// acc += G b over column tiles of 32 (FP64 bordered inverse, column-major); acc zero on entry
template <typename T>
__device__ __noinline__ void phase_coarse(const MGLevelDesc<T>& C, double* bs) {
  constexpr int CT = 32;
  const int D = C.D, nr = (D + PT - 1) / PT, nc = (D + CT - 1) / CT;
  const long long nvb = (long long)nr * nc;
  for (long long vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
    const int bx = (int)(vb % nr), by = (int)(vb / nr);
    const int c0 = by * CT, cn = min(CT, D - c0);
    if (threadIdx.x < CT) bs[threadIdx.x] = threadIdx.x < cn ? (double)__ldcg(C.b + c0 + threadIdx.x) : 0.0;
    __syncthreads();
    const int row = bx * PT + threadIdx.x;
    if (row < D) {
      const double* g = C.G + (size_t)c0 * D + row;
      double s[4] = {0.0, 0.0, 0.0, 0.0};
      if (cn == CT) {
        double v[CT];
#pragma unroll
        for (int c = 0; c < CT; ++c) v[c] = __ldg(g + (size_t)c * D);
#pragma unroll
        for (int c = 0; c < CT; ++c) s[c & 3] += v[c] * bs[c];
      } else {
        for (int c = 0; c < cn; ++c) s[0] += __ldg(g + (size_t)c * D) * bs[c];
      }
      atomicAdd(C.acc + row, (s[0] + s[1]) + (s[2] + s[3]));
    }
    __syncthreads();
  }
}

// x_c = acc (rounded to T), acc = 0 again for the next V-cycle
template <typename T>
__device__ __noinline__ void phase_finish(const MGLevelDesc<T>& C) {
  for (long long i = item_first(); i < C.D; i += item_stride()) {
    C.x[i] = (T)__ldcg(C.acc + i);
    C.acc[i] = 0.0;
  }
}

}  // namespace

template <typename T>
__global__ void __launch_bounds__(PT, 2) k_mg_persist(const MGLevelDesc<T>* __restrict__ Ld, int nl, int nu1, int nu2,
                                                   unsigned* bar, int* err) {
  // phases use one shared scratch at a time: the sweep's patch residuals, or a level's
  // operator tables, or its transfer tables (the barrier between phases separates them)
  constexpr size_t SCR = sizeof(T) * 1024 > sizeof(ApplyRegParams<T>)
                             ? (sizeof(T) * 1024 > sizeof(TransferParams<T>) ? sizeof(T) * 1024 : sizeof(TransferParams<T>))
                             : (sizeof(ApplyRegParams<T>) > sizeof(TransferParams<T>) ? sizeof(ApplyRegParams<T>)
                                                                                        : sizeof(TransferParams<T>));
  __shared__ __align__(16) unsigned char scratch[SCR];
  T* rs = reinterpret_cast<T*>(scratch);
  ApplyRegParams<T>* sap = reinterpret_cast<ApplyRegParams<T>*>(scratch);
  TransferParams<T>* stp = reinterpret_cast<TransferParams<T>*>(scratch);
  __shared__ T tsh[2 * PT];
  __shared__ double bs[32];
  __shared__ int sh_ok;
  unsigned* count = bar;
  volatile unsigned* gen = bar + 1;
#define STMG_SYNC() \
  if (!pbarrier(count, gen, err, &sh_ok)) return
  // ---- down
  for (int l = 0; l + 1 < nl; ++l) {
    const MGLevelDesc<T>& L = Ld[l];
    const long long nv = L.size;              // the residual is scatter-added: all of r zero first
    for (int it = 0; it < nu1; ++it) {
      if (it == 0) {
        phase_sweep(L, L.b, rs);                 // x = 0: the residual is b
      } else {
        phase_residual(L, sap);
        STMG_SYNC();
        phase_sweep(L, L.r, rs);
        STMG_SYNC();
      }
      zero_fill(L.r, nv);                        // r: scatter-added next
      STMG_SYNC();
    }
    if (nu1 > 0) {
      phase_residual(L, sap);
      STMG_SYNC();
      phase_restrict(L, L.r, Ld[l + 1], tsh, stp);    // next level: b = P^T r, x = 0
    } else {
      phase_restrict(L, L.b, Ld[l + 1], tsh, stp);    // no presmoothing: the residual is b
    }
    STMG_SYNC();
  }
  // ---- coarsest level: x = G b
  phase_coarse(Ld[nl - 1], bs);
  STMG_SYNC();
  phase_finish(Ld[nl - 1]);
  STMG_SYNC();
  // ---- up
  for (int l = nl - 2; l >= 0; --l) {
    const MGLevelDesc<T>& L = Ld[l];
    const long long nv = L.size;
    phase_prolongate(L, Ld[l + 1], stp);
    zero_fill(L.r, nv);
    STMG_SYNC();
    for (int it = 0; it < nu2; ++it) {
      phase_residual(L, sap);
      STMG_SYNC();
      phase_sweep(L, L.r, rs);
      if (it + 1 < nu2) {
        STMG_SYNC();
        zero_fill(L.r, nv);
      }
      if (l > 0 || it + 1 < nu2) STMG_SYNC();
    }
  }
#undef STMG_SYNC
}

// resident blocks per SM of the persistent kernel (at most 2; 0: not available)
template <typename T>
int mg_persist_blocks(int n_sm) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mg_persist<T>, PT, 0) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return 0;
  }
  (void)n_sm;
  return per_sm < 2 ? per_sm : 2;
}

template <typename T>
cudaError_t launch_mg_persist(const MGLevelDesc<T>* levels, int nl, int nu1, int nu2, unsigned* bar, int* err,
                              int nblocks, cudaStream_t st) {
  if (nl < 2 || nblocks < 1) return cudaErrorInvalidValue;
  k_mg_persist<T><<<nblocks, PT, 0, st>>>(levels, nl, nu1, nu2, bar, err);
  return cudaGetLastError();
}

template int mg_persist_blocks<float>(int);
template int mg_persist_blocks<double>(int);
template cudaError_t launch_mg_persist<float>(const MGLevelDesc<float>*, int, int, int, unsigned*, int*, int,
                                              cudaStream_t);
template cudaError_t launch_mg_persist<double>(const MGLevelDesc<double>*, int, int, int, unsigned*, int*, int,
                                               cudaStream_t);

}  // namespace stmg

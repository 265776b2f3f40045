// Grid transfers of the hp space-time multigrid (App. A: Eq. DefPrRe, DeftTps, DeftTrs,
// DefPrRer, DefPrRek, DefoTsl).  Prolongation is the canonical embedding of the coarse
// space-time function into the fine space; restriction is its transpose.
//
// One thread block handles `cpb` coarse cells.  Per coarse cell:
//   velocity  fine values at the ns^d fine nodes under the cell =
//             (P1 (x) P1 (x) P1) applied to the cell's coarse nodes, with
//             P1[s, j] = ell_j^coarse(position of fine node s) (h: two children, p: same
//             cell), after the temporal map Pt[af, ac] = phi_ac^coarse(t_af^fine);
//   pressure  h: per child o, the 1D child maps E^o[i', i] = int L_i((o+xi)/2) L_i'(xi);
//             p: Legendre modes are nested, so embedding pads and restriction truncates.
// Fine nodes on coarse-cell faces belong to several coarse cells: each cell contributes
// with weight 1/multiplicity and the contributions meet in atomics, which reproduces
// the global P and P^T exactly.  Boundary (Dirichlet) velocity entries are neither read
// nor written.
#include <cuda_runtime.h>

#include "internal.h"

namespace stmg {

namespace {

template <typename T>
__device__ __forceinline__ void coarse_cell(const TransferParams<T>& P, int c, int* cc) {
  cc[0] = c % P.nc;
  cc[1] = (c / P.nc) % P.nc;
  cc[2] = P.dim == 3 ? c / (P.nc * P.nc) : 0;
}

// global fine scalar node index and flags for span position (sx, sy, sz) of coarse cell cc
template <typename T>
__device__ __forceinline__ long long fine_node(const TransferParams<T>& P, const int* cc, int sx, int sy, int sz,
                                               bool* dir, int* mult) {
  const int s[3] = {sx, sy, sz};
  long long g = 0, stride = 1;
  bool d = false;
  int m = 1;
  for (int k = 0; k < P.dim; ++k) {
    const int gk = cc[k] * (P.ns - 1) + s[k];
    d = d || gk == 0 || gk == P.Gf - 1;
    if ((s[k] == 0 && cc[k] > 0) || (s[k] == P.ns - 1 && cc[k] < P.nc - 1)) m *= 2;
    g += gk * stride;
    stride *= P.Gf;
  }
  *dir = d;
  *mult = m;
  return g;
}

template <typename T>
__device__ __forceinline__ long long coarse_node(const TransferParams<T>& P, const int* cc, int jx, int jy, int jz,
                                                 bool* dir) {
  const int j[3] = {jx, jy, jz};
  long long g = 0, stride = 1;
  bool d = false;
  for (int k = 0; k < P.dim; ++k) {
    const int gk = cc[k] * (P.npc - 1) + j[k];
    d = d || gk == 0 || gk == P.Gc - 1;
    g += gk * stride;
    stride *= P.Gc;
  }
  *dir = d;
  return g;
}

// fine cell index of child o (bits per dimension) of coarse cell cc (h), or the same cell (p)
template <typename T>
__device__ __forceinline__ long long fine_cell(const TransferParams<T>& P, const int* cc, int o) {
  long long f = 0, stride = 1;
  for (int k = 0; k < P.dim; ++k) {
    const int fk = P.h_type ? 2 * cc[k] + ((o >> k) & 1) : cc[k];
    f += fk * stride;
    stride *= P.nf;
  }
  return f;
}

// pressure child map coefficient between fine mode mf and coarse mode mc for child o
template <typename T>
__device__ __forceinline__ T pres_map(const TransferParams<T>& P, int o, int mf, int mc) {
  if (P.h_type) {
    T v = 1;
    const int rc1 = P.rc + 1;
    for (int k = 0; k < P.dim; ++k) {
      const int ef = P.modes_f[mf][k], ec = P.modes_c[mc][k];
      if (ef > ec) return T(0);
      v *= P.E[(o >> k) & 1][ef * rc1 + ec];
    }
    return v;
  }
  for (int k = 0; k < 3; ++k)
    if (P.modes_f[mf][k] != P.modes_c[mc][k]) return T(0);
  return T(1);
}

}  // namespace

// x_f += P y_c
template <typename T>
__global__ void k_prolongate(const TransferParams<T> P, const T* __restrict__ yc, T* __restrict__ xf) {
  const int dim = P.dim, npc = P.npc, ns = P.ns, ktc = P.ktc, ktf = P.ktf;
  const int ncd = dim == 2 ? P.nc * P.nc : P.nc * P.nc * P.nc;
  const int c = blockIdx.x;
  if (c >= ncd) return;
  const int nqc = dim == 2 ? npc * npc : npc * npc * npc;
  const int nsd = dim == 2 ? ns * ns : ns * ns * ns;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* C0 = reinterpret_cast<T*>(smraw);       // [ktc][dim][nqc]
  T* C1 = C0 + ktc * dim * nqc;              // [ktf][dim][nqc]
  T* X1 = C1 + ktf * dim * nqc;              // [ktf][dim][ns^d] (pass buffers)
  T* X2 = X1 + ktf * dim * nsd;
  T* PC = X2 + ktf * dim * nsd;              // [ktc][npmc]
  T* PT = PC + ktc * P.npmc;                 // [ktf][npmc]
  int cc[3];
  coarse_cell(P, c, cc);
  for (int w = threadIdx.x; w < ktc * dim * nqc; w += blockDim.x) {
    const int node = w % nqc, t = w / nqc, comp = t % dim, a = t / dim;
    const int jx = node % npc, jy = (node / npc) % npc, jz = dim == 3 ? node / (npc * npc) : 0;
    bool dir;
    const long long g = coarse_node(P, cc, jx, jy, jz, &dir);
    C0[w] = dir ? T(0) : yc[a * P.nvc + comp * P.nnc + g];
  }
  for (int w = threadIdx.x; w < ktc * P.npmc; w += blockDim.x) {
    const int m = w % P.npmc, a = w / P.npmc;
    PC[w] = yc[(long long)ktc * P.nvc + a * P.npc_tot + (long long)c * P.npmc + m];
  }
  __syncthreads();
  for (int w = threadIdx.x; w < ktf * dim * nqc; w += blockDim.x) {
    const int r = w % (dim * nqc), af = w / (dim * nqc);
    T s = 0;
    for (int ac = 0; ac < ktc; ++ac) s += P.Pt[af * MAXKT + ac] * C0[ac * dim * nqc + r];
    C1[w] = s;
  }
  for (int w = threadIdx.x; w < ktf * P.npmc; w += blockDim.x) {
    const int m = w % P.npmc, af = w / P.npmc;
    T s = 0;
    for (int ac = 0; ac < ktc; ++ac) s += P.Pt[af * MAXKT + ac] * PC[ac * P.npmc + m];
    PT[w] = s;
  }
  __syncthreads();
  // x-pass: [.][jz][jy][jx] -> [.][jz][jy][sx]
  const int n1 = dim == 2 ? npc * ns : npc * npc * ns;
  for (int w = threadIdx.x; w < ktf * dim * n1; w += blockDim.x) {
    const int e = w % n1, t = w / n1;
    const int sx = e % ns, rest = e / ns;            // rest = jy + npc jz
    const T* src = C1 + t * nqc + rest * npc;
    T s = 0;
    for (int jx = 0; jx < npc; ++jx) s += P.P1[sx * MAXNP + jx] * src[jx];
    X1[t * nsd + e] = s;
  }
  __syncthreads();
  // y-pass: [.][jz][jy][sx] -> [.][jz][sy][sx]
  const int n2 = dim == 2 ? ns * ns : npc * ns * ns;
  for (int w = threadIdx.x; w < ktf * dim * n2; w += blockDim.x) {
    const int e = w % n2, t = w / n2;
    const int sx = e % ns, sy = (e / ns) % ns, jz = e / (ns * ns);
    const T* src = X1 + t * nsd + jz * npc * ns + sx;
    T s = 0;
    for (int jy = 0; jy < npc; ++jy) s += P.P1[sy * MAXNP + jy] * src[jy * ns];
    X2[t * nsd + e] = s;
  }
  __syncthreads();
  T* XF = X2;
  if (dim == 3) {
    // z-pass: [.][jz][sy][sx] -> [.][sz][sy][sx]
    for (int w = threadIdx.x; w < ktf * dim * nsd; w += blockDim.x) {
      const int e = w % nsd, t = w / nsd;
      const int sxy = e % (ns * ns), sz = e / (ns * ns);
      const T* src = X2 + t * nsd + sxy;
      T s = 0;
      for (int jz = 0; jz < npc; ++jz) s += P.P1[sz * MAXNP + jz] * src[jz * ns * ns];
      X1[t * nsd + e] = s;
    }
    __syncthreads();
    XF = X1;
  }
  for (int w = threadIdx.x; w < ktf * dim * nsd; w += blockDim.x) {
    const int e = w % nsd, t = w / nsd, comp = t % dim, af = t / dim;
    const int sx = e % ns, sy = (e / ns) % ns, sz = dim == 3 ? e / (ns * ns) : 0;
    bool dir;
    int mult;
    const long long g = fine_node(P, cc, sx, sy, sz, &dir, &mult);
    if (dir) continue;
    atomicAdd(xf + af * P.nvf + comp * P.nnf + g, XF[w] / T(mult));
  }
  const int nchild = P.h_type ? (1 << dim) : 1;
  for (int w = threadIdx.x; w < ktf * nchild * P.npmf; w += blockDim.x) {
    const int mf = w % P.npmf, t = w / P.npmf, o = t % nchild, af = t / nchild;
    T s = 0;
    for (int mc = 0; mc < P.npmc; ++mc) s += pres_map(P, o, mf, mc) * PT[af * P.npmc + mc];
    const long long fc = fine_cell(P, cc, o);
    xf[(long long)ktf * P.nvf + af * P.npf_tot + fc * P.npmf + mf] += s;
  }
}

// b_c = P^T r_f  (b_c must be zero on entry for the velocity part; pressure is stored)
template <typename T>
__global__ void k_restrict(const TransferParams<T> P, const T* __restrict__ rf, T* __restrict__ bc) {
  const int dim = P.dim, npc = P.npc, ns = P.ns, ktc = P.ktc, ktf = P.ktf;
  const int ncd = dim == 2 ? P.nc * P.nc : P.nc * P.nc * P.nc;
  const int c = blockIdx.x;
  if (c >= ncd) return;
  const int nqc = dim == 2 ? npc * npc : npc * npc * npc;
  const int nsd = dim == 2 ? ns * ns : ns * ns * ns;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* F0 = reinterpret_cast<T*>(smraw);       // [ktf][dim][nsd]
  T* F1 = F0 + ktf * dim * nsd;              // [ktf][dim][nsd]
  T* C1 = F1 + ktf * dim * nsd;              // [ktf][dim][nqc]
  T* PF = C1 + ktf * dim * nqc;              // [ktf][npmc]
  int cc[3];
  coarse_cell(P, c, cc);
  for (int w = threadIdx.x; w < ktf * dim * nsd; w += blockDim.x) {
    const int e = w % nsd, t = w / nsd, comp = t % dim, af = t / dim;
    const int sx = e % ns, sy = (e / ns) % ns, sz = dim == 3 ? e / (ns * ns) : 0;
    bool dir;
    int mult;
    const long long g = fine_node(P, cc, sx, sy, sz, &dir, &mult);
    F0[w] = dir ? T(0) : rf[af * P.nvf + comp * P.nnf + g] / T(mult);
  }
  // pressure: coarse mode mc at fine temporal dof af = sum_o sum_mf E(o, mf, mc) r_f
  const int nchild = P.h_type ? (1 << dim) : 1;
  for (int w = threadIdx.x; w < ktf * P.npmc; w += blockDim.x) {
    const int mc = w % P.npmc, af = w / P.npmc;
    T s = 0;
    for (int o = 0; o < nchild; ++o) {
      const long long fc = fine_cell(P, cc, o);
      const T* r = rf + (long long)ktf * P.nvf + af * P.npf_tot + fc * P.npmf;
      for (int mf = 0; mf < P.npmf; ++mf) s += pres_map(P, o, mf, mc) * r[mf];
    }
    PF[w] = s;
  }
  __syncthreads();
  if (dim == 3) {
    // z: [.][sz][sy][sx] -> [.][jz][sy][sx]
    for (int w = threadIdx.x; w < ktf * dim * npc * ns * ns; w += blockDim.x) {
      const int e = w % (npc * ns * ns), t = w / (npc * ns * ns);
      const int sxy = e % (ns * ns), jz = e / (ns * ns);
      const T* src = F0 + t * nsd + sxy;
      T s = 0;
      for (int sz = 0; sz < ns; ++sz) s += P.P1[sz * MAXNP + jz] * src[sz * ns * ns];
      F1[t * nsd + e] = s;
    }
    __syncthreads();
  }
  const T* FY = dim == 3 ? F1 : F0;
  T* FYo = dim == 3 ? F0 : F1;
  // y: [.][jz][sy][sx] -> [.][jz][jy][sx]
  const int ny = dim == 2 ? npc * ns : npc * npc * ns;
  for (int w = threadIdx.x; w < ktf * dim * ny; w += blockDim.x) {
    const int e = w % ny, t = w / ny;
    const int sx = e % ns, jy = (e / ns) % npc, jz = e / (ns * npc);
    const T* src = FY + t * nsd + jz * ns * ns + sx;
    T s = 0;
    for (int sy = 0; sy < ns; ++sy) s += P.P1[sy * MAXNP + jy] * src[sy * ns];
    FYo[t * nsd + e] = s;
  }
  __syncthreads();
  // x: [.][jz][jy][sx] -> [.][jz][jy][jx]
  for (int w = threadIdx.x; w < ktf * dim * nqc; w += blockDim.x) {
    const int e = w % nqc, t = w / nqc;
    const int jx = e % npc, rest = e / npc;
    const T* src = FYo + t * nsd + rest * ns;
    T s = 0;
    for (int sx = 0; sx < ns; ++sx) s += P.P1[sx * MAXNP + jx] * src[sx];
    C1[t * nqc + e] = s;
  }
  __syncthreads();
  for (int w = threadIdx.x; w < ktc * dim * nqc; w += blockDim.x) {
    const int node = w % nqc, t = w / nqc, comp = t % dim, ac = t / dim;
    const int jx = node % npc, jy = (node / npc) % npc, jz = dim == 3 ? node / (npc * npc) : 0;
    bool dir;
    const long long g = coarse_node(P, cc, jx, jy, jz, &dir);
    if (dir) continue;
    T s = 0;
    for (int af = 0; af < ktf; ++af) s += P.Pt[af * MAXKT + ac] * C1[(af * dim + comp) * nqc + node];
    atomicAdd(bc + ac * P.nvc + comp * P.nnc + g, s);
  }
  for (int w = threadIdx.x; w < ktc * P.npmc; w += blockDim.x) {
    const int mc = w % P.npmc, ac = w / P.npmc;
    T s = 0;
    for (int af = 0; af < ktf; ++af) s += P.Pt[af * MAXKT + ac] * PF[af * P.npmc + mc];
    bc[(long long)ktc * P.nvc + ac * P.npc_tot + (long long)c * P.npmc + mc] = s;
  }
}

template <typename T>
static size_t prolong_smem(const TransferParams<T>& p) {
  const int nqc = p.dim == 2 ? p.npc * p.npc : p.npc * p.npc * p.npc;
  const int nsd = p.dim == 2 ? p.ns * p.ns : p.ns * p.ns * p.ns;
  return sizeof(T) * ((size_t)p.ktc * p.dim * nqc + (size_t)p.ktf * p.dim * nqc + 2 * (size_t)p.ktf * p.dim * nsd +
                      (size_t)(p.ktc + p.ktf) * p.npmc);
}

template <typename T>
static size_t restrict_smem(const TransferParams<T>& p) {
  const int nqc = p.dim == 2 ? p.npc * p.npc : p.npc * p.npc * p.npc;
  const int nsd = p.dim == 2 ? p.ns * p.ns : p.ns * p.ns * p.ns;
  return sizeof(T) * (2 * (size_t)p.ktf * p.dim * nsd + (size_t)p.ktf * p.dim * nqc + (size_t)p.ktf * p.npmc);
}

template <typename T>
cudaError_t launch_prolongate(const TransferParams<T>& p, const T* yc, T* xf, cudaStream_t st) {
  const int ncd = p.dim == 2 ? p.nc * p.nc : p.nc * p.nc * p.nc;
  const size_t smem = prolong_smem(p);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_prolongate<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_prolongate<T><<<ncd, 128, smem, st>>>(p, yc, xf);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restrict(const TransferParams<T>& p, const T* rf, T* bc, cudaStream_t st) {
  const int ncd = p.dim == 2 ? p.nc * p.nc : p.nc * p.nc * p.nc;
  const size_t smem = restrict_smem(p);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_restrict<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_restrict<T><<<ncd, 128, smem, st>>>(p, rf, bc);
  return cudaGetLastError();
}

template cudaError_t launch_prolongate<double>(const TransferParams<double>&, const double*, double*, cudaStream_t);
template cudaError_t launch_prolongate<float>(const TransferParams<float>&, const float*, float*, cudaStream_t);
template cudaError_t launch_restrict<double>(const TransferParams<double>&, const double*, double*, cudaStream_t);
template cudaError_t launch_restrict<float>(const TransferParams<float>&, const float*, float*, cudaStream_t);

}  // namespace stmg

// Grid transfers of the hp space-time multigrid (App. A: Eq. DefPrRe, DeftTps, DeftTrs,
// DefPrRer, DefPrRek, DefoTsl).  Prolongation is the canonical embedding of the coarse
// space-time function into the fine space; restriction is its transpose.
//
// One thread block handles `cpb` coarse cells (every phase runs over cell x entry).
// Per coarse cell:
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
#include "mg_device.cuh"

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

}  // namespace

// x_f += P y_c; one block handles P.cpb coarse cells, every phase runs over (cell, entry)
template <typename T>
__global__ void k_prolongate(const TransferParams<T> P, const T* __restrict__ yc, T* __restrict__ xf) {
  const int dim = P.dim, npc = P.npc, ns = P.ns, ktc = P.ktc, ktf = P.ktf, cpb = P.cpb;
  const int ncd = dim == 2 ? P.nc * P.nc : P.nc * P.nc * P.nc;
  const int c0 = blockIdx.x * cpb;
  const int ncl = min(cpb, ncd - c0);
  if (ncl <= 0) return;
  const int nqc = dim == 2 ? npc * npc : npc * npc * npc;
  const int nsd = dim == 2 ? ns * ns : ns * ns * ns;
  const int s0 = ktc * dim * nqc, s1 = ktf * dim * nqc, sx = ktf * dim * nsd;
  const int sp0 = ktc * P.npmc, sp1 = ktf * P.npmc;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* C0 = reinterpret_cast<T*>(smraw);       // [cell][ktc][dim][nqc]
  T* C1 = C0 + cpb * s0;                     // [cell][ktf][dim][nqc]
  T* X1 = C1 + cpb * s1;                     // [cell][ktf][dim][ns^d] (pass buffers)
  T* X2 = X1 + cpb * sx;
  T* PC = X2 + cpb * sx;                     // [cell][ktc][npmc]
  T* PT = PC + cpb * sp0;                    // [cell][ktf][npmc]
  for (int w = threadIdx.x; w < ncl * s0; w += blockDim.x) {
    const int cl = w / s0, r = w % s0;
    const int node = r % nqc, t = r / nqc, comp = t % dim, a = t / dim;
    int cc[3];
    coarse_cell(P, c0 + cl, cc);
    const int jx = node % npc, jy = (node / npc) % npc, jz = dim == 3 ? node / (npc * npc) : 0;
    bool dir;
    const long long g = coarse_node(P, cc, jx, jy, jz, &dir);
    C0[w] = dir ? T(0) : yc[a * P.nvc + comp * P.nnc + g];
  }
  for (int w = threadIdx.x; w < ncl * sp0; w += blockDim.x) {
    const int cl = w / sp0, r = w % sp0;
    const int m = r % P.npmc, a = r / P.npmc;
    PC[w] = yc[(long long)ktc * P.nvc + a * P.npc_tot + (long long)(c0 + cl) * P.npmc + m];
  }
  __syncthreads();
  for (int w = threadIdx.x; w < ncl * s1; w += blockDim.x) {
    const int cl = w / s1, r = w % s1;
    const int q = r % (dim * nqc), af = r / (dim * nqc);
    T s = 0;
    for (int ac = 0; ac < ktc; ++ac) s += P.Pt[af * MAXKT + ac] * C0[cl * s0 + ac * dim * nqc + q];
    C1[w] = s;
  }
  for (int w = threadIdx.x; w < ncl * sp1; w += blockDim.x) {
    const int cl = w / sp1, r = w % sp1;
    const int m = r % P.npmc, af = r / P.npmc;
    T s = 0;
    for (int ac = 0; ac < ktc; ++ac) s += P.Pt[af * MAXKT + ac] * PC[cl * sp0 + ac * P.npmc + m];
    PT[w] = s;
  }
  __syncthreads();
  // x-pass: [.][jz][jy][jx] -> [.][jz][jy][sx]
  const int n1 = dim == 2 ? npc * ns : npc * npc * ns;
  const int kd = ktf * dim;
  for (int w = threadIdx.x; w < ncl * kd * n1; w += blockDim.x) {
    const int e = w % n1, t = w / n1;                // t = cl * kd + (af, comp)
    const int sxx = e % ns, rest = e / ns;
    const T* src = C1 + t * nqc + rest * npc;
    T s = 0;
    for (int jx = 0; jx < npc; ++jx) s += P.P1[sxx * MAXNP + jx] * src[jx];
    X1[t * nsd + e] = s;
  }
  __syncthreads();
  // y-pass: [.][jz][jy][sx] -> [.][jz][sy][sx]
  const int n2 = dim == 2 ? ns * ns : npc * ns * ns;
  for (int w = threadIdx.x; w < ncl * kd * n2; w += blockDim.x) {
    const int e = w % n2, t = w / n2;
    const int sxx = e % ns, sy = (e / ns) % ns, jz = e / (ns * ns);
    const T* src = X1 + t * nsd + jz * npc * ns + sxx;
    T s = 0;
    for (int jy = 0; jy < npc; ++jy) s += P.P1[sy * MAXNP + jy] * src[jy * ns];
    X2[t * nsd + e] = s;
  }
  __syncthreads();
  T* XF = X2;
  if (dim == 3) {
    // z-pass: [.][jz][sy][sx] -> [.][sz][sy][sx]
    for (int w = threadIdx.x; w < ncl * kd * nsd; w += blockDim.x) {
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
  for (int w = threadIdx.x; w < ncl * kd * nsd; w += blockDim.x) {
    const int e = w % nsd, t = w / nsd;
    const int cl = t / kd, tt = t % kd, comp = tt % dim, af = tt / dim;
    int cc[3];
    coarse_cell(P, c0 + cl, cc);
    const int sxx = e % ns, sy = (e / ns) % ns, sz = dim == 3 ? e / (ns * ns) : 0;
    bool dir;
    int mult;
    const long long g = fine_node(P, cc, sxx, sy, sz, &dir, &mult);
    if (dir) continue;
    atomicAdd(xf + af * P.nvf + comp * P.nnf + g, XF[w] / T(mult));
  }
  const int nchild = P.h_type ? (1 << dim) : 1;
  const int spf = ktf * nchild * P.npmf;
  for (int w = threadIdx.x; w < ncl * spf; w += blockDim.x) {
    const int cl = w / spf, r = w % spf;
    const int mf = r % P.npmf, t = r / P.npmf, o = t % nchild, af = t / nchild;
    int cc[3];
    coarse_cell(P, c0 + cl, cc);
    T s = 0;
    for (int mc = 0; mc < P.npmc; ++mc) s += pres_map(P, o, mf, mc) * PT[cl * sp1 + af * P.npmc + mc];
    const long long fc = fine_cell(P, cc, o);
    xf[(long long)ktf * P.nvf + af * P.npf_tot + fc * P.npmf + mf] += s;
  }
}

// b_c = P^T r_f (b_c must be zero on entry for the velocity part; pressure is stored)
template <typename T>
__global__ void k_restrict(const TransferParams<T> P, const T* __restrict__ rf, T* __restrict__ bc) {
  const int dim = P.dim, npc = P.npc, ns = P.ns, ktc = P.ktc, ktf = P.ktf, cpb = P.cpb;
  const int ncd = dim == 2 ? P.nc * P.nc : P.nc * P.nc * P.nc;
  const int c0 = blockIdx.x * cpb;
  const int ncl = min(cpb, ncd - c0);
  if (ncl <= 0) return;
  const int nqc = dim == 2 ? npc * npc : npc * npc * npc;
  const int nsd = dim == 2 ? ns * ns : ns * ns * ns;
  const int kd = ktf * dim;
  const int sf = kd * nsd, sc = kd * nqc, sp = ktf * P.npmc;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* F0 = reinterpret_cast<T*>(smraw);       // [cell][ktf][dim][nsd]
  T* F1 = F0 + cpb * sf;                     // [cell][ktf][dim][nsd]
  T* C1 = F1 + cpb * sf;                     // [cell][ktf][dim][nqc]
  T* PF = C1 + cpb * sc;                     // [cell][ktf][npmc]
  for (int w = threadIdx.x; w < ncl * sf; w += blockDim.x) {
    const int cl = w / sf, r = w % sf;
    const int e = r % nsd, t = r / nsd, comp = t % dim, af = t / dim;
    int cc[3];
    coarse_cell(P, c0 + cl, cc);
    const int sxx = e % ns, sy = (e / ns) % ns, sz = dim == 3 ? e / (ns * ns) : 0;
    bool dir;
    int mult;
    const long long g = fine_node(P, cc, sxx, sy, sz, &dir, &mult);
    F0[w] = dir ? T(0) : rf[af * P.nvf + comp * P.nnf + g] / T(mult);
  }
  // pressure: coarse mode mc at fine temporal dof af = sum_o sum_mf E(o, mf, mc) r_f
  const int nchild = P.h_type ? (1 << dim) : 1;
  for (int w = threadIdx.x; w < ncl * sp; w += blockDim.x) {
    const int cl = w / sp, r = w % sp;
    const int mc = r % P.npmc, af = r / P.npmc;
    int cc[3];
    coarse_cell(P, c0 + cl, cc);
    T s = 0;
    for (int o = 0; o < nchild; ++o) {
      const long long fc = fine_cell(P, cc, o);
      const T* rr = rf + (long long)ktf * P.nvf + af * P.npf_tot + fc * P.npmf;
      for (int mf = 0; mf < P.npmf; ++mf) s += pres_map(P, o, mf, mc) * rr[mf];
    }
    PF[w] = s;
  }
  __syncthreads();
  if (dim == 3) {
    // z: [.][sz][sy][sx] -> [.][jz][sy][sx]
    const int nz = npc * ns * ns;
    for (int w = threadIdx.x; w < ncl * kd * nz; w += blockDim.x) {
      const int e = w % nz, t = w / nz;
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
  for (int w = threadIdx.x; w < ncl * kd * ny; w += blockDim.x) {
    const int e = w % ny, t = w / ny;
    const int sxx = e % ns, jy = (e / ns) % npc, jz = e / (ns * npc);
    const T* src = FY + t * nsd + jz * ns * ns + sxx;
    T s = 0;
    for (int sy = 0; sy < ns; ++sy) s += P.P1[sy * MAXNP + jy] * src[sy * ns];
    FYo[t * nsd + e] = s;
  }
  __syncthreads();
  // x: [.][jz][jy][sx] -> [.][jz][jy][jx]
  for (int w = threadIdx.x; w < ncl * kd * nqc; w += blockDim.x) {
    const int e = w % nqc, t = w / nqc;
    const int jx = e % npc, rest = e / npc;
    const T* src = FYo + t * nsd + rest * ns;
    T s = 0;
    for (int sxx = 0; sxx < ns; ++sxx) s += P.P1[sxx * MAXNP + jx] * src[sxx];
    C1[t * nqc + e] = s;
  }
  __syncthreads();
  const int sco = ktc * dim * nqc;
  for (int w = threadIdx.x; w < ncl * sco; w += blockDim.x) {
    const int cl = w / sco, r = w % sco;
    const int node = r % nqc, t = r / nqc, comp = t % dim, ac = t / dim;
    int cc[3];
    coarse_cell(P, c0 + cl, cc);
    const int jx = node % npc, jy = (node / npc) % npc, jz = dim == 3 ? node / (npc * npc) : 0;
    bool dir;
    const long long g = coarse_node(P, cc, jx, jy, jz, &dir);
    if (dir) continue;
    T s = 0;
    for (int af = 0; af < ktf; ++af) s += P.Pt[af * MAXKT + ac] * C1[cl * sc + (af * dim + comp) * nqc + node];
    atomicAdd(bc + ac * P.nvc + comp * P.nnc + g, s);
  }
  const int spc = ktc * P.npmc;
  for (int w = threadIdx.x; w < ncl * spc; w += blockDim.x) {
    const int cl = w / spc, r = w % spc;
    const int mc = r % P.npmc, ac = r / P.npmc;
    T s = 0;
    for (int af = 0; af < ktf; ++af) s += P.Pt[af * MAXKT + ac] * PF[cl * sp + af * P.npmc + mc];
    bc[(long long)ktc * P.nvc + ac * P.npc_tot + (long long)(c0 + cl) * P.npmc + mc] = s;
  }
}

// Specialisations with the cell shape fixed at compile time (index arithmetic by
// constants); same arithmetic as the generic kernels.
template <typename T, int DIMc, int NPFc, int NPCc, int HTc>
__global__ void __launch_bounds__(512) k_prolongate_s(const TransferParams<T> P, const T* __restrict__ yc, T* __restrict__ xf) {
  constexpr int dim = DIMc, npc = NPCc, ns = HTc ? 2 * (NPFc - 1) + 1 : NPFc;
  const int ktc = P.ktc, ktf = P.ktf, cpb = P.cpb;
  const int ncd = dim == 2 ? P.nc * P.nc : P.nc * P.nc * P.nc;
  const int c0 = blockIdx.x * cpb;
  const int ncl = min(cpb, ncd - c0);
  if (ncl <= 0) return;
  constexpr int nqc = dim == 2 ? npc * npc : npc * npc * npc;
  constexpr int nsd = dim == 2 ? ns * ns : ns * ns * ns;
  const int s0 = ktc * dim * nqc, s1 = ktf * dim * nqc, sx = ktf * dim * nsd;
  const int sp0 = ktc * P.npmc, sp1 = ktf * P.npmc;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* C0 = reinterpret_cast<T*>(smraw);       // [cell][ktc][dim][nqc]
  T* C1 = C0 + cpb * s0;                     // [cell][ktf][dim][nqc]
  T* X1 = C1 + cpb * s1;                     // [cell][ktf][dim][ns^d] (pass buffers)
  T* X2 = X1 + cpb * sx;
  T* PC = X2 + cpb * sx;                     // [cell][ktc][npmc]
  T* PT = PC + cpb * sp0;                    // [cell][ktf][npmc]
  for (int w = threadIdx.x; w < ncl * s0; w += blockDim.x) {
    const int cl = w / s0, r = w % s0;
    const int node = r % nqc, t = r / nqc, comp = t % dim, a = t / dim;
    int cc[3];
    coarse_cell(P, c0 + cl, cc);
    const int jx = node % npc, jy = (node / npc) % npc, jz = dim == 3 ? node / (npc * npc) : 0;
    bool dir;
    const long long g = coarse_node(P, cc, jx, jy, jz, &dir);
    C0[w] = dir ? T(0) : yc[a * P.nvc + comp * P.nnc + g];
  }
  for (int w = threadIdx.x; w < ncl * sp0; w += blockDim.x) {
    const int cl = w / sp0, r = w % sp0;
    const int m = r % P.npmc, a = r / P.npmc;
    PC[w] = yc[(long long)ktc * P.nvc + a * P.npc_tot + (long long)(c0 + cl) * P.npmc + m];
  }
  __syncthreads();
  for (int w = threadIdx.x; w < ncl * s1; w += blockDim.x) {
    const int cl = w / s1, r = w % s1;
    const int q = r % (dim * nqc), af = r / (dim * nqc);
    T s = 0;
    for (int ac = 0; ac < ktc; ++ac) s += P.Pt[af * MAXKT + ac] * C0[cl * s0 + ac * dim * nqc + q];
    C1[w] = s;
  }
  for (int w = threadIdx.x; w < ncl * sp1; w += blockDim.x) {
    const int cl = w / sp1, r = w % sp1;
    const int m = r % P.npmc, af = r / P.npmc;
    T s = 0;
    for (int ac = 0; ac < ktc; ++ac) s += P.Pt[af * MAXKT + ac] * PC[cl * sp0 + ac * P.npmc + m];
    PT[w] = s;
  }
  __syncthreads();
  // x-pass: [.][jz][jy][jx] -> [.][jz][jy][sx]
  constexpr int n1 = dim == 2 ? npc * ns : npc * npc * ns;
  const int kd = ktf * dim;
  for (int w = threadIdx.x; w < ncl * kd * n1; w += blockDim.x) {
    const int e = w % n1, t = w / n1;                // t = cl * kd + (af, comp)
    const int sxx = e % ns, rest = e / ns;
    const T* src = C1 + t * nqc + rest * npc;
    T s = 0;
    _Pragma("unroll") for (int jx = 0; jx < npc; ++jx) s += P.P1[sxx * MAXNP + jx] * src[jx];
    X1[t * nsd + e] = s;
  }
  __syncthreads();
  // y-pass: [.][jz][jy][sx] -> [.][jz][sy][sx]
  constexpr int n2 = dim == 2 ? ns * ns : npc * ns * ns;
  for (int w = threadIdx.x; w < ncl * kd * n2; w += blockDim.x) {
    const int e = w % n2, t = w / n2;
    const int sxx = e % ns, sy = (e / ns) % ns, jz = e / (ns * ns);
    const T* src = X1 + t * nsd + jz * npc * ns + sxx;
    T s = 0;
    _Pragma("unroll") for (int jy = 0; jy < npc; ++jy) s += P.P1[sy * MAXNP + jy] * src[jy * ns];
    X2[t * nsd + e] = s;
  }
  __syncthreads();
  T* XF = X2;
  if (dim == 3) {
    // z-pass: [.][jz][sy][sx] -> [.][sz][sy][sx]
    for (int w = threadIdx.x; w < ncl * kd * nsd; w += blockDim.x) {
      const int e = w % nsd, t = w / nsd;
      const int sxy = e % (ns * ns), sz = e / (ns * ns);
      const T* src = X2 + t * nsd + sxy;
      T s = 0;
      _Pragma("unroll") for (int jz = 0; jz < npc; ++jz) s += P.P1[sz * MAXNP + jz] * src[jz * ns * ns];
      X1[t * nsd + e] = s;
    }
    __syncthreads();
    XF = X1;
  }
  for (int w = threadIdx.x; w < ncl * kd * nsd; w += blockDim.x) {
    const int e = w % nsd, t = w / nsd;
    const int cl = t / kd, tt = t % kd, comp = tt % dim, af = tt / dim;
    int cc[3];
    coarse_cell(P, c0 + cl, cc);
    const int sxx = e % ns, sy = (e / ns) % ns, sz = dim == 3 ? e / (ns * ns) : 0;
    bool dir;
    int mult;
    const long long g = fine_node(P, cc, sxx, sy, sz, &dir, &mult);
    if (dir) continue;
    atomicAdd(xf + af * P.nvf + comp * P.nnf + g, XF[w] / T(mult));
  }
  constexpr int nchild = HTc ? (1 << dim) : 1;
  const int spf = ktf * nchild * P.npmf;
  for (int w = threadIdx.x; w < ncl * spf; w += blockDim.x) {
    const int cl = w / spf, r = w % spf;
    const int mf = r % P.npmf, t = r / P.npmf, o = t % nchild, af = t / nchild;
    int cc[3];
    coarse_cell(P, c0 + cl, cc);
    T s = 0;
    for (int mc = 0; mc < P.npmc; ++mc) s += pres_map(P, o, mf, mc) * PT[cl * sp1 + af * P.npmc + mc];
    const long long fc = fine_cell(P, cc, o);
    xf[(long long)ktf * P.nvf + af * P.npf_tot + fc * P.npmf + mf] += s;
  }
}


template <typename T, int DIMc, int NPFc, int NPCc, int HTc>
__global__ void __launch_bounds__(512) k_restrict_s(const TransferParams<T> P, const T* __restrict__ rf, T* __restrict__ bc) {
  constexpr int dim = DIMc, npc = NPCc, ns = HTc ? 2 * (NPFc - 1) + 1 : NPFc;
  const int ktc = P.ktc, ktf = P.ktf, cpb = P.cpb;
  const int ncd = dim == 2 ? P.nc * P.nc : P.nc * P.nc * P.nc;
  const int c0 = blockIdx.x * cpb;
  const int ncl = min(cpb, ncd - c0);
  if (ncl <= 0) return;
  constexpr int nqc = dim == 2 ? npc * npc : npc * npc * npc;
  constexpr int nsd = dim == 2 ? ns * ns : ns * ns * ns;
  const int kd = ktf * dim;
  const int sf = kd * nsd, sc = kd * nqc, sp = ktf * P.npmc;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* F0 = reinterpret_cast<T*>(smraw);       // [cell][ktf][dim][nsd]
  T* F1 = F0 + cpb * sf;                     // [cell][ktf][dim][nsd]
  T* C1 = F1 + cpb * sf;                     // [cell][ktf][dim][nqc]
  T* PF = C1 + cpb * sc;                     // [cell][ktf][npmc]
  for (int w = threadIdx.x; w < ncl * sf; w += blockDim.x) {
    const int cl = w / sf, r = w % sf;
    const int e = r % nsd, t = r / nsd, comp = t % dim, af = t / dim;
    int cc[3];
    coarse_cell(P, c0 + cl, cc);
    const int sxx = e % ns, sy = (e / ns) % ns, sz = dim == 3 ? e / (ns * ns) : 0;
    bool dir;
    int mult;
    const long long g = fine_node(P, cc, sxx, sy, sz, &dir, &mult);
    F0[w] = dir ? T(0) : rf[af * P.nvf + comp * P.nnf + g] / T(mult);
  }
  // pressure: coarse mode mc at fine temporal dof af = sum_o sum_mf E(o, mf, mc) r_f
  constexpr int nchild = HTc ? (1 << dim) : 1;
  for (int w = threadIdx.x; w < ncl * sp; w += blockDim.x) {
    const int cl = w / sp, r = w % sp;
    const int mc = r % P.npmc, af = r / P.npmc;
    int cc[3];
    coarse_cell(P, c0 + cl, cc);
    T s = 0;
    for (int o = 0; o < nchild; ++o) {
      const long long fc = fine_cell(P, cc, o);
      const T* rr = rf + (long long)ktf * P.nvf + af * P.npf_tot + fc * P.npmf;
      for (int mf = 0; mf < P.npmf; ++mf) s += pres_map(P, o, mf, mc) * rr[mf];
    }
    PF[w] = s;
  }
  __syncthreads();
  if (dim == 3) {
    // z: [.][sz][sy][sx] -> [.][jz][sy][sx]
    constexpr int nz = npc * ns * ns;
    for (int w = threadIdx.x; w < ncl * kd * nz; w += blockDim.x) {
      const int e = w % nz, t = w / nz;
      const int sxy = e % (ns * ns), jz = e / (ns * ns);
      const T* src = F0 + t * nsd + sxy;
      T s = 0;
      _Pragma("unroll") for (int sz = 0; sz < ns; ++sz) s += P.P1[sz * MAXNP + jz] * src[sz * ns * ns];
      F1[t * nsd + e] = s;
    }
    __syncthreads();
  }
  const T* FY = dim == 3 ? F1 : F0;
  T* FYo = dim == 3 ? F0 : F1;
  // y: [.][jz][sy][sx] -> [.][jz][jy][sx]
  constexpr int ny = dim == 2 ? npc * ns : npc * npc * ns;
  for (int w = threadIdx.x; w < ncl * kd * ny; w += blockDim.x) {
    const int e = w % ny, t = w / ny;
    const int sxx = e % ns, jy = (e / ns) % npc, jz = e / (ns * npc);
    const T* src = FY + t * nsd + jz * ns * ns + sxx;
    T s = 0;
    _Pragma("unroll") for (int sy = 0; sy < ns; ++sy) s += P.P1[sy * MAXNP + jy] * src[sy * ns];
    FYo[t * nsd + e] = s;
  }
  __syncthreads();
  // x: [.][jz][jy][sx] -> [.][jz][jy][jx]
  for (int w = threadIdx.x; w < ncl * kd * nqc; w += blockDim.x) {
    const int e = w % nqc, t = w / nqc;
    const int jx = e % npc, rest = e / npc;
    const T* src = FYo + t * nsd + rest * ns;
    T s = 0;
    _Pragma("unroll") for (int sxx = 0; sxx < ns; ++sxx) s += P.P1[sxx * MAXNP + jx] * src[sxx];
    C1[t * nqc + e] = s;
  }
  __syncthreads();
  const int sco = ktc * dim * nqc;
  for (int w = threadIdx.x; w < ncl * sco; w += blockDim.x) {
    const int cl = w / sco, r = w % sco;
    const int node = r % nqc, t = r / nqc, comp = t % dim, ac = t / dim;
    int cc[3];
    coarse_cell(P, c0 + cl, cc);
    const int jx = node % npc, jy = (node / npc) % npc, jz = dim == 3 ? node / (npc * npc) : 0;
    bool dir;
    const long long g = coarse_node(P, cc, jx, jy, jz, &dir);
    if (dir) continue;
    T s = 0;
    for (int af = 0; af < ktf; ++af) s += P.Pt[af * MAXKT + ac] * C1[cl * sc + (af * dim + comp) * nqc + node];
    atomicAdd(bc + ac * P.nvc + comp * P.nnc + g, s);
  }
  const int spc = ktc * P.npmc;
  for (int w = threadIdx.x; w < ncl * spc; w += blockDim.x) {
    const int cl = w / spc, r = w % spc;
    const int mc = r % P.npmc, ac = r / P.npmc;
    T s = 0;
    for (int af = 0; af < ktf; ++af) s += P.Pt[af * MAXKT + ac] * PF[cl * sp + af * P.npmc + mc];
    bc[(long long)ktc * P.nvc + ac * P.npc_tot + (long long)(c0 + cl) * P.npmc + mc] = s;
  }
}

// ------------------------------------------------------------------------------------
// Gather form (2D): one thread per output value, no shared-memory phases, no atomics
// (bodies in mg_device.cuh, shared with the persistent multigrid kernel).  On the small
// levels the per-cell form is bound by the latency of its phases; this form is one phase.
// ------------------------------------------------------------------------------------
template <typename T, int NPF, int NPC, int HT>
__global__ void __launch_bounds__(256) k_prolongate_g(const TransferParams<T> P, const T* __restrict__ yc,
                                                      T* __restrict__ xf) {
  prolongate_g_thread<T, NPF, NPC, HT, false>(P, yc, xf, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

template <typename T, int NPF, int NPC, int HT>
__global__ void __launch_bounds__(256) k_restrict_g(const TransferParams<T> P, const T* __restrict__ rf,
                                                    T* __restrict__ bc, T* __restrict__ zc) {
  __shared__ T tsh[512];
  restrict_g_block<T, NPF, NPC, HT, false>(P, rf, bc, zc, blockIdx.x, tsh);
}

template <typename T>
size_t transfer_smem(const TransferParams<T>& p, int restrict_) {
  const int nqc = p.dim == 2 ? p.npc * p.npc : p.npc * p.npc * p.npc;
  const int nsd = p.dim == 2 ? p.ns * p.ns : p.ns * p.ns * p.ns;
  size_t per;
  if (!restrict_)
    per = (size_t)p.ktc * p.dim * nqc + (size_t)p.ktf * p.dim * nqc + 2 * (size_t)p.ktf * p.dim * nsd +
          (size_t)(p.ktc + p.ktf) * p.npmc;
  else
    per = 2 * (size_t)p.ktf * p.dim * nsd + (size_t)p.ktf * p.dim * nqc + (size_t)p.ktf * p.npmc;
  return sizeof(T) * per * (p.cpb > 0 ? p.cpb : 1);
}

template <typename T>
static int transfer_threads(const TransferParams<T>& p) {
  const int nsd = p.dim == 2 ? p.ns * p.ns : p.ns * p.ns * p.ns;
  int t = p.cpb * p.ktf * p.dim * nsd / 2;
  t = (t + 31) / 32 * 32;
  return t < 64 ? 64 : (t > 512 ? 512 : t);
}

template <typename K, typename T>
static cudaError_t launch_one(K kern, const TransferParams<T>& p, size_t smem, const T* in, T* out, cudaStream_t st) {
  const int ncd = p.dim == 2 ? p.nc * p.nc : p.nc * p.nc * p.nc;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<(ncd + p.cpb - 1) / p.cpb, transfer_threads(p), smem, st>>>(p, in, out);
  return cudaGetLastError();
}

// the (dim, fine nodes, coarse nodes, h/p) shapes of the default hierarchies
#define STMG_TRANSFER_SHAPES(X) \
  X(2, 4, 3, 0) X(2, 5, 3, 0) X(2, 6, 4, 0) X(2, 3, 3, 0) X(2, 3, 3, 1) \
  X(3, 4, 3, 0) X(3, 5, 3, 0) X(3, 6, 4, 0) X(3, 3, 3, 0) X(3, 3, 3, 1)
// the 2D shapes of the gather form
#define STMG_GATHER_SHAPES(X) X(4, 3, 0) X(5, 3, 0) X(6, 4, 0) X(3, 3, 0) X(3, 3, 1)

template <typename T>
bool transfer_gather_supported(const TransferParams<T>& p) {
  if (p.dim != 2 || 2 * p.ktf > 256 || p.ktc > p.ktf) return false;
#define STMG_G(F, C, H) if (p.npf == F && p.npc == C && p.h_type == H) return true;
  STMG_GATHER_SHAPES(STMG_G)
#undef STMG_G
  return false;
}

template <typename T>
cudaError_t launch_prolongate(const TransferParams<T>& p, const T* yc, T* xf, cudaStream_t st) {
  if (p.variant == 2 && transfer_gather_supported(p)) {
    const long long tot = prolongate_g_items(p);
    const unsigned blocks = (unsigned)((tot + 255) / 256);
#define STMG_PG(F, C, H) \
    if (p.npf == F && p.npc == C && p.h_type == H) { \
      k_prolongate_g<T, F, C, H><<<blocks, 256, 0, st>>>(p, yc, xf); \
      return cudaGetLastError(); \
    }
    STMG_GATHER_SHAPES(STMG_PG)
#undef STMG_PG
  }
  const size_t smem = transfer_smem(p, 0);
#define STMG_P(D, F, C, H) \
  if (p.dim == D && p.npf == F && p.npc == C && p.h_type == H) return launch_one(k_prolongate_s<T, D, F, C, H>, p, smem, yc, xf, st);
  STMG_TRANSFER_SHAPES(STMG_P)
#undef STMG_P
  return launch_one(k_prolongate<T>, p, smem, yc, xf, st);
}

// b_c = P^T r_f.  The per-cell form needs the velocity part of b_c zero on entry; the
// gather form writes all of b_c.
template <typename T>
cudaError_t launch_restrict(const TransferParams<T>& p, const T* rf, T* bc, T* zc, cudaStream_t st) {
  if (p.variant == 2 && transfer_gather_supported(p)) {
    const unsigned blocks = (unsigned)restrict_g_blocks(p);
#define STMG_RG(F, C, H) \
    if (p.npf == F && p.npc == C && p.h_type == H) { \
      k_restrict_g<T, F, C, H><<<blocks, 256, 0, st>>>(p, rf, bc, zc); \
      return cudaGetLastError(); \
    }
    STMG_GATHER_SHAPES(STMG_RG)
#undef STMG_RG
  }
  const size_t smem = transfer_smem(p, 1);
#define STMG_R(D, F, C, H) \
  if (p.dim == D && p.npf == F && p.npc == C && p.h_type == H) return launch_one(k_restrict_s<T, D, F, C, H>, p, smem, rf, bc, st);
  STMG_TRANSFER_SHAPES(STMG_R)
#undef STMG_R
  return launch_one(k_restrict<T>, p, smem, rf, bc, st);
}

template bool transfer_gather_supported<double>(const TransferParams<double>&);
template bool transfer_gather_supported<float>(const TransferParams<float>&);
template size_t transfer_smem<double>(const TransferParams<double>&, int);
template size_t transfer_smem<float>(const TransferParams<float>&, int);
template cudaError_t launch_prolongate<double>(const TransferParams<double>&, const double*, double*, cudaStream_t);
template cudaError_t launch_prolongate<float>(const TransferParams<float>&, const float*, float*, cudaStream_t);
template cudaError_t launch_restrict<double>(const TransferParams<double>&, const double*, double*, double*,
                                            cudaStream_t);
template cudaError_t launch_restrict<float>(const TransferParams<float>&, const float*, float*, float*, cudaStream_t);

}  // namespace stmg

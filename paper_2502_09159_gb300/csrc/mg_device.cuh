// Device bodies shared by the one-kernel-per-operation path and the persistent multigrid
// kernel (k_mg_persist.cu): the register-resident 2D operator and the gather-form grid
// transfers of 2D levels.
//
// Each body takes the index of its thread (or of its block) explicitly, so that a launch
// with one block per work item and a persistent launch looping over the items run the same
// code.  Template flag CG: the vectors that the persistent kernel itself wrote earlier in
// the same launch (iterates, residuals, right-hand sides) are read through L2 (ld.global.cg),
// never from a possibly stale L1 line of another phase; the standalone kernels read them
// through the read-only path.  Tables, inverses and patch lists are read-only everywhere.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace stmg {

template <bool CG, typename T>
__device__ __forceinline__ T ldv(const T* p) {
  if (CG) return __ldcg(p);
  return __ldg(p);
}

template <typename T>
__device__ __forceinline__ T pres_map(const TransferParams<T>& P, int o, int mf, int mc);

// ------------------------------------------------------------------------------------
// Register-resident 2D operator (Sec. 4.5): thread t -> (temporal dof a, velocity
// component d, cell c), cells fastest, so that a warp covers consecutive cells of one
// (a, d) and its loads are unit-stride runs.  See k_apply2d_reg.cu for the arithmetic.
// Every row of y is scatter-added (y zero on entry): the velocity rows of component d by
// the cells holding the node, the pressure rows of a cell by its two component threads
// (continuity is a sum over the components).
//
// With NPC > 0 (single precision, RESIDUAL mode) the thread first prolongates the coarser
// level's correction ec onto its cell (App. A: the coarse function of NPC x NPC nodes per
// coarse cell evaluated at the fine nodes, HT = 1 for a coarse cell of 2 x 2 fine cells,
// combined in time with the temporal map; the pressure through the child map), forms
// x2 = x + P ec on the fly, computes r = b - S x2 from it, and writes x2 (each velocity
// node by the thread of its owner cell with a equal to the node's temporal dof, each
// pressure dof by the d = 0 thread).  x is only read, so the cells sharing a node all see
// the old value.
//
// With RST (single precision, RESIDUAL mode) the thread restricts its cell's residual to
// the coarser level instead of scattering it (App. A: P^T, the transpose of the same
// interpolation): the residual rows of the cell's non-Dirichlet nodes, b through the
// owner cell, times the coarse basis functions of the parent cell at those nodes and the
// temporal map, are added to bc (zero on entry) at the parent's non-Dirichlet coarse
// nodes; the pressure rows through the child map.  The sum over the cells sharing a fine
// node is the node's full residual, so bc = P^T (b - S x).  The (0, 0) child of each
// coarse cell also zeroes the coarse iterate xc at the coarse dofs the coarse cell owns.
// ------------------------------------------------------------------------------------
template <typename T, int NP, int KT, bool CG, int NPC = 0, int HT = 0, bool RST = false>
__device__ __forceinline__ void apply2d_reg_thread(const ApplyRegParams<T>& P, const T* __restrict__ x,
                                                   const T* __restrict__ b, T* __restrict__ y, int mode,
                                                   long long t, const TransferParams<T>* tp = nullptr,
                                                   const T* __restrict__ ec = nullptr, T* __restrict__ x2 = nullptr,
                                                   T* __restrict__ bc = nullptr, T* __restrict__ xc = nullptr) {
  constexpr bool PRO = NPC > 0 && !RST;
  static_assert(NPC > 0 || !RST, "the fused restriction needs the coarse shape");
  static_assert(NPC == 0 || sizeof(T) == 4, "the fused transfers are a single-precision path");
  constexpr int E = NP - 1, NQ = NP * NP;
  constexpr int NPM = NP * (NP - 1) / 2;            // C(r + 2, 2) pressure modes, r = NP - 2
  const int n = P.n, G = P.G;
  const long long ncells = (long long)n * n;
  if (t >= ncells * KT * 2) return;
  const long long ad = t / ncells;
  const long long c = t - ad * ncells;
  const int a = (int)(ad >> 1), d = (int)(ad & 1);
  const int cx = (int)(c % n), cy = (int)(c / n);
  const long long nvel = P.n_vel, nnod = P.n_nodes;
  const long long poff = (long long)KT * nvel;
  const bool res = mode == RESIDUAL || mode == LIFT;
  const bool lift = mode == LIFT;
  const bool tr = mode == APPLY_T;
  const long long base = (long long)(cy * E) * G + cx * E;      // global index of the cell's node (0, 0)
  // boundary lines of the cell's nodes (the mesh boundary crosses a cell only at its outer lines)
  const bool bx0 = cx == 0, bx1 = cx == n - 1, by0 = cy == 0, by1 = cy == n - 1;
  const T* fx = &P.FX[d][0];                        // [ex * NP + ix]: B_h factor along x of component d
  const T* fy = &P.FY[d][0];                        // [ey * NP + iy]: along y

  // the prolongated coarse correction at this cell's nodes, component d, every temporal dof
  T pe[PRO ? KT : 1][PRO ? NQ : 1];
  if constexpr (PRO) {
    const TransferParams<T>& Q = *tp;
    const int Gc = Q.Gc, ccx = HT ? cx >> 1 : cx, ccy = HT ? cy >> 1 : cy;
    const int ox = HT ? (cx & 1) * (NP - 1) : 0, oy = HT ? (cy & 1) * (NP - 1) : 0;
    T ct[KT][NPC * NPC];                            // coarse nodal values, combined in time
#pragma unroll
    for (int bb = 0; bb < KT; ++bb)
#pragma unroll
      for (int q = 0; q < NPC * NPC; ++q) ct[bb][q] = 0;
    const T* src = ec + d * Q.nnc + (long long)(ccy * (NPC - 1)) * Gc + ccx * (NPC - 1);
#pragma unroll
    for (int ac = 0; ac < KT; ++ac) {
      if (ac < Q.ktc) {
        T cv[NPC * NPC];
#pragma unroll
        for (int jy = 0; jy < NPC; ++jy)
#pragma unroll
          for (int jx = 0; jx < NPC; ++jx) {
            const int Jx = ccx * (NPC - 1) + jx, Jy = ccy * (NPC - 1) + jy;
            const bool dirc = Jx == 0 || Jx == Gc - 1 || Jy == 0 || Jy == Gc - 1;
            cv[jy * NPC + jx] = dirc ? T(0) : ldv<CG>(src + ac * Q.nvc + (long long)jy * Gc + jx);
          }
#pragma unroll
        for (int bb = 0; bb < KT; ++bb) {
          const T w = Q.Pt[bb * MAXKT + ac];
#pragma unroll
          for (int q = 0; q < NPC * NPC; ++q) ct[bb][q] += w * cv[q];
        }
      }
    }
    T wx[NP][NPC], wy[NP][NPC];
#pragma unroll
    for (int i = 0; i < NP; ++i)
#pragma unroll
      for (int j = 0; j < NPC; ++j) {
        wx[i][j] = Q.P1[(ox + i) * MAXNP + j];
        wy[i][j] = Q.P1[(oy + i) * MAXNP + j];
      }
#pragma unroll
    for (int bb = 0; bb < KT; ++bb) {
      T tx[NPC][NP];                                // along x first, then along y
#pragma unroll
      for (int jy = 0; jy < NPC; ++jy)
#pragma unroll
        for (int ix = 0; ix < NP; ++ix) {
          T s = 0;
#pragma unroll
          for (int jx = 0; jx < NPC; ++jx) s += wx[ix][jx] * ct[bb][jy * NPC + jx];
          tx[jy][ix] = s;
        }
#pragma unroll
      for (int iy = 0; iy < NP; ++iy)
#pragma unroll
        for (int ix = 0; ix < NP; ++ix) {
          T s = 0;
#pragma unroll
          for (int jy = 0; jy < NPC; ++jy) s += wy[iy][jy] * tx[jy][ix];
          pe[bb][iy * NP + ix] = s;
        }
    }
  }

  T ut[NQ], ua[NQ], p[NPM];
#pragma unroll
  for (int q = 0; q < NQ; ++q) { ut[q] = 0; ua[q] = 0; }
  T kt_row[KT];
#pragma unroll
  for (int bb = 0; bb < KT; ++bb) kt_row[bb] = tr ? P.Kt[bb * MAXKT + a] : P.Kt[a * MAXKT + bb];
  // the KT slices of the thread's component: in single precision all loads at once; in
  // double precision slice by slice (the registers of all KT slices at once would spill)
  auto slice = [&](int bb) {
    const T* xb = x + bb * nvel + d * nnod + base;
    const T kb = kt_row[bb];
#pragma unroll
    for (int iy = 0; iy < NP; ++iy) {
      const bool dy = (iy == 0 && by0) || (iy == E && by1);
#pragma unroll
      for (int ix = 0; ix < NP; ++ix) {
        const bool dir = dy || (ix == 0 && bx0) || (ix == E && bx1);
        const bool take = lift ? dir : !dir;
        T v = take ? ldv<CG>(xb + iy * G + ix) : T(0);
        if constexpr (PRO) {
          if (!dir) v += pe[bb % KT][iy * NP + ix];
          const bool own = (iy < E || by1) && (ix < E || bx1);
          if (own && bb == a) x2[bb * nvel + d * nnod + base + iy * G + ix] = dir ? ldv<CG>(xb + iy * G + ix) : v;
        }
        ut[iy * NP + ix] += kb * v;
        if (bb == a) ua[iy * NP + ix] = v;
      }
    }
  };
  if (sizeof(T) == 4) {
#pragma unroll
    for (int bb = 0; bb < KT; ++bb) slice(bb);
  } else {
#pragma unroll 1
    for (int bb = 0; bb < KT; ++bb) slice(bb);
  }
#pragma unroll
  for (int m = 0; m < NPM; ++m) p[m] = lift ? T(0) : ldv<CG>(x + poff + (long long)a * P.n_pres + c * NPM + m);
  if constexpr (PRO) {
    // the parent cell's pressure modes through the child map, combined in time
    const TransferParams<T>& Q = *tp;
    constexpr int NPMC = NPC * (NPC - 1) / 2;
    const int o = HT ? ((cx & 1) | ((cy & 1) << 1)) : 0;
    const long long cc = HT ? (long long)(cy >> 1) * Q.nc + (cx >> 1) : c;
    T pc[NPMC];
#pragma unroll
    for (int mc = 0; mc < NPMC; ++mc) pc[mc] = 0;
#pragma unroll
    for (int ac = 0; ac < KT; ++ac)
      if (ac < Q.ktc) {
        const T w = Q.Pt[a * MAXKT + ac];
        const T* srcp = ec + (long long)Q.ktc * Q.nvc + ac * Q.npc_tot + cc * NPMC;
#pragma unroll
        for (int mc = 0; mc < NPMC; ++mc) pc[mc] += w * ldv<CG>(srcp + mc);
      }
#pragma unroll
    for (int m = 0; m < NPM; ++m) {
      T s = 0;
#pragma unroll
      for (int mc = 0; mc < NPMC; ++mc) s += pres_map(Q, o, m, mc) * pc[mc];
      p[m] += s;
      if (d == 0) x2[poff + (long long)a * P.n_pres + c * NPM + m] = p[m];
    }
  }
  // the right-hand side rows this thread adds b to (residual / lift): loaded with x in
  // single precision (latency bound); in double precision the registers are scarcer and the
  // FP64 arithmetic hides the later loads
  constexpr bool HOIST_B = sizeof(T) == 4;
  T bv[HOIST_B ? NQ : 1], bp[HOIST_B ? NPM : 1];
  const T* bd = b + a * nvel + d * nnod + base;
  if (HOIST_B) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int iy = q / NP, i = q % NP;
      const bool own = (iy < E || by1) && (i < E || bx1);
      bv[q] = own && res ? ldv<CG>(bd + (long long)iy * G + i) : T(0);
    }
#pragma unroll
    for (int m = 0; m < NPM; ++m) bp[m] = res && d == 0 ? ldv<CG>(b + poff + (long long)a * P.n_pres + c * NPM + m) : T(0);
  }
  auto bvel = [&](int iy, int i) -> T { return HOIST_B ? bv[(iy * NP + i) % (HOIST_B ? NQ : 1)] : ldv<CG>(bd + (long long)iy * G + i); };
  auto bpre = [&](int m) -> T {
    return HOIST_B ? bp[m % (HOIST_B ? NPM : 1)] : ldv<CG>(b + poff + (long long)a * P.n_pres + c * NPM + m);
  };
  const T beta = P.beta[a], bsc = P.bscale[a], hd = P.hd;
  // continuity rows: this component's share, sum-factorised over the modes (ex, ey) of
  // degree ex + ey <= R: cont[m(ex, ey)] = sum_iy fy[ey][iy] sum_ix fx[ex][ix] ua[iy][ix]
  constexpr int R = NP - 2;
  T cont[NPM];
  {
    T tx[R + 1][NP];
#pragma unroll
    for (int ex = 0; ex <= R; ++ex)
#pragma unroll
      for (int iy = 0; iy < NP; ++iy) {
        T s = 0;
#pragma unroll
        for (int ix = 0; ix < NP; ++ix) s += fx[ex * NP + ix] * ua[iy * NP + ix];
        tx[ex][iy] = s;
      }
#pragma unroll
    for (int ex = 0; ex <= R; ++ex)
#pragma unroll
      for (int ey = 0; ey <= R - ex; ++ey) {
        T s = 0;
#pragma unroll
        for (int iy = 0; iy < NP; ++iy) s += fy[ey * NP + iy] * tx[ex][iy];
        cont[mode_index(ex, ey)] = s;
      }
  }
  // pressure gradient factor: sp[ex][iy] = sum_ey fy[ey][iy] p[m(ex, ey)], so that the
  // B_h^T term of node (iy, ix) is sum_ex fx[ex][ix] sp[ex][iy]
  T sp[R + 1][NP];
#pragma unroll
  for (int ex = 0; ex <= R; ++ex)
#pragma unroll
    for (int iy = 0; iy < NP; ++iy) {
      T s = 0;
#pragma unroll
      for (int ey = 0; ey <= R - ex; ++ey) s += fy[ey * NP + iy] * p[mode_index(ex, ey)];
      sp[ex][iy] = s;
    }
  // y-pass: A1 = hd M1y ut + beta K1y ua, A2 = M1y ua (column by column)
  T A1[NQ], A2[NQ];
#pragma unroll
  for (int ix = 0; ix < NP; ++ix) {
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      T m1 = 0, k1 = 0, m2 = 0;
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        m1 += P.M1[i * NP + j] * ut[j * NP + ix];
        k1 += P.K1[i * NP + j] * ua[j * NP + ix];
        m2 += P.M1[i * NP + j] * ua[j * NP + ix];
      }
      A1[i * NP + ix] = hd * m1 + beta * k1;
      A2[i * NP + ix] = m2;
    }
  }
  // x-pass, pressure gradient, scatter (row by row)
  T* yd = y + a * nvel + d * nnod + base;
  const T* xd = x + a * nvel + d * nnod + base;
  T rl[RST ? NQ : 1];                               // RST: the cell's residual rows, slice a
#pragma unroll
  for (int iy = 0; iy < NP; ++iy) {
    const bool dy = (iy == 0 && by0) || (iy == E && by1);
    const bool oy = iy < E || by1;                      // this cell owns the node row (for boundary rows)
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      const bool dir = dy || (i == 0 && bx0) || (i == E && bx1);
      const bool own = oy && (i < E || bx1);
      const long long off = (long long)iy * G + i;
      if (dir) {
        if constexpr (RST) {
          rl[(iy * NP + i) % (RST ? NQ : 1)] = T(0);   // the restriction reads no fine Dirichlet row
        } else if (own) {
          const T xv = ldv<CG>(xd + off);
          atomicAdd(yd + off, mode == RESIDUAL ? bvel(iy, i) - xv : xv);   // identity row, by its owner
        }
        continue;
      }
      T m1 = 0, k1 = 0;
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        m1 += P.M1[i * NP + j] * A1[iy * NP + j];
        k1 += P.K1[i * NP + j] * A2[iy * NP + j];
      }
      T bt = 0;
#pragma unroll
      for (int ex = 0; ex <= R; ++ex) bt += fx[ex * NP + i] * sp[ex][iy];
      T v = m1 + beta * k1 + bsc * bt;
      if (res) v = own ? bvel(iy, i) - v : -v;           // b enters once, through the owner
      if constexpr (RST)
        rl[(iy * NP + i) % (RST ? NQ : 1)] = v;
      else
        atomicAdd(yd + off, v);
    }
  }
  // pressure rows of the cell: this component's share (b through component 0)
  T rp[RST ? NPM : 1];
#pragma unroll
  for (int m = 0; m < NPM; ++m) {
    const long long gi = poff + (long long)a * P.n_pres + c * NPM + m;
    T v = bsc * cont[m];
    if (res) v = d == 0 ? bpre(m) - v : -v;
    if constexpr (RST)
      rp[m % (RST ? NPM : 1)] = v;
    else
      atomicAdd(y + gi, v);
  }
  if constexpr (RST) {
    const TransferParams<T>& Q = *tp;
    constexpr int NPMC = NPC * (NPC - 1) / 2;
    const int Gc = Q.Gc, nc = Q.nc, ktc = Q.ktc;
    const int ccx = HT ? cx >> 1 : cx, ccy = HT ? cy >> 1 : cy;
    const int ox = HT ? (cx & 1) * (NP - 1) : 0, oy = HT ? (cy & 1) * (NP - 1) : 0;
    // velocity: S[jy][jx] = sum_iy wy[iy][jy] sum_ix wx[ix][jx] rl[iy][ix]
    T tx[NP][NPC];
#pragma unroll
    for (int iy = 0; iy < NP; ++iy)
#pragma unroll
      for (int jx = 0; jx < NPC; ++jx) {
        T s = 0;
#pragma unroll
        for (int ix = 0; ix < NP; ++ix) s += Q.P1[(ox + ix) * MAXNP + jx] * rl[(iy * NP + ix) % (RST ? NQ : 1)];
        tx[iy][jx] = s;
      }
    const bool zero_owner = HT ? ((cx & 1) == 0 && (cy & 1) == 0) : true;
#pragma unroll
    for (int jy = 0; jy < NPC; ++jy)
#pragma unroll
      for (int jx = 0; jx < NPC; ++jx) {
        T s = 0;
#pragma unroll
        for (int iy = 0; iy < NP; ++iy) s += Q.P1[(oy + iy) * MAXNP + jy] * tx[iy][jx];
        const int Jx = ccx * (NPC - 1) + jx, Jy = ccy * (NPC - 1) + jy;
        const long long J = (long long)Jy * Gc + Jx;
        const bool dirc = Jx == 0 || Jx == Gc - 1 || Jy == 0 || Jy == Gc - 1;
#pragma unroll
        for (int ac = 0; ac < KT; ++ac)
          if (ac < ktc && !dirc) atomicAdd(bc + ac * Q.nvc + d * Q.nnc + J, Q.Pt[a * MAXKT + ac] * s);
        const bool ownc = (jx < NPC - 1 || ccx == nc - 1) && (jy < NPC - 1 || ccy == nc - 1);
        if (zero_owner && ownc && a < ktc) xc[a * Q.nvc + d * Q.nnc + J] = T(0);
      }
    // pressure: the parent's coarse modes through the child map
    const int o = HT ? ((cx & 1) | ((cy & 1) << 1)) : 0;
    const long long cc = (long long)ccy * nc + ccx;
#pragma unroll
    for (int mc = 0; mc < NPMC; ++mc) {
      T s = 0;
#pragma unroll
      for (int m = 0; m < NPM; ++m) s += pres_map(Q, o, m, mc) * rp[m % (RST ? NPM : 1)];
#pragma unroll
      for (int ac = 0; ac < KT; ++ac)
        if (ac < ktc) atomicAdd(bc + (long long)ktc * Q.nvc + ac * Q.npc_tot + cc * NPMC + mc, Q.Pt[a * MAXKT + ac] * s);
      if (zero_owner && d == 0 && a < ktc) xc[(long long)ktc * Q.nvc + a * Q.npc_tot + cc * NPMC + mc] = T(0);
    }
  }
}

// ------------------------------------------------------------------------------------
// Pair-split form of the register-resident 2D operator (NP even): the work of one
// (cell, a, d) on two adjacent lanes.  Lane half hh = t & 1 owns the node columns
// ix = hh * HC + il, il < HC = NP / 2.  Each lane
//   - loads and combines in time its own columns (all rows),
//   - runs the y-pass (along y, within a column) on them,
//   - takes the partner's y-pass results of each row by shuffles and runs the x-pass for
//     its own output columns,
//   - forms the continuity sums of its columns; one shuffle-add completes them, and the
//     pair splits the pressure rows between its lanes (even modes: lane 0).
// The arithmetic per output is that of apply2d_reg_thread (the continuity sums add their
// two column halves last); the serial chain per lane is half as long and there are twice
// as many lanes, which spreads a level of few cells over more warps.  Every lane of a
// warp takes part in the shuffles: lanes past the last item compute on cell 0 and store
// nothing.
// ------------------------------------------------------------------------------------
template <typename T, int NP, int KT, bool CG>
__device__ __forceinline__ void apply2d_pair_thread(const ApplyRegParams<T>& P, const T* __restrict__ x,
                                                    const T* __restrict__ b, T* __restrict__ y, int mode,
                                                    long long t) {
  static_assert(NP % 2 == 0, "the pair split halves the node columns");
  constexpr int E = NP - 1, R = NP - 2, HC = NP / 2;
  constexpr int NPM = NP * (NP - 1) / 2;
  constexpr unsigned FULL = 0xffffffffu;
  const int n = P.n, G = P.G;
  const long long ncells = (long long)n * n;
  const long long tp = t >> 1;
  const int hh = (int)(t & 1);
  const bool live = tp < ncells * KT * 2;
  const long long tq = live ? tp : 0;
  const long long ad = tq / ncells;
  const long long c = tq - ad * ncells;
  const int a = (int)(ad >> 1), d = (int)(ad & 1);
  const int cx = (int)(c % n), cy = (int)(c / n);
  const long long nvel = P.n_vel, nnod = P.n_nodes;
  const long long poff = (long long)KT * nvel;
  const bool res = mode == RESIDUAL || mode == LIFT;
  const bool lift = mode == LIFT;
  const bool tr = mode == APPLY_T;
  const int c0 = hh * HC;                                         // first column of this lane
  const long long base = (long long)(cy * E) * G + cx * E + c0;   // node (0, c0) of the cell
  const bool bx0 = cx == 0, bx1 = cx == n - 1, by0 = cy == 0, by1 = cy == n - 1;
  auto dirn = [&](int iy, int il) -> bool {
    const int ix = c0 + il;
    return (iy == 0 && by0) || (iy == E && by1) || (ix == 0 && bx0) || (ix == E && bx1);
  };
  const T* fy = &P.FY[d][0];
  T fxo[R + 1][HC];                                 // x factors of this lane's columns
#pragma unroll
  for (int ex = 0; ex <= R; ++ex)
#pragma unroll
    for (int il = 0; il < HC; ++il) fxo[ex][il] = P.FX[d][ex * NP + c0 + il];

  T ut[NP][HC], ua[NP][HC], p[NPM];
#pragma unroll
  for (int iy = 0; iy < NP; ++iy)
#pragma unroll
    for (int il = 0; il < HC; ++il) { ut[iy][il] = 0; ua[iy][il] = 0; }
  T kt_row[KT];
#pragma unroll
  for (int bb = 0; bb < KT; ++bb) kt_row[bb] = tr ? P.Kt[bb * MAXKT + a] : P.Kt[a * MAXKT + bb];
#pragma unroll
  for (int bb = 0; bb < KT; ++bb) {
    const T* xb = x + bb * nvel + d * nnod + base;
    const T kb = kt_row[bb];
#pragma unroll
    for (int iy = 0; iy < NP; ++iy)
#pragma unroll
      for (int il = 0; il < HC; ++il) {
        const bool dir = dirn(iy, il);
        const bool take = lift ? dir : !dir;
        const T v = take ? ldv<CG>(xb + iy * G + il) : T(0);
        ut[iy][il] += kb * v;
        if (bb == a) ua[iy][il] = v;
      }
  }
#pragma unroll
  for (int m = 0; m < NPM; ++m) p[m] = lift ? T(0) : ldv<CG>(x + poff + (long long)a * P.n_pres + c * NPM + m);
  const T beta = P.beta[a], bsc = P.bscale[a], hd = P.hd;

  // continuity: sum over this lane's columns, then the partner's half
  T cont[NPM];
  {
    T ty[R + 1][HC];
#pragma unroll
    for (int ey = 0; ey <= R; ++ey)
#pragma unroll
      for (int il = 0; il < HC; ++il) {
        T s = 0;
#pragma unroll
        for (int iy = 0; iy < NP; ++iy) s += fy[ey * NP + iy] * ua[iy][il];
        ty[ey][il] = s;
      }
#pragma unroll
    for (int ex = 0; ex <= R; ++ex)
#pragma unroll
      for (int ey = 0; ey <= R - ex; ++ey) {
        T s = 0;
#pragma unroll
        for (int il = 0; il < HC; ++il) s += fxo[ex][il] * ty[ey][il];
        cont[mode_index(ex, ey)] = s + __shfl_xor_sync(FULL, s, 1);
      }
  }
  T sp[R + 1][NP];
#pragma unroll
  for (int ex = 0; ex <= R; ++ex)
#pragma unroll
    for (int iy = 0; iy < NP; ++iy) {
      T s = 0;
#pragma unroll
      for (int ey = 0; ey <= R - ex; ++ey) s += fy[ey * NP + iy] * p[mode_index(ex, ey)];
      sp[ex][iy] = s;
    }
  // y-pass on this lane's columns
  T A1[NP][HC], A2[NP][HC];
#pragma unroll
  for (int il = 0; il < HC; ++il)
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      T m1 = 0, k1 = 0, m2 = 0;
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        m1 += P.M1[i * NP + j] * ut[j][il];
        k1 += P.K1[i * NP + j] * ua[j][il];
        m2 += P.M1[i * NP + j] * ua[j][il];
      }
      A1[i][il] = hd * m1 + beta * k1;
      A2[i][il] = m2;
    }
  // rows of M1 and K1 of this lane's output columns
  T m1o[HC][NP], k1o[HC][NP];
#pragma unroll
  for (int io = 0; io < HC; ++io)
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      m1o[io][j] = P.M1[(c0 + io) * NP + j];
      k1o[io][j] = P.K1[(c0 + io) * NP + j];
    }
  // x-pass, pressure gradient, scatter
  T* yd = y + a * nvel + d * nnod + base;
  const T* xd = x + a * nvel + d * nnod + base;
  const T* bd = b + a * nvel + d * nnod + base;
#pragma unroll
  for (int iy = 0; iy < NP; ++iy) {
    T f1[NP], f2[NP];                               // row iy of A1, A2 in column order
#pragma unroll
    for (int jl = 0; jl < HC; ++jl) {
      const T o1 = __shfl_xor_sync(FULL, A1[iy][jl], 1), o2 = __shfl_xor_sync(FULL, A2[iy][jl], 1);
      f1[jl] = hh ? o1 : A1[iy][jl];
      f1[HC + jl] = hh ? A1[iy][jl] : o1;
      f2[jl] = hh ? o2 : A2[iy][jl];
      f2[HC + jl] = hh ? A2[iy][jl] : o2;
    }
    const bool dy = (iy == 0 && by0) || (iy == E && by1);
    const bool oy = iy < E || by1;
#pragma unroll
    for (int io = 0; io < HC; ++io) {
      const int ix = c0 + io;
      const bool dir = dy || (ix == 0 && bx0) || (ix == E && bx1);
      const bool own = oy && (ix < E || bx1);
      const long long off = (long long)iy * G + io;
      if (dir) {
        if (own && live) {
          const T xv = ldv<CG>(xd + off);
          atomicAdd(yd + off, mode == RESIDUAL ? ldv<CG>(bd + off) - xv : xv);
        }
        continue;
      }
      T m1 = 0, k1 = 0, bt = 0;
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        m1 += m1o[io][j] * f1[j];
        k1 += k1o[io][j] * f2[j];
      }
#pragma unroll
      for (int ex = 0; ex <= R; ++ex) bt += fxo[ex][io] * sp[ex][iy];
      T v = m1 + beta * k1 + bsc * bt;
      if (res) v = own ? ldv<CG>(bd + off) - v : -v;
      if (live) atomicAdd(yd + off, v);
    }
  }
  // pressure rows of the cell: this component's share, modes split between the lanes
#pragma unroll
  for (int m = 0; m < NPM; ++m) {
    if ((m & 1) != hh || !live) continue;
    const long long gi = poff + (long long)a * P.n_pres + c * NPM + m;
    T v = bsc * cont[m];
    if (res) v = d == 0 ? ldv<CG>(b + gi) - v : -v;
    atomicAdd(y + gi, v);
  }
}

// ------------------------------------------------------------------------------------
// Gather-form grid transfers of 2D levels (App. A).
//   prolongation  a fine velocity node takes the coarse function's value in the coarse
//                 cell that contains it (on a coarse-cell face, either cell: the coarse
//                 function is continuous, so both give the same value);
//   restriction   a coarse velocity node sums its basis function's values at the fine
//                 nodes of its support, each fine node once: per direction the fine nodes
//                 of the one or two coarse cells that contain the node, weighted by P1 of
//                 the cell that contains the fine node.
// Coarse Dirichlet nodes read as 0 (identity columns), fine Dirichlet nodes are neither
// written (prolongation) nor read (restriction); the restriction writes every coarse
// value, Dirichlet ones as 0 (and, if zc is given, zc = 0 at the same entries).
// ------------------------------------------------------------------------------------

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

// threads of the prolongation: one per fine node for the velocity (both components), then
// one per (fine cell, fine mode) for the pressure
template <typename T>
__host__ __device__ __forceinline__ long long prolongate_g_items(const TransferParams<T>& P) {
  return (long long)P.Gf * P.Gf + (long long)P.nf * P.nf * P.npmf;
}

template <typename T, int NPF, int NPC, int HT, bool CG>
__device__ __forceinline__ void prolongate_g_thread(const TransferParams<T>& P, const T* __restrict__ yc,
                                                    T* __restrict__ xf, long long t) {
  constexpr int NS = HT ? 2 * (NPF - 1) + 1 : NPF;
  const int Gf = P.Gf, Gc = P.Gc, nc = P.nc, ktc = P.ktc, ktf = P.ktf;
  const long long nvt = (long long)Gf * Gf;                   // fine nodes, both components each
  if (t < nvt) {
    const int g = (int)t;
    const int gy = g / Gf, gx = g - gy * Gf;
    if (gx == 0 || gx == Gf - 1 || gy == 0 || gy == Gf - 1) return;
    const int cx = min(gx / (NS - 1), nc - 1), cy = min(gy / (NS - 1), nc - 1);
    const int sx = gx - cx * (NS - 1), sy = gy - cy * (NS - 1);
    T wx[NPC], wy[NPC];
    bool dx[NPC], dy[NPC];
#pragma unroll
    for (int j = 0; j < NPC; ++j) {
      wx[j] = P.P1[sx * MAXNP + j];
      wy[j] = P.P1[sy * MAXNP + j];
      const int Jx = cx * (NPC - 1) + j, Jy = cy * (NPC - 1) + j;
      dx[j] = Jx == 0 || Jx == Gc - 1;
      dy[j] = Jy == 0 || Jy == Gc - 1;
    }
    // the coarse values of both components share the addresses (offset nnc): one address,
    // two loads
    const long long cbase = (long long)(cy * (NPC - 1)) * Gc + cx * (NPC - 1);
    T s0[MAXKT], s1[MAXKT];
#pragma unroll
    for (int ac = 0; ac < MAXKT; ++ac) {
      s0[ac] = T(0);
      s1[ac] = T(0);
      if (ac < ktc) {
        const T* yv = yc + ac * P.nvc + cbase;
        T a0 = 0, a1 = 0;
#pragma unroll
        for (int jy = 0; jy < NPC; ++jy) {
          T row0 = 0, row1 = 0;
#pragma unroll
          for (int jx = 0; jx < NPC; ++jx) {
            const bool z = dx[jx] || dy[jy];
            const T* q = yv + jy * Gc + jx;
            row0 += wx[jx] * (z ? T(0) : ldv<CG>(q));
            row1 += wx[jx] * (z ? T(0) : ldv<CG>(q + P.nnc));
          }
          a0 += wy[jy] * row0;
          a1 += wy[jy] * row1;
        }
        s0[ac] = a0;
        s1[ac] = a1;
      }
    }
    T old0[MAXKT], old1[MAXKT];                       // the fine values first, all at once
#pragma unroll
    for (int af = 0; af < MAXKT; ++af) {
      old0[af] = af < ktf ? ldv<CG>(xf + af * P.nvf + g) : T(0);
      old1[af] = af < ktf ? ldv<CG>(xf + af * P.nvf + P.nnf + g) : T(0);
    }
#pragma unroll
    for (int af = 0; af < MAXKT; ++af) {
      if (af < ktf) {
        T o0 = 0, o1 = 0;
#pragma unroll
        for (int ac = 0; ac < MAXKT; ++ac)
          if (ac < ktc) {
            const T pt = P.Pt[af * MAXKT + ac];
            o0 += pt * s0[ac];
            o1 += pt * s1[ac];
          }
        xf[af * P.nvf + g] = old0[af] + o0;
        xf[af * P.nvf + P.nnf + g] = old1[af] + o1;
      }
    }
    return;
  }
  // pressure: one thread per (fine cell, fine mode), every fine temporal dof; the parent
  // cell's coarse modes of every coarse temporal dof are loaded first, all at once
  constexpr int NPMC = NPC * (NPC - 1) / 2;           // 2D pressure modes of the coarse degree
  const long long tq = t - nvt;
  if (tq >= (long long)P.nf * P.nf * P.npmf) return;
  const int fc = (int)(tq / P.npmf), mf = (int)(tq - (long long)fc * P.npmf);
  const int fx = fc % P.nf, fy = fc / P.nf;
  const int ccx = HT ? fx / 2 : fx, ccy = HT ? fy / 2 : fy;
  const int o = HT ? ((fx & 1) | ((fy & 1) << 1)) : 0;
  const long long cc = (long long)ccy * nc + ccx;
  // the child map's coefficients of this thread's fine mode, once (each is a chain of
  // dependent table reads; they do not depend on the temporal dof)
  T pm[NPMC];
#pragma unroll
  for (int mc = 0; mc < NPMC; ++mc) pm[mc] = pres_map(P, o, mf, mc);
  T u[MAXKT];
#pragma unroll
  for (int ac = 0; ac < MAXKT; ++ac) {
    T yv[NPMC];
    const T* src = yc + (long long)ktc * P.nvc + ac * P.npc_tot + cc * NPMC;
#pragma unroll
    for (int mc = 0; mc < NPMC; ++mc) yv[mc] = ac < ktc ? ldv<CG>(src + mc) : T(0);
    T s = 0;
#pragma unroll
    for (int mc = 0; mc < NPMC; ++mc) s += pm[mc] * yv[mc];
    u[ac] = s;
  }
  T old[MAXKT];
#pragma unroll
  for (int af = 0; af < MAXKT; ++af)
    old[af] = af < ktf ? ldv<CG>(xf + (long long)ktf * P.nvf + af * P.npf_tot + (long long)fc * P.npmf + mf) : T(0);
#pragma unroll
  for (int af = 0; af < MAXKT; ++af) {
    if (af < ktf) {
      T v = 0;
#pragma unroll
      for (int ac = 0; ac < MAXKT; ++ac)
        if (ac < ktc) v += P.Pt[af * MAXKT + ac] * u[ac];
      xf[(long long)ktf * P.nvf + af * P.npf_tot + (long long)fc * P.npmf + mf] = old[af] + v;
    }
  }
}

// 1D support of coarse node J: first fine node i0, count n (<= BX) and weights w[m] of the
// fine nodes i0 + m (0 at fine Dirichlet nodes)
template <typename T, int NPC, int NS, int BX>
__device__ __forceinline__ void support_1d(const TransferParams<T>& P, int J, int* i0, int* n, T* w) {
  const int q = J / (NPC - 1), rem = J - q * (NPC - 1);
  int c0 = q, c1 = q;
  if (rem == 0) {
    c0 = q - 1 < 0 ? 0 : q - 1;
    c1 = q < P.nc - 1 ? q : P.nc - 1;
  }
  *i0 = c0 * (NS - 1);
  *n = (c1 - c0 + 1) * (NS - 1) + 1;
#pragma unroll
  for (int m = 0; m < BX; ++m) {
    const int i = *i0 + m;
    int ci = i / (NS - 1);
    ci = ci < c0 ? c0 : (ci > c1 ? c1 : ci);
    int s = i - ci * (NS - 1), jl = J - ci * (NPC - 1);
    s = s < 0 ? 0 : (s > NS - 1 ? NS - 1 : s);               // in range whenever m < n;
    jl = jl < 0 ? 0 : (jl > NPC - 1 ? NPC - 1 : jl);         // clamped so no index leaves P1
    const T v = P.P1[s * MAXNP + jl];
    w[m] = (m >= *n || i == 0 || i == P.Gf - 1) ? T(0) : v;
  }
}

// blocks of the restriction (256 threads): the velocity blocks first, one thread per
// (coarse node, fine temporal dof), the latter fastest, both components per thread (the
// two share every address), meeting in tsh[512] for the temporal restriction; then one
// thread per (coarse cell, coarse mode, coarse temporal dof).
template <typename T>
__host__ __device__ __forceinline__ long long restrict_g_velocity_blocks(const TransferParams<T>& P) {
  const int npb = 256 / P.ktf;
  return ((long long)P.Gc * P.Gc + npb - 1) / npb;
}

template <typename T>
__host__ __device__ __forceinline__ long long restrict_g_blocks(const TransferParams<T>& P) {
  const long long npt = (long long)P.nc * P.nc * P.npmc * P.ktc;
  return restrict_g_velocity_blocks(P) + (npt + 255) / 256;
}

// tsh: 512 values of shared memory
template <typename T, int NPF, int NPC, int HT, bool CG>
__device__ __forceinline__ void restrict_g_block(const TransferParams<T>& P, const T* __restrict__ rf,
                                                 T* __restrict__ bc, T* __restrict__ zc, long long vb, T* tsh) {
  constexpr int NS = HT ? 2 * (NPF - 1) + 1 : NPF;
  constexpr int BX = 2 * (NS - 1) + 1;
  const int Gf = P.Gf, Gc = P.Gc, ktc = P.ktc, ktf = P.ktf;
  const int npb = 256 / ktf;                                   // coarse nodes per block
  const long long nnodes = (long long)Gc * Gc;
  const long long nvb = restrict_g_velocity_blocks(P);
  if (vb < nvb) {
    const int nl = threadIdx.x / ktf, af = threadIdx.x - nl * ktf;
    const long long Gi = vb * (long long)npb + nl;
    const bool active = nl < npb && Gi < nnodes;
    bool dirc = true;
    if (active) {
      const int Jx = (int)(Gi % Gc), Jy = (int)(Gi / Gc);
      dirc = Jx == 0 || Jx == Gc - 1 || Jy == 0 || Jy == Gc - 1;
      T acc0 = 0, acc1 = 0;
      if (!dirc) {
        int ix0, nx, iy0, ny;
        T wx[BX], wy[BX];
        support_1d<T, NPC, NS, BX>(P, Jx, &ix0, &nx, wx);
        support_1d<T, NPC, NS, BX>(P, Jy, &iy0, &ny, wy);
        (void)nx; (void)ny;
        // every load unconditional (indices clamped into the grid, weights 0 outside the
        // support), so that all of them are in flight at once
        int col[BX];
#pragma unroll
        for (int mx = 0; mx < BX; ++mx) col[mx] = min(ix0 + mx, Gf - 1);
        const T* r0 = rf + af * P.nvf;
        const T* r1 = r0 + P.nnf;
#pragma unroll
        for (int my = 0; my < BX; ++my) {
          const long long ro = (long long)min(iy0 + my, Gf - 1) * Gf;
          T row0 = 0, row1 = 0;
#pragma unroll
          for (int mx = 0; mx < BX; ++mx) {
            row0 += wx[mx] * ldv<CG>(r0 + ro + col[mx]);
            row1 += wx[mx] * ldv<CG>(r1 + ro + col[mx]);
          }
          acc0 += wy[my] * row0;
          acc1 += wy[my] * row1;
        }
      }
      tsh[2 * threadIdx.x] = acc0;
      tsh[2 * threadIdx.x + 1] = acc1;
    }
    __syncthreads();
    if (active && af < ktc) {
      const int a = af;
      T o0 = 0, o1 = 0;
      if (!dirc)
        for (int f = 0; f < ktf; ++f) {
          const T pt = P.Pt[f * MAXKT + a];
          o0 += pt * tsh[2 * (nl * ktf + f)];
          o1 += pt * tsh[2 * (nl * ktf + f) + 1];
        }
      bc[a * P.nvc + Gi] = o0;
      bc[a * P.nvc + P.nnc + Gi] = o1;
      if (zc) {
        zc[a * P.nvc + Gi] = T(0);
        zc[a * P.nvc + P.nnc + Gi] = T(0);
      }
    }
    __syncthreads();                                           // tsh is reused by the next block
    return;
  }
  // pressure: one thread per (coarse cell, coarse mode, coarse temporal dof)
  const long long tq = (vb - nvb) * 256 + threadIdx.x;
  const long long ncc = (long long)P.nc * P.nc;
  if (tq >= ncc * P.npmc * ktc) return;
  const int ac = (int)(tq % ktc);
  const long long rest = tq / ktc;
  const int mc = (int)(rest % P.npmc);
  const long long cc = rest / P.npmc;
  const int ccx = (int)(cc % P.nc), ccy = (int)(cc / P.nc);
  // the children's fine modes of one fine temporal dof are loaded together, then combined
  constexpr int nchild = HT ? 4 : 1;
  constexpr int NPMF = NPF * (NPF - 1) / 2;           // 2D pressure modes of the fine degree
  long long fcs[nchild];
#pragma unroll
  for (int o = 0; o < nchild; ++o) {
    const int fx = HT ? 2 * ccx + (o & 1) : ccx, fy = HT ? 2 * ccy + ((o >> 1) & 1) : ccy;
    fcs[o] = (long long)fy * P.nf + fx;
  }
  // the child map's coefficients of this thread's coarse mode, once (each is a chain of
  // dependent table reads; they do not depend on the temporal dof)
  T pm[nchild][NPMF];
#pragma unroll
  for (int o = 0; o < nchild; ++o)
#pragma unroll
    for (int mf = 0; mf < NPMF; ++mf) pm[o][mf] = pres_map(P, o, mf, mc);
  // fine temporal dofs in groups of four, every load of a group in flight at once
  T v = 0;
  for (int a0 = 0; a0 < ktf; a0 += 4) {
    T rv[4][nchild][NPMF];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int o = 0; o < nchild; ++o) {
        const T* rr = rf + (long long)ktf * P.nvf + (a0 + q) * P.npf_tot + fcs[o] * NPMF;
#pragma unroll
        for (int mf = 0; mf < NPMF; ++mf) rv[q][o][mf] = a0 + q < ktf ? ldv<CG>(rr + mf) : T(0);
      }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (a0 + q < ktf) {
        T u = 0;
#pragma unroll
        for (int o = 0; o < nchild; ++o)
#pragma unroll
          for (int mf = 0; mf < NPMF; ++mf) u += pm[o][mf] * rv[q][o][mf];
        v += P.Pt[(a0 + q) * MAXKT + ac] * u;
      }
    }
  }
  bc[(long long)ktc * P.nvc + ac * P.npc_tot + cc * P.npmc + mc] = v;
  if (zc) zc[(long long)ktc * P.nvc + ac * P.npc_tot + cc * P.npmc + mc] = T(0);
}

}  // namespace stmg

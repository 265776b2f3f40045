// Host-side numerics of libstmg: quadrature rules, 1D reference tables, temporal DG(k)
// matrices.  Quadrature nodes come from root isolation (sign scan + bisection + Newton)
// on the Legendre three-term recurrence; weights from exact integration of the
// Lagrange basis.
#include <array>
#include <cmath>
#include <cstring>
#include <stdexcept>
#include <vector>

#include "internal.h"

namespace stmg {

namespace {

// P_n(x) and P_n'(x) by the three-term recurrence.
void legendre(int n, double x, double* p, double* dp) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (n == 0) { *p = 1.0; *dp = 0.0; return; }
  for (int m = 2; m <= n; ++m) {
    double p2 = ((2.0 * m - 1.0) * x * p1 - (m - 1.0) * p0) / m;
    double d2 = d0 + (2.0 * m - 1.0) * p1;          // P_m' = P_{m-2}' + (2m-1) P_{m-1}
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  *p = p1; *dp = d1;
}

// all roots of f in (a, b): scan for sign changes, then bisection.
template <typename F>
std::vector<double> roots_in(F f, double a, double b, int scan = 4000) {
  std::vector<double> out;
  double xl = a, fl = f(a);
  for (int i = 1; i <= scan; ++i) {
    double xr = a + (b - a) * i / scan, fr = f(xr);
    if (fl == 0.0) { out.push_back(xl); }
    else if (fl * fr < 0.0) {
      double lo = xl, hi = xr, flo = fl;
      for (int it = 0; it < 200 && hi - lo > 1e-17; ++it) {
        double mid = 0.5 * (lo + hi), fm = f(mid);
        if (fm == 0.0) { lo = hi = mid; break; }
        if ((fm < 0) == (flo < 0)) { lo = mid; flo = fm; } else { hi = mid; }
      }
      out.push_back(0.5 * (lo + hi));
    }
    xl = xr; fl = fr;
  }
  return out;
}

double lagrange_deriv(const double* nodes, int n, int j, double t) {
  double s = 0.0;
  for (int m = 0; m < n; ++m) {
    if (m == j) continue;
    double term = 1.0 / (nodes[j] - nodes[m]);
    for (int l = 0; l < n; ++l)
      if (l != j && l != m) term *= (t - nodes[l]) / (nodes[j] - nodes[l]);
    s += term;
  }
  return s;
}

void interpolatory_weights(const double* x, int n, double* w) {
  double gx[16], gw[16];
  gauss_legendre(n + 1, gx, gw);
  for (int j = 0; j < n; ++j) {
    double s = 0.0;
    for (int q = 0; q <= n; ++q) s += gw[q] * lagrange_eval(x, n, j, gx[q]);
    w[j] = s;
  }
}

}  // namespace

void gauss_legendre(int n, double* x, double* w) {
  auto f = [n](double t) { double p, dp; legendre(n, t, &p, &dp); return p; };
  std::vector<double> r = roots_in(f, -1.0, 1.0);
  if ((int)r.size() != n) throw std::runtime_error("gauss_legendre: root count");
  for (int i = 0; i < n; ++i) {
    double t = r[i], p, dp;
    for (int it = 0; it < 3; ++it) { legendre(n, t, &p, &dp); t -= p / dp; }
    legendre(n, t, &p, &dp);
    x[i] = t;
    w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
  }
}

double lagrange_eval(const double* nodes, int n, int j, double t) {
  double v = 1.0;
  for (int m = 0; m < n; ++m)
    if (m != j) v *= (t - nodes[m]) / (nodes[j] - nodes[m]);
  return v;
}

double legendre_unit(int i, double xi) {
  double p, dp;
  legendre(i, 2.0 * xi - 1.0, &p, &dp);
  return std::sqrt(2.0 * i + 1.0) * p;
}

void pressure_modes(int dim, int r, std::vector<std::array<int, 3>>* out) {
  out->clear();
  for (int s = 0; s <= r; ++s) {
    if (dim == 2) {
      for (int j = 0; j <= s; ++j) out->push_back({s - j, j, 0});
    } else {
      for (int l = 0; l <= s; ++l)
        for (int j = 0; j <= s - l; ++j) out->push_back({s - l - j, j, l});
    }
  }
}

Tables1D make_tables_1d(int r) {
  Tables1D t;
  const int np = r + 2;
  t.np = np;
  t.r = r;
  // Gauss-Lobatto nodes: -1, roots of P'_{np-1}, +1; mapped to [0,1]
  {
    auto f = [np](double s) { double p, dp; legendre(np - 1, s, &p, &dp); return dp; };
    std::vector<double> in = roots_in(f, -1.0, 1.0);
    if ((int)in.size() != np - 2) throw std::runtime_error("gauss_lobatto: root count");
    t.xi[0] = 0.0;
    for (int i = 0; i < np - 2; ++i) t.xi[i + 1] = 0.5 * (in[i] + 1.0);
    t.xi[np - 1] = 1.0;
  }
  double gx[16], gw[16];
  const int nq = np + 1;            // exact for degree 2 np - 1 >= 2 (r + 1)
  gauss_legendre(nq, gx, gw);
  std::memset(t.M1, 0, sizeof(t.M1));
  std::memset(t.K1, 0, sizeof(t.K1));
  std::memset(t.G1, 0, sizeof(t.G1));
  std::memset(t.N1, 0, sizeof(t.N1));
  for (int q = 0; q < nq; ++q) {
    const double xq = 0.5 * (gx[q] + 1.0), wq = 0.5 * gw[q];
    double l[MAXNP], dl[MAXNP], L[MAXNP];
    for (int j = 0; j < np; ++j) { l[j] = lagrange_eval(t.xi, np, j, xq); dl[j] = lagrange_deriv(t.xi, np, j, xq); }
    for (int i = 0; i <= r; ++i) L[i] = legendre_unit(i, xq);
    for (int i = 0; i < np; ++i)
      for (int j = 0; j < np; ++j) {
        t.M1[i * np + j] += wq * l[i] * l[j];
        t.K1[i * np + j] += wq * dl[i] * dl[j];
      }
    for (int i = 0; i <= r; ++i)
      for (int p = 0; p < np; ++p) {
        t.G1[i * np + p] += wq * L[i] * dl[p];
        t.N1[i * np + p] += wq * L[i] * l[p];
      }
  }
  return t;
}

// One DG(k) subinterval (Eq. DefKMC), then the system of nsub subintervals (Eq. GloSys
// over a macro step, Remark rem:GLSP): K block-bidiagonal with K1 on the diagonal and
// -C1 below it (C1[a][b] = delta_{b,k} phi_a(-1)), M block diagonal, nodes of subinterval
// j shifted by 2 j, the coupling to the previous system only on the first subinterval.
TimeTables make_time_tables(int k, double tau, int nsub) {
  if (nsub < 1 || nsub * (k + 1) > MAXKT) throw std::runtime_error("time tables: too many temporal dofs");
  TimeTables t;
  const int kt = k + 1;
  t.kt = kt;
  // right Radau: roots of P_k - P_{k+1}, the last is +1
  if (k == 0) {
    t.nodes[0] = 1.0;
  } else {
    auto f = [k](double s) { double a, b, da, db; legendre(k, s, &a, &da); legendre(k + 1, s, &b, &db); return a - b; };
    std::vector<double> in = roots_in(f, -1.0, 1.0 - 1e-9);
    if ((int)in.size() != k) throw std::runtime_error("radau: root count");
    for (int i = 0; i < k; ++i) t.nodes[i] = in[i];
    t.nodes[k] = 1.0;
  }
  interpolatory_weights(t.nodes, kt, t.weights);
  double gx[16], gw[16];
  gauss_legendre(kt + 1, gx, gw);
  for (int a = 0; a < kt; ++a) {
    t.phi_left[a] = lagrange_eval(t.nodes, kt, a, -1.0);
    double m = 0.0;
    for (int q = 0; q <= kt; ++q) m += gw[q] * lagrange_eval(t.nodes, kt, a, gx[q]) * lagrange_eval(t.nodes, kt, a, gx[q]);
    t.M[a] = 0.5 * tau * m;
    for (int b = 0; b < kt; ++b) {
      double s = 0.0;
      for (int q = 0; q <= kt; ++q)
        s += gw[q] * lagrange_eval(t.nodes, kt, a, gx[q]) * lagrange_deriv(t.nodes, kt, b, gx[q]);
      t.K[a * kt + b] = s;       // phi_b(-1) phi_a(-1) added below
    }
  }
  for (int a = 0; a < kt; ++a)
    for (int b = 0; b < kt; ++b) t.K[a * kt + b] += t.phi_left[a] * t.phi_left[b];
  t.k1 = kt;
  t.nsub = 1;
  for (int a = 0; a < kt; ++a) t.nodes1[a] = t.nodes[a];
  if (nsub == 1) return t;
  TimeTables m = t;
  const int KT = nsub * kt;
  m.kt = KT;
  m.nsub = nsub;
  for (int i = 0; i < MAXKT * MAXKT; ++i) m.K[i] = 0.0;
  for (int j = 0; j < nsub; ++j)
    for (int a = 0; a < kt; ++a) {
      const int A = j * kt + a;
      m.nodes[A] = t.nodes[a] + 2.0 * j;
      m.weights[A] = t.weights[a];
      m.M[A] = t.M[a];
      m.phi_left[A] = j == 0 ? t.phi_left[a] : 0.0;
      for (int b = 0; b < kt; ++b) m.K[A * KT + j * kt + b] = t.K[a * kt + b];
      if (j > 0) m.K[A * KT + (j - 1) * kt + (kt - 1)] = -t.phi_left[a];
    }
  return m;
}

}  // namespace stmg

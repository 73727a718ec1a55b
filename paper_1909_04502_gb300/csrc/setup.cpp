// Host-side FP64 construction of the RLBM lattice tables.
//
// Sec. 5.2 (orthonormal polynomials under the weight omega), Sec. 5.3
// (quadratures with prescribed abscissas, Eq. mj-orthogonal-conditions,
// Eq. quadrature-problem), App. B (Maxwell-Juttner moments via the Z
// integrals), App. H (stencils and massless tables) of arXiv:1909.04502.
#include "setup.h"

#include <array>
#include <functional>
#include <set>

#include "dd.h"

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <set>
#include <utility>

namespace rlbm {

namespace {
constexpr double kPi = 3.14159265358979323846;
}

std::vector<Monomial> moment_basis(int order) {
  std::vector<Monomial> out;
  for (int deg = 0; deg <= order; ++deg) {
    // p0 times a degree-(deg-1) monomial in (px, py), then pure (px, py) monomials
    if (deg >= 1)
      for (int a = deg - 1; a >= 0; --a) out.push_back({1, a, deg - 1 - a});
    for (int a = deg; a >= 0; --a) out.push_back({0, a, deg - a});
  }
  // order 2: 1 | p0 px py | p0px p0py pxpx pxpy pypy (K = 9); order 3 adds
  // p0pxpx p0pxpy p0pypy pxpxpx pxpxpy pxpypy pypypy (K = 16)
  return out;
}

void gauss_laguerre(int n, std::vector<double>& x, std::vector<double>& w) {
  // Roots of L_n by Newton iteration from the usual asymptotic starting
  // values; weights w_j = x_j / ((n+1)^2 L_{n+1}(x_j)^2).
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  double z = 0.0;
  for (int i = 0; i < n; ++i) {
    if (i == 0) z = 3.0 / (1.0 + 2.4 * n);
    else if (i == 1) z += 15.0 / (1.0 + 2.5 * n);
    else {
      double ai = i - 1;
      z += ((1.0 + 2.55 * ai) / (1.9 * ai)) * (z - x[i - 2]);
    }
    for (int it = 0; it < 100; ++it) {
      double l0 = 1.0, l1 = 1.0 - z;
      for (int k = 1; k < n; ++k) {
        double l2 = ((2.0 * k + 1.0 - z) * l1 - k * l0) / (k + 1.0);
        l0 = l1;
        l1 = l2;
      }
      // l1 = L_n(z), l0 = L_{n-1}(z); z L_n' = n (L_n - L_{n-1})
      double dl = n * (l1 - l0) / z;
      double dz = l1 / dl;
      z -= dz;
      if (std::fabs(dz) <= 1e-15 * std::fabs(z)) break;
    }
    x[i] = z;
    double l0 = 1.0, l1 = 1.0 - z;
    for (int k = 1; k <= n; ++k) {
      double l2 = ((2.0 * k + 1.0 - z) * l1 - k * l0) / (k + 1.0);
      l0 = l1;
      l1 = l2;
    }
    w[i] = z / ((n + 1.0) * (n + 1.0) * l1 * l1);
  }
}

double omega_moment(int c, int a, int b, double m) {
  if ((a & 1) || (b & 1)) return 0.0;
  // d^2p / p0 = dp0 dtheta on the mass shell; p0 = m + s, |p|^2 = s (2m + s).
  static thread_local std::vector<double> xs, ws;
  if (xs.empty()) gauss_laguerre(16, xs, ws);   // exact for polynomials of degree <= 31
  double radial = 0.0;
  const int k2 = (a + b) / 2;
  for (size_t j = 0; j < xs.size(); ++j) {
    double s = xs[j];
    radial += ws[j] * std::pow(m + s, c) * std::pow(s * (2.0 * m + s), k2);
  }
  const int nth = 64;                             // exact for trig degree < 64
  double ang = 0.0;
  for (int j = 0; j < nth; ++j) {
    double th = 2.0 * kPi * j / nth;
    ang += std::pow(std::cos(th), a) * std::pow(std::sin(th), b);
  }
  ang /= nth;
  return ang * radial;
}

std::vector<double> gram_matrix(int order, double m) {
  auto B = moment_basis(order);
  const int K = (int)B.size();
  std::vector<double> G(K * K);
  for (int i = 0; i < K; ++i)
    for (int j = 0; j < K; ++j)
      G[i * K + j] = omega_moment(B[i].e + B[j].e, B[i].a + B[j].a, B[i].b + B[j].b, m);
  return G;
}

namespace {

// Well-conditioned working basis phi'_k = s^e (px/sg)^a (py/sg)^b with
// s = p0 - m and sg = sqrt(m + 1) (the scale of App. F's J^(1)_x).  It spans
// the same space as moment_basis, phi = A phi'.
// E_omega[s^c (px/sg)^a (py/sg)^b] in double-double.  With p0 = m + s,
// |p|^2 = s (2m + s) and d^2p/p0 = ds dtheta, the radial integrand expands
// into positive terms s^q e^{-s} (int = q!), the angular factor is
// (a-1)!!(b-1)!!/(a+b)!! for even a, b and zero otherwise.
dd omega_moment_shifted_dd(int c, int a, int b, double m) {
  if ((a & 1) || (b & 1)) return dd(0.0);
  const int k2 = (a + b) / 2;
  dd ang(1.0);
  for (int k = a - 1; k > 0; k -= 2) ang = ang * dd((double)k);
  for (int k = b - 1; k > 0; k -= 2) ang = ang * dd((double)k);
  dd den(1.0);
  for (int k = a + b; k > 0; k -= 2) den = den * dd((double)k);
  ang = ang / den;
  // (2m + s)^k2 = sum_j C(k2, j) (2m)^(k2-j) s^j
  dd radial(0.0);
  dd binom(1.0);
  for (int j = 0; j <= k2; ++j) {
    if (j > 0) binom = binom * dd((double)(k2 - j + 1)) / dd((double)j);
    dd pw(1.0);
    for (int t = 0; t < k2 - j; ++t) pw = pw * dd(2.0 * m);
    dd fact(1.0);
    for (int t = 2; t <= c + k2 + j; ++t) fact = fact * dd((double)t);
    radial = radial + binom * pw * fact;
  }
  dd sg2 = dd(m) + dd(1.0);
  dd scale(1.0);
  for (int t = 0; t < k2; ++t) scale = scale * sg2;
  return ang * radial / scale;
}

std::vector<dd> gram_shifted_dd(int order, double m) {
  auto B = moment_basis(order);
  const int K = (int)B.size();
  std::vector<dd> G(K * K);
  for (int i = 0; i < K; ++i)
    for (int j = 0; j < K; ++j)
      G[i * K + j] = omega_moment_shifted_dd(B[i].e + B[j].e, B[i].a + B[j].a, B[i].b + B[j].b, m);
  return G;
}

std::vector<double> gram_shifted(int order, double m) {
  std::vector<dd> g = gram_shifted_dd(order, m);
  std::vector<double> out(g.size());
  for (size_t i = 0; i < g.size(); ++i) out[i] = g[i].to_double();
  return out;
}

// Inverse of a symmetric positive definite matrix in double-double
// (Cholesky, then forward and back substitution per column).
bool spd_inverse_dd(const std::vector<dd>& a, int n, std::vector<dd>* inv) {
  std::vector<dd> L = a;
  for (int j = 0; j < n; ++j) {
    dd d = L[j * n + j];
    for (int k = 0; k < j; ++k) d = d - L[j * n + k] * L[j * n + k];
    if (!(d.hi > 0.0)) return false;
    d = dd_sqrt(d);
    L[j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      dd s = L[i * n + j];
      for (int k = 0; k < j; ++k) s = s - L[i * n + k] * L[j * n + k];
      L[i * n + j] = s / d;
    }
  }
  inv->assign(n * n, dd(0.0));
  std::vector<dd> y(n);
  for (int c = 0; c < n; ++c) {
    for (int i = 0; i < n; ++i) {
      dd s((i == c) ? 1.0 : 0.0);
      for (int k = 0; k < i; ++k) s = s - L[i * n + k] * y[k];
      y[i] = s / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      dd s = y[i];
      for (int k = i + 1; k < n; ++k) s = s - L[k * n + i] * (*inv)[k * n + c];
      (*inv)[i * n + c] = s / L[i * n + i];
    }
  }
  return true;
}

void eval_shifted(const std::vector<Monomial>& B, double m, double p0, double px, double py, double* out) {
  const double sg = std::sqrt(m + 1.0);
  const double s = p0 - m, qx = px / sg, qy = py / sg;
  for (size_t k = 0; k < B.size(); ++k) {
    double r = B[k].e ? s : 1.0;
    for (int i = 0; i < B[k].a; ++i) r *= qx;
    for (int i = 0; i < B[k].b; ++i) r *= qy;
    out[k] = r;
  }
}

}  // namespace

bool cholesky(std::vector<double>& a, int n) {
  for (int j = 0; j < n; ++j) {
    double d = a[j * n + j];
    for (int k = 0; k < j; ++k) d -= a[j * n + k] * a[j * n + k];
    if (!(d > 0.0)) return false;
    d = std::sqrt(d);
    a[j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double s = a[i * n + j];
      for (int k = 0; k < j; ++k) s -= a[i * n + k] * a[j * n + k];
      a[i * n + j] = s / d;
    }
    for (int k = j + 1; k < n; ++k) a[j * n + k] = 0.0;
  }
  return true;
}

std::vector<double> spd_inverse(const std::vector<double>& a, int n, bool* ok) {
  std::vector<double> L = a;
  std::vector<double> inv(n * n, 0.0);
  if (!cholesky(L, n)) {
    *ok = false;
    return inv;
  }
  // solve L L^T X = I column by column
  std::vector<double> y(n);
  for (int c = 0; c < n; ++c) {
    for (int i = 0; i < n; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) s -= L[i * n + k] * y[k];
      y[i] = s / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double s = y[i];
      for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * inv[k * n + c];
      inv[i * n + c] = s / L[i * n + i];
    }
  }
  *ok = true;
  return inv;
}

// ---------------------------------------------------------------------------
// Stencils
// ---------------------------------------------------------------------------

namespace {

// Full-symmetric group of a generator vector: all sign flips and the swap of
// the two components, without repetitions (Sec. 5.3).
std::vector<std::pair<int, int>> fs_group(int gx, int gy) {
  std::set<std::pair<int, int>> s;
  const int sx[2] = {1, -1};
  for (int swap = 0; swap < 2; ++swap) {
    int u = swap ? gy : gx, v = swap ? gx : gy;
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) s.insert({sx[a] * u, sx[b] * v});
  }
  return std::vector<std::pair<int, int>>(s.begin(), s.end());
}


// Least squares min ||A w - b|| by Householder QR (A: rows x cols, row-major).
bool least_squares(std::vector<double> A, std::vector<double> b, int rows, int cols,
                   std::vector<double>* x) {
  if (rows < cols) return false;
  for (int k = 0; k < cols; ++k) {
    double nrm = 0.0;
    for (int i = k; i < rows; ++i) nrm += A[i * cols + k] * A[i * cols + k];
    nrm = std::sqrt(nrm);
    if (nrm == 0.0) return false;
    double alpha = A[k * cols + k] > 0 ? -nrm : nrm;
    std::vector<double> v(rows - k);
    for (int i = k; i < rows; ++i) v[i - k] = A[i * cols + k];
    v[0] -= alpha;
    double vn = 0.0;
    for (double t : v) vn += t * t;
    if (vn == 0.0) continue;
    for (int j = k; j < cols; ++j) {
      double s = 0.0;
      for (int i = k; i < rows; ++i) s += v[i - k] * A[i * cols + j];
      s = 2.0 * s / vn;
      for (int i = k; i < rows; ++i) A[i * cols + j] -= s * v[i - k];
    }
    double s = 0.0;
    for (int i = k; i < rows; ++i) s += v[i - k] * b[i];
    s = 2.0 * s / vn;
    for (int i = k; i < rows; ++i) b[i] -= s * v[i - k];
  }
  x->assign(cols, 0.0);
  for (int i = cols - 1; i >= 0; --i) {
    double s = b[i];
    for (int j = i + 1; j < cols; ++j) s -= A[i * cols + j] * (*x)[j];
    if (std::fabs(A[i * cols + i]) < 1e-300) return false;
    (*x)[i] = s / A[i * cols + i];
  }
  return true;
}

}  // namespace

bool massless_quadrature(int order, Quadrature* q, std::string* err) {
  // App. H, ultra-relativistic regime, (2+1) dimensions.  Stencil
  // {(+-3, +-4)FS, (+-5, 0)FS}; shell energies are the printed p0_j.  The
  // printed weight column is read shell by shell, the (+-5, 0) group first
  // and the (+-3, +-4) group second; this reading satisfies the
  // orthonormality conditions (the literal group-by-group reading does not).
  static const double s2[3] = {0.4157745567834790, 2.2942803602790417, 6.2899450829374791};
  static const double c2[6] = {0.0, 0.0888866262411466, 0.0, 0.0348147166961551,
                               0.0017535654166088, 0.0004218743543938};
  static const double s3[4] = {0.3225476896193923, 1.7457611011583465, 4.5366202969211279,
                               9.3950709123011331};
  static const double c3[8] = {0.0, 0.0753942630427042, 0.0410206173754781,
                               0.0241670278669858, 0.0044457884155769, 0.0026380943565871,
                               0.0000616926157132, 0.0000365655303385};
  const double* shells;
  const double* col;
  int ns;
  if (order == 2) { shells = s2; col = c2; ns = 3; }
  else if (order == 3) { shells = s3; col = c3; ns = 4; }
  else { *err = "massless quadrature: order must be 2 or 3"; return false; }
  *q = Quadrature();
  q->m = 0.0;
  q->order = order;
  // Orbit order (the kernels' symmetric evaluation relies on it): for each
  // shell with weight, the eight images of (3, 4) as two sign quartets
  // (a, b), (-a, b), (a, -b), (-a, -b) of (3, 4) and of its swap (4, 3);
  // then for each shell with weight the four images of (5, 0):
  // (5, 0), (-5, 0), (0, 5), (0, -5).
  static const int fam8[8][2] = {{3, 4}, {-3, 4}, {3, -4}, {-3, -4}, {4, 3}, {-4, 3}, {4, -3}, {-4, -3}};
  static const int fam4[4][2] = {{5, 0}, {-5, 0}, {0, 5}, {0, -5}};
  auto push = [&](int vx, int vy, int j, double wgt) {
    q->nx.push_back(vx);
    q->ny.push_back(vy);
    q->p0.push_back(shells[j]);
    q->px.push_back(shells[j] * vx / 5.0);
    q->py.push_back(shells[j] * vy / 5.0);
    q->w.push_back(wgt);
  };
  for (int j = 0; j < ns; ++j)
    if (col[2 * j + 1] != 0.0)
      for (auto& v : fam8) push(v[0], v[1], j, col[2 * j + 1]);
  for (int j = 0; j < ns; ++j)
    if (col[2 * j] != 0.0)
      for (auto& v : fam4) push(v[0], v[1], j, col[2 * j]);
  q->Q = (int)q->w.size();
  return true;
}

namespace {

// Group weights of Eq. mj-orthogonal-conditions in double-double.  The
// orthonormal basis is J = L^{-1} phi' with L the Cholesky factor of the
// shifted Gram matrix; s = p0 - m is formed as m v^2 / (r (1 + r)),
// r = sqrt(1 - v^2), so no digits cancel; the conditions are summed per FS
// group and solved in the least-squares sense through the column-equilibrated
// normal equations.  At order 3 the same construction in double loses up to
// 1e-9 of a weight (m~ = 20) to the conditioning of the basis; this one is
// limited by the final rounding to double.
bool group_weights_dd(const std::vector<int>& groups, double m, double v0, int order,
                      std::vector<double>* wg_out, double* residual) {
  const int ng = (int)groups.size() / 2;
  auto B = moment_basis(order);
  const int K = (int)B.size();
  std::vector<dd> L = gram_shifted_dd(order, m);
  for (int j = 0; j < K; ++j) {
    dd d = L[j * K + j];
    for (int k = 0; k < j; ++k) d = d - L[j * K + k] * L[j * K + k];
    if (!(d.hi > 0.0)) return false;
    d = dd_sqrt(d);
    L[j * K + j] = d;
    for (int i = j + 1; i < K; ++i) {
      dd t = L[i * K + j];
      for (int k = 0; k < j; ++k) t = t - L[i * K + k] * L[j * K + k];
      L[i * K + j] = t / d;
    }
  }
  const dd mm(m), sg = dd_sqrt(mm + dd(1.0));
  const int rows = K * (K + 1) / 2;
  std::vector<dd> A((size_t)rows * ng, dd(0.0)), J(K), phi(K);
  for (int g = 0; g < ng; ++g)
    for (auto v : fs_group(groups[2 * g], groups[2 * g + 1])) {
      const dd vx = dd(v0) * dd((double)v.first), vy = dd(v0) * dd((double)v.second);
      const dd v2 = vx * vx + vy * vy;
      if (!(v2.hi < 1.0)) return false;
      const dd r = dd_sqrt(dd(1.0) - v2);
      const dd s = mm * v2 / (r * (dd(1.0) + r));
      const dd qx = mm * vx / (r * sg), qy = mm * vy / (r * sg);
      for (int k = 0; k < K; ++k) {
        dd t = B[k].e ? s : dd(1.0);
        for (int i = 0; i < B[k].a; ++i) t = t * qx;
        for (int i = 0; i < B[k].b; ++i) t = t * qy;
        phi[k] = t;
      }
      for (int k = 0; k < K; ++k) {
        dd t = phi[k];
        for (int j = 0; j < k; ++j) t = t - L[k * K + j] * J[j];
        J[k] = t / L[k * K + k];
      }
      int rr = 0;
      for (int l = 0; l < K; ++l)
        for (int k = l; k < K; ++k, ++rr) A[(size_t)rr * ng + g] = A[(size_t)rr * ng + g] + J[l] * J[k];
    }
  // column scales D (powers of two, so scaling is exact), then (AD)^T (AD) y = (AD)^T b
  std::vector<dd> D(ng);
  for (int g = 0; g < ng; ++g) {
    double n2 = 0.0;
    for (int rr = 0; rr < rows; ++rr) n2 += A[(size_t)rr * ng + g].hi * A[(size_t)rr * ng + g].hi;
    if (!(n2 > 0.0)) return false;
    int e;
    std::frexp(std::sqrt(n2), &e);
    D[g] = dd(std::ldexp(1.0, -e));
  }
  std::vector<dd> N((size_t)ng * ng, dd(0.0)), y(ng, dd(0.0));
  {
    int rr = 0;
    for (int l = 0; l < K; ++l)
      for (int k = l; k < K; ++k, ++rr) {
        const dd* a = &A[(size_t)rr * ng];
        for (int i = 0; i < ng; ++i) {
          const dd ai = a[i] * D[i];
          if (l == k) y[i] = y[i] + ai;
          for (int j = 0; j < ng; ++j) N[(size_t)i * ng + j] = N[(size_t)i * ng + j] + ai * (a[j] * D[j]);
        }
      }
  }
  std::vector<dd> Ni;
  if (!spd_inverse_dd(N, ng, &Ni)) return false;
  wg_out->assign(ng, 0.0);
  std::vector<dd> w(ng);
  for (int i = 0; i < ng; ++i) {
    dd t(0.0);
    for (int j = 0; j < ng; ++j) t = t + Ni[(size_t)i * ng + j] * y[j];
    w[i] = t * D[i];
    (*wg_out)[i] = w[i].to_double();
  }
  double res = 0.0;
  int rr = 0;
  for (int l = 0; l < K; ++l)
    for (int k = l; k < K; ++k, ++rr) {
      dd t(l == k ? -1.0 : 0.0);
      for (int g = 0; g < ng; ++g) t = t + A[(size_t)rr * ng + g] * w[g];
      res = std::max(res, std::fabs(t.to_double()));
    }
  *residual = res;
  return true;
}

}  // namespace

bool massive_quadrature(const std::vector<int>& groups, double m, double v0, int order,
                        Quadrature* q, double* residual, std::vector<double>* group_w,
                        bool precise) {
  const int ng = (int)groups.size() / 2;
  auto B = moment_basis(order);
  const int K = (int)B.size();
  std::vector<double> L = gram_shifted(order, m);
  if (!cholesky(L, K)) return false;
  // stencil and momenta, Eq. discrete-momentum-vectors / discrete-p0
  std::vector<int> vx, vy, gid;
  for (int g = 0; g < ng; ++g)
    for (auto v : fs_group(groups[2 * g], groups[2 * g + 1])) {
      vx.push_back(v.first);
      vy.push_back(v.second);
      gid.push_back(g);
    }
  const int Qf = (int)vx.size();
  std::vector<double> p0(Qf), px(Qf), py(Qf), J((size_t)Qf * K);
  for (int i = 0; i < Qf; ++i) {
    double v2 = v0 * v0 * (vx[i] * vx[i] + vy[i] * vy[i]);
    if (v2 >= 1.0) return false;
    double gam = 1.0 / std::sqrt(1.0 - v2);
    p0[i] = m * gam;
    px[i] = m * gam * v0 * vx[i];
    py[i] = m * gam * v0 * vy[i];
    // orthonormal basis J = L^{-1} phi' (G' = L L^T)
    std::vector<double> phi(K);
    eval_shifted(B, m, p0[i], px[i], py[i], phi.data());
    for (int k = 0; k < K; ++k) {
      double s = phi[k];
      for (int j = 0; j < k; ++j) s -= L[k * K + j] * J[(size_t)i * K + j];
      J[(size_t)i * K + k] = s / L[k * K + k];
    }
  }
  // Eq. mj-orthogonal-conditions, one unknown per FS group
  const int rows = K * (K + 1) / 2;
  std::vector<double> A((size_t)rows * ng, 0.0), b(rows, 0.0);
  int r = 0;
  for (int l = 0; l < K; ++l)
    for (int k = l; k < K; ++k, ++r) {
      for (int i = 0; i < Qf; ++i) A[(size_t)r * ng + gid[i]] += J[(size_t)i * K + l] * J[(size_t)i * K + k];
      b[r] = (l == k) ? 1.0 : 0.0;
    }
  std::vector<double> wg;
  double res = 0.0;
  if (precise) {
    if (!group_weights_dd(groups, m, v0, order, &wg, &res)) return false;
  } else {
    if (!least_squares(A, b, rows, ng, &wg)) return false;
    for (int rr = 0; rr < rows; ++rr) {
      double s = -b[rr];
      for (int g = 0; g < ng; ++g) s += A[(size_t)rr * ng + g] * wg[g];
      res = std::max(res, std::fabs(s));
    }
  }
  *residual = res;
  if (group_w) *group_w = wg;
  *q = Quadrature();
  q->m = m;
  q->order = order;
  q->v0 = v0;
  q->groups = groups;
  // Populations in orbit order (the kernels' symmetric evaluation relies on
  // it), each type in group order: eight-member orbits as the sign quartets
  // (a, b), (-a, b), (a, -b), (-a, -b) of the generator and of its swap; axis
  // quartets (p, 0), (-p, 0), (0, p), (0, -p); diagonal quartets (a, a),
  // (-a, a), (a, -a), (-a, -a); the rest population.
  auto emit = [&](int nx, int ny, double wgt) {
    const double v2 = v0 * v0 * (nx * nx + ny * ny);
    const double gam = 1.0 / std::sqrt(1.0 - v2);
    q->nx.push_back(nx);
    q->ny.push_back(ny);
    q->p0.push_back(m * gam);
    q->px.push_back(m * gam * v0 * nx);
    q->py.push_back(m * gam * v0 * ny);
    q->w.push_back(wgt);
  };
  for (int type = 0; type < 4; ++type) {
    for (int g = 0; g < ng; ++g) {
      if (wg[g] == 0.0) continue;
      const int a = std::abs(groups[2 * g]), b = std::abs(groups[2 * g + 1]);
      const int t = (a == 0 && b == 0) ? 3 : (a == 0 || b == 0) ? 1 : (a == b) ? 2 : 0;
      if (t != type) continue;
      if (t == 0) {
        const int sg[4][2] = {{1, 1}, {-1, 1}, {1, -1}, {-1, -1}};
        for (auto& z : sg) emit(z[0] * a, z[1] * b, wg[g]);
        for (auto& z : sg) emit(z[0] * b, z[1] * a, wg[g]);
      } else if (t == 1) {
        const int p = std::max(a, b);
        emit(p, 0, wg[g]); emit(-p, 0, wg[g]); emit(0, p, wg[g]); emit(0, -p, wg[g]);
      } else if (t == 2) {
        emit(a, a, wg[g]); emit(-a, a, wg[g]); emit(a, -a, wg[g]); emit(-a, -a, wg[g]);
      } else {
        emit(0, 0, wg[g]);
      }
    }
  }
  q->Q = (int)q->w.size();
  return true;
}

bool search_v0(const std::vector<int>& groups, double m, int order, double* v0_out,
               double* lo_out, double* hi_out) {
  double nmax = 0.0;
  for (size_t g = 0; g + 1 < groups.size(); g += 2)
    nmax = std::max(nmax, std::hypot((double)groups[g], (double)groups[g + 1]));
  if (nmax == 0.0) return false;
  const double vmax = 1.0 / nmax;
  const int npts = 4000;
  int best_lo = -1, best_hi = -1, run_lo = -1;
  for (int j = 1; j <= npts; ++j) {
    double v0 = vmax * j / (npts + 1.0);
    Quadrature q;
    double res = 1.0;
    std::vector<double> wg;
    bool ok = massive_quadrature(groups, m, v0, order, &q, &res, &wg) && res < 1e-9;
    if (ok)
      for (double x : wg) ok = ok && x >= 0.0;
    if (ok) {
      if (run_lo < 0) run_lo = j;
      if (best_lo < 0 || j - run_lo > best_hi - best_lo) { best_lo = run_lo; best_hi = j; }
    } else {
      run_lo = -1;
    }
  }
  if (best_lo < 0) return false;
  double lo = vmax * best_lo / (npts + 1.0), hi = vmax * best_hi / (npts + 1.0);
  *v0_out = 0.5 * (lo + hi);
  if (lo_out) *lo_out = lo;
  if (hi_out) *hi_out = hi;
  return true;
}

bool builtin_massive(double m, int order, Quadrature* q, std::string* err) {
  // the v0 scan is the expensive part: remember results per (m, order)
  static std::mutex mtx;
  static std::map<std::pair<double, int>, Quadrature> memo;
  {
    std::lock_guard<std::mutex> lock(mtx);
    auto it = memo.find({m, order});
    if (it != memo.end()) {
      *q = it->second;
      return true;
    }
  }
  const bool ok = builtin_massive_search(m, order, q, err);
  if (ok) {
    std::lock_guard<std::mutex> lock(mtx);
    memo[{m, order}] = *q;
  }
  return ok;
}

bool builtin_massive_search(double m, int order, Quadrature* q, std::string* err) {
  // Candidate stencils: the Sec. 5.3 worked example (order 2) and the five
  // (2+1)-d columns of App. H for the requested order.
  static const std::vector<std::vector<int>> o2 = {
      {0, 0, 1, 0, 1, 1, 2, 1, 2, 2, 3, 1},   // Sec. 5.3 example (m~ = 5)
      {0, 0, 1, 0, 1, 1, 2, 0, 2, 1, 2, 2},   // App. H G_A^(o2)
      {0, 0, 1, 0, 1, 1, 2, 2, 3, 2, 4, 0},   // G_B^(o2)
      {0, 0, 3, 3, 4, 2, 4, 3, 5, 0, 5, 1},   // G_C^(o2)
      {0, 0, 3, 1, 4, 2, 4, 3, 5, 0, 5, 1},   // G_D^(o2)
      {0, 0, 5, 2, 5, 3, 5, 4, 6, 0, 6, 2}};  // G_E^(o2)
  static const std::vector<std::vector<int>> o3 = {
      {0, 0, 1, 1, 4, 2, 5, 4, 5, 5, 6, 2, 6, 3, 6, 4, 7, 1, 7, 2},   // G_A^(o3)
      {0, 0, 1, 1, 2, 2, 4, 3, 5, 0, 5, 5, 6, 2, 6, 3, 6, 4, 7, 1},   // G_B^(o3)
      {0, 0, 1, 0, 2, 0, 2, 2, 3, 0, 3, 2, 3, 3, 4, 0, 4, 1, 4, 2},   // G_C^(o3)
      {0, 0, 1, 0, 1, 1, 2, 0, 2, 1, 3, 1, 3, 2, 3, 3, 4, 0, 4, 2},   // G_D^(o3)
      {0, 0, 1, 0, 1, 1, 2, 0, 2, 1, 2, 2, 3, 0, 3, 1, 3, 2, 3, 3}};  // G_E^(o3)
  const auto& cands = (order == 2) ? o2 : o3;
  if (order != 2 && order != 3) { *err = "order must be 2 or 3"; return false; }
  for (const auto& g : cands) {
    double v0;
    if (!search_v0(g, m, order, &v0, nullptr, nullptr)) continue;
    double res;
    if (massive_quadrature(g, m, v0, order, q, &res, nullptr, true) && res < 1e-9) return true;
  }
  *err = "no built-in stencil yields a non-negative quadrature for this mass and order";
  return false;
}

bool equilibrium_matrix(const Quadrature& q, std::vector<double>* H, std::string* err) {
  // H = W Phi G^{-1} in the basis of moment_basis; evaluated through the
  // shifted basis phi' = A^{-1} phi as H = W Phi' G'^{-1} A^{-1}, in
  // double-double and rounded once at the end.
  auto B = moment_basis(q.order);
  const int K = (int)B.size();
  std::vector<dd> Gi;
  if (!spd_inverse_dd(gram_shifted_dd(q.order, q.m), K, &Gi)) {
    *err = "Gram matrix not positive definite";
    return false;
  }
  const dd sg = dd_sqrt(dd(q.m) + dd(1.0));
  std::vector<int> partner(K, -1);
  for (int k = 0; k < K; ++k)
    if (B[k].e == 1)
      for (int j = 0; j < K; ++j)
        if (B[j].e == 0 && B[j].a == B[k].a && B[j].b == B[k].b) partner[k] = j;
  H->assign((size_t)q.Q * K, 0.0);
  std::vector<dd> phi(K), r(K), row(K);
  for (int i = 0; i < q.Q; ++i) {
    const dd s = dd(q.p0[i]) - dd(q.m), qx = dd(q.px[i]) / sg, qy = dd(q.py[i]) / sg;
    for (int k = 0; k < K; ++k) {
      dd v = B[k].e ? s : dd(1.0);
      for (int t = 0; t < B[k].a; ++t) v = v * qx;
      for (int t = 0; t < B[k].b; ++t) v = v * qy;
      phi[k] = v;
    }
    for (int k = 0; k < K; ++k) {
      dd t(0.0);
      for (int j = 0; j < K; ++j) t = t + phi[j] * Gi[j * K + k];
      r[k] = t;
    }
    for (int k = 0; k < K; ++k) row[k] = dd(0.0);
    // multiply by A^{-1}: phi'_k = sg^{-(a+b)} (phi_k - m phi_partner(k)) for e = 1.
    // Order 3 keeps the shifted p0 monomials (p0 - m) p^a p^b as the basis
    // (only the px, py scale is undone): the moments of that basis are
    // evaluated without cancellation, while those of p0^e p^a p^b at large m
    // cancel to a part in 1e3-1e4 in f^eq.
    const bool keep_shift = q.order == 3;
    for (int k = 0; k < K; ++k) {
      dd sc = dd(q.w[i]) * r[k];
      for (int t = 0; t < B[k].a + B[k].b; ++t) sc = sc / sg;
      row[k] = row[k] + sc;
      if (B[k].e == 1 && !keep_shift) row[partner[k]] = row[partner[k]] - dd(q.m) * sc;
    }
    for (int k = 0; k < K; ++k) (*H)[(size_t)i * K + k] = row[k].to_double();
  }
  return true;
}

void mj_moments_shifted3(double m, double n, const double U[3], double T, double* M) {
  // App. B moments (see mj_moments) of the order-3 basis with shifted p0
  // monomials: for X = 1, px, py, pxpx, pxpy, pypy,
  //   <(p0 - m) X> = <p0 X> - m <X>,
  // rewritten with U0 - 1 = |u|^2 / (U0 + 1), r2 - m = T (2m + 3T)/(m + T) and
  // r3 - m r2 = 3T (m^2 + 4mT + 5T^2)/(m + T) so that every term is positive.
  const double U0 = U[0], Ux = U[1], Uy = U[2];
  const double u0m1 = (Ux * Ux + Uy * Uy) / (U0 + 1.0);
  const double mT = m + T;
  const double r2 = (m * m + 3.0 * m * T + 3.0 * T * T) / mT;
  const double r3 = (m * m * m + 6.0 * m * m * T + 15.0 * m * T * T + 15.0 * T * T * T) / mT;
  const double A2 = r2 * u0m1 + T * (2.0 * m + 3.0 * T) / mT;                       // r2 U0 - m
  const double A3 = r3 * u0m1 + 3.0 * T * (m * m + 4.0 * m * T + 5.0 * T * T) / mT;  // r3 U0 - m r2
  M[0] = n / mT;
  M[1] = n * (u0m1 + T / mT);
  M[2] = n * Ux;
  M[3] = n * Uy;
  M[4] = n * Ux * A2;
  M[5] = n * Uy * A2;
  M[6] = n * (r2 * Ux * Ux + T);
  M[7] = n * r2 * Ux * Uy;
  M[8] = n * (r2 * Uy * Uy + T);
  M[9] = n * (Ux * Ux * A3 + T * A2);
  M[10] = n * Ux * Uy * A3;
  M[11] = n * (Uy * Uy * A3 + T * A2);
  M[12] = n * (r3 * Ux * Ux * Ux + 3.0 * T * r2 * Ux);
  M[13] = n * (r3 * Ux * Ux * Uy + T * r2 * Uy);
  M[14] = n * (r3 * Ux * Uy * Uy + T * r2 * Ux);
  M[15] = n * (r3 * Uy * Uy * Uy + 3.0 * T * r2 * Uy);
}

void mj_moments(int order, double m, double n, const double U[3], double T, double* M) {
  if (order == 3) {
    mj_moments_shifted3(m, n, U, T, M);
    return;
  }
  // App. B: B Z^{a1..ar} = n T^{r-1} sum_k (-1)^k (A_{r-k}/A_1) <U_{r-2k} eta_k>,
  // with, for d = 2 (half-integer Bessel functions are elementary):
  //   A_0/(A_1 T) = 1/(m + T), T A_2/A_1 = (m^2 + 3mT + 3T^2)/(m + T),
  //   T^2 A_3/A_1 = (m^3 + 6m^2 T + 15 m T^2 + 15 T^3)/(m + T).
  const double eta[3] = {1.0, -1.0, -1.0};
  const double r0 = 1.0 / (m + T);
  const double r2 = (m * m + 3.0 * m * T + 3.0 * T * T) / (m + T);
  const double r3 = (m * m * m + 6.0 * m * m * T + 15.0 * m * T * T + 15.0 * T * T * T) / (m + T);
  auto Bs = moment_basis(order);
  for (size_t k = 0; k < Bs.size(); ++k) {
    int idx[4], r = 0;
    for (int i = 0; i < Bs[k].e; ++i) idx[r++] = 0;
    for (int i = 0; i < Bs[k].a; ++i) idx[r++] = 1;
    for (int i = 0; i < Bs[k].b; ++i) idx[r++] = 2;
    double v;
    if (r == 0) v = n * r0;
    else if (r == 1) v = n * U[idx[0]];
    else if (r == 2) {
      double e01 = idx[0] == idx[1] ? eta[idx[0]] : 0.0;
      v = n * (r2 * U[idx[0]] * U[idx[1]] - T * e01);
    } else {
      int a = idx[0], b = idx[1], c = idx[2];
      double eab = a == b ? eta[a] : 0.0, eac = a == c ? eta[a] : 0.0, ebc = b == c ? eta[b] : 0.0;
      v = n * (r3 * U[a] * U[b] * U[c] - T * r2 * (eab * U[c] + eac * U[b] + ebc * U[a]));
    }
    M[k] = v;
  }
}

// ---------------------------------------------------------------------------
// (3+1)-d massless tables, order 2 (App. H "(3+1) dimensions").
// ---------------------------------------------------------------------------

namespace {

dd dd_factorial(int k) {
  dd r(1.0);
  for (int t = 2; t <= k; ++t) r = r * dd((double)t);
  return r;
}

dd dd_dfact(int k) {
  dd r(1.0);
  for (int t = k; t > 1; t -= 2) r = r * dd((double)t);
  return r;
}

// E_omega[p0^c0 px^a py^b pz^c] for omega = e^{-p0} on the light cone
// (d^3p/p0 = p0 dp0 dOmega), normalised to 1: the angular mean of
// nx^a ny^b nz^c, (a-1)!!(b-1)!!(c-1)!!/(a+b+c+1)!! for even a, b, c, times
// (c0+a+b+c+1)!.
dd omega_moment3_dd(int c0, int a, int b, int c) {
  if ((a & 1) || (b & 1) || (c & 1)) return dd(0.0);
  return dd_dfact(a - 1) * dd_dfact(b - 1) * dd_dfact(c - 1) / dd_dfact(a + b + c + 1) *
         dd_factorial(c0 + a + b + c + 1);
}

}  // namespace

const int kBasis3[14][4] = {{0, 0, 0, 0}, {1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, 1, 0}, {0, 0, 0, 1},
                             {1, 1, 0, 0}, {1, 0, 1, 0}, {1, 0, 0, 1}, {0, 2, 0, 0}, {0, 1, 1, 0},
                             {0, 1, 0, 1}, {0, 0, 2, 0}, {0, 0, 1, 1}, {0, 0, 0, 2}};
const int kBasis3o3[30][4] = {
    {0, 0, 0, 0}, {1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, 1, 0}, {0, 0, 0, 1},
    {1, 1, 0, 0}, {1, 0, 1, 0}, {1, 0, 0, 1}, {0, 2, 0, 0}, {0, 1, 1, 0},
    {0, 1, 0, 1}, {0, 0, 2, 0}, {0, 0, 1, 1}, {0, 0, 0, 2},
    {1, 2, 0, 0}, {1, 1, 1, 0}, {1, 1, 0, 1}, {1, 0, 2, 0}, {1, 0, 1, 1}, {1, 0, 0, 2},
    {0, 3, 0, 0}, {0, 2, 1, 0}, {0, 2, 0, 1}, {0, 1, 2, 0}, {0, 1, 1, 1}, {0, 1, 0, 2},
    {0, 0, 3, 0}, {0, 0, 2, 1}, {0, 0, 1, 2}, {0, 0, 0, 3}};

bool massless3_tables(int order, Quadrature3* q, std::string* err) {
  // Order 2: stencil {(+-2, +-2, +-1)FS, (+-3, 0, 0)FS} (all of length 3: the
  // printed first group, (+-2, +-1, +-1), is not of the common length a
  // massless stencil needs), weights read shell by shell, per shell the
  // (2, 2, 1) group then the (3, 0, 0) group.  Order 3: stencil {(+-4, +-4,
  // +-3)FS, (+-5, +-4, 0)FS, (+-6, +-2, +-1)FS} (length sqrt(41)), weights shell
  // by shell, per shell the groups in that order.  These readings integrate
  // the weight's moments up to degree 2N; the others do not.  Shell energies
  // p0_j as printed; p_ij = p0_j (1, n_i / |n_i|).
  static const double sh2[3] = {0.9358222275240878, 3.3054072893322786, 7.7587704831436335};
  static const double col2[6] = {0.0245283950433191, 0.0, 0.0163006691342629, 0.0,
                                 0.0003891858228425, 0.0017936666649682};
  static const int gen2[2][3] = {{2, 2, 1}, {3, 0, 0}};
  static const double sh3[4] = {0.7432919279814314, 2.5716350076462784, 5.7311787516890996,
                                10.953894312683190};
  static const double col3[12] = {0.0, 0.0, 0.0093098040253911, 0.0085195569675087, 0.0,
                                  0.0056909667738262, 0.0013041770173120, 0.0, 0.0008932820065742,
                                  0.0000029126213348, 0.0000338363537565, 0.0000090390475856};
  static const int gen3[3][3] = {{4, 4, 3}, {5, 4, 0}, {6, 2, 1}};
  if (order != 2 && order != 3) { *err = "3-d order must be 2 or 3"; return false; }
  const int ns = order == 2 ? 3 : 4, ng = order == 2 ? 2 : 3;
  const double* shells = order == 2 ? sh2 : sh3;
  const double* col = order == 2 ? col2 : col3;
  *q = Quadrature3();
  q->order = order;
  q->K = order == 2 ? 14 : 30;
  for (int j = 0; j < ns; ++j)
    for (int g = 0; g < ng; ++g) {
      const double wgt = col[ng * j + g];
      if (wgt == 0.0) continue;
      const int* gen = order == 2 ? gen2[g] : gen3[g];
      // the distinct permutations of |gen| (descending), each followed by its
      // sign variants: member s negates component k where bit k of s is set,
      // s running over the subsets of the non-zero components
      std::set<std::array<int, 3>, std::greater<std::array<int, 3>>> pats;
      int perm[3] = {0, 1, 2};
      do {
        pats.insert({gen[perm[0]], gen[perm[1]], gen[perm[2]]});
      } while (std::next_permutation(perm, perm + 3));
      for (const auto& a : pats) {
        int mask = 0;
        for (int k = 0; k < 3; ++k) mask |= (a[k] != 0) << k;
        q->orbit_mask.push_back(mask);
        const double len = std::sqrt((double)(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]));
        for (int sgn = 0; sgn < 8; ++sgn) {
          if (sgn & ~mask) continue;
          for (int k = 0; k < 3; ++k) q->n.push_back(((sgn >> k) & 1 ? -1 : 1) * a[k]);
          q->p.push_back(shells[j]);
          for (int k = 0; k < 3; ++k) q->p.push_back(shells[j] * (((sgn >> k) & 1 ? -1 : 1) * a[k]) / len);
          q->w.push_back(wgt);
        }
      }
    }
  q->Q = (int)q->w.size();
  if (q->Q > (order == 2 ? kMaxQ3 : kMaxQ3o3)) { *err = "3-d stencil larger than the kernels accept"; return false; }
  // H = W Phi G^{-1} in double-double, Phi and G in the basis kBasis3 / kBasis3o3
  const int K = q->K;
  const int (*B)[4] = order == 2 ? kBasis3 : kBasis3o3;
  std::vector<dd> G(K * K), Gi;
  for (int k = 0; k < K; ++k)
    for (int l = 0; l < K; ++l)
      G[k * K + l] = omega_moment3_dd(B[k][0] + B[l][0], B[k][1] + B[l][1], B[k][2] + B[l][2], B[k][3] + B[l][3]);
  if (!spd_inverse_dd(G, K, &Gi)) { *err = "3-d Gram matrix not positive definite"; return false; }
  q->H.assign((size_t)q->Q * K, 0.0);
  std::vector<dd> phi(K);
  for (int i = 0; i < q->Q; ++i) {
    const double* pi = &q->p[4 * i];
    for (int k = 0; k < K; ++k) {
      dd v(1.0);
      for (int c = 0; c < 4; ++c)
        for (int t = 0; t < B[k][c]; ++t) v = v * dd(pi[c]);
      phi[k] = v;
    }
    for (int k = 0; k < K; ++k) {
      dd t(0.0);
      for (int l = 0; l < K; ++l) t = t + phi[l] * Gi[l * K + k];
      q->H[(size_t)i * K + k] = (dd(q->w[i]) * t).to_double();
    }
  }
  // the sign-orbit identities of H, checked exactly
  q->sym = true;
  for (size_t r = 0, i0 = 0; r < q->orbit_mask.size(); ++r) {
    const int mask = q->orbit_mask[r];
    int s = 0;
    for (int sgn = 0; sgn < 8; ++sgn) {
      if (sgn & ~mask) continue;
      const size_t i = i0 + s++;
      for (int k = 0; k < K; ++k) {
        int par = 0;
        for (int c = 0; c < 3; ++c) par ^= ((sgn >> c) & 1) & (B[k][1 + c] & 1);
        const double want = par ? -q->H[i0 * K + k] : q->H[i0 * K + k];
        if (q->H[i * K + k] != want) q->sym = false;
      }
    }
    i0 += s;
  }
  return true;
}

}  // namespace rlbm

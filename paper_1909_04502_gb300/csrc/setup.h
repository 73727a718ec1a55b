// Host-side FP64 construction of the RLBM lattice tables (Sec. 5.2-5.3,
// App. F-H of arXiv:1909.04502).  No CUDA in here.
#pragma once
#include <string>
#include <vector>

namespace rlbm {

constexpr int kMaxQ = 72;   // largest population count the kernels accept
constexpr int kMaxK = 16;   // moment-vector length at order 3

// One discrete momentum set {n_i, p_i^mu, w_i} (App. H, Eq. discrete-momentum-vectors,
// Eq. ur-discrete-momentum-vectors).
struct Quadrature {
  int Q = 0;
  std::vector<int> nx, ny;            // integer stencil vectors n_i
  std::vector<double> p0, px, py, w;  // momenta p~_i^mu and weights
  double m = 0.0;                     // rest mass m~
  int order = 2;                      // expansion order N
  double v0 = 0.0;                    // massive parametrisation (0 for m~ = 0)
  std::vector<int> groups;            // generator vectors (x, y) of the FS stencil (massive)
};

// Monomial basis of the equilibrium moment vector: p0^e px^a py^b with e in
// {0, 1} and e + a + b <= order.  On the mass shell p0^2 = m^2 + px^2 + py^2,
// so these span every polynomial of degree <= order in p^mu.
struct Monomial { int e, a, b; };
std::vector<Monomial> moment_basis(int order);

// Gauss-Laguerre rule with n nodes (weight e^{-s} on [0, inf)).
void gauss_laguerre(int n, std::vector<double>& x, std::vector<double>& w);

// E_omega[p0^c px^a py^b] for d = 2 with the App. F weight e^m/(2 pi) e^{-p0}
// (normalised to one, Eq. numerical-normalization-cond).
double omega_moment(int c, int a, int b, double m);

// Gram matrix of moment_basis(order) under omega (row-major K x K).
std::vector<double> gram_matrix(int order, double m);

// Symmetric positive definite helpers (row-major n x n).
bool cholesky(std::vector<double>& a, int n);              // in place, lower factor
std::vector<double> spd_inverse(const std::vector<double>& a, int n, bool* ok);

// Massless 2-d tables of App. H (order 2 or 3).
bool massless_quadrature(int order, Quadrature* q, std::string* err);

// Massive quadrature on the FS stencil generated by groups (Sec. 5.3):
// weights per group from Eq. mj-orthogonal-conditions by least squares.
// Returns the largest residual of the conditions in *residual.  precise
// solves in double-double (the tables a lattice runs on); the fast double
// solve serves the v0 scan, which needs only the residual and the signs.
bool massive_quadrature(const std::vector<int>& groups, double m, double v0, int order,
                        Quadrature* q, double* residual, std::vector<double>* group_w,
                        bool precise = false);

// Line search of Sec. 5.3: scan v0 over (0, 1/max||n||) and return the middle
// of the widest interval where the conditions hold and every weight is >= 0.
bool search_v0(const std::vector<int>& groups, double m, int order, double* v0_out,
               double* lo_out, double* hi_out);

// Built-in stencil choice for a mass and order (tries a fixed candidate list
// of App. H stencils and the Sec. 5.3 example).
bool builtin_massive(double m, int order, Quadrature* q, std::string* err);
bool builtin_massive_search(double m, int order, Quadrature* q, std::string* err);   // uncached

// Equilibrium matrix H (Q x K, row-major) with f^eq_i = sum_k H_ik M_k(n, U, T),
// M the Maxwell-Juttner moments of moment_basis(order), where at order 3 the
// monomials with p0 are taken shifted, (p0 - m) p^a p^b:
// H = W Phi G^{-1}  (Eq. mj-discrete-feq with J = C phi and C^T C = G^{-1}).
bool equilibrium_matrix(const Quadrature& q, std::vector<double>* H, std::string* err);

// Maxwell-Juttner moments of that basis for (n, U, T) (App. B); order 3
// through mj_moments_shifted3.
void mj_moments(int order, double m, double n, const double U[3], double T, double* M);
void mj_moments_shifted3(double m, double n, const double U[3], double T, double* M);


// (3+1)-d massless stencils of orders 2 and 3 (App. H, read as in setup.cpp)
// with their equilibrium matrices: f^eq_i = sum_k H_ik M_k, M the MJ moments
// of the basis kBasis3 (order 2) or kBasis3o3 (order 3).
constexpr int kMaxQ3 = 80;       // order 2 (Q = 78)
constexpr int kMaxQ3o3 = 288;    // order 3
struct Quadrature3 {
  int Q = 0, order = 2, K = 14;
  std::vector<int> n;       // 3 Q stencil vectors
  std::vector<double> p;    // 4 Q momenta (p0, px, py, pz)
  std::vector<double> w;    // Q weights
  std::vector<double> H;    // Q x K
  // Sign orbits: populations come in runs that share |n_i|, p0 and w; member
  // s of a run negates component k where bit k of s is set (s over the
  // components that are not zero, in increasing order).  orbit_mask[r] holds
  // the run's non-zero components (bit k: component k); sym is true when
  // every run also satisfies H_{s,k} = sigma_k(s) H_{0,k} exactly, sigma_k(s)
  // the sign the basis member k takes under the flips of s.
  std::vector<int> orbit_mask;
  bool sym = false;
};
extern const int kBasis3[14][4];     // order 2: 1 | p0 px py pz | p0px p0py p0pz pxpx pxpy pxpz pypy pypz pzpz
extern const int kBasis3o3[30][4];   // order 3: the 14 above, then p0 x (pxpx pxpy pxpz pypy pypz pzpz) and
                                     // pxpxpx pxpxpy pxpxpz pxpypy pxpypz pxpzpz pypypy pypypz pypzpz pzpzpz
bool massless3_tables(int order, Quadrature3* q, std::string* err);

}  // namespace rlbm

// Reference-element construction (host, FP64).  See fr_ref.hpp.
//
// Point sets (Section 2, Fig. 1): tensor Gauss-Legendre points on the
// hexahedron and on quadrilateral faces; alpha-optimised warp-and-blend
// nodes (Hesthaven & Warburton 2008) on the tetrahedron; triangular faces
// carry the face restriction of the tetrahedron set (3D alpha of the same
// order), so tetrahedron flux points are a subset of its solution points as
// Fig. 1(b,c) shows; prisms use the 2D-optimised triangle set tensored with
// Gauss-Legendre points along the axis.
//
// Correction (Eq. FRfinal): the DG choice of Huynh (2007), written for every
// element type as the DG lift  int v div~g_s = int_face v l_s  for all v in
// the solution space, evaluated with exact Gauss rules on the faces.
#include "fr_ref.hpp"

#include <algorithm>
#include <cmath>
#include <stdexcept>

namespace frgb {

static const double kAlpha2D[15] = {0.0, 0.0, 1.4152, 0.1001, 0.2751, 0.9800,
                                    1.0999, 1.2832, 1.3648, 1.4773, 1.4959,
                                    1.5743, 1.5770, 1.6223, 1.6258};
static const double kAlpha3D[15] = {0.0, 0.0, 0.0, 0.1002, 1.1332, 1.5608,
                                    1.3413, 1.2577, 1.1603, 1.10153, 0.6080,
                                    0.4523, 0.8856, 0.8717, 0.9655};

// ---------------------------------------------------------------- 1D tools
double jacobi_p(int n, double a, double b, double x) {
  // orthonormal Jacobi polynomial by the three-term recurrence
  double g0 = std::pow(2.0, a + b + 1) / (a + b + 1) * std::tgamma(a + 1) *
              std::tgamma(b + 1) / std::tgamma(a + b + 1);
  double p0 = 1.0 / std::sqrt(g0);
  if (n == 0) return p0;
  double g1 = (a + 1) * (b + 1) / (a + b + 3) * g0;
  double p1 = ((a + b + 2) * x / 2 + (a - b) / 2) / std::sqrt(g1);
  if (n == 1) return p1;
  double aold = 2 / (2 + a + b) * std::sqrt((a + 1) * (b + 1) / (a + b + 3));
  for (int i = 1; i < n; ++i) {
    double h1 = 2 * i + a + b;
    double anew = 2 / (h1 + 2) *
                  std::sqrt((i + 1) * (i + 1 + a + b) * (i + 1 + a) *
                            (i + 1 + b) / (h1 + 1) / (h1 + 3));
    double bnew = -(a * a - b * b) / h1 / (h1 + 2);
    double p2 = (-aold * p0 + (x - bnew) * p1) / anew;
    p0 = p1;
    p1 = p2;
    aold = anew;
  }
  return p1;
}

double jacobi_dp(int n, double a, double b, double x) {
  if (n == 0) return 0.0;
  return std::sqrt(n * (n + a + b + 1)) * jacobi_p(n - 1, a + 1, b + 1, x);
}

static void legendre(int n, double x, double* pn, double* dpn) {
  double p0 = 1.0, p1 = x;
  if (n == 0) {
    *pn = 1.0;
    *dpn = 0.0;
    return;
  }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  *pn = p1;
  *dpn = n * (x * p1 - p0) / (x * x - 1.0);
}

void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = -std::cos(M_PI * (4.0 * i + 3.0) / (4.0 * n + 2.0));
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(n, z, &p, &dp);
      double dz = p / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p, dp;
    legendre(n, z, &p, &dp);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  // sort ascending
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (x[j] < x[i]) {
        std::swap(x[i], x[j]);
        std::swap(w[i], w[j]);
      }
}

void gauss_lobatto(int n, double* x) {
  // n points; interior ones are the roots of P'_{n-1}
  x[0] = -1.0;
  x[n - 1] = 1.0;
  int m = n - 1;
  for (int i = 1; i < n - 1; ++i) {
    double z = -std::cos(M_PI * i / m);
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(m, z, &p, &dp);
      double d2 = (2 * z * dp - m * (m + 1) * p) / (1 - z * z);
      double dz = dp / d2;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
  }
}

void gauss_jacobi(int n, double a, double b, double* x, double* w) {
  // Nodes: roots of the degree-n orthonormal Jacobi polynomial by Newton's
  // method, each iteration deflated by the roots already found.  Weights:
  // Christoffel numbers 1 / sum_{k<n} p_k(x_i)^2 of the orthonormal family.
  for (int k = 0; k < n; ++k) {
    double z = -std::cos(M_PI * (2.0 * k + 1.0) / (2.0 * n));
    if (k > 0) z = 0.5 * (z + x[k - 1]);
    for (int it = 0; it < 200; ++it) {
      double s = 0.0;
      for (int j = 0; j < k; ++j) s += 1.0 / (z - x[j]);
      const double p = jacobi_p(n, a, b, z);
      const double dz = -p / (jacobi_dp(n, a, b, z) - p * s);
      z += dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[k] = z;
  }
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (x[j] < x[i]) std::swap(x[i], x[j]);
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) {
      const double p = jacobi_p(k, a, b, x[i]);
      s += p * p;
    }
    w[i] = 1.0 / s;
  }
}

void aa_rule(int kind, int qdeg, std::vector<double>& xq, std::vector<double>& wq) {
  const int n = qdeg / 2 + 1;
  std::vector<double> xa(n), wa(n), xb(n), wb(n), xc(n), wc(n);
  gauss_legendre(n, xa.data(), wa.data());
  if (kind == EK_HEX) {
    xb = xc = xa;
    wb = wc = wa;
  } else if (kind == EK_PRI) {
    gauss_jacobi(n, 1.0, 0.0, xb.data(), wb.data());
    xc = xa;
    wc = wa;
  } else {
    gauss_jacobi(n, 1.0, 0.0, xb.data(), wb.data());
    gauss_jacobi(n, 2.0, 0.0, xc.data(), wc.data());
  }
  xq.clear();
  wq.clear();
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        const double A = xa[i], B = xb[j], C = xc[k];
        const double w = wa[i] * wb[j] * wc[k];
        if (kind == EK_HEX) {
          xq.insert(xq.end(), {A, B, C});
          wq.push_back(w);
        } else if (kind == EK_PRI) {  // (a, b) -> triangle, Jacobian (1-b)/2
          xq.insert(xq.end(), {0.5 * (1 + A) * (1 - B) - 1, B, C});
          wq.push_back(0.5 * w);
        } else {  // Jacobian (1-b)(1-c)^2 / 8: weights of the Jacobi factors
          xq.insert(xq.end(), {0.25 * (1 + A) * (1 - B) * (1 - C) - 1,
                               0.5 * (1 + B) * (1 - C) - 1, C});
          wq.push_back(0.125 * w);
        }
      }
}

void aa_operators(const RefElement& R, const std::vector<double>& xq,
                  const std::vector<double>& wq, std::vector<double>& B,
                  std::vector<double>& P) {
  const int nu = R.nupts, nq = int(wq.size());
  std::vector<double> phi(size_t(nq) * nu), V(size_t(nu) * nu);
  R.basis(nq, xq.data(), phi.data());
  R.basis(nu, R.upts.data(), V.data());
  B.assign(size_t(nq) * nu, 0.0);
  for (int q = 0; q < nq; ++q)
    for (int z = 0; z < nu; ++z) {
      double s = 0.0;
      for (int k = 0; k < nu; ++k) s += phi[size_t(q) * nu + k] * R.vdm_inv[size_t(k) * nu + z];
      B[size_t(q) * nu + z] = s;
    }
  P.assign(size_t(nu) * nq, 0.0);
  for (int z = 0; z < nu; ++z)
    for (int q = 0; q < nq; ++q) {
      double s = 0.0;
      for (int k = 0; k < nu; ++k) s += V[size_t(z) * nu + k] * phi[size_t(q) * nu + k];
      P[size_t(z) * nq + q] = s * wq[q];
    }
}

bool invert(int n, const double* A, double* Ainv) {
  std::vector<double> a(A, A + n * n);
  std::vector<int> piv(n);
  for (int i = 0; i < n * n; ++i) Ainv[i] = 0.0;
  for (int i = 0; i < n; ++i) Ainv[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int r = c;
    for (int k = c + 1; k < n; ++k)
      if (std::fabs(a[k * n + c]) > std::fabs(a[r * n + c])) r = k;
    if (std::fabs(a[r * n + c]) < 1e-300) return false;
    if (r != c)
      for (int k = 0; k < n; ++k) {
        std::swap(a[r * n + k], a[c * n + k]);
        std::swap(Ainv[r * n + k], Ainv[c * n + k]);
      }
    double d = 1.0 / a[c * n + c];
    for (int k = 0; k < n; ++k) {
      a[c * n + k] *= d;
      Ainv[c * n + k] *= d;
    }
    for (int r2 = 0; r2 < n; ++r2) {
      if (r2 == c) continue;
      double f = a[r2 * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        a[r2 * n + k] -= f * a[c * n + k];
        Ainv[r2 * n + k] -= f * Ainv[c * n + k];
      }
    }
  }
  return true;
}

// ----------------------------------------------------- warp-and-blend sets
static double warp1d(int n, double r) {
  // (GLL - equispaced) interpolated at r and divided by 1 - r^2
  std::vector<double> gll(n + 1), req(n + 1);
  gauss_lobatto(n + 1, gll.data());
  for (int i = 0; i <= n; ++i) req[i] = -1.0 + 2.0 * i / n;
  double w = 0.0;
  for (int i = 0; i <= n; ++i) {
    double l = 1.0;
    for (int j = 0; j <= n; ++j)
      if (j != i) l *= (r - req[j]) / (req[i] - req[j]);
    w += l * (gll[i] - req[i]);
  }
  if (std::fabs(r) < 1.0 - 1e-10) w /= (1.0 - r * r);
  else w = 0.0;
  return w;
}

static void tri_shift(int n, double alpha, double l1, double l2, double l3,
                      double* dx, double* dy) {
  double w1 = warp1d(n, l3 - l2), w2 = warp1d(n, l1 - l3),
         w3 = warp1d(n, l2 - l1);
  double f1 = 4 * l2 * l3 * w1 * (1 + (alpha * l1) * (alpha * l1));
  double f2 = 4 * l1 * l3 * w2 * (1 + (alpha * l2) * (alpha * l2));
  double f3 = 4 * l1 * l2 * w3 * (1 + (alpha * l3) * (alpha * l3));
  double c2 = std::cos(2 * M_PI / 3), s2 = std::sin(2 * M_PI / 3);
  double c4 = std::cos(4 * M_PI / 3), s4 = std::sin(4 * M_PI / 3);
  *dx = f1 + c2 * f2 + c4 * f3;
  *dy = s2 * f2 + s4 * f3;
}

// triangle nodes on the reference triangle (-1,-1),(1,-1),(-1,1)
static std::vector<double> tri_nodes(int n, double alpha) {
  std::vector<double> out;
  if (n == 0) return {-1.0 / 3.0, -1.0 / 3.0};
  const double s3 = std::sqrt(3.0);
  for (int i = 0; i <= n; ++i)
    for (int j = 0; j <= n - i; ++j) {
      double l1 = double(i) / n, l3 = double(j) / n, l2 = 1.0 - l1 - l3;
      double x = -l2 + l3, y = (-l2 - l3 + 2 * l1) / s3;
      double dx, dy;
      tri_shift(n, alpha, l1, l2, l3, &dx, &dy);
      x += dx;
      y += dy;
      double b1 = (s3 * y + 1.0) / 3.0;
      double b2 = (-3.0 * x - s3 * y + 2.0) / 6.0;
      double b3 = (3.0 * x - s3 * y + 2.0) / 6.0;
      out.push_back(-b2 + b3 - b1);
      out.push_back(-b2 - b3 + b1);
    }
  return out;
}

static double eval_warp(int n, const std::vector<double>& xn, double xo) {
  std::vector<double> xeq(n + 1);
  for (int i = 0; i <= n; ++i) xeq[i] = -1.0 + 2.0 * (n - i) / n;
  double w = 0.0;
  for (int i = 0; i <= n; ++i) {
    double d = xn[i] - xeq[i];
    for (int j = 1; j < n; ++j)
      if (i != j) d *= (xo - xeq[j]) / (xeq[i] - xeq[j]);
    if (i != 0) d = -d / (xeq[i] - xeq[0]);
    if (i != n) d = d / (xeq[i] - xeq[n]);
    w += d;
  }
  return w;
}

static void eval_shift(int n, double alpha, double l1, double l2, double l3,
                       double* dx, double* dy) {
  std::vector<double> g(n + 1);
  gauss_lobatto(n + 1, g.data());
  for (auto& v : g) v = -v;
  double w1 = eval_warp(n, g, l3 - l2), w2 = eval_warp(n, g, l1 - l3),
         w3 = eval_warp(n, g, l2 - l1);
  double f1 = 4 * l2 * l3 * w1 * (1 + (alpha * l1) * (alpha * l1));
  double f2 = 4 * l3 * l1 * w2 * (1 + (alpha * l2) * (alpha * l2));
  double f3 = 4 * l1 * l2 * w3 * (1 + (alpha * l3) * (alpha * l3));
  double c2 = std::cos(2 * M_PI / 3), s2 = std::sin(2 * M_PI / 3);
  double c4 = std::cos(4 * M_PI / 3), s4 = std::sin(4 * M_PI / 3);
  *dx = f1 + c2 * f2 + c4 * f3;
  *dy = s2 * f2 + s4 * f3;
}

static std::vector<double> tet_nodes(int n) {
  if (n == 0) return {-0.5, -0.5, -0.5};
  double alpha = n <= 15 ? kAlpha3D[n - 1] : 1.0;
  const double tol = 1e-10;
  double v[4][3] = {{-1.0, -1.0 / std::sqrt(3.0), -1.0 / std::sqrt(6.0)},
                    {1.0, -1.0 / std::sqrt(3.0), -1.0 / std::sqrt(6.0)},
                    {0.0, 2.0 / std::sqrt(3.0), -1.0 / std::sqrt(6.0)},
                    {0.0, 0.0, 3.0 / std::sqrt(6.0)}};
  double t1[4][3], t2[4][3];
  for (int k = 0; k < 3; ++k) {
    t1[0][k] = v[1][k] - v[0][k];
    t1[1][k] = v[1][k] - v[0][k];
    t1[2][k] = v[2][k] - v[1][k];
    t1[3][k] = v[2][k] - v[0][k];
    t2[0][k] = v[2][k] - 0.5 * (v[0][k] + v[1][k]);
    t2[1][k] = v[3][k] - 0.5 * (v[0][k] + v[1][k]);
    t2[2][k] = v[3][k] - 0.5 * (v[1][k] + v[2][k]);
    t2[3][k] = v[3][k] - 0.5 * (v[0][k] + v[2][k]);
  }
  for (int f = 0; f < 4; ++f) {
    double a = std::sqrt(t1[f][0] * t1[f][0] + t1[f][1] * t1[f][1] +
                         t1[f][2] * t1[f][2]);
    double b = std::sqrt(t2[f][0] * t2[f][0] + t2[f][1] * t2[f][1] +
                         t2[f][2] * t2[f][2]);
    for (int k = 0; k < 3; ++k) {
      t1[f][k] /= a;
      t2[f][k] /= b;
    }
  }
  // inverse of the equilateral frame [v1-v0, v2-v0, v3-v0]
  double A[9], Ai[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) A[r * 3 + c] = v[c + 1][r] - v[0][r];
  invert(3, A, Ai);
  std::vector<double> out;
  for (int k = 0; k <= n; ++k)
    for (int j = 0; j <= n - k; ++j)
      for (int i = 0; i <= n - k - j; ++i) {
        double r = -1.0 + 2.0 * i / n, s = -1.0 + 2.0 * j / n,
               t = -1.0 + 2.0 * k / n;
        double L1 = (1 + t) / 2, L2 = (1 + s) / 2, L3 = -(1 + r + s + t) / 2,
               L4 = (1 + r) / 2;
        double X[3], sh[3] = {0, 0, 0};
        for (int c = 0; c < 3; ++c)
          X[c] = L3 * v[0][c] + L4 * v[1][c] + L2 * v[2][c] + L1 * v[3][c];
        double La_[4] = {L1, L2, L3, L4};
        int perm[4][4] = {{0, 1, 2, 3}, {1, 0, 2, 3}, {2, 0, 3, 1}, {3, 0, 2, 1}};
        for (int f = 0; f < 4; ++f) {
          double La = La_[perm[f][0]], Lb = La_[perm[f][1]],
                 Lc = La_[perm[f][2]], Ld = La_[perm[f][3]];
          double w1, w2;
          eval_shift(n, alpha, Lb, Lc, Ld, &w1, &w2);
          double blend = Lb * Lc * Ld;
          double den = (Lb + 0.5 * La) * (Lc + 0.5 * La) * (Ld + 0.5 * La);
          if (den > tol) blend = (1 + (alpha * La) * (alpha * La)) * blend / den;
          int nz = (Lb > tol) + (Lc > tol) + (Ld > tol);
          if (La < tol && nz < 3) {
            for (int c = 0; c < 3; ++c) sh[c] = w1 * t1[f][c] + w2 * t2[f][c];
          } else {
            for (int c = 0; c < 3; ++c)
              sh[c] += blend * w1 * t1[f][c] + blend * w2 * t2[f][c];
          }
        }
        double d[3];
        for (int c = 0; c < 3; ++c) d[c] = X[c] + sh[c] - v[0][c];
        for (int r2 = 0; r2 < 3; ++r2) {
          double lam = Ai[r2 * 3 + 0] * d[0] + Ai[r2 * 3 + 1] * d[1] +
                       Ai[r2 * 3 + 2] * d[2];
          out.push_back(-1.0 + 2.0 * lam);
        }
      }
  return out;
}

// ------------------------------------------------------------ modal bases
static void tri_collapse(double r, double s, double* a, double* b) {
  *a = std::fabs(1.0 - s) > 1e-14 ? 2.0 * (1.0 + r) / (1.0 - s) - 1.0 : -1.0;
  *b = s;
}

static int tri_nm(int p) { return (p + 1) * (p + 2) / 2; }

// value and gradient of the orthonormal triangle basis, mode order (i, j)
static void tri_eval(int p, double r, double s, double* v, double* dr,
                     double* ds) {
  double a, b;
  tri_collapse(r, s, &a, &b);
  int m = 0;
  for (int i = 0; i <= p; ++i)
    for (int j = 0; j <= p - i; ++j, ++m) {
      double fa = jacobi_p(i, 0, 0, a), dfa = jacobi_dp(i, 0, 0, a);
      double gb = jacobi_p(j, 2 * i + 1, 0, b),
             dgb = jacobi_dp(j, 2 * i + 1, 0, b);
      double h = 0.5 * (1.0 - b);
      v[m] = std::sqrt(2.0) * fa * gb * std::pow(1.0 - b, i);
      if (dr) {
        double mr = dfa * gb, ms = dfa * gb * 0.5 * (1.0 + a);
        if (i > 0) {
          mr *= std::pow(h, i - 1);
          ms *= std::pow(h, i - 1);
        }
        double tmp = dgb * std::pow(h, i);
        if (i > 0) tmp -= 0.5 * i * gb * std::pow(h, i - 1);
        ms += fa * tmp;
        double sc = std::pow(2.0, i + 0.5);
        dr[m] = mr * sc;
        ds[m] = ms * sc;
      }
    }
}

static void tet_eval(int p, const double* x, double* v, double* g0,
                     double* g1, double* g2) {
  double r = x[0], s = x[1], t = x[2];
  double a = std::fabs(s + t) > 1e-14 ? 2.0 * (1.0 + r) / (-s - t) - 1.0 : -1.0;
  double b = std::fabs(1.0 - t) > 1e-14 ? 2.0 * (1.0 + s) / (1.0 - t) - 1.0
                                         : -1.0;
  double c = t;
  int m = 0;
  for (int i = 0; i <= p; ++i)
    for (int j = 0; j <= p - i; ++j)
      for (int k = 0; k <= p - i - j; ++k, ++m) {
        double fa = jacobi_p(i, 0, 0, a), dfa = jacobi_dp(i, 0, 0, a);
        double gb = jacobi_p(j, 2 * i + 1, 0, b),
               dgb = jacobi_dp(j, 2 * i + 1, 0, b);
        double hc = jacobi_p(k, 2 * (i + j) + 2, 0, c),
               dhc = jacobi_dp(k, 2 * (i + j) + 2, 0, c);
        v[m] = 2.0 * std::sqrt(2.0) * fa * gb * std::pow(1.0 - b, i) * hc *
               std::pow(1.0 - c, i + j);
        if (!g0) continue;
        double hb = 0.5 * (1.0 - b), hcc = 0.5 * (1.0 - c);
        double vr = dfa * gb * hc;
        if (i > 0) vr *= std::pow(hb, i - 1);
        if (i + j > 0) vr *= std::pow(hcc, i + j - 1);
        double vs = 0.5 * (1.0 + a) * vr;
        double tmp = dgb * std::pow(hb, i);
        if (i > 0) tmp -= 0.5 * i * gb * std::pow(hb, i - 1);
        if (i + j > 0) tmp *= std::pow(hcc, i + j - 1);
        tmp = fa * tmp * hc;
        vs += tmp;
        double vt = 0.5 * (1.0 + a) * vr + 0.5 * (1.0 + b) * tmp;
        tmp = dhc * std::pow(hcc, i + j);
        if (i + j > 0) tmp -= 0.5 * (i + j) * hc * std::pow(hcc, i + j - 1);
        tmp = fa * gb * tmp * std::pow(hb, i);
        vt += tmp;
        double sc = std::pow(2.0, 2 * i + j + 1.5);
        g0[m] = vr * sc;
        g1[m] = vs * sc;
        g2[m] = vt * sc;
      }
}

void RefElement::basis(int npts, const double* x, double* out) const {
  int nm = nupts;
  for (int q = 0; q < npts; ++q) {
    const double* xq = x + 3 * q;
    double* o = out + size_t(q) * nm;
    if (kind == EK_HEX) {
      int m = 0;
      for (int k = 0; k <= p; ++k)
        for (int j = 0; j <= p; ++j)
          for (int i = 0; i <= p; ++i, ++m)
            o[m] = jacobi_p(i, 0, 0, xq[0]) * jacobi_p(j, 0, 0, xq[1]) *
                   jacobi_p(k, 0, 0, xq[2]);
    } else if (kind == EK_PRI) {
      int nt = tri_nm(p);
      std::vector<double> tv(nt);
      tri_eval(p, xq[0], xq[1], tv.data(), nullptr, nullptr);
      for (int k = 0; k <= p; ++k)
        for (int m = 0; m < nt; ++m)
          o[k * nt + m] = tv[m] * jacobi_p(k, 0, 0, xq[2]);
    } else {
      tet_eval(p, xq, o, nullptr, nullptr, nullptr);
    }
  }
}

void RefElement::grad(int npts, const double* x, double* out) const {
  int nm = nupts;
  size_t stride = size_t(npts) * nm;
  for (int q = 0; q < npts; ++q) {
    const double* xq = x + 3 * q;
    double* o0 = out + size_t(q) * nm;
    double* o1 = o0 + stride;
    double* o2 = o1 + stride;
    if (kind == EK_HEX) {
      int m = 0;
      for (int k = 0; k <= p; ++k)
        for (int j = 0; j <= p; ++j)
          for (int i = 0; i <= p; ++i, ++m) {
            double a = jacobi_p(i, 0, 0, xq[0]), da = jacobi_dp(i, 0, 0, xq[0]);
            double b = jacobi_p(j, 0, 0, xq[1]), db = jacobi_dp(j, 0, 0, xq[1]);
            double c = jacobi_p(k, 0, 0, xq[2]), dc = jacobi_dp(k, 0, 0, xq[2]);
            o0[m] = da * b * c;
            o1[m] = a * db * c;
            o2[m] = a * b * dc;
          }
    } else if (kind == EK_PRI) {
      int nt = tri_nm(p);
      std::vector<double> tv(nt), tr(nt), ts(nt);
      tri_eval(p, xq[0], xq[1], tv.data(), tr.data(), ts.data());
      for (int k = 0; k <= p; ++k) {
        double l = jacobi_p(k, 0, 0, xq[2]), dl = jacobi_dp(k, 0, 0, xq[2]);
        for (int m = 0; m < nt; ++m) {
          o0[k * nt + m] = tr[m] * l;
          o1[k * nt + m] = ts[m] * l;
          o2[k * nt + m] = tv[m] * dl;
        }
      }
    } else {
      std::vector<double> v(nm);
      tet_eval(p, xq, v.data(), o0, o1, o2);
    }
  }
}

void RefElement::shape(const double* x, double* N) const {
  if (kind == EK_HEX) {
    static const int sg[8][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1},
                                 {-1, 1, -1},  {-1, -1, 1}, {1, -1, 1},
                                 {1, 1, 1},    {-1, 1, 1}};
    for (int v = 0; v < 8; ++v)
      N[v] = (1 + sg[v][0] * x[0]) * (1 + sg[v][1] * x[1]) *
             (1 + sg[v][2] * x[2]) / 8.0;
  } else if (kind == EK_PRI) {
    double l[3] = {-(x[0] + x[1]) / 2, (1 + x[0]) / 2, (1 + x[1]) / 2};
    for (int v = 0; v < 3; ++v) {
      N[v] = l[v] * (1 - x[2]) / 2;
      N[v + 3] = l[v] * (1 + x[2]) / 2;
    }
  } else {
    N[0] = -(1 + x[0] + x[1] + x[2]) / 2;
    N[1] = (1 + x[0]) / 2;
    N[2] = (1 + x[1]) / 2;
    N[3] = (1 + x[2]) / 2;
  }
}

void RefElement::dshape(const double* x, double* dN) const {
  if (kind == EK_HEX) {
    static const int sg[8][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1},
                                 {-1, 1, -1},  {-1, -1, 1}, {1, -1, 1},
                                 {1, 1, 1},    {-1, 1, 1}};
    for (int v = 0; v < 8; ++v) {
      double f[3];
      for (int k = 0; k < 3; ++k) f[k] = 1 + sg[v][k] * x[k];
      dN[0 * 8 + v] = sg[v][0] * f[1] * f[2] / 8.0;
      dN[1 * 8 + v] = sg[v][1] * f[0] * f[2] / 8.0;
      dN[2 * 8 + v] = sg[v][2] * f[0] * f[1] / 8.0;
    }
  } else if (kind == EK_PRI) {
    double l[3] = {-(x[0] + x[1]) / 2, (1 + x[0]) / 2, (1 + x[1]) / 2};
    double dl0[3] = {-0.5, 0.5, 0.0}, dl1[3] = {-0.5, 0.0, 0.5};
    double zl = (1 - x[2]) / 2, zh = (1 + x[2]) / 2;
    for (int v = 0; v < 3; ++v) {
      dN[0 * 6 + v] = dl0[v] * zl;
      dN[0 * 6 + v + 3] = dl0[v] * zh;
      dN[1 * 6 + v] = dl1[v] * zl;
      dN[1 * 6 + v + 3] = dl1[v] * zh;
      dN[2 * 6 + v] = -0.5 * l[v];
      dN[2 * 6 + v + 3] = 0.5 * l[v];
    }
  } else {
    static const double b[3][4] = {{-0.5, 0.5, 0.0, 0.0},
                                   {-0.5, 0.0, 0.5, 0.0},
                                   {-0.5, 0.0, 0.0, 0.5}};
    for (int j = 0; j < 3; ++j)
      for (int v = 0; v < 4; ++v) dN[j * 4 + v] = b[j][v];
  }
}

// --------------------------------------------------------- face geometry
static RefFace mkface(bool tri, std::initializer_list<int> verts,
                      std::array<double, 3> o, std::array<double, 3> ds,
                      std::array<double, 3> dt, std::array<double, 3> n) {
  RefFace f{};
  f.tri = tri;
  f.nv = int(verts.size());
  int i = 0;
  for (int v : verts) f.verts[i++] = v;
  for (int k = 0; k < 3; ++k) {
    f.origin[k] = o[k];
    f.ds[k] = ds[k];
    f.dt[k] = dt[k];
    f.normal[k] = n[k];
  }
  double c[3] = {ds[1] * dt[2] - ds[2] * dt[1], ds[2] * dt[0] - ds[0] * dt[2],
                 ds[0] * dt[1] - ds[1] * dt[0]};
  f.scale = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
  return f;
}

// 2D face point sets in face coordinates (s, t)
// 1D line points of a tensor direction: Gauss-Legendre, or Gauss-Lobatto
static std::vector<double> line_points(int p, int family) {
  std::vector<double> x(p + 1), w(p + 1);
  if (family == 1)
    gauss_lobatto(p + 1, x.data());
  else
    gauss_legendre(p + 1, x.data(), w.data());
  return x;
}

static std::vector<double> face_points(const RefFace& f, int p, int family) {
  if (f.tri) {
    double a = p <= 15 ? kAlpha3D[std::max(p, 1) - 1] : 1.0;
    return tri_nodes(p, a);
  }
  std::vector<double> x = line_points(p, family), out;
  for (int j = 0; j <= p; ++j)
    for (int i = 0; i <= p; ++i) {
      out.push_back(x[i]);
      out.push_back(x[j]);
    }
  return out;
}

// orthonormal 2D face basis values at (s, t) points
static void face_basis(const RefFace& f, int p, int npts, const double* st,
                       double* out) {
  int nm = f.tri ? tri_nm(p) : (p + 1) * (p + 1);
  for (int q = 0; q < npts; ++q) {
    double* o = out + size_t(q) * nm;
    if (f.tri) {
      tri_eval(p, st[2 * q], st[2 * q + 1], o, nullptr, nullptr);
    } else {
      int m = 0;
      for (int j = 0; j <= p; ++j)
        for (int i = 0; i <= p; ++i, ++m)
          o[m] = jacobi_p(i, 0, 0, st[2 * q]) * jacobi_p(j, 0, 0, st[2 * q + 1]);
    }
  }
}

// exact Gauss rule on a face (collapsed Gauss-Legendre on triangles)
static void face_rule(const RefFace& f, int n, std::vector<double>& st,
                      std::vector<double>& w) {
  std::vector<double> x(n), wx(n);
  gauss_legendre(n, x.data(), wx.data());
  st.clear();
  w.clear();
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      if (f.tri) {
        double a = x[i], b = x[j];
        st.push_back(0.5 * (1 + a) * (1 - b) - 1);
        st.push_back(b);
        w.push_back(wx[i] * wx[j] * 0.5 * (1 - b));
      } else {
        st.push_back(x[i]);
        st.push_back(x[j]);
        w.push_back(wx[i] * wx[j]);
      }
    }
}

static void volume_rule(int kind, int n, std::vector<double>& xq,
                        std::vector<double>& wq) {
  std::vector<double> x(n), w(n);
  gauss_legendre(n, x.data(), w.data());
  xq.clear();
  wq.clear();
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < n; ++k) {
        double a = x[i], b = x[j], c = x[k];
        if (kind == EK_HEX) {
          xq.insert(xq.end(), {a, b, c});
          wq.push_back(w[i] * w[j] * w[k]);
        } else if (kind == EK_PRI) {
          xq.insert(xq.end(), {0.5 * (1 + a) * (1 - b) - 1, b, c});
          wq.push_back(w[i] * w[j] * w[k] * 0.5 * (1 - b));
        } else {
          xq.insert(xq.end(), {0.25 * (1 + a) * (1 - b) * (1 - c) - 1,
                               0.5 * (1 + b) * (1 - c) - 1, c});
          wq.push_back(w[i] * w[j] * w[k] * (1 - b) * (1 - c) * (1 - c) / 8.0);
        }
      }
}

std::vector<double> curl_nodes(const RefElement& R) {
  const int p = R.p;
  std::vector<double> g(p + 1), out;
  gauss_lobatto(p + 1, g.data());
  if (R.kind == EK_HEX) {
    for (int k = 0; k <= p; ++k)
      for (int j = 0; j <= p; ++j)
        for (int i = 0; i <= p; ++i) out.insert(out.end(), {g[i], g[j], g[k]});
  } else if (R.kind == EK_TET) {
    out = tet_nodes(p);
  } else {
    const double a = p <= 15 ? kAlpha3D[std::max(p, 1) - 1] : 1.0;
    const std::vector<double> t = tri_nodes(p, a);
    const int nt = int(t.size() / 2);
    for (int k = 0; k <= p; ++k)
      for (int m = 0; m < nt; ++m) out.insert(out.end(), {t[2 * m], t[2 * m + 1], g[k]});
  }
  return out;
}

RefElement make_ref(int kind, int p, int family) {
  if (p < 1 || p > 8) throw std::invalid_argument("order out of range");
  if (family != 0 && (family != 1 || kind != EK_HEX))
    throw std::invalid_argument("Gauss-Lobatto points are for hexahedra only");
  RefElement e;
  e.kind = kind;
  e.p = p;
  e.family = family;
  const double r2 = 1.0 / std::sqrt(2.0), r3 = 1.0 / std::sqrt(3.0);
  if (kind == EK_HEX) {
    e.nverts = 8;
    e.faces = {mkface(false, {0, 3, 7, 4}, {-1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {-1, 0, 0}),
               mkface(false, {1, 2, 6, 5}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 0, 0}),
               mkface(false, {0, 1, 5, 4}, {0, -1, 0}, {1, 0, 0}, {0, 0, 1}, {0, -1, 0}),
               mkface(false, {3, 2, 6, 7}, {0, 1, 0}, {1, 0, 0}, {0, 0, 1}, {0, 1, 0}),
               mkface(false, {0, 1, 2, 3}, {0, 0, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, -1}),
               mkface(false, {4, 5, 6, 7}, {0, 0, 1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1})};
    std::vector<double> x = line_points(p, family);
    for (int k = 0; k <= p; ++k)
      for (int j = 0; j <= p; ++j)
        for (int i = 0; i <= p; ++i) e.upts.insert(e.upts.end(), {x[i], x[j], x[k]});
  } else if (kind == EK_PRI) {
    e.nverts = 6;
    e.faces = {mkface(true, {0, 1, 2}, {0, 0, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, -1}),
               mkface(true, {3, 4, 5}, {0, 0, 1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}),
               mkface(false, {0, 1, 4, 3}, {0, -1, 0}, {1, 0, 0}, {0, 0, 1}, {0, -1, 0}),
               mkface(false, {1, 2, 5, 4}, {0, 0, 0}, {-1, 1, 0}, {0, 0, 1}, {r2, r2, 0}),
               mkface(false, {0, 2, 5, 3}, {-1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {-1, 0, 0})};
    auto t = tri_nodes(p, p <= 15 ? kAlpha2D[p - 1] : 5.0 / 3.0);
    std::vector<double> z(p + 1), w(p + 1);
    gauss_legendre(p + 1, z.data(), w.data());
    int nt = int(t.size() / 2);
    for (int k = 0; k <= p; ++k)
      for (int m = 0; m < nt; ++m) e.upts.insert(e.upts.end(), {t[2 * m], t[2 * m + 1], z[k]});
  } else {
    e.nverts = 4;
    e.faces = {mkface(true, {0, 1, 2}, {0, 0, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, -1}),
               mkface(true, {0, 1, 3}, {0, -1, 0}, {1, 0, 0}, {0, 0, 1}, {0, -1, 0}),
               mkface(true, {0, 2, 3}, {-1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {-1, 0, 0}),
               mkface(true, {1, 2, 3}, {-1, 0, 0}, {-1, 1, 0}, {-1, 0, 1}, {r3, r3, r3})};
    e.upts = tet_nodes(p);
  }
  e.nupts = int(e.upts.size() / 3);
  e.nfaces = int(e.faces.size());
  // total degree of every mode, in the order of RefElement::basis
  if (kind == EK_HEX) {
    for (int k = 0; k <= p; ++k)
      for (int j = 0; j <= p; ++j)
        for (int i = 0; i <= p; ++i) e.mdeg.push_back(i + j + k);
  } else if (kind == EK_PRI) {
    for (int k = 0; k <= p; ++k)
      for (int i = 0; i <= p; ++i)
        for (int j = 0; j <= p - i; ++j) e.mdeg.push_back(i + j + k);
  } else {
    for (int i = 0; i <= p; ++i)
      for (int j = 0; j <= p - i; ++j)
        for (int k = 0; k <= p - i - j; ++k) e.mdeg.push_back(i + j + k);
  }
  // flux points face by face
  e.face_start.push_back(0);
  std::vector<std::vector<double>> fst(e.nfaces);
  for (int fi = 0; fi < e.nfaces; ++fi) {
    const RefFace& f = e.faces[fi];
    fst[fi] = face_points(f, p, family);
    int n = int(fst[fi].size() / 2);
    for (int q = 0; q < n; ++q) {
      double s = fst[fi][2 * q], t = fst[fi][2 * q + 1];
      for (int k = 0; k < 3; ++k)
        e.fpts.push_back(f.origin[k] + s * f.ds[k] + t * f.dt[k]);
      for (int k = 0; k < 3; ++k) e.fnorm.push_back(f.normal[k]);
      e.fpts_face.push_back(fi);
    }
    e.face_start.push_back(e.face_start.back() + n);
  }
  e.nfpts = int(e.fpts.size() / 3);
  const int nu = e.nupts, nf = e.nfpts;
  // Vandermonde and its inverse
  std::vector<double> V(nu * nu);
  e.basis(nu, e.upts.data(), V.data());
  e.vdm_inv.resize(nu * nu);
  if (!invert(nu, V.data(), e.vdm_inv.data()))
    throw std::runtime_error("singular Vandermonde matrix");
  auto mul = [&](const double* A, int n, const double* B, double* C) {
    // C[n][nu] = A[n][nu] * vdm_inv[nu][nu]
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < nu; ++c) {
        double s = 0.0;
        for (int k = 0; k < nu; ++k) s += A[size_t(r) * nu + k] * B[size_t(k) * nu + c];
        C[size_t(r) * nu + c] = s;
      }
  };
  std::vector<double> Vf(size_t(nf) * nu);
  e.basis(nf, e.fpts.data(), Vf.data());
  e.M0.resize(size_t(nf) * nu);
  mul(Vf.data(), nf, e.vdm_inv.data(), e.M0.data());
  std::vector<double> G(3 * size_t(nu) * nu);
  e.grad(nu, e.upts.data(), G.data());
  e.D.resize(3 * size_t(nu) * nu);
  for (int d = 0; d < 3; ++d)
    mul(G.data() + d * size_t(nu) * nu, nu, e.vdm_inv.data(),
        e.D.data() + d * size_t(nu) * nu);
  // DG lift: LIFT[:, s] = V * b_s, b_s[k] = int_face psi_k l_s dGamma
  e.LIFT.assign(size_t(nu) * nf, 0.0);
  for (int fi = 0; fi < e.nfaces; ++fi) {
    const RefFace& f = e.faces[fi];
    std::vector<double> st, wq;
    face_rule(f, p + 3, st, wq);
    int nq = int(wq.size());
    std::vector<double> xq(3 * nq);
    for (int q = 0; q < nq; ++q)
      for (int k = 0; k < 3; ++k)
        xq[3 * q + k] = f.origin[k] + st[2 * q] * f.ds[k] + st[2 * q + 1] * f.dt[k];
    std::vector<double> psi(size_t(nq) * nu);
    e.basis(nq, xq.data(), psi.data());
    int nfp = e.face_start[fi + 1] - e.face_start[fi];
    std::vector<double> Vfp(size_t(nfp) * nfp), Vfpi(size_t(nfp) * nfp),
        Vq(size_t(nq) * nfp);
    face_basis(f, p, nfp, fst[fi].data(), Vfp.data());
    if (!invert(nfp, Vfp.data(), Vfpi.data()))
      throw std::runtime_error("singular face Vandermonde matrix");
    face_basis(f, p, nq, st.data(), Vq.data());
    // face Lagrange basis at the quadrature points: lq = Vq * Vfpi
    std::vector<double> lq(size_t(nq) * nfp, 0.0);
    for (int q = 0; q < nq; ++q)
      for (int c = 0; c < nfp; ++c) {
        double s = 0.0;
        for (int k = 0; k < nfp; ++k) s += Vq[size_t(q) * nfp + k] * Vfpi[size_t(k) * nfp + c];
        lq[size_t(q) * nfp + c] = s;
      }
    for (int c = 0; c < nfp; ++c) {
      std::vector<double> bk(nu, 0.0);
      for (int q = 0; q < nq; ++q) {
        double wl = wq[q] * f.scale * lq[size_t(q) * nfp + c];
        for (int k = 0; k < nu; ++k) bk[k] += psi[size_t(q) * nu + k] * wl;
      }
      int col = e.face_start[fi] + c;
      for (int z = 0; z < nu; ++z) {
        double s = 0.0;
        for (int k = 0; k < nu; ++k) s += V[size_t(z) * nu + k] * bk[k];
        e.LIFT[size_t(z) * nf + col] = s;
      }
    }
  }
  // integration weights W[z] = int l_z
  {
    std::vector<double> xq, wq;
    volume_rule(kind, p + 2, xq, wq);
    int nq = int(wq.size());
    std::vector<double> B(size_t(nq) * nu);
    e.basis(nq, xq.data(), B.data());
    e.W.assign(nu, 0.0);
    for (int q = 0; q < nq; ++q)
      for (int z = 0; z < nu; ++z) {
        double l = 0.0;
        for (int k = 0; k < nu; ++k) l += B[size_t(q) * nu + k] * e.vdm_inv[size_t(k) * nu + z];
        e.W[z] += wq[q] * l;
      }
  }
  if (kind == EK_HEX) {
    int n = p + 1;
    e.x1 = line_points(p, family);
    e.d1.resize(n * n);
    e.lm.resize(n);
    e.lp.resize(n);
    for (int m = 0; m < n; ++m) {
      double am = 1.0, ap = 1.0;
      for (int j = 0; j < n; ++j)
        if (j != m) {
          am *= (-1.0 - e.x1[j]) / (e.x1[m] - e.x1[j]);
          ap *= (1.0 - e.x1[j]) / (e.x1[m] - e.x1[j]);
        }
      e.lm[m] = am;
      e.lp[m] = ap;
    }
    for (int a = 0; a < n; ++a)
      for (int m = 0; m < n; ++m) {
        // l_m'(x_a) = sum_k prod_{j != m, k} ...
        double s = 0.0;
        for (int k = 0; k < n; ++k) {
          if (k == m) continue;
          double t = 1.0 / (e.x1[m] - e.x1[k]);
          for (int j = 0; j < n; ++j)
            if (j != m && j != k) t *= (e.x1[a] - e.x1[j]) / (e.x1[m] - e.x1[j]);
          s += t;
        }
        e.d1[a * n + m] = s;
      }
    // correction weights read back from the lift columns of the x faces
    e.gl.resize(n);
    e.gr.resize(n);
    for (int a = 0; a < n; ++a) {
      int z = a;                       // solution point (a, 0, 0)
      int sm = e.face_start[0];        // x=-1 face, point (y_0, z_0)
      int sp = e.face_start[1];        // x=+1 face, point (y_0, z_0)
      e.gl[a] = e.LIFT[size_t(z) * nf + sm];
      e.gr[a] = e.LIFT[size_t(z) * nf + sp];
    }
  }
  return e;
}

}  // namespace frgb

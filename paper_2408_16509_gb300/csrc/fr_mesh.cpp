// Host-side mesh geometry and interface pairing.  See fr_mesh.hpp.
#include "fr_mesh.hpp"

#include <algorithm>
#include <cmath>
#include <numeric>
#include <system_error>
#include <thread>
#include <unordered_map>

namespace frgb {

namespace {

struct FaceRec {
  int t;
  int64_t e;
  int f;
  int64_t key[4];
};

bool key_less(const FaceRec& a, const FaceRec& b) {
  for (int k = 0; k < 4; ++k)
    if (a.key[k] != b.key[k]) return a.key[k] < b.key[k];
  return false;
}

bool key_eq(const int64_t* a, const int64_t* b) {
  for (int k = 0; k < 4; ++k)
    if (a[k] != b[k]) return false;
  return true;
}

struct Key3Hash {
  size_t operator()(const std::array<int64_t, 3>& k) const {
    uint64_t h = 1469598103934665603ull;
    for (int i = 0; i < 3; ++i) {
      h ^= uint64_t(k[i]);
      h *= 1099511628211ull;
    }
    return size_t(h);
  }
};

struct Key4Hash {
  size_t operator()(const std::array<int64_t, 4>& k) const {
    uint64_t h = 1469598103934665603ull;
    for (int i = 0; i < 4; ++i) {
      h ^= uint64_t(k[i]);
      h *= 1099511628211ull;
    }
    return size_t(h);
  }
};

void geometry(HostType& T, const double* nodes) {
  const RefElement& R = T.ref;
  const int nv = R.nverts, nu = R.nupts, nf = R.nfpts;
  T.verts.resize(size_t(T.ne) * nv * 3);
  for (int64_t e = 0; e < T.ne; ++e)
    for (int v = 0; v < nv; ++v)
      for (int k = 0; k < 3; ++k)
        T.verts[(size_t(e) * nv + v) * 3 + k] = nodes[T.conn[size_t(e) * nv + v] * 3 + k];
  std::vector<double> Nu(size_t(nu) * nv), dNu(size_t(nu) * 3 * nv);
  std::vector<double> Nf(size_t(nf) * nv), dNf(size_t(nf) * 3 * nv);
  for (int q = 0; q < nu; ++q) {
    R.shape(&R.upts[3 * q], &Nu[size_t(q) * nv]);
    R.dshape(&R.upts[3 * q], &dNu[size_t(q) * 3 * nv]);
  }
  for (int q = 0; q < nf; ++q) {
    R.shape(&R.fpts[3 * q], &Nf[size_t(q) * nv]);
    R.dshape(&R.fpts[3 * q], &dNf[size_t(q) * 3 * nv]);
  }
  T.upts_x.resize(size_t(T.ne) * nu * 3);
  T.smat.resize(size_t(T.ne) * 9 * nu);
  T.rcpdjac.resize(size_t(T.ne) * nu);
  T.fpts_x.resize(size_t(T.ne) * nf * 3);
  T.fnvec.resize(size_t(T.ne) * nf * 3);
  auto metric = [&](const double* X, const double* dN, double S[3][3],
                    double* det) {
    double a[3][3];  // a[j] = d x / d x~_j
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) {
        double s = 0.0;
        for (int v = 0; v < nv; ++v) s += dN[j * nv + v] * X[v * 3 + k];
        a[j][k] = s;
      }
    for (int i = 0; i < 3; ++i) {
      const double* b = a[(i + 1) % 3];
      const double* c = a[(i + 2) % 3];
      S[i][0] = b[1] * c[2] - b[2] * c[1];
      S[i][1] = b[2] * c[0] - b[0] * c[2];
      S[i][2] = b[0] * c[1] - b[1] * c[0];
    }
    *det = a[0][0] * S[0][0] + a[0][1] * S[0][1] + a[0][2] * S[0][2];
  };
  for (int64_t e = 0; e < T.ne; ++e) {
    const double* X = &T.verts[size_t(e) * nv * 3];
    for (int q = 0; q < nu; ++q) {
      for (int k = 0; k < 3; ++k) {
        double s = 0.0;
        for (int v = 0; v < nv; ++v) s += Nu[size_t(q) * nv + v] * X[v * 3 + k];
        T.upts_x[(size_t(e) * nu + q) * 3 + k] = s;
      }
      double S[3][3], det;
      metric(X, &dNu[size_t(q) * 3 * nv], S, &det);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
          T.smat[(size_t(e) * 9 + i * 3 + j) * nu + q] = S[i][j];
      T.rcpdjac[size_t(e) * nu + q] = det > 0 ? 1.0 / det : -1.0;
    }
    for (int q = 0; q < nf; ++q) {
      for (int k = 0; k < 3; ++k) {
        double s = 0.0;
        for (int v = 0; v < nv; ++v) s += Nf[size_t(q) * nv + v] * X[v * 3 + k];
        T.fpts_x[(size_t(e) * nf + q) * 3 + k] = s;
      }
      double S[3][3], det;
      metric(X, &dNf[size_t(q) * 3 * nv], S, &det);
      const double* n = &R.fnorm[3 * q];
      for (int j = 0; j < 3; ++j)
        T.fnvec[(size_t(e) * nf + q) * 3 + j] =
            S[0][j] * n[0] + S[1][j] * n[1] + S[2][j] * n[2];
    }
  }
}

// Curved hexahedra ("Curved Elements", Section 3.4): the map is the
// triquadratic interpolant of 27 nodes, node a + 3b + 9c at (-1+a, -1+b,
// -1+c).  Positions and det J come from that map exactly.  The metric terms
// det J dxi_i/dx_n are taken in the conservative curl form
//   S[i][n] = -(curl_xi I(X_l grad_xi X_m))_i,   (n, m, l) cyclic,
// I the order-p tensor Lagrange interpolant on the (p+1)^3 Gauss-Lobatto
// nodes.  Its discrete divergence vanishes (a uniform flow stays uniform) and,
// because the Gauss-Lobatto set has nodes on every face, the normal component
// on a face depends on that face's nodes only, so both sides of an interface
// see the same normal.
struct Quad1D {  // 1D quadratic Lagrange factors on {-1, 0, 1}
  static void val(double s, double* l) {
    l[0] = 0.5 * s * (s - 1.0);
    l[1] = 1.0 - s * s;
    l[2] = 0.5 * s * (s + 1.0);
  }
  static void der(double s, double* d) {
    d[0] = s - 0.5;
    d[1] = -2.0 * s;
    d[2] = s + 0.5;
  }
};

// x_k(pt) and a[j][k] = d x_k / d xi_j of a tensor hexahedron map of
// order k (nodes a + (k+1) b + (k+1)^2 c at equispaced reference points).
void lagrange1d(int n, const double* g, double s, double* l, double* d);
void hexk_eval(int order, const double* X, const double* pt, double x[3], double a[3][3]) {
  const int n = order + 1;
  double g[8], l[3][8], d[3][8];
  for (int i = 0; i < n; ++i) g[i] = -1.0 + 2.0 * i / order;
  for (int i = 0; i < 3; ++i) lagrange1d(n, g, pt[i], l[i], d[i]);
  for (int k = 0; k < 3; ++k) {
    x[k] = 0.0;
    for (int j = 0; j < 3; ++j) a[j][k] = 0.0;
  }
  for (int c = 0; c < n; ++c)
    for (int b = 0; b < n; ++b)
      for (int aa = 0; aa < n; ++aa) {
        const double* P = &X[(aa + n * (b + n * c)) * 3];
        const double N = l[0][aa] * l[1][b] * l[2][c];
        const double g0 = d[0][aa] * l[1][b] * l[2][c];
        const double g1 = l[0][aa] * d[1][b] * l[2][c];
        const double g2 = l[0][aa] * l[1][b] * d[2][c];
        for (int k = 0; k < 3; ++k) {
          x[k] += N * P[k];
          a[0][k] += g0 * P[k];
          a[1][k] += g1 * P[k];
          a[2][k] += g2 * P[k];
        }
      }
}

// x_k(pt) and a[j][k] = d x_k / d xi_j of a 27-node map X[27][3].
void q2_eval(const double* X, const double* pt, double x[3], double a[3][3]) {
  double l[3][3], d[3][3];
  for (int i = 0; i < 3; ++i) {
    Quad1D::val(pt[i], l[i]);
    Quad1D::der(pt[i], d[i]);
  }
  for (int k = 0; k < 3; ++k) {
    x[k] = 0.0;
    for (int j = 0; j < 3; ++j) a[j][k] = 0.0;
  }
  for (int c = 0; c < 3; ++c)
    for (int b = 0; b < 3; ++b)
      for (int aa = 0; aa < 3; ++aa) {
        const double* P = &X[(aa + 3 * b + 9 * c) * 3];
        const double N = l[0][aa] * l[1][b] * l[2][c];
        const double g0 = d[0][aa] * l[1][b] * l[2][c];
        const double g1 = l[0][aa] * d[1][b] * l[2][c];
        const double g2 = l[0][aa] * l[1][b] * d[2][c];
        for (int k = 0; k < 3; ++k) {
          x[k] += N * P[k];
          a[0][k] += g0 * P[k];
          a[1][k] += g1 * P[k];
          a[2][k] += g2 * P[k];
        }
      }
}

// Lagrange basis of the nodes g[0..n) at s: values l[n] and derivatives d[n].
void lagrange1d(int n, const double* g, double s, double* l, double* d) {
  for (int i = 0; i < n; ++i) {
    double v = 1.0, dv = 0.0;
    for (int k = 0; k < n; ++k) {
      if (k == i) continue;
      const double r = 1.0 / (g[i] - g[k]);
      dv = dv * (s - g[k]) * r + v * r;
      v *= (s - g[k]) * r;
    }
    l[i] = v;
    d[i] = dv;
  }
}

// Nodal fields w[n][j][node] = X_l d X_m / d xi_j ((n, m, l) cyclic) of a
// 27-node map at the Gauss-Lobatto tensor nodes g (n1 per direction).
void curl_fields(const double* X, const std::vector<double>& g, double* w, int order = 2) {
  const int n1 = int(g.size()), ng = n1 * n1 * n1;
  for (int c = 0; c < n1; ++c)
    for (int b = 0; b < n1; ++b)
      for (int a = 0; a < n1; ++a) {
        const int node = a + n1 * (b + n1 * c);
        const double pt[3] = {g[a], g[b], g[c]};
        double x[3], J[3][3];
        hexk_eval(order, X, pt, x, J);
        for (int n = 0; n < 3; ++n) {
          const int m = (n + 1) % 3, l = (n + 2) % 3;
          for (int j = 0; j < 3; ++j) w[(size_t(n) * 3 + j) * ng + node] = x[l] * J[j][m];
        }
      }
}

// S[i][n] = -(curl_xi I(w^n))_i at one point, from its 1D Lagrange factors
// L[3][n1] (values) and dL[3][n1] (derivatives) on the nodes.
void curl_eval(int n1, const double* L, const double* dL, const double* w,
               double S[3][3]) {
  const int ng = n1 * n1 * n1;
  double dw[3][3][3] = {};  // dw[n][j][i] = d_i I(w^n_j)
  for (int c = 0; c < n1; ++c)
    for (int b = 0; b < n1; ++b)
      for (int a = 0; a < n1; ++a) {
        const int node = a + n1 * (b + n1 * c);
        const double B[3] = {dL[a] * L[n1 + b] * L[2 * n1 + c],
                             L[a] * dL[n1 + b] * L[2 * n1 + c],
                             L[a] * L[n1 + b] * dL[2 * n1 + c]};
        for (int n = 0; n < 3; ++n)
          for (int j = 0; j < 3; ++j) {
            const double v = w[(size_t(n) * 3 + j) * ng + node];
            for (int i = 0; i < 3; ++i) dw[n][j][i] += B[i] * v;
          }
      }
  for (int i = 0; i < 3; ++i) {
    const int j = (i + 1) % 3, k = (i + 2) % 3;
    for (int n = 0; n < 3; ++n) S[i][n] = dw[n][j][k] - dw[n][k][j];
  }
}

// 1D Lagrange factors of the Gauss-Lobatto nodes at np points: [np][3][n1].
void curl_factors(const std::vector<double>& g, int np, const double* pts,
                  std::vector<double>& L, std::vector<double>& dL) {
  const int n1 = int(g.size());
  L.resize(size_t(np) * 3 * n1);
  dL.resize(size_t(np) * 3 * n1);
  for (int q = 0; q < np; ++q)
    for (int i = 0; i < 3; ++i)
      lagrange1d(n1, g.data(), pts[3 * q + i], &L[(size_t(q) * 3 + i) * n1],
                 &dL[(size_t(q) * 3 + i) * n1]);
}

std::vector<double> gll_nodes(int n1) {
  std::vector<double> g(n1);
  gauss_lobatto(n1, g.data());
  return g;
}

// Runs body(e0, e1) over [0, ne) split across host threads; elements write
// disjoint slices.  Falls back to the calling thread when none can start.
template <typename F>
void parallel_elements(int64_t ne, F body) {
  const int64_t nthr = std::max<int64_t>(
      1, std::min<int64_t>(std::thread::hardware_concurrency(), ne / 64));
  std::vector<std::thread> pool;
  int64_t t = 1;
  try {
    for (; t < nthr; ++t)
      pool.emplace_back(body, ne * t / nthr, ne * (t + 1) / nthr);
  } catch (const std::system_error&) {  // no more threads: the rest runs here
    body(ne * t / nthr, ne);
  }
  body(0, ne / nthr);
  for (auto& th : pool) th.join();
}

// Number of map nodes of a curved element of map order 2 or 3 and the map
// node of each vertex.
int map_nodes(int kind, int order) {
  if (kind == EK_HEX) return (order + 1) * (order + 1) * (order + 1);
  if (kind == EK_PRI) return order == 3 ? 40 : 18;
  return order == 3 ? 20 : 10;
}
const int* map_corners(int kind, int order) {
  static const int hexc[8] = {0, 2, 8, 6, 18, 20, 26, 24};
  static const int hex3[8] = {0, 3, 15, 12, 48, 51, 63, 60};
  static const int pric[6] = {0, 1, 2, 12, 13, 14};
  static const int pri3[6] = {0, 1, 2, 30, 31, 32};
  static const int tetc[4] = {0, 1, 2, 3};
  if (kind == EK_HEX) return order == 3 ? hex3 : hexc;
  if (kind == EK_PRI) return order == 3 ? pri3 : pric;
  return tetc;
}

// Cubic Lagrange basis of a triangle (nv = 3) or tetrahedron (nv = 4) from
// its barycentric coordinates lam[nv], whose gradients dl[nv][3] are
// constant.  Nodes: the vertices; two per edge (a, b), at barycentric
// (2/3, 1/3) then (1/3, 2/3) of a and b; the centroid of each face.  Basis:
// l (3l - 1)(3l - 2) / 2 at a vertex, 9/2 l_a l_b (3 l_a - 1) at an edge
// node nearer a, 27 l_a l_b l_c at a centroid.  N[n], dN[3][kMaxSimplexMap].
constexpr int kMaxSimplexMap = 20;
int cubic_simplex(int nv, const double* lam, const double (*dl)[3], int nedge,
                  const int (*E)[2], int nface, const int (*F)[3], double* N,
                  double (*dN)[kMaxSimplexMap]) {
  int k = 0;
  for (int v = 0; v < nv; ++v, ++k) {
    const double l = lam[v], g = 0.5 * (27 * l * l - 18 * l + 2);
    N[k] = 0.5 * l * (3 * l - 1) * (3 * l - 2);
    for (int j = 0; j < 3; ++j) dN[j][k] = g * dl[v][j];
  }
  for (int e = 0; e < nedge; ++e)
    for (int side = 0; side < 2; ++side, ++k) {
      const int a = E[e][side], b = E[e][1 - side];
      const double la = lam[a], lb = lam[b];
      N[k] = 4.5 * la * lb * (3 * la - 1);
      const double ga = 4.5 * lb * (6 * la - 1), gb = 4.5 * la * (3 * la - 1);
      for (int j = 0; j < 3; ++j) dN[j][k] = ga * dl[a][j] + gb * dl[b][j];
    }
  for (int f = 0; f < nface; ++f, ++k) {
    const int a = F[f][0], b = F[f][1], c = F[f][2];
    const double la = lam[a], lb = lam[b], lc = lam[c];
    N[k] = 27 * la * lb * lc;
    for (int j = 0; j < 3; ++j)
      dN[j][k] = 27 * (lb * lc * dl[a][j] + la * lc * dl[b][j] + la * lb * dl[c][j]);
  }
  return k;
}

// x_k(pt) and a[j][k] = d x_k / d xi_j of a curved prism or tetrahedron.
// Quadratic prism (18 nodes): triangle node + 6 layer, triangle nodes v0 v1
// v2 and the midpoints of edges 01, 12, 02, layers z = -1, 0, 1; quadratic
// tetrahedron (10 nodes): the vertices, then the midpoints of edges 01, 12,
// 02, 03, 13, 23.  Cubic prism (40 nodes): triangle node + 10 layer, the
// cubic triangle of cubic_simplex on edges 01, 12, 02 and face 012, layers
// z = -1, -1/3, 1/3, 1; cubic tetrahedron (20 nodes): cubic_simplex on
// edges 01, 12, 02, 03, 13, 23 and faces 012, 013, 023, 123.
void simplex_map_eval(int kind, int order, const double* X, const double* pt, double x[3],
                      double a[3][3]) {
  double N[40], dN[3][40];
  int nn;
  static const int TE[6][2] = {{0, 1}, {1, 2}, {0, 2}, {0, 3}, {1, 3}, {2, 3}};
  if (kind == EK_TET) {
    const double lam[4] = {-(1 + pt[0] + pt[1] + pt[2]) / 2, (1 + pt[0]) / 2,
                           (1 + pt[1]) / 2, (1 + pt[2]) / 2};
    const double dl[4][3] = {{-0.5, -0.5, -0.5}, {0.5, 0, 0}, {0, 0.5, 0}, {0, 0, 0.5}};
    if (order == 3) {
      static const int TF[4][3] = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};
      double Nc[kMaxSimplexMap], dNc[3][kMaxSimplexMap];
      nn = cubic_simplex(4, lam, dl, 6, TE, 4, TF, Nc, dNc);
      for (int v = 0; v < nn; ++v) {
        N[v] = Nc[v];
        for (int j = 0; j < 3; ++j) dN[j][v] = dNc[j][v];
      }
    } else {
      nn = 10;
      for (int v = 0; v < 4; ++v) {
        N[v] = lam[v] * (2 * lam[v] - 1);
        for (int j = 0; j < 3; ++j) dN[j][v] = (4 * lam[v] - 1) * dl[v][j];
      }
      for (int e = 0; e < 6; ++e) {
        const int p0 = TE[e][0], p1 = TE[e][1];
        N[4 + e] = 4 * lam[p0] * lam[p1];
        for (int j = 0; j < 3; ++j) dN[j][4 + e] = 4 * (dl[p0][j] * lam[p1] + lam[p0] * dl[p1][j]);
      }
    }
  } else {
    const double lam[3] = {-(pt[0] + pt[1]) / 2, (1 + pt[0]) / 2, (1 + pt[1]) / 2};
    const double dl[3][3] = {{-0.5, -0.5, 0.0}, {0.5, 0.0, 0.0}, {0.0, 0.5, 0.0}};
    double T[kMaxSimplexMap], dT[3][kMaxSimplexMap], L[4], dL[4];
    int nt, nl;
    const double t = pt[2];
    if (order == 3) {
      static const int E[3][2] = {{0, 1}, {1, 2}, {0, 2}};
      static const int F[1][3] = {{0, 1, 2}};
      static const double g3[4] = {-1.0, -1.0 / 3.0, 1.0 / 3.0, 1.0};
      nt = cubic_simplex(3, lam, dl, 3, E, 1, F, T, dT);
      nl = 4;
      lagrange1d(4, g3, t, L, dL);
    } else {
      nt = 6;
      nl = 3;
      for (int v = 0; v < 3; ++v) {
        T[v] = lam[v] * (2 * lam[v] - 1);
        for (int j = 0; j < 2; ++j) dT[j][v] = (4 * lam[v] - 1) * dl[v][j];
      }
      for (int e = 0; e < 3; ++e) {
        const int p0 = TE[e][0], p1 = TE[e][1];  // edges 01, 12, 02
        T[3 + e] = 4 * lam[p0] * lam[p1];
        for (int j = 0; j < 2; ++j) dT[j][3 + e] = 4 * (dl[p0][j] * lam[p1] + lam[p0] * dl[p1][j]);
      }
      L[0] = 0.5 * t * (t - 1);
      L[1] = 1 - t * t;
      L[2] = 0.5 * t * (t + 1);
      dL[0] = t - 0.5;
      dL[1] = -2 * t;
      dL[2] = t + 0.5;
    }
    nn = nt * nl;
    for (int l = 0; l < nl; ++l)
      for (int q = 0; q < nt; ++q) {
        N[q + nt * l] = T[q] * L[l];
        dN[0][q + nt * l] = dT[0][q] * L[l];
        dN[1][q + nt * l] = dT[1][q] * L[l];
        dN[2][q + nt * l] = T[q] * dL[l];
      }
  }
  for (int k = 0; k < 3; ++k) {
    x[k] = 0.0;
    for (int j = 0; j < 3; ++j) a[j][k] = 0.0;
  }
  for (int v = 0; v < nn; ++v)
    for (int k = 0; k < 3; ++k) {
      x[k] += N[v] * X[3 * v + k];
      for (int j = 0; j < 3; ++j) a[j][k] += dN[j][v] * X[3 * v + k];
    }
}

// Curl-form interpolant of a prism or tetrahedron through its modal basis:
// the derivative d_i of the interpolant on the curl nodes, at np points,
// dB[np][3][ng].
struct CurlSimplex {
  int ng = 0;
  std::vector<double> G;     // [ng][3] curl nodes
  std::vector<double> Vinv;  // [nm][ng] modal <- nodal on the curl nodes
  explicit CurlSimplex(const RefElement& R) : G(curl_nodes(R)) {
    ng = int(G.size() / 3);
    std::vector<double> V(size_t(ng) * ng);
    R.basis(ng, G.data(), V.data());
    Vinv.resize(V.size());
    invert(ng, V.data(), Vinv.data());
  }
  void deriv(const RefElement& R, int np, const double* pts, std::vector<double>& dB) const {
    std::vector<double> g(size_t(3) * np * ng);
    R.grad(np, pts, g.data());
    dB.assign(size_t(np) * 3 * ng, 0.0);
    for (int q = 0; q < np; ++q)
      for (int i = 0; i < 3; ++i)
        for (int m = 0; m < ng; ++m) {
          const double gv = g[(size_t(i) * np + q) * ng + m];
          if (gv == 0.0) continue;
          for (int node = 0; node < ng; ++node)
            dB[(size_t(q) * 3 + i) * ng + node] += gv * Vinv[size_t(m) * ng + node];
        }
  }
  // w[n][j][node] = X_l d X_m / d xi_j ((n, m, l) cyclic) at the curl nodes
  void fields(int kind, int order, const double* X, double* w) const {
    for (int node = 0; node < ng; ++node) {
      double x[3], J[3][3];
      simplex_map_eval(kind, order, X, &G[3 * node], x, J);
      for (int n = 0; n < 3; ++n) {
        const int m = (n + 1) % 3, l = (n + 2) % 3;
        for (int j = 0; j < 3; ++j) w[(size_t(n) * 3 + j) * ng + node] = x[l] * J[j][m];
      }
    }
  }
  // S[i][n] = -(curl_xi I(w^n))_i at one point from its dB row [3][ng]
  void eval(const double* dBq, const double* w, double S[3][3]) const {
    double dw[3][3][3];
    for (int n = 0; n < 3; ++n)
      for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) {
          double s = 0.0;
          for (int node = 0; node < ng; ++node)
            s += dBq[size_t(i) * ng + node] * w[(size_t(n) * 3 + j) * ng + node];
          dw[n][j][i] = s;
        }
    for (int i = 0; i < 3; ++i) {
      const int j = (i + 1) % 3, k = (i + 2) % 3;
      for (int n = 0; n < 3; ++n) S[i][n] = dw[n][j][k] - dw[n][k][j];
    }
  }
};

void curved_geometry_simplex(HostType& T) {
  const RefElement& R = T.ref;
  const int nu = R.nupts, nf = R.nfpts, nmap = map_nodes(T.kind, T.map_order);
  const CurlSimplex C(R);
  std::vector<double> dBu, dBf;
  C.deriv(R, nu, R.upts.data(), dBu);
  C.deriv(R, nf, R.fpts.data(), dBf);
  T.upts_x.resize(size_t(T.ne) * nu * 3);
  T.smat.resize(size_t(T.ne) * 9 * nu);
  T.rcpdjac.resize(size_t(T.ne) * nu);
  T.fpts_x.resize(size_t(T.ne) * nf * 3);
  T.fnvec.resize(size_t(T.ne) * nf * 3);
  parallel_elements(T.ne, [&](int64_t e0, int64_t e1) {
    std::vector<double> w(size_t(9) * C.ng);
    for (int64_t e = e0; e < e1; ++e) {
      const double* X = &T.mapx[size_t(e) * nmap * 3];
      C.fields(T.kind, T.map_order, X, w.data());
      for (int q = 0; q < nu; ++q) {
        double x[3], J[3][3], S[3][3];
        simplex_map_eval(T.kind, T.map_order, X, &R.upts[3 * q], x, J);
        for (int k = 0; k < 3; ++k) T.upts_x[(size_t(e) * nu + q) * 3 + k] = x[k];
        const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                           J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                           J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        C.eval(&dBu[size_t(q) * 3 * C.ng], w.data(), S);
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) T.smat[(size_t(e) * 9 + i * 3 + j) * nu + q] = S[i][j];
        T.rcpdjac[size_t(e) * nu + q] = det > 0 ? 1.0 / det : -1.0;
      }
      for (int q = 0; q < nf; ++q) {
        double x[3], J[3][3], S[3][3];
        simplex_map_eval(T.kind, T.map_order, X, &R.fpts[3 * q], x, J);
        for (int k = 0; k < 3; ++k) T.fpts_x[(size_t(e) * nf + q) * 3 + k] = x[k];
        C.eval(&dBf[size_t(q) * 3 * C.ng], w.data(), S);
        const double* n = &R.fnorm[3 * q];
        for (int j = 0; j < 3; ++j)
          T.fnvec[(size_t(e) * nf + q) * 3 + j] =
              S[0][j] * n[0] + S[1][j] * n[1] + S[2][j] * n[2];
      }
    }
  });
}

void curved_geometry(HostType& T) {
  if (T.kind != EK_HEX) {
    curved_geometry_simplex(T);
    return;
  }
  const RefElement& R = T.ref;
  const int nu = R.nupts, nf = R.nfpts, n1 = R.p + 1, ng = n1 * n1 * n1;
  const std::vector<double> g = gll_nodes(n1);
  std::vector<double> Lu, dLu, Lf, dLf;
  curl_factors(g, nu, R.upts.data(), Lu, dLu);
  curl_factors(g, nf, R.fpts.data(), Lf, dLf);
  T.upts_x.resize(size_t(T.ne) * nu * 3);
  T.smat.resize(size_t(T.ne) * 9 * nu);
  T.rcpdjac.resize(size_t(T.ne) * nu);
  T.fpts_x.resize(size_t(T.ne) * nf * 3);
  T.fnvec.resize(size_t(T.ne) * nf * 3);
  parallel_elements(T.ne, [&](int64_t e0, int64_t e1) {
    std::vector<double> w(size_t(9) * ng);
    const int nmap = map_nodes(EK_HEX, T.map_order);
    for (int64_t e = e0; e < e1; ++e) {
      const double* X = &T.mapx[size_t(e) * nmap * 3];
      curl_fields(X, g, w.data(), T.map_order);
      for (int q = 0; q < nu; ++q) {
        double x[3], J[3][3], S[3][3];
        hexk_eval(T.map_order, X, &R.upts[3 * q], x, J);
        for (int k = 0; k < 3; ++k) T.upts_x[(size_t(e) * nu + q) * 3 + k] = x[k];
        const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                           J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                           J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        curl_eval(n1, &Lu[size_t(q) * 3 * n1], &dLu[size_t(q) * 3 * n1], w.data(), S);
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) T.smat[(size_t(e) * 9 + i * 3 + j) * nu + q] = S[i][j];
        T.rcpdjac[size_t(e) * nu + q] = det > 0 ? 1.0 / det : -1.0;
      }
      for (int q = 0; q < nf; ++q) {
        double x[3], J[3][3], S[3][3];
        hexk_eval(T.map_order, X, &R.fpts[3 * q], x, J);
        for (int k = 0; k < 3; ++k) T.fpts_x[(size_t(e) * nf + q) * 3 + k] = x[k];
        curl_eval(n1, &Lf[size_t(q) * 3 * n1], &dLf[size_t(q) * 3 * n1], w.data(), S);
        const double* n = &R.fnorm[3 * q];
        for (int j = 0; j < 3; ++j)
          T.fnvec[(size_t(e) * nf + q) * 3 + j] =
              S[0][j] * n[0] + S[1][j] * n[1] + S[2][j] * n[2];
      }
    }
  });
}

}  // namespace

void metric_points(const HostType& T, int np, const double* pts,
                   std::vector<double>& S) {
  const RefElement& R = T.ref;
  S.assign(size_t(T.ne) * 9 * np, 0.0);
  if (T.map_order >= 2 && T.kind != EK_HEX) {
    const CurlSimplex C(R);
    std::vector<double> dB;
    C.deriv(R, np, pts, dB);
    const int nmap = map_nodes(T.kind, T.map_order);
    parallel_elements(T.ne, [&](int64_t e0, int64_t e1) {
      std::vector<double> w(size_t(9) * C.ng);
      for (int64_t e = e0; e < e1; ++e) {
        C.fields(T.kind, T.map_order, &T.mapx[size_t(e) * nmap * 3], w.data());
        for (int q = 0; q < np; ++q) {
          double M[3][3];
          C.eval(&dB[size_t(q) * 3 * C.ng], w.data(), M);
          for (int r = 0; r < 9; ++r) S[(size_t(e) * 9 + r) * np + q] = M[r / 3][r % 3];
        }
      }
    });
    return;
  }
  if (T.map_order >= 2) {
    const int n1 = R.p + 1, ng = n1 * n1 * n1;
    const std::vector<double> g = gll_nodes(n1);
    std::vector<double> L, dL;
    curl_factors(g, np, pts, L, dL);
    parallel_elements(T.ne, [&](int64_t e0, int64_t e1) {
      std::vector<double> w(size_t(9) * ng);
      for (int64_t e = e0; e < e1; ++e) {
        curl_fields(&T.mapx[size_t(e) * map_nodes(EK_HEX, T.map_order) * 3], g, w.data(),
                    T.map_order);
        for (int q = 0; q < np; ++q) {
          double M[3][3];
          curl_eval(n1, &L[size_t(q) * 3 * n1], &dL[size_t(q) * 3 * n1], w.data(), M);
          for (int r = 0; r < 9; ++r) S[(size_t(e) * 9 + r) * np + q] = M[r / 3][r % 3];
        }
      }
    });
    return;
  }
  const int nv = R.nverts;
  std::vector<double> dN(size_t(np) * 3 * nv);
  for (int q = 0; q < np; ++q) R.dshape(&pts[3 * q], &dN[size_t(q) * 3 * nv]);
  for (int64_t e = 0; e < T.ne; ++e) {
    const double* X = &T.verts[size_t(e) * nv * 3];
    for (int q = 0; q < np; ++q) {
      double a[3][3];  // a[j] = d x / d x~_j
      for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) {
          double v = 0.0;
          for (int i = 0; i < nv; ++i) v += dN[(size_t(q) * 3 + j) * nv + i] * X[i * 3 + k];
          a[j][k] = v;
        }
      for (int i = 0; i < 3; ++i) {
        const double* b = a[(i + 1) % 3];
        const double* c = a[(i + 2) % 3];
        const double row[3] = {b[1] * c[2] - b[2] * c[1], b[2] * c[0] - b[0] * c[2],
                               b[0] * c[1] - b[1] * c[0]};
        for (int j = 0; j < 3; ++j) S[(size_t(e) * 9 + i * 3 + j) * np + q] = row[j];
      }
    }
  }
}

std::string build_mesh(const MeshInput& in, std::vector<HostType>& types,
                       HostConn& conn, bool* err_mesh) {
  *err_mesh = false;
  types.clear();
  for (auto& t : in.types) {
    if (t.second.first <= 0) continue;
    HostType T;
    T.kind = t.first;
    T.ne = t.second.first;
    T.ref = make_ref(T.kind, in.order, T.kind == EK_HEX ? in.family : 0);
    const int nv = T.ref.nverts;
    T.conn.assign(t.second.second, t.second.second + size_t(T.ne) * nv);
    for (int64_t v : T.conn)
      if (v < 0 || v >= in.n_nodes) return "connectivity refers to a missing node";
    int64_t span = T.ne * 5 * int64_t(T.ref.nfpts);
    if (span >= (int64_t(1) << 29)) return "too many elements of one type";
    const size_t ti = size_t(&t - in.types.data());
    if (ti < in.map_order.size() && in.map_order[ti] >= 2) {
      T.map_order = in.map_order[ti];
      const int nmap = map_nodes(T.kind, T.map_order);
      const int* corner = map_corners(T.kind, T.map_order);
      T.map_conn.assign(in.map_conn[ti], in.map_conn[ti] + size_t(T.ne) * nmap);
      for (int64_t e = 0; e < T.ne; ++e) {
        for (int v = 0; v < nmap; ++v) {
          const int64_t id = T.map_conn[size_t(e) * nmap + v];
          if (id < 0 || id >= in.n_nodes) return "map connectivity refers to a missing node";
        }
        for (int v = 0; v < nv; ++v)
          if (T.map_conn[size_t(e) * nmap + corner[v]] != T.conn[size_t(e) * nv + v])
            return "map corner nodes differ from the element vertices";
      }
      T.mapx.resize(size_t(T.ne) * nmap * 3);
      T.verts.resize(size_t(T.ne) * nv * 3);
      for (int64_t e = 0; e < T.ne; ++e) {
        for (int v = 0; v < nmap; ++v)
          for (int k = 0; k < 3; ++k)
            T.mapx[(size_t(e) * nmap + v) * 3 + k] =
                in.nodes[T.map_conn[size_t(e) * nmap + v] * 3 + k];
        for (int v = 0; v < nv; ++v)
          for (int k = 0; k < 3; ++k)
            T.verts[(size_t(e) * nv + v) * 3 + k] = T.mapx[(size_t(e) * nmap + corner[v]) * 3 + k];
      }
      curved_geometry(T);
    } else {
      geometry(T, in.nodes);
    }
    for (double r : T.rcpdjac)
      if (r <= 0) {
        *err_mesh = true;
        return "element with non-positive Jacobian";
      }
    types.push_back(std::move(T));
  }
  if (types.empty()) return "mesh has no elements";
  // ---- faces keyed by sorted vertex ids
  std::vector<FaceRec> faces;
  for (int t = 0; t < int(types.size()); ++t) {
    const HostType& T = types[t];
    const int nv = T.ref.nverts;
    for (int64_t e = 0; e < T.ne; ++e)
      for (int f = 0; f < T.ref.nfaces; ++f) {
        const RefFace& F = T.ref.faces[f];
        FaceRec r{t, e, f, {-1, -1, -1, -1}};
        int64_t ids[4];
        for (int i = 0; i < F.nv; ++i) ids[i] = T.conn[size_t(e) * nv + F.verts[i]];
        std::sort(ids, ids + F.nv);
        for (int i = 0; i < F.nv; ++i) r.key[4 - F.nv + i] = ids[i];
        faces.push_back(r);
      }
  }
  std::vector<size_t> order(faces.size());
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](size_t a, size_t b) {
    return key_less(faces[a], faces[b]);
  });
  struct FacePair {
    size_t a, b;
    double T[3];
  };
  std::vector<FacePair> fpairs;
  std::vector<char> matched(faces.size(), 0);
  for (size_t i = 0; i + 1 < order.size(); ++i) {
    const FaceRec& A = faces[order[i]];
    const FaceRec& B = faces[order[i + 1]];
    if (!key_eq(A.key, B.key)) continue;
    if (i + 2 < order.size() && key_eq(B.key, faces[order[i + 2]].key)) {
      *err_mesh = true;
      return "a face is shared by more than two elements";
    }
    matched[order[i]] = matched[order[i + 1]] = 1;
    fpairs.push_back({order[i], order[i + 1], {0, 0, 0}});
    ++i;
  }
  // ---- periodic pairing of left-over faces by translated centroids
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t n = 0; n < in.n_nodes; ++n)
    for (int k = 0; k < 3; ++k) {
      lo[k] = std::min(lo[k], in.nodes[3 * n + k]);
      hi[k] = std::max(hi[k], in.nodes[3 * n + k]);
    }
  double scale = std::max({hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]});
  const double tol = 1e-8 * scale;
  std::vector<size_t> left;
  for (size_t i = 0; i < faces.size(); ++i)
    if (!matched[i]) left.push_back(i);
  std::vector<std::array<double, 3>> cent(left.size());
  for (size_t i = 0; i < left.size(); ++i) {
    const FaceRec& r = faces[left[i]];
    double c[3] = {0, 0, 0};
    int n = 0;
    for (int k = 0; k < 4; ++k)
      if (r.key[k] >= 0) {
        for (int d = 0; d < 3; ++d) c[d] += in.nodes[3 * r.key[k] + d];
        ++n;
      }
    for (int d = 0; d < 3; ++d) cent[i][d] = c[d] / n;
  }
  std::vector<char> used(left.size(), 0);
  if (!in.periodic.empty() && !left.empty()) {
    const double q = 1e3 * tol;  // hash cell, far above rounding noise
    std::unordered_multimap<std::array<int64_t, 3>, size_t, Key3Hash> grid;
    auto cell = [&](const double* x) {
      return std::array<int64_t, 3>{int64_t(std::floor(x[0] / q)),
                                    int64_t(std::floor(x[1] / q)),
                                    int64_t(std::floor(x[2] / q))};
    };
    for (size_t i = 0; i < left.size(); ++i) grid.emplace(cell(cent[i].data()), i);
    for (auto& T : in.periodic)
      for (size_t i = 0; i < left.size(); ++i) {
        if (used[i]) continue;
        double x[3] = {cent[i][0] + T[0], cent[i][1] + T[1], cent[i][2] + T[2]};
        auto c0 = cell(x);
        size_t found = size_t(-1);
        for (int dx = -1; dx <= 1 && found == size_t(-1); ++dx)
          for (int dy = -1; dy <= 1 && found == size_t(-1); ++dy)
            for (int dz = -1; dz <= 1 && found == size_t(-1); ++dz) {
              auto rng = grid.equal_range({c0[0] + dx, c0[1] + dy, c0[2] + dz});
              for (auto it = rng.first; it != rng.second; ++it) {
                size_t j = it->second;
                if (used[j] || j == i) continue;
                double d2 = 0;
                for (int k = 0; k < 3; ++k) d2 += (cent[j][k] - x[k]) * (cent[j][k] - x[k]);
                if (d2 < tol * tol) {
                  found = j;
                  break;
                }
              }
            }
        if (found == size_t(-1)) continue;
        bool ta = faces[left[i]].key[0] < 0, tb = faces[left[found]].key[0] < 0;
        if (ta != tb) {
          *err_mesh = true;
          return "periodic faces of different kinds";
        }
        used[i] = used[found] = 1;
        fpairs.push_back({left[i], left[found], {T[0], T[1], T[2]}});
      }
  }
  // ---- element adjacency across every paired face (periodic ones too)
  {
    std::vector<int64_t> goff(types.size(), 0);
    for (size_t t = 1; t < types.size(); ++t) goff[t] = goff[t - 1] + types[t - 1].ne;
    for (auto& T : types) T.nbr.assign(size_t(T.ne) * T.ref.nfaces, -1);
    for (auto& fp : fpairs) {
      const FaceRec& A = faces[fp.a];
      const FaceRec& B = faces[fp.b];
      types[A.t].nbr[size_t(A.e) * types[A.t].ref.nfaces + A.f] = goff[B.t] + B.e;
      types[B.t].nbr[size_t(B.e) * types[B.t].ref.nfaces + B.f] = goff[A.t] + A.e;
    }
  }
  // ---- boundary faces
  std::unordered_map<std::array<int64_t, 4>, int, Key4Hash> bkey;
  for (int64_t b = 0; b < in.n_bfaces; ++b) {
    std::array<int64_t, 4> k;
    int n = 0;
    int64_t ids[4];
    for (int i = 0; i < 4; ++i)
      if (in.bface_nodes[4 * b + i] >= 0) ids[n++] = in.bface_nodes[4 * b + i];
    std::sort(ids, ids + n);
    k = {-1, -1, -1, -1};
    for (int i = 0; i < n; ++i) k[4 - n + i] = ids[i];
    int tag = in.bface_tags[b];
    int bc = -1;
    for (size_t i = 0; i < in.bc_tags.size(); ++i)
      if (in.bc_tags[i] == tag) bc = int(i);
    if (bc < 0) return "boundary face tag without a boundary condition";
    bkey[k] = bc;
  }
  struct BFace {
    size_t rec;
    int bc;
  };
  std::vector<BFace> bfaces;
  for (size_t i = 0; i < left.size(); ++i) {
    if (used[i]) continue;
    const FaceRec& r = faces[left[i]];
    std::array<int64_t, 4> k = {r.key[0], r.key[1], r.key[2], r.key[3]};
    auto it = bkey.find(k);
    if (it == bkey.end()) {
      *err_mesh = true;
      return "unmatched face (non-conforming mesh)";
    }
    bfaces.push_back({left[i], it->second});
  }
  // ---- flux-point pairing by physical coordinates
  conn = HostConn();
  struct PairRec {
    int32_t l, r;
    double n[4], mr;
  };
  std::vector<PairRec> prs;
  std::vector<int64_t> eoff(types.size(), 0);
  for (size_t t = 1; t < types.size(); ++t) eoff[t] = eoff[t - 1] + types[t - 1].ne;
  for (auto& fp0 : fpairs) {
    // orientation: the "-" (left) side is the element with the lower global
    // index, the lower face for an element paired with itself
    FacePair fp = fp0;
    {
      const FaceRec& a = faces[fp.a];
      const FaceRec& b = faces[fp.b];
      const int64_t ga = eoff[a.t] + a.e, gb = eoff[b.t] + b.e;
      if (gb < ga || (gb == ga && b.f < a.f)) {
        std::swap(fp.a, fp.b);
        for (int k = 0; k < 3; ++k) fp.T[k] = -fp.T[k];
      }
    }
    const FaceRec& A = faces[fp.a];
    const FaceRec& B = faces[fp.b];
    const HostType& TA = types[A.t];
    const HostType& TB = types[B.t];
    int a0 = TA.ref.face_start[A.f], na = TA.ref.face_start[A.f + 1] - a0;
    int b0 = TB.ref.face_start[B.f], nb = TB.ref.face_start[B.f + 1] - b0;
    if (na != nb) {
      *err_mesh = true;
      return "face kinds differ across an interface";
    }
    const int nfa = TA.ref.nfpts, nfb = TB.ref.nfpts;
    std::vector<char> taken(nb, 0);
    for (int i = 0; i < na; ++i) {
      const double* xa = &TA.fpts_x[(size_t(A.e) * nfa + a0 + i) * 3];
      double x[3] = {xa[0] + fp.T[0], xa[1] + fp.T[1], xa[2] + fp.T[2]};
      int best = -1;
      double bd = 1e300;
      for (int j = 0; j < nb; ++j) {
        const double* xb = &TB.fpts_x[(size_t(B.e) * nfb + b0 + j) * 3];
        double d2 = 0;
        for (int k = 0; k < 3; ++k) d2 += (x[k] - xb[k]) * (x[k] - xb[k]);
        if (d2 < bd) {
          bd = d2;
          best = j;
        }
      }
      if (bd > tol * tol || taken[best]) {
        *err_mesh = true;
        return "flux points do not conform across a face";
      }
      taken[best] = 1;
      PairRec pr;
      pr.l = encode_fp(A.t, A.e, nfa, a0 + i);
      pr.r = encode_fp(B.t, B.e, nfb, b0 + best);
      const double* na_ = &TA.fnvec[(size_t(A.e) * nfa + a0 + i) * 3];
      const double* nb_ = &TB.fnvec[(size_t(B.e) * nfb + b0 + best) * 3];
      double ma = std::sqrt(na_[0] * na_[0] + na_[1] * na_[1] + na_[2] * na_[2]);
      double mb = std::sqrt(nb_[0] * nb_[0] + nb_[1] * nb_[1] + nb_[2] * nb_[2]);
      for (int k = 0; k < 3; ++k) {
        pr.n[k] = na_[k] / ma;
        if (std::fabs(pr.n[k] + nb_[k] / mb) > 1e-8) {
          *err_mesh = true;
          return "interface normals do not match";
        }
      }
      pr.n[3] = ma;
      pr.mr = mb;
      prs.push_back(pr);
    }
  }
  std::sort(prs.begin(), prs.end(),
            [](const PairRec& a, const PairRec& b) { return a.l < b.l; });
  for (auto& p : prs) {
    conn.pl.push_back(p.l);
    conn.pr.push_back(p.r);
    conn.pn.insert(conn.pn.end(), p.n, p.n + 4);
    conn.pmr.push_back(p.mr);
  }
  for (auto& bf : bfaces) {
    const FaceRec& A = faces[bf.rec];
    const HostType& TA = types[A.t];
    int a0 = TA.ref.face_start[A.f], na = TA.ref.face_start[A.f + 1] - a0;
    const int nfa = TA.ref.nfpts;
    for (int i = 0; i < na; ++i) {
      conn.bidx.push_back(encode_fp(A.t, A.e, nfa, a0 + i));
      conn.bbc.push_back(bf.bc);
      const double* n = &TA.fnvec[(size_t(A.e) * nfa + a0 + i) * 3];
      double m = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
      conn.bn.insert(conn.bn.end(), {n[0] / m, n[1] / m, n[2] / m, m});
    }
  }
  return "";
}

}  // namespace frgb

// Reference-element data for the FR library (host side, FP64).
//
// Builds, for each element type and order p, the point sets and operator
// matrices of the Flux Reconstruction method (PyFR v2.0.3, Section 2):
//   M0   [nfpts][nupts]   interpolation to flux points, Eq. (disu)
//   D    [3][nupts][nupts] derivative of the nodal basis, Eq. (FRfinal)
//   LIFT [nupts][nfpts]   divergence of the DG correction function g_s at
//                         the solution points, Eq. (FRfinal)
// and, for the hexahedron, the 1D factors used by the sum-factorised kernels.
#pragma once
#include <array>
#include <cstdint>
#include <vector>

namespace frgb {

enum ElemKind { EK_HEX = 0, EK_PRI = 1, EK_TET = 2 };

struct RefFace {
  bool tri;                    // triangle (else quadrilateral)
  int nv;                      // 3 or 4 vertices
  int verts[4];                // local vertex ids
  double origin[3], ds[3], dt[3];  // x~ = origin + s ds + t dt
  double normal[3];            // reference unit outward normal
  double scale;                // |ds x dt|
};

struct RefElement {
  int kind = 0, p = 0, nverts = 0, nupts = 0, nfpts = 0, nfaces = 0;
  std::vector<RefFace> faces;
  std::vector<double> upts;        // [nupts][3]
  std::vector<double> fpts;        // [nfpts][3]
  std::vector<int> fpts_face;      // [nfpts]
  std::vector<int> face_start;     // [nfaces+1]
  std::vector<double> fnorm;       // [nfpts][3]
  std::vector<double> M0;          // [nfpts][nupts]
  std::vector<double> D;           // [3][nupts][nupts]
  std::vector<double> LIFT;        // [nupts][nfpts]
  std::vector<double> W;           // [nupts]  integration weights
  std::vector<double> vdm_inv;     // [nupts][nupts] modal <- nodal
  std::vector<int> mdeg;           // [nupts] total degree of each mode
  // hexahedron only: 1D factors on the line points x1
  std::vector<double> x1;          // [p+1]
  std::vector<double> d1;          // [p+1][p+1]  l_m'(x_a)
  std::vector<double> lm, lp;      // [p+1]  l_m(-1), l_m(+1)
  int family = 0;                  // 0 Gauss-Legendre, 1 Gauss-Lobatto lines
  std::vector<double> gl, gr;      // [p+1]  correction derivative weights:
                                   //  -g_L'(x_a) on x=-1, g_R'(x_a) on x=+1
  // vertex map of the element type
  void shape(const double* x, double* N) const;            // N[nverts]
  void dshape(const double* x, double* dN) const;          // dN[3][nverts]
  // orthonormal basis (modal) at points
  void basis(int npts, const double* x, double* out) const;           // [npts][nm]
  void grad(int npts, const double* x, double* out) const;            // [3][npts][nm]
};

// family 0: Gauss-Legendre line points; 1: Gauss-Lobatto (hexahedra only)
RefElement make_ref(int kind, int p, int family = 0);

// Nodes of the interpolant of the curl-form metric of curved elements
// ([n][3], n = the element's number of modes, nodes on every face so that a
// face's normal depends on that face alone): the Gauss-Lobatto tensor nodes
// (hexahedra), the warp-and-blend nodes (tetrahedra), the tetrahedron's
// face nodes times Gauss-Lobatto points along z (prisms).
std::vector<double> curl_nodes(const RefElement& R);

// 1D helpers (exposed for unit use)
void gauss_legendre(int n, double* x, double* w);
void gauss_lobatto(int n, double* x);
// n-point Gauss rule of the weight (1-x)^a (1+x)^b on [-1, 1], ascending.
void gauss_jacobi(int n, double a, double b, double* x, double* w);
// Anti-aliasing (Section 3.2): volume rule exact to degree qdeg, n = qdeg/2+1
// points per direction (n^3 points on every type): tensor Gauss-Legendre on
// the hexahedron; collapsed products with Gauss-Jacobi (1,0) / (2,0) factors
// on the prism's triangle and the tetrahedron.  xq [nq][3], wq [nq].
void aa_rule(int kind, int qdeg, std::vector<double>& xq, std::vector<double>& wq);
// B [nq][nupts]: l_z(x_q);  P [nupts][nq]: least-squares projection onto the
// solution space, P = V Phi_q^T diag(w) with the orthonormal basis Phi.
void aa_operators(const RefElement& R, const std::vector<double>& xq,
                  const std::vector<double>& wq, std::vector<double>& B,
                  std::vector<double>& P);
double jacobi_p(int n, double a, double b, double x);
double jacobi_dp(int n, double a, double b, double x);
bool invert(int n, const double* A, double* Ainv);

}  // namespace frgb

// Host-side mesh geometry and interface pairing for the FR library.
//
// Section 2 of the paper: the domain is a conforming tessellation; each
// element is the image of a reference element under x = M_n(x~) with
// Jacobian J; the transformed flux is f~ = J J^{-1} f = S f.  Flux points of
// adjoining elements conform.  Section 3.4: for linear elements the metric
// terms follow from the vertices alone.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "fr_ref.hpp"

namespace frgb {

struct HostType {
  int kind = 0;
  int64_t ne = 0;
  RefElement ref;
  std::vector<int64_t> conn;     // [ne][nv]
  int map_order = 1;             // 2: quadratic, 3: cubic map
  std::vector<int64_t> map_conn; // [ne][n_map] (map_order 2 or 3)
  std::vector<double> mapx;      // [ne][n_map][3] map node coordinates (map_order 2 or 3)
  // anti-aliasing (Section 3.2): rule of degree aa_qdeg and its operators
  int aa_qdeg = 0;
  std::vector<double> aa_x, aa_w;  // [nq][3], [nq]
  std::vector<double> aa_B;        // [nq][nupts]
  std::vector<double> aa_P;        // [nupts][nq]
  std::vector<double> verts;     // [ne][nv][3]
  std::vector<double> upts_x;    // [ne][nupts][3]
  std::vector<double> smat;      // [ne][9][nupts]   S[i][j] = row i, col j
  std::vector<double> rcpdjac;   // [ne][nupts]
  std::vector<double> fpts_x;    // [ne][nfpts][3]
  std::vector<double> fnvec;     // [ne][nfpts][3]  S^T n~ at flux points
  std::vector<int64_t> nbr;      // [ne][nfaces] neighbour element across each
                                 // face (global index: types in order hex,
                                 // prism, tet, then element), -1 on a boundary
};

// One side of a flux-point pair: element type in bits 29..30, offset of
// variable 0 (e * 5 * nfpts + f) in the low 29 bits.
inline int32_t encode_fp(int t, int64_t e, int nf, int f) {
  return int32_t((int64_t(t) << 29) | (e * 5 * nf + f));
}

struct HostConn {
  std::vector<int32_t> pl, pr;   // interior pairs (sorted by pl)
  std::vector<double> pn;        // [np][4]  unit normal from L side, |S^T n~| L
  std::vector<double> pmr;       // [np]     |S^T n~| on the R side
  std::vector<int32_t> bidx;     // boundary flux points
  std::vector<int32_t> bbc;      // boundary-condition index per point
  std::vector<double> bn;        // [nb][4]
};

struct MeshInput {
  int64_t n_nodes = 0;
  const double* nodes = nullptr;
  int order = 0;
  int family = 0;                       // hexahedron line points: 0 GL, 1 GLL
  std::vector<std::pair<int, std::pair<int64_t, const int64_t*>>> types;
  std::vector<int> map_order;               // per entry of types: 1, 2 or 3
  std::vector<const int64_t*> map_conn;     // per entry: [ne][n_map] or null
  std::vector<std::array<double, 3>> periodic;
  int64_t n_bfaces = 0;
  const int64_t* bface_nodes = nullptr;  // [n][4], -1 pads triangles
  const int* bface_tags = nullptr;
  std::vector<int> bc_tags;              // tag of bc index i
};

// S = det J J^{-1} of every element at reference points pts [np][3], laid
// out [ne][9][np]: the curl form on curved elements, the map's cross
// products on straight ones (the metric the mesh itself uses).
void metric_points(const HostType& T, int np, const double* pts,
                   std::vector<double>& S);

// Partition all elements (global index as in HostType::nbr) into nparts by
// recursive coordinate bisection of the element centroids.  mode 0
// (weighted): one bisection of all elements, element of kind k weighing
// w[k]; mode 1 (balanced): each element type bisected on its own, so every
// part gets the same number of elements of each type (to within one).
std::string partition_elements(const std::vector<HostType>& types, int nparts,
                               int mode, const double w[3],
                               std::vector<int32_t>& part);

// Returns an empty string on success, else an error message.  ``err_mesh``
// is set when the failure is a non-conforming / unmatched mesh.
std::string build_mesh(const MeshInput& in, std::vector<HostType>& types,
                       HostConn& conn, bool* err_mesh);

}  // namespace frgb

// Host-side mesh geometry and interface pairing.  See fr_mesh.hpp.
#include "fr_mesh.hpp"

#include <algorithm>
#include <cmath>
#include <numeric>
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

}  // namespace

std::string build_mesh(const MeshInput& in, std::vector<HostType>& types,
                       HostConn& conn, bool* err_mesh) {
  *err_mesh = false;
  types.clear();
  for (auto& t : in.types) {
    if (t.second.first <= 0) continue;
    HostType T;
    T.kind = t.first;
    T.ne = t.second.first;
    T.ref = make_ref(T.kind, in.order);
    const int nv = T.ref.nverts;
    T.conn.assign(t.second.second, t.second.second + size_t(T.ne) * nv);
    for (int64_t v : T.conn)
      if (v < 0 || v >= in.n_nodes) return "connectivity refers to a missing node";
    int64_t span = T.ne * 5 * int64_t(T.ref.nfpts);
    if (span >= (int64_t(1) << 29)) return "too many elements of one type";
    geometry(T, in.nodes);
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
  for (auto& fp : fpairs) {
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

// Internals of the FR library: device state of a mesh, kernel launch
// sequences and CUDA-graph replay of Runge-Kutta steps (templated on the
// value type T and the RK-register type TR).  Included by the C ABI unit
// fr_api.cu and by one unit per precision (fr_prec_*.cu), which alone
// instantiate the templates; see include/frgb.h for the ABI.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <array>
#include <memory>
#include <unordered_map>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/frgb.h"
#include "fr_aa.cuh"
#include "fr_dense_tc.cuh"
#include "fr_filter.cuh"
#include "fr_hex.cuh"
#include "fr_kernels.cuh"
#include "fr_prism.cuh"
#include "fr_err.hpp"
#include "fr_mesh.hpp"

using namespace frgb;

namespace frgb {


// Compile-time (nupts, nfpts) for every supported (element kind, order).
template <class F>
bool dispatch(int kind, int p, F&& f) {
  switch (kind * 16 + p) {
#define FR_CASE(K, P, NU, NF)                                              \
  case K * 16 + P:                                                         \
    f(std::integral_constant<int, NU>{}, std::integral_constant<int, NF>{}); \
    return true;
    FR_CASE(0, 1, 8, 24)
    FR_CASE(0, 2, 27, 54)
    FR_CASE(0, 3, 64, 96)
    FR_CASE(0, 4, 125, 150)
    FR_CASE(1, 1, 6, 18)
    FR_CASE(1, 2, 18, 39)
    FR_CASE(1, 3, 40, 68)
    FR_CASE(1, 4, 75, 105)
    FR_CASE(2, 1, 4, 12)
    FR_CASE(2, 2, 10, 24)
    FR_CASE(2, 3, 20, 40)
    FR_CASE(2, 4, 35, 60)
#undef FR_CASE
  }
  return false;
}

template <int NU>
constexpr int epb() {
  return NU >= 128 ? 1 : 128 / NU;
}

// elements per CTA of the persistent dense kernels
template <int NU>
constexpr int dense_epb() {
  return NU >= 256 ? 1 : 256 / NU;
}

template <typename T, int NU, int NF>
constexpr size_t dense_grad_smem() {
  return (size_t(DenseLayout<T, NU, NF>::kStagedCount) +
          size_t(dense_epb<NU>()) * size_t(DenseLayout<T, NU, NF>::kGradElem)) * sizeof(T);
}

template <typename T, int NU, int NF>
constexpr size_t dense_vol_smem() {
  return (size_t(DenseLayout<T, NU, NF>::kStagedCount) +
          size_t(dense_epb<NU>()) * size_t(DenseLayout<T, NU, NF>::kVolElem)) * sizeof(T);
}

struct DevType {
  int kind = 0, nu = 0, nf = 0;
  long long ne = 0;
  long long off_f = 0;      // offset of this type in the flux-point buffers
  void* X = nullptr;        // solution register        [ne][5][nu]
  void* Y = nullptr;        // stage register
  void* A = nullptr;        // RK4 accumulator
  void* R = nullptr;        // right-hand side (fr_rhs)
  void* smat = nullptr;     // [ne][9][nu]
  void* rcpdjac = nullptr;  // [ne][nu]
  void* grad = nullptr;     // [ne][15][nu] (NS)
  void* M0T = nullptr;
  void* DT = nullptr;
  void* LIFTT = nullptr;
  void* NREF = nullptr;
  HexOps<double> hx64{};
  HexOps<float> hx32{};
  // entropy filter (allocated by fr_filter_enable)
  void* fVinvT = nullptr;
  void* fVT = nullptr;
  void* fdeg = nullptr;
  void* fW = nullptr;
  int32_t* fpartner = nullptr;
  int32_t* flist = nullptr;  // [ne] elements that fail the zeta = 0 test
  int* fcount = nullptr;     // their number
  double* smin = nullptr;
  float* zeta_last = nullptr;
  int* evals_last = nullptr;
  int grad_ctas = 1, vol_ctas = 1;  // resident CTAs per SM (dense kernels)
  // prisms: operators in the structured form of fr_prism.cuh (device image
  // of PriLayout: values, then the column indices)
  bool pri_ok = false;
  int pri_nm = 0, pri_nl = 0;
  void* pri_img = nullptr;
  int pri_grad_ctas = 1, pri_vol_ctas = 1;
  // tetrahedra: M0 by its nonzeros (every flux point is a solution point)
  int32_t* m0c = nullptr;
  void* m0v = nullptr;
  int m0_nm = 0;
  // tiles picked by the autotuner (0: the default, the largest): elements per
  // CTA of the hexahedron kernels, persistent CTAs per SM of the dense ones
  int tile_grad = 0, tile_vol = 0;
  void* fnv = nullptr;       // [ne][3][nf] S^T n~ at flux points (NS)
  int8_t* fbc = nullptr;     // [ne][nf] boundary-condition index or -1 (NS)
  int32_t* fbi = nullptr;    // [ne][nf] boundary-point index or -1 (NS, prescribed states)
  void* verts = nullptr;     // [ne][8][3] vertices minus vertex 0 (hex, FP32)
  bool curved = false;       // quadratic map: metrics only from the tables
  // anti-aliasing (Section 3.2): operators, metric at the quadrature
  // points, and the projected transformed flux
  void* aaBT = nullptr;      // [nu][nq]
  void* aaPT = nullptr;      // [nq][nu]
  void* aasmq = nullptr;     // [ne][9][nq]
  void* tf = nullptr;        // [ne][3][5][nu]
  int aa_nq = 0, aa_ctas = 1;
  bool aa_hex = false;        // sum-factorised hexahedron form fits
  bool aa_dense = false;      // dense form fits
  bool aa_dv = false;         // vectorised dense form (operators resident)
  int aa_epb = 1, aa_dv_ctas = 1;
  int aa_hex_ctas = 1;
  HexAaOps<double> hxaa64{};
  HexAaOps<float> hxaa32{};
  // tensor-core kernels (prisms / tetrahedra, FP32 values)
  bool tc_ok = false;
  bool tca_ok = false;       // data-as-A volume kernel available
  bool tc_grad_on = true;    // kernels on the tensor cores when the family
  bool tc_vol_on = true;     //   is TENSOR (the tuner decides per type)
  void* tcimg = nullptr;     // split-TF32 operator image
  void* E = nullptr;         // embedded-error register (adaptive steps)
  void* Xs = nullptr;        // solution at the start of an adaptive step
  void* tcaimg = nullptr;    // the same, output points padded to 16
  TcGeom tcgeo{};
  int tc_vol_ctas = 1, tc_grad_ctas = 1;
};

inline void free_all(std::vector<void*>& v) {
  for (void* p : v)
    if (p) cudaFree(p);
  v.clear();
}

}  // namespace frgb

struct fr_mesh {
  int device = 0, precision = FR_FP64, physics = FR_EULER, order = 0;
  bool host_only = false;
  int num_sms = 152;
  size_t wsize = 8;   // bytes of a trace / flux / stage value
  size_t rsize = 8;   // bytes of a solution-register value
  cudaStream_t stream = nullptr, own_stream = nullptr;
  double gamma = 1.4, mu = 0.0, prandtl = 0.72;
  std::vector<HostType> host;
  HostConn conn;
  std::vector<DevType> types;
  int type_of_kind[3] = {-1, -1, -1};
  TypeTab tt{};
  BCTab<double> bc64{};
  BCTab<float> bc32{};
  long long nf_total = 0;
  void* uf = nullptr;
  void* fc = nullptr;
  void* du = nullptr;
  void* gradf = nullptr;
  int32_t* pl = nullptr;
  int32_t* pr = nullptr;
  void* pn = nullptr;
  void* pmr = nullptr;
  int32_t* bidx = nullptr;
  int32_t* bbc = nullptr;
  void* bn = nullptr;
  int np = 0, nb = 0;
  double* d_dt = nullptr;
  int* d_flag = nullptr;
  double h_dt = 0.0;
  bool uf_valid = false;
  // RK step graphs: FR_RK4, FR_RK45, and the adaptive RK45 step (index 2)
  cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};
  cudaStream_t graph_stream[3] = {nullptr, nullptr, nullptr};
  int variant = FR_VARIANT_AUTO;   // requested kernel family
  int active = FR_VARIANT_SUMFACT; // family in use (the tuner's choice)
  bool tuned = false;
  float tune_ms[5] = {0, 0, 0, 0, 0}; // ms per step of each family tried
  long long epoch = 0;            // bumped by every change of launch config
  long long graph_epoch[3] = {-1, -1, -1};
  int aa_qdeg = 0;            // anti-aliasing rule degree (0: collocation)
  double ldg_beta = 0.0, ldg_tau = 0.0;  // viscous coupling (0, 0: BR1)
  // exchange boundary points (partitioned meshes): receive buffers filled
  // by the group's push kernels, indexed by boundary point
  bool has_exch = false;
  bool has_presc = false;          // a boundary condition FR_BC_PRESCRIBED
  std::vector<int> bc_tags;        // tag of boundary condition i
  std::vector<char> presc_set;     // per condition: fr_set_bc_state called
  bool in_group = false;
  void* xu = nullptr;         // [nb][5] partner solution traces
  void* xg = nullptr;         // [nb][15] partner gradients (FP64) or [nb][5] q (FP32)
  void* xm = nullptr;         // [nb] partner |S^T n~|
  // boundary points [nb_x0, nb) are the exchange points; elements [0,
  // n_int[t]) of type t own none of them (the interior part of a stage)
  long long nb_x0 = 0;
  std::vector<long long> n_int;
  // exchange with other processes (fr_exchange_setup): own exchange points
  // (boundary-point indices) in message order, partners ascending
  int32_t* x_list = nullptr;
  long long n_xlist = 0;
  std::vector<long long> x_counts;  // points exchanged with each rank
  std::vector<int32_t> x_list_host;
  std::vector<double> periodic;  // [n][3] translation vectors
  bool err_on = false;        // stage epilogues accumulate the embedded error
  double* d_errpart = nullptr;  // per-block partial sums of the error norm
  double* d_errsum = nullptr;   // total
  double* d_tol = nullptr;      // atol, rtol
  double h_tol[2] = {0.0, 0.0};
  int n_errpart = 0;
  bool filter_on = false;
  bool mlp_on = false;
  FilterStats* d_fstats = nullptr;
  float* d_samples = nullptr;
  unsigned long long sample_cap = 0;
  __nv_bfloat16* d_mlp = nullptr;
  float* d_mlp_norm = nullptr;
  double mlp_ratio = 1.25;
  // fr_stats: call counters and device time of the timed calls (fr_rhs,
  // fr_rk_step, fr_rk_adaptive_step), measured with pairs of events on the
  // handle's stream and harvested once they have completed
  unsigned long long n_rhs = 0, n_steps = 0, n_attempts = 0, n_rejected = 0,
                     n_stages = 0;
  double ms_device = 0.0, t_last = 0.0;
  static constexpr int kEvRing = 32;
  cudaEvent_t ev_a[kEvRing] = {}, ev_b[kEvRing] = {};
  int ev_head = 0, ev_count = 0;
  double prof_ms[FR_KC_COUNT] = {};
  int prof_launches[FR_KC_COUNT] = {};
  // schedule picked by the autotuner: threads per CTA of the interface and
  // boundary kernels, and whether the per-type kernels of a phase run as
  // parallel branches (streams forked and joined inside the captured graph)
  int face_tb = 256;
  bool par_types = false;
  std::vector<cudaStream_t> par_st;
  std::vector<cudaEvent_t> par_ev;
  float sched_ms[2] = {0.f, 0.f};  // step time before / after tile tuning
  std::vector<void*> allocs;
  void* d_staging = nullptr;   // host-layout FP64 staging for set/get
  size_t staging_bytes = 0;

  ~fr_mesh() {
    if (x_list) cudaFree(x_list);
    for (cudaStream_t st : par_st)
      if (st) cudaStreamDestroy(st);
    for (cudaEvent_t ev : par_ev)
      if (ev) cudaEventDestroy(ev);
    for (int i = 0; i < kEvRing; ++i) {
      if (ev_a[i]) cudaEventDestroy(ev_a[i]);
      if (ev_b[i]) cudaEventDestroy(ev_b[i]);
    }
    for (int i = 0; i < 3; ++i)
      if (graph[i]) cudaGraphExecDestroy(graph[i]);
    free_all(allocs);
    if (d_staging) cudaFree(d_staging);
    if (d_samples) cudaFree(d_samples);
    if (own_stream) cudaStreamDestroy(own_stream);
  }
};

namespace {

template <typename T>
int dev_upload(fr_mesh* m, const std::vector<double>& h, void** out) {
  *out = nullptr;
  if (h.empty()) return FR_OK;
  std::vector<T> t(h.begin(), h.end());
  CK(cudaMalloc(out, t.size() * sizeof(T)));
  m->allocs.push_back(*out);
  CK(cudaMemcpy(*out, t.data(), t.size() * sizeof(T), cudaMemcpyHostToDevice));
  return FR_OK;
}

int dev_upload_i32(fr_mesh* m, const std::vector<int32_t>& h, int32_t** out) {
  *out = nullptr;
  if (h.empty()) return FR_OK;
  CK(cudaMalloc((void**)out, h.size() * sizeof(int32_t)));
  m->allocs.push_back(*out);
  CK(cudaMemcpy(*out, h.data(), h.size() * 4, cudaMemcpyHostToDevice));
  return FR_OK;
}

// The prism's operators in the structured form of fr_prism.cuh, read out of
// its dense operators: D_xi and D_eta must act within a level of the
// triangle x line point set (identical blocks on every level) and D_zeta
// along a line (the same 1D operator for every triangle point); M0 and LIFT
// are stored by their nonzeros.  Entries below 1e-12 of an operator's
// largest are structural zeros (the rounding of the dense construction).
// Returns false (the dense kernels stay) when the structure does not hold
// or a row has more nonzeros than the kernels are built for.
inline bool build_prism_ops(const RefElement& R, std::vector<double>& tv,
                            std::vector<int32_t>& ti, int* nm_out, int* nl_out) {
  const int p = R.p, NT = (p + 1) * (p + 2) / 2, NL = p + 1;
  const int NU = R.nupts, NF = R.nfpts;
  if (R.kind != EK_PRI || NU != NT * NL || NF != 2 * NT + 3 * NL * NL) return false;
  auto amax = [](const std::vector<double>& v) {
    double a = 0.0;
    for (double x : v) a = std::max(a, std::fabs(x));
    return a;
  };
  const double td = 1e-12 * amax(R.D);
  auto Dv = [&](int d, int r, int c) { return R.D[(size_t(d) * NU + r) * NU + c]; };
  for (int r = 0; r < NU; ++r)
    for (int c = 0; c < NU; ++c) {
      const int zr = r / NT, tr = r % NT, zc = c / NT, tc = c % NT;
      for (int d = 0; d < 2; ++d) {
        const double ref = zr == zc ? Dv(d, tr, tc) : 0.0;
        if (std::fabs(Dv(d, r, c) - ref) > td) return false;
      }
      const double rz = tr == tc ? Dv(2, zr * NT, zc * NT) : 0.0;
      if (std::fabs(Dv(2, r, c) - rz) > td) return false;
    }
  const double tm = 1e-12 * amax(R.M0), tl = 1e-12 * amax(R.LIFT);
  int nm = 0, nl = 0;
  for (int f = 0; f < NF; ++f) {
    int c = 0;
    for (int q = 0; q < NU; ++q) c += std::fabs(R.M0[size_t(f) * NU + q]) > tm;
    nm = std::max(nm, c);
  }
  for (int z = 0; z < NU; ++z) {
    int c = 0;
    for (int f = 0; f < NF; ++f) c += std::fabs(R.LIFT[size_t(z) * NF + f]) > tl;
    nl = std::max(nl, c);
  }
  if (nm < 1 || nl < 1 || nm > kPriMaxM0 || nl > kPriMaxLift) return false;
  tv.assign(size_t(2 * NT * NT + NL * NL + NF * nm + NU * nl + 3 * NF), 0.0);
  ti.assign(size_t(NF * nm + NU * nl), 0);
  double* axi = tv.data();
  double* aeta = axi + NT * NT;
  double* b = aeta + NT * NT;
  double* mv = b + NL * NL;
  double* lv = mv + NF * nm;
  double* nr = lv + NU * nl;
  int32_t* mc = ti.data();
  int32_t* lc = mc + NF * nm;
  for (int t = 0; t < NT; ++t)
    for (int t2 = 0; t2 < NT; ++t2) {
      axi[t * NT + t2] = Dv(0, t, t2);
      aeta[t * NT + t2] = Dv(1, t, t2);
    }
  for (int z = 0; z < NL; ++z)
    for (int z2 = 0; z2 < NL; ++z2) b[z * NL + z2] = Dv(2, z * NT, z2 * NT);
  for (int f = 0; f < NF; ++f) {
    int j = 0;
    for (int q = 0; q < NU; ++q) {
      const double v = R.M0[size_t(f) * NU + q];
      if (std::fabs(v) > tm) {
        mc[f * nm + j] = q;
        mv[f * nm + j] = v;
        ++j;
      }
    }
  }
  for (int z = 0; z < NU; ++z) {
    int j = 0;
    for (int f = 0; f < NF; ++f) {
      const double v = R.LIFT[size_t(z) * NF + f];
      if (std::fabs(v) > tl) {
        lc[z * nl + j] = f;
        lv[z * nl + j] = v;
        ++j;
      }
    }
  }
  for (int i = 0; i < 3 * NF; ++i) nr[i] = R.fnorm[i];
  *nm_out = nm;
  *nl_out = nl;
  return true;
}

// PriOps over the device image of a prism type (PriLayout order)
template <typename T>
PriOps<T> pri_ops_of(const fr_mesh* m, const DevType& D) {
  const int p = m->order, NT = (p + 1) * (p + 2) / 2, NL = p + 1;
  const int NU = D.nu, NF = D.nf, nm = D.pri_nm, nl = D.pri_nl;
  const T* t = static_cast<const T*>(D.pri_img);
  const T* axi = t;
  const T* aeta = axi + NT * NT;
  const T* b = aeta + NT * NT;
  const T* mv = b + NL * NL;
  const T* lv = mv + NF * nm;
  const T* nr = lv + NU * nl;
  const int tcount = 2 * NT * NT + NL * NL + NF * nm + NU * nl + 3 * NF;
  const int* ib = reinterpret_cast<const int*>(
      static_cast<const char*>(D.pri_img) + (size_t(tcount) * sizeof(T) + 15) / 16 * 16);
  return PriOps<T>{axi, aeta, b, ib, mv, ib + NF * nm, lv, nr, nm, nl};
}

int dev_zeros(fr_mesh* m, size_t bytes, void** out) {
  *out = nullptr;
  if (!bytes) return FR_OK;
  CK(cudaMalloc(out, bytes));
  m->allocs.push_back(*out);
  CK(cudaMemset(*out, 0, bytes));
  return FR_OK;
}

template <typename T>
HexOps<T> hex_ops(const RefElement& R) {
  HexOps<T> h{};
  const int n = R.p + 1;
  for (int a = 0; a < n; ++a) {
    for (int m = 0; m < n; ++m) h.d1[a][m] = T(R.d1[a * n + m]);
    h.lm[a] = T(R.lm[a]);
    h.lp[a] = T(R.lp[a]);
    h.gl[a] = T(R.gl[a]);
    h.gr[a] = T(R.gr[a]);
    h.xg[a] = T(R.x1[a]);
  }
  h.gather = R.family == 1;
  return h;
}

// TF32 value of x rounded to nearest, ties away from zero (the rounding of
// cvt.rna.tf32.f32): the low 13 mantissa bits become zero.
float tf32_rna_host(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7f800000u) != 0x7f800000u) {
    u += 0x1000u;
    u &= 0xffffe000u;
  }
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

// Face-aligned flux-point order of the tensor-core kernels for a prism or
// tetrahedron (layout documented in fr_dense_tc.cuh).  False when the
// element does not have the expected face structure (contiguous faces with
// one reference normal each).
bool build_tc_geo(const RefElement& R, TcGeom& geo, std::vector<int>& fpad) {
  const int nu = R.nupts, nf = R.nfpts;
  const int KFP = tc_kfp(nu, nf), NFACE = tc_nface(nu, nf);
  if (KFP == 0 || KFP > 128 || nf > 128 || nu > 128 || R.nfaces != NFACE ||
      int(R.face_start.size()) != NFACE + 1)
    return false;
  geo = TcGeom{};
  fpad.assign(nf, -1);
  int kofs = 0;
  for (int fa = 0; fa < NFACE; ++fa) {
    const int f0 = R.face_start[fa], f1 = R.face_start[fa + 1];
    geo.fslice[fa] = kofs / 8;
    for (int f = f0; f < f1; ++f) {
      fpad[f] = kofs + (f - f0);
      for (int d = 0; d < 3; ++d)
        if (R.fnorm[size_t(f) * 3 + d] != R.faces[fa].normal[d]) return false;
    }
    for (int d = 0; d < 3; ++d) geo.nface[fa][d] = float(R.faces[fa].normal[d]);
    kofs += tc_ru(f1 - f0, 8);
  }
  geo.fslice[NFACE] = kofs / 8;
  if (kofs != KFP) return false;
  std::vector<bool> used(KFP, false);
  for (int f = 0; f < nf; ++f) {
    if (fpad[f] < 0) return false;
    geo.fpad[f] = uint8_t(fpad[f]);
    used[fpad[f]] = true;
  }
  geo.npad = 0;
  for (int k = 0; k < KFP; ++k)
    if (!used[k]) geo.pad[geo.npad++] = uint8_t(k);
  return true;
}

// Split-TF32 operator image (hi plane, then lo plane, per operator) with the
// operators' output points padded to mf rows (M0) and mu rows (D, LIFT):
//   M0  mf x KU    M0[f][q]
//   D3  mu x 3KU   D_d[z][q] at column d KU + q
//   L   mu x KFP   LIFT[z][f] at column fpad[f]
void build_tc_image(const RefElement& R, const std::vector<int>& fpad, int mf, int mu,
                    std::vector<double>& img) {
  const int nu = R.nupts, nf = R.nfpts;
  const int KU = tc_ru(nu, 8), K3 = 3 * KU, KFP = tc_kfp(nu, nf);
  const size_t sm0 = size_t(mf) * KU, sd3 = size_t(mu) * K3, sl = size_t(mu) * KFP;
  img.assign(2 * (sm0 + sd3 + sl), 0.0);
  auto put = [&](size_t base, size_t plane, int off, double x) {
    const float h = tf32_rna_host(float(x));
    img[base + off] = h;
    img[base + plane + off] = tf32_rna_host(float(x - double(h)));
  };
  const size_t b_m0 = 0, b_d3 = 2 * sm0, b_l = 2 * (sm0 + sd3);
  for (int f = 0; f < nf; ++f)
    for (int q = 0; q < nu; ++q)
      put(b_m0, sm0, tc_offset(f, q, KU), R.M0[size_t(f) * nu + q]);
  for (int d = 0; d < 3; ++d)
    for (int z = 0; z < nu; ++z)
      for (int q = 0; q < nu; ++q)
        put(b_d3, sd3, tc_offset(z, d * KU + q, K3), R.D[(size_t(d) * nu + z) * nu + q]);
  for (int z = 0; z < nu; ++z)
    for (int f = 0; f < nf; ++f)
      put(b_l, sl, tc_offset(z, fpad[f], KFP), R.LIFT[size_t(z) * nf + f]);
}

// Compile-time tile of the tensor-core kernels for (NU, NF); false when the
// type has no tensor-core form (then the CUDA-core dense kernels run).
template <int NU, int NF>
constexpr bool tc_supported() {
  return tc_vol_epb<NU, NF>() > 0 && tc_grad_epb<NU, NF>() > 0;
}

// the data-as-A volume kernel: its MMA height when 128 rows (25 elements)
// fit, else 0 (with 64 rows it was no faster than k_vol_tc on prisms)
template <int NU, int NF>
constexpr int tca_supported() {
  return tc_supported<NU, NF>() && tca_m<NU, NF>() == 128 ? 128 : 0;
}

// precisions with tensor-core kernels: FP32 values and registers
template <typename T, typename TR>
constexpr bool tc_types() {
  return std::is_same<T, float>::value && std::is_same<TR, float>::value;
}

// T: storage/compute type of traces, fluxes and stage values;
// TR: type of the RK solution and accumulator registers (X, A).
template <typename T, typename TR>
int setup_device(fr_mesh* m) {
  int rc;
  long long off = 0;
  for (size_t t = 0; t < m->host.size(); ++t) {
    const HostType& H = m->host[t];
    DevType D;
    D.kind = H.kind;
    D.curved = H.map_order >= 2;
    D.nu = H.ref.nupts;
    D.nf = H.ref.nfpts;
    D.ne = H.ne;
    D.off_f = off;
    off += D.ne * 5 * D.nf;
    m->tt.nf[t] = D.nf;
    m->tt.off_f[t] = D.off_f;
    m->type_of_kind[D.kind] = int(t);
    size_t n = size_t(D.ne) * 5 * D.nu;
    if ((rc = dev_zeros(m, n * sizeof(TR), &D.X))) return rc;
    if ((rc = dev_zeros(m, n * sizeof(T), &D.Y))) return rc;
    if ((rc = dev_zeros(m, n * sizeof(TR), &D.A))) return rc;
    if ((rc = dev_zeros(m, n * sizeof(T), &D.R))) return rc;
    if (m->physics == FR_NAVIER_STOKES &&
        (rc = dev_zeros(m, 3 * n * sizeof(T), &D.grad)))
      return rc;
    if ((rc = dev_upload<T>(m, H.smat, &D.smat))) return rc;
    if ((rc = dev_upload<T>(m, H.rcpdjac, &D.rcpdjac))) return rc;
    const RefElement& R = H.ref;
    std::vector<double> m0t(size_t(D.nu) * D.nf), dt(3 * size_t(D.nu) * D.nu),
        lt(size_t(D.nf) * D.nu);
    for (int f = 0; f < D.nf; ++f)
      for (int z = 0; z < D.nu; ++z) {
        m0t[size_t(z) * D.nf + f] = R.M0[size_t(f) * D.nu + z];
        lt[size_t(f) * D.nu + z] = R.LIFT[size_t(z) * D.nf + f];
      }
    for (int d = 0; d < 3; ++d)
      for (int z = 0; z < D.nu; ++z)
        for (int v = 0; v < D.nu; ++v)
          dt[(size_t(d) * D.nu + v) * D.nu + z] =
              R.D[(size_t(d) * D.nu + z) * D.nu + v];
    if ((rc = dev_upload<T>(m, m0t, &D.M0T))) return rc;
    if ((rc = dev_upload<T>(m, dt, &D.DT))) return rc;
    if ((rc = dev_upload<T>(m, lt, &D.LIFTT))) return rc;
    if ((rc = dev_upload<T>(m, R.fnorm, &D.NREF))) return rc;
    if (D.kind == EK_TET) {
      // M0 rows with at most a quarter of the points nonzero: stored by
      // their nonzeros (a gather when the flux points are solution points)
      const int NU = D.nu, NF = D.nf;
      double mx = 0.0;
      for (double x : R.M0) mx = std::max(mx, std::fabs(x));
      int nm = 0;
      for (int f = 0; f < NF; ++f) {
        int c = 0;
        for (int q = 0; q < NU; ++q) c += std::fabs(R.M0[size_t(f) * NU + q]) > 1e-12 * mx;
        nm = std::max(nm, c);
      }
      if (nm >= 1 && 4 * nm <= NU) {
        std::vector<int32_t> mc(size_t(NF) * nm, 0);
        std::vector<double> mv(size_t(NF) * nm, 0.0);
        for (int f = 0; f < NF; ++f) {
          int j = 0;
          for (int q = 0; q < NU; ++q) {
            const double v = R.M0[size_t(f) * NU + q];
            if (std::fabs(v) > 1e-12 * mx) {
              mc[size_t(f) * nm + j] = q;
              mv[size_t(f) * nm + j] = v;
              ++j;
            }
          }
        }
        if ((rc = dev_upload_i32(m, mc, &D.m0c))) return rc;
        if ((rc = dev_upload<T>(m, mv, &D.m0v))) return rc;
        D.m0_nm = nm;
      }
    }
    if (D.kind == EK_PRI) {
      std::vector<double> tv;
      std::vector<int32_t> ti;
      if (build_prism_ops(R, tv, ti, &D.pri_nm, &D.pri_nl)) {
        // one device image: the values as T, padded to 16 bytes, then the
        // column indices (the shared-memory layout of the kernels)
        const size_t tb = (tv.size() * sizeof(T) + 15) / 16 * 16;
        std::vector<unsigned char> img(tb + ti.size() * 4, 0);
        for (size_t i = 0; i < tv.size(); ++i) {
          const T v = T(tv[i]);
          std::memcpy(img.data() + i * sizeof(T), &v, sizeof(T));
        }
        std::memcpy(img.data() + tb, ti.data(), ti.size() * 4);
        CK(cudaMalloc(&D.pri_img, img.size()));
        m->allocs.push_back(D.pri_img);
        CK(cudaMemcpy(D.pri_img, img.data(), img.size(), cudaMemcpyHostToDevice));
        D.pri_ok = true;
      }
    }
    if (sizeof(T) == 4 && D.kind != EK_HEX) {
      bool fits = false;
      int tca = 0;
      bool order_ok = true;  // host face order = the compile-time one
      dispatch(D.kind, m->order, [&](auto nu, auto nf) {
        constexpr int NU = decltype(nu)::value, NF = decltype(nf)::value;
        fits = tc_supported<NU, NF>();
        tca = tca_supported<NU, NF>();
      });
      std::vector<double> img;
      std::vector<int> fpad;
      if (fits && build_tc_geo(R, D.tcgeo, fpad)) {
        build_tc_image(R, fpad, D.nf <= 64 ? 64 : 128, D.nu <= 64 ? 64 : 128, img);
        if ((rc = dev_upload<float>(m, img, &D.tcimg))) return rc;
        D.tc_ok = true;
        for (int f = 0; f < D.nf; ++f) order_ok &= fpad[f] == tc_fpad(D.nu, D.nf, f);
        if (tca && order_ok) {
          build_tc_image(R, fpad, tc_ru(D.nf, 16), tc_ru(D.nu, 16), img);
          if ((rc = dev_upload<float>(m, img, &D.tcaimg))) return rc;
          D.tca_ok = true;
        }
      }
    }
    if (D.kind == EK_HEX) {
      D.hx64 = hex_ops<double>(R);
      D.hx32 = hex_ops<float>(R);
      if (sizeof(T) == 4 && !D.curved) {  // vertex metrics for the FP32-value kernels
        std::vector<double> xv(size_t(D.ne) * 24);
        for (long long e = 0; e < D.ne; ++e)
          for (int v = 0; v < 8; ++v)
            for (int k = 0; k < 3; ++k)
              xv[size_t(e) * 24 + v * 3 + k] = H.verts[(size_t(e) * 8 + v) * 3 + k] -
                                               H.verts[size_t(e) * 24 + k];
        if ((rc = dev_upload<T>(m, xv, &D.verts))) return rc;
      }
    }
    if (m->physics == FR_NAVIER_STOKES) {
      std::vector<double> nv(size_t(D.ne) * 3 * D.nf);
      for (long long e = 0; e < D.ne; ++e)
        for (int f = 0; f < D.nf; ++f)
          for (int j = 0; j < 3; ++j)
            nv[(size_t(e) * 3 + j) * D.nf + f] = H.fnvec[(size_t(e) * D.nf + f) * 3 + j];
      if ((rc = dev_upload<T>(m, nv, &D.fnv))) return rc;
      std::vector<int8_t> fbc(size_t(D.ne) * D.nf, -1);
      for (size_t i = 0; i < m->conn.bidx.size(); ++i) {
        int32_t code = m->conn.bidx[i];
        if ((code >> 29) != int(t)) continue;
        long long l = code & ((1 << 29) - 1);
        long long e = l / (5 * D.nf);
        int f = int(l - e * 5 * D.nf);
        fbc[size_t(e) * D.nf + f] = int8_t(m->conn.bbc[i]);
      }
      void* p = nullptr;
      CK(cudaMalloc(&p, fbc.size()));
      m->allocs.push_back(p);
      CK(cudaMemcpy(p, fbc.data(), fbc.size(), cudaMemcpyHostToDevice));
      D.fbc = (int8_t*)p;
      if (m->has_presc) {  // boundary-point index of every prescribed flux point
        std::vector<int32_t> fbi(size_t(D.ne) * D.nf, -1);
        for (size_t ib = 0; ib < m->conn.bidx.size(); ++ib) {
          int32_t code = m->conn.bidx[ib];
          if ((code >> 29) != int(t) || m->bc64.kind[m->conn.bbc[ib]] != FR_BC_PRESCRIBED) continue;
          long long l = code & ((1 << 29) - 1);
          long long e = l / (5 * D.nf);
          int f = int(l - e * 5 * D.nf);
          fbi[size_t(e) * D.nf + f] = int32_t(ib);
        }
        if ((rc = dev_upload_i32(m, fbi, &D.fbi))) return rc;
      }
    }
    m->types.push_back(D);
  }
  m->nf_total = off;
  size_t fb = size_t(off) * sizeof(T);
  if ((rc = dev_zeros(m, fb, &m->uf))) return rc;
  if ((rc = dev_zeros(m, fb, &m->fc))) return rc;
  if (m->physics == FR_NAVIER_STOKES) {
    if ((rc = dev_zeros(m, fb, &m->du))) return rc;
    // FP32 values: viscous normal flux q (5 per flux point); FP64: the 15
    // gradient components at flux points
    if ((rc = dev_zeros(m, (sizeof(T) == 4 ? 1 : 3) * fb, &m->gradf))) return rc;
  }
  const HostConn& C = m->conn;
  m->np = int(C.pl.size());
  m->nb = int(C.bidx.size());
  if ((rc = dev_upload_i32(m, C.pl, &m->pl))) return rc;
  if ((rc = dev_upload_i32(m, C.pr, &m->pr))) return rc;
  if ((rc = dev_upload<T>(m, C.pn, &m->pn))) return rc;
  if ((rc = dev_upload<T>(m, C.pmr, &m->pmr))) return rc;
  if ((rc = dev_upload_i32(m, C.bidx, &m->bidx))) return rc;
  if ((rc = dev_upload_i32(m, C.bbc, &m->bbc))) return rc;
  if ((rc = dev_upload<T>(m, C.bn, &m->bn))) return rc;
  CK(cudaMalloc((void**)&m->d_dt, sizeof(double)));
  m->allocs.push_back(m->d_dt);
  CK(cudaMalloc((void**)&m->d_flag, sizeof(int)));
  m->allocs.push_back(m->d_flag);
  CK(cudaMemset(m->d_flag, 0, sizeof(int)));
  return FR_OK;
}

template <typename T>
Phys<T> phys(const fr_mesh* m) {
  Phys<T> p;
  p.gamma = T(m->gamma);
  p.gm1 = T(m->gamma - 1.0);
  p.mu = T(m->mu);
  p.kappa = T(m->mu * m->gamma / m->prandtl);
  p.beta = T(m->ldg_beta);
  p.tau = T(m->ldg_tau);
  return p;
}

template <typename T>
const BCTab<T>& bctab(const fr_mesh* m);
template <>
const BCTab<double>& bctab<double>(const fr_mesh* m) {
  return m->bc64;
}
template <>
const BCTab<float>& bctab<float>(const fr_mesh* m) {
  return m->bc32;
}

template <typename T>
const HexOps<T>& hexops(const DevType& D);
template <>
const HexOps<double>& hexops<double>(const DevType& D) {
  return D.hx64;
}
template <>
const HexOps<float>& hexops<float>(const DevType& D) {
  return D.hx32;
}

template <typename T>
DenseOps<T> ops_of(const DevType& D) {
  return DenseOps<T>{(const T*)D.M0T, (const T*)D.DT, (const T*)D.LIFTT,
                     (const T*)D.NREF};
}

// tetrahedra outside the DENSE family: M0 by its nonzeros
bool use_m0s(const fr_mesh* m, const DevType& D) {
  return D.kind == EK_TET && D.m0_nm > 0 && m->active != FR_VARIANT_DENSE;
}

template <typename T>
DenseOps<T> stage_ops_of(const fr_mesh* m, const DevType& D) {
  DenseOps<T> o = ops_of<T>(D);
  if (use_m0s(m, D)) {
    o.Mc = D.m0c;
    o.Mv = (const T*)D.m0v;
    o.nm = D.m0_nm;
  }
  return o;
}

inline unsigned nblk(long long n, int b) { return unsigned((n + b - 1) / b); }

// hexahedron kernels: N = p + 1 solution points per line
template <class F>
bool hex_dispatch(int p, F&& f) {
  switch (p) {
    case 1: f(std::integral_constant<int, 2>{}); return true;
    case 2: f(std::integral_constant<int, 3>{}); return true;
    case 3: f(std::integral_constant<int, 4>{}); return true;
    case 4: f(std::integral_constant<int, 5>{}); return true;
  }
  return false;
}

template <int N>
constexpr int hex_epb() {
  return (N * N * N) >= 256 ? 1 : 256 / (N * N * N);
}

template <typename T, typename TR, int N>
constexpr size_t hex_vol_smem() {
  return size_t(hex_epb<N>()) * size_t(hex_vol_bytes_per_elem<T, TR, N>());
}

template <typename T, int N>
constexpr size_t hex_grad_smem() {
  return size_t(hex_epb<N>()) * size_t(hex_grad_bytes_per_elem<T, N, sizeof(T) == 4>());
}

bool use_hex(const fr_mesh* m, const DevType& D) {
  return D.kind == EK_HEX && m->active != FR_VARIANT_DENSE;
}

bool use_tc_grad(const fr_mesh* m, const DevType& D) {
  return D.tc_ok && D.tc_grad_on && m->active == FR_VARIANT_TENSOR;
}

bool use_tc_vol(const fr_mesh* m, const DevType& D) {
  return D.tc_ok && D.tc_vol_on && m->active == FR_VARIANT_TENSOR && m->aa_qdeg == 0;
}

// prisms on the structured kernels of fr_prism.cuh: every family but DENSE
// (which keeps the dense operator products), no anti-aliasing
bool use_pri(const fr_mesh* m, const DevType& D) {
  return D.kind == EK_PRI && D.pri_ok && m->active != FR_VARIANT_DENSE && m->aa_qdeg == 0;
}

template <typename T, int NU, int NF>
size_t pri_grad_smem(const DevType& D) {
  return size_t(PriLayout<T, NU, NF>::bytes(D.pri_nm, D.pri_nl)) +
         size_t(dense_epb<NU>()) * size_t(DenseLayout<T, NU, NF>::kGradElem) * sizeof(T);
}

template <typename T, int NU, int NF>
size_t pri_vol_smem(const DevType& D) {
  return size_t(PriLayout<T, NU, NF>::bytes(D.pri_nm, D.pri_nl)) +
         size_t(dense_epb<NU>()) * size_t(DenseLayout<T, NU, NF>::kVolElem) * sizeof(T);
}

// Anti-aliased transformed flux of one element type (Section 3.2) into D.tf;
// the volume kernel then reads it instead of collocating the flux.
template <typename T>
const HexAaOps<T>& hexaa_of(const DevType& D) {
  if constexpr (sizeof(T) == 8) return D.hxaa64;
  else return D.hxaa32;
}

template <typename T, typename TR>
void launch_aa_flux(fr_mesh* m, const DevType& D, cudaStream_t s, bool from_x,
                    bool ns, const Phys<T>& ph) {
  if (D.ne == 0) return;
  const bool hexk = use_hex(m, D);
  const T* uin = hexk ? (from_x ? nullptr : (const T*)D.Y)
                      : (from_x ? (const T*)D.X : (const T*)D.Y);
  const TR* X = hexk ? (const TR*)D.X : nullptr;
  if (hexk && D.aa_hex) {
    const HexAaOps<T>& hop = hexaa_of<T>(D);
    hex_dispatch(m->order, [&](auto n) {
      constexpr int N = decltype(n)::value;
      const unsigned grid = unsigned(std::min<long long>(D.ne, (long long)m->num_sms * D.aa_hex_ctas));
      const size_t sm = hex_aa_smem<T>(N, hop.q);
      auto go = [&](auto qt) {
        constexpr int QT = decltype(qt)::value;
        if (ns)
          k_hex_aa_flux<T, TR, N, QT, true><<<grid, kAaThreads, sm, s>>>(
              D.ne, uin, X, (const T*)D.grad, (const T*)D.aasmq, hop, ph, (T*)D.tf);
        else
          k_hex_aa_flux<T, TR, N, QT, false><<<grid, kAaThreads, sm, s>>>(
              D.ne, uin, X, nullptr, (const T*)D.aasmq, hop, ph, (T*)D.tf);
      };
      // compile-time point counts for FP32 values (the FP64 form is bound by
      // FP64 arithmetic, where the coefficient loads cost nothing extra)
      if constexpr (sizeof(T) == 4) {
        if (hop.q == N + 1) return go(std::integral_constant<int, N + 1>{});
        if (hop.q == N + 2) return go(std::integral_constant<int, N + 2>{});
      }
      go(std::integral_constant<int, 0>{});
    });
    return;
  }
  const AaOps<T> op{(const T*)D.aaBT, (const T*)D.aaPT, D.aa_nq};
  dispatch(D.kind, m->order, [&](auto nu, auto nf) {
    constexpr int NU = decltype(nu)::value;
    if (D.aa_dv) {
      const long long groups = (D.ne + D.aa_epb - 1) / D.aa_epb;
      const unsigned grid = unsigned(std::min<long long>(groups, (long long)m->num_sms * D.aa_dv_ctas));
      const size_t sm = aa_dense_v_smem<T, NU>(D.aa_nq, D.aa_epb);
      if (ns)
        k_aa_flux_dense_v<T, TR, NU, true><<<grid, kAaVThreads, sm, s>>>(
            D.ne, D.aa_epb, uin, X, (const T*)D.grad, (const T*)D.aasmq, op, ph, (T*)D.tf);
      else
        k_aa_flux_dense_v<T, TR, NU, false><<<grid, kAaVThreads, sm, s>>>(
            D.ne, D.aa_epb, uin, X, nullptr, (const T*)D.aasmq, op, ph, (T*)D.tf);
      return;
    }
    const unsigned grid = unsigned(std::min<long long>(D.ne, (long long)m->num_sms * D.aa_ctas));
    const size_t sm = aa_dense_smem<T, NU>(D.aa_nq);
    if (ns)
      k_aa_flux_dense<T, TR, NU, true><<<grid, kAaThreads, sm, s>>>(
          D.ne, uin, X, (const T*)D.grad, (const T*)D.aasmq, op, ph, (T*)D.tf);
    else
      k_aa_flux_dense<T, TR, NU, false><<<grid, kAaThreads, sm, s>>>(
          D.ne, uin, X, nullptr, (const T*)D.aasmq, op, ph, (T*)D.tf);
  });
}

// Tensor-core gradient kernel of a prism / tetrahedron type (FP32 values).
template <typename T, typename TR>
void launch_grad_tc(fr_mesh* m, const DevType& D, cudaStream_t s, bool from_x,
                    const T* du, const ViscArgs<T>& va, const BCTab<T>& bc,
                    const Phys<T>& ph) {
  if constexpr (tc_types<T, TR>()) {
    if (D.ne == 0) return;
    dispatch(D.kind, m->order, [&](auto nu, auto nf) {
      constexpr int NU = decltype(nu)::value, NF = decltype(nf)::value;
      if constexpr (tc_supported<NU, NF>()) {
        constexpr int EG = tc_grad_epb<NU, NF>();
        constexpr int BG = tc_minb_grad<NU, NF, EG>();
        const long long tiles = (D.ne + EG - 1) / EG;
        const unsigned grid = unsigned(
            std::min<long long>(tiles, (long long)m->num_sms * D.tc_grad_ctas));
        k_grad_tc<NU, NF, EG, TR, BG>
            <<<grid, kTcThreads, TcGradCfg<NU, NF, EG>::SMEM, s>>>(
                D.ne, from_x ? nullptr : (const float*)D.Y, (const TR*)D.X, du,
                (const float*)D.smat, (const float*)D.rcpdjac,
                (const float*)D.tcimg, D.tcgeo, (float*)D.grad, va, bc, ph,
                m->d_flag);
      }
    });
  }
}

// Tensor-core volume kernel of a prism / tetrahedron type (FP32 values).
template <typename T, typename TR>
void launch_vol_tc(fr_mesh* m, const DevType& D, cudaStream_t s, bool from_x,
                   bool ns, const T* fc, const Phys<T>& ph,
                   const HexStage<T, TR>& sa) {
  if constexpr (tc_types<T, TR>()) {
    if (D.ne == 0) return;
    dispatch(D.kind, m->order, [&](auto nu, auto nf) {
      constexpr int NU = decltype(nu)::value, NF = decltype(nf)::value;
      constexpr int MA = tca_supported<NU, NF>();
      if constexpr (MA > 0) {
        if (D.tca_ok) {
          using CA = TcaVolCfg<NU, NF, MA>;
          const long long tiles = (D.ne + CA::E - 1) / CA::E;
          const unsigned grid = unsigned(std::min<long long>(tiles, (long long)m->num_sms));
          const float* uin = from_x ? nullptr : (const float*)D.Y;
          if (ns)
            k_vol_tca<NU, NF, MA, true><<<grid, kTcThreads, CA::SMEM, s>>>(
                D.ne, uin, (const float*)D.grad, fc, (const float*)D.smat,
                (const float*)D.rcpdjac, (const float*)D.tcaimg, (const float*)D.NREF, ph,
                sa);
          else
            k_vol_tca<NU, NF, MA, false><<<grid, kTcThreads, CA::SMEM, s>>>(
                D.ne, uin, nullptr, fc, (const float*)D.smat, (const float*)D.rcpdjac,
                (const float*)D.tcaimg, (const float*)D.NREF, ph, sa);
          return;
        }
      }
      if constexpr (tc_supported<NU, NF>()) {
        constexpr int EV = tc_vol_epb<NU, NF>();
        constexpr int BV = tc_minb_vol<NU, NF, EV>();
        const long long tiles = (D.ne + EV - 1) / EV;
        const unsigned grid = unsigned(
            std::min<long long>(tiles, (long long)m->num_sms * D.tc_vol_ctas));
        const size_t sm = TcVolCfg<NU, NF, EV>::SMEM;
        const float* uin = from_x ? nullptr : (const float*)D.Y;
        if (ns)
          k_vol_tc<NU, NF, EV, true, TR, BV><<<grid, kTcThreads, sm, s>>>(
              D.ne, uin, (const float*)D.grad, fc, (const float*)D.smat,
              (const float*)D.rcpdjac, (const float*)D.tcimg,
              (const float*)D.NREF, D.tcgeo, ph, sa);
        else
          k_vol_tc<NU, NF, EV, false, TR, BV><<<grid, kTcThreads, sm, s>>>(
              D.ne, uin, nullptr, fc, (const float*)D.smat,
              (const float*)D.rcpdjac, (const float*)D.tcimg,
              (const float*)D.NREF, D.tcgeo, ph, sa);
      }
    });
  }
}

// shared memory of the FP32-value hexahedron kernels (vertex metrics,
// recomputed gradients)
template <typename T, int N>
constexpr size_t hexv_grad_smem() {
  return size_t(hex_epb<N>()) * size_t(hexv_grad_bytes_per_elem<T, N>());
}

template <typename T, typename TR, int N>
constexpr size_t hexv_vol_smem() {
  return size_t(hex_epb<N>()) * size_t(hexv_vol_bytes_per_elem<T, TR, N>());
}

// Opt in to > 48 KB of dynamic shared memory where a kernel needs it.  Runs
// once per handle outside any stream capture.
template <typename T, typename TR>
int prepare_kernels(fr_mesh* m) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, dev);
  for (auto& D : m->types) {
    dispatch(D.kind, m->order, [&](auto nu, auto nf) {
      constexpr int NU = decltype(nu)::value, NF = decltype(nf)::value;
      constexpr int E = dense_epb<NU>();
      auto kg = k_grad_dense<T, NU, NF, E, sizeof(T) == 4>;
      auto kv0 = k_vol_dense<T, NU, NF, E, false>;
      auto kv1 = k_vol_dense<T, NU, NF, E, true>;
      const int sg = int(dense_grad_smem<T, NU, NF>()), sv = int(dense_vol_smem<T, NU, NF>());
      cudaFuncSetAttribute(kg, cudaFuncAttributeMaxDynamicSharedMemorySize, sg);
      cudaFuncSetAttribute(kv0, cudaFuncAttributeMaxDynamicSharedMemorySize, sv);
      cudaFuncSetAttribute(kv1, cudaFuncAttributeMaxDynamicSharedMemorySize, sv);
      cudaFuncSetAttribute(k_vol_dense<T, NU, NF, E, false, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, sv);
      cudaFuncSetAttribute(k_vol_dense<T, NU, NF, E, true, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, sv);
      int a = 0, b = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, kg, E * NU, sg);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kv1, E * NU, sv);
      D.grad_ctas = a > 0 ? a : 1;
      D.vol_ctas = b > 0 ? b : 1;
      if constexpr (pri_order(NU, NF) > 0) {
        if (D.pri_ok) {
          auto pg = k_grad_pri<T, NU, NF, E, sizeof(T) == 4>;
          auto pv0 = k_vol_pri<T, NU, NF, E, false>;
          auto pv1 = k_vol_pri<T, NU, NF, E, true>;
          const int psg = int(pri_grad_smem<T, NU, NF>(D)), psv = int(pri_vol_smem<T, NU, NF>(D));
          cudaFuncSetAttribute(pg, cudaFuncAttributeMaxDynamicSharedMemorySize, psg);
          cudaFuncSetAttribute(pv0, cudaFuncAttributeMaxDynamicSharedMemorySize, psv);
          cudaFuncSetAttribute(pv1, cudaFuncAttributeMaxDynamicSharedMemorySize, psv);
          int pa = 0, pb = 0;
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pa, pg, E * NU, psg);
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pb, pv1, E * NU, psv);
          D.pri_grad_ctas = pa > 0 ? pa : 1;
          D.pri_vol_ctas = pb > 0 ? pb : 1;
        }
      }
      if constexpr (tc_types<T, TR>() && tc_supported<NU, NF>()) {
        if (D.tc_ok) {
          constexpr int EV = tc_vol_epb<NU, NF>(), EG = tc_grad_epb<NU, NF>();
          constexpr int BV = tc_minb_vol<NU, NF, EV>(), BG = tc_minb_grad<NU, NF, EG>();
          auto tv0 = k_vol_tc<NU, NF, EV, false, TR, BV>;
          auto tv1 = k_vol_tc<NU, NF, EV, true, TR, BV>;
          auto tg = k_grad_tc<NU, NF, EG, TR, BG>;
          const int smv = int(TcVolCfg<NU, NF, EV>::SMEM);
          const int smg = int(TcGradCfg<NU, NF, EG>::SMEM);
          cudaFuncSetAttribute(tv0, cudaFuncAttributeMaxDynamicSharedMemorySize, smv);
          cudaFuncSetAttribute(tv1, cudaFuncAttributeMaxDynamicSharedMemorySize, smv);
          cudaFuncSetAttribute(tg, cudaFuncAttributeMaxDynamicSharedMemorySize, smg);
          for (auto fn : {(const void*)tv0, (const void*)tv1, (const void*)tg})
            cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 int(cudaSharedmemCarveoutMaxShared));
          // resident CTAs per SM as designed: shared memory (the MINB bound
          // of the kernel's launch bounds) and the 512 TMEM columns.  (The
          // occupancy calculator reports one CTA for these kernels although
          // two fit; a grid that is too large would only run in two waves.)
          D.tc_vol_ctas = std::max(1, std::min(BV, 512 / TcVolCfg<NU, NF, EV>::TCOLS));
          D.tc_grad_ctas = std::max(1, std::min(BG, 512 / TcGradCfg<NU, NF, EG>::TCOLS));
          constexpr int MA = tca_supported<NU, NF>();
          if constexpr (MA > 0) {
            if (D.tca_ok) {
              const int sma = int(TcaVolCfg<NU, NF, MA>::SMEM);
              for (auto fn : {(const void*)k_vol_tca<NU, NF, MA, true>,
                              (const void*)k_vol_tca<NU, NF, MA, false>}) {
                cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, sma);
                cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     int(cudaSharedmemCarveoutMaxShared));
              }
            }
          }
        }
      }
    });
    if (D.kind != EK_HEX) continue;
    hex_dispatch(m->order, [&](auto n) {
      constexpr int N = decltype(n)::value;
      constexpr int E = hex_epb<N>();
      cudaFuncSetAttribute(k_hex_vol<T, TR, N, E, false>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(hex_vol_smem<T, TR, N>()));
      cudaFuncSetAttribute(k_hex_vol<T, TR, N, E, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(hex_vol_smem<T, TR, N>()));
      cudaFuncSetAttribute(k_hex_vol<T, TR, N, E, false, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(hex_vol_smem<T, TR, N>()));
      cudaFuncSetAttribute(k_hex_vol<T, TR, N, E, true, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(hex_vol_smem<T, TR, N>()));
      cudaFuncSetAttribute(k_hex_grad<T, TR, N, E, sizeof(T) == 4>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(hex_grad_smem<T, N>()));
      cudaFuncSetAttribute(k_hex_grad_v<T, TR, N, E>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(hexv_grad_smem<T, N>()));
      cudaFuncSetAttribute(k_hex_vol_v<T, TR, N, E, false>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(hexv_vol_smem<T, TR, N>()));
      cudaFuncSetAttribute(k_hex_vol_v<T, TR, N, E, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(hexv_vol_smem<T, TR, N>()));
    });
  }
  CK(cudaGetLastError());
  return FR_OK;
}

template <typename T, typename TR>
void launch_interp(fr_mesh* m, cudaStream_t s) {
  for (auto& D : m->types) {
    T* uf = (T*)m->uf + D.off_f;
    if (use_hex(m, D)) {
      hex_dispatch(m->order, [&](auto n) {
        constexpr int N = decltype(n)::value;
        constexpr int E = hex_epb<N>();
        k_hex_interp<T, TR, N, E><<<nblk(D.ne, E), E * N * N * N, 0, s>>>(
            D.ne, (const TR*)D.X, hexops<T>(D), uf);
      });
      continue;
    }
    dispatch(D.kind, m->order, [&](auto nu, auto nf) {
      constexpr int NU = decltype(nu)::value, NF = decltype(nf)::value;
      constexpr int E = epb<NU>();
      k_interp_dense<T, NU, NF, E><<<nblk(D.ne, E), E * NU, 0, s>>>(
          D.ne, (const T*)D.X, ops_of<T>(D), uf);
    });
  }
}

// Optional per-launch event recorder used by fr_profile_step.
struct Prof {
  std::vector<int> cls;
  std::vector<cudaEvent_t> ev;  // pairs (start, end)
  void mark(int c, cudaStream_t s, bool start) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, s);
    ev.push_back(e);
    if (start) cls.push_back(c);
  }
};

#define PROF_BEGIN(c) \
  if (prof) prof->mark(c, s, true)
#define PROF_END(c) \
  if (prof) prof->mark(c, s, false)

template <typename T, typename TR>
void launch_entropy_min(fr_mesh* m, cudaStream_t s, bool from_x);
template <typename T, typename TR>
void launch_filter(fr_mesh* m, cudaStream_t s, DevType& D, bool last_stage);

// Streams and events of the parallel per-type branches (created once).
inline int ensure_par(fr_mesh* m) {
  const size_t nt = m->types.size();
  while (m->par_st.size() < nt) {
    cudaStream_t st = nullptr;
    CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    m->par_st.push_back(st);
  }
  while (m->par_ev.size() < nt + 1) {
    cudaEvent_t ev = nullptr;
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    m->par_ev.push_back(ev);
  }
  return FR_OK;
}

// Largest elements-per-CTA tile of the hexahedron kernels at order p (the
// kernels' launch bound) and the tiles the autotuner tries: its divisors
// down to one element.
inline int hex_tile_max(int p) {
  const int nu = (p + 1) * (p + 1) * (p + 1);
  return nu >= 256 ? 1 : 256 / nu;
}

inline std::vector<int> tile_candidates(const fr_mesh* m, const DevType& D, bool grad) {
  std::vector<int> c;
  if (D.kind == EK_HEX && m->active != FR_VARIANT_DENSE) {
    const int e = hex_tile_max(m->order);
    for (int k = e; k >= 1; k = k > 1 ? (k % 2 == 0 ? k / 2 : (k % 3 == 0 ? k / 3 : 1)) : 0) {
      c.push_back(k);
      if (k == 1) break;
    }
  } else {
    const int mx = use_pri(m, D) ? (grad ? D.pri_grad_ctas : D.pri_vol_ctas)
                                 : (grad ? D.grad_ctas : D.vol_ctas);
    for (int k = mx; k >= 1; k /= 2) c.push_back(k);
  }
  return c;
}

// Elements [e0, e0 + n) of a type as a type of their own: every
// per-element array shifted, flux-point regions included.  The kernels then
// run on that range unchanged.
inline DevType sub_view(const fr_mesh* m, const DevType& D, long long e0, long long n) {
  DevType V = D;
  V.ne = n;
  const size_t w = m->wsize, r = m->rsize, nu = size_t(D.nu), nf = size_t(D.nf);
  auto sh = [&](void* p, size_t per) -> void* {
    return p ? static_cast<void*>(static_cast<char*>(p) + size_t(e0) * per) : nullptr;
  };
  V.X = sh(D.X, 5 * nu * r);
  V.A = sh(D.A, 5 * nu * r);
  V.E = sh(D.E, 5 * nu * r);
  V.Xs = sh(D.Xs, 5 * nu * r);
  V.Y = sh(D.Y, 5 * nu * w);
  V.R = sh(D.R, 5 * nu * w);
  V.smat = sh(D.smat, 9 * nu * w);
  V.rcpdjac = sh(D.rcpdjac, nu * w);
  V.grad = sh(D.grad, 15 * nu * w);
  V.fnv = sh(D.fnv, 3 * nf * w);
  V.fbc = static_cast<int8_t*>(sh(D.fbc, nf));
  V.fbi = static_cast<int32_t*>(sh(D.fbi, nf * sizeof(int32_t)));
  V.verts = sh(D.verts, 24 * w);
  V.aasmq = sh(D.aasmq, 9 * size_t(D.aa_nq) * w);
  V.tf = sh(D.tf, 15 * nu * w);
  V.off_f = D.off_f + e0 * 5 * (long long)nf;
  return V;
}

// Launch one RK stage (or a bare right-hand side when mode == 0).  phase
// bit 1: the NS common solution and gradients; bit 2: the common fluxes and
// the volume kernels.  A partitioned group exchanges the gradient traces
// between the two (and the solution traces before bit 1).  part 1: only the
// interior pairs, the boundary points that are not exchange points and the
// elements that own no exchange point; part 2: the rest (exchange points and
// the elements [n_int, ne)); 0: everything.
template <typename T, typename TR>
void launch_stage(fr_mesh* m, cudaStream_t s, int mode, int stage,
                  Prof* prof = nullptr, int phase = 3, int part = 0) {
  const bool ns = m->physics == FR_NAVIER_STOKES;
  const Phys<T> ph = phys<T>(m);
  const BCTab<T>& bc = bctab<T>(m);
  const int tb = m->face_tb;
  // the per-type kernels of a phase: in order on s, or (schedule par_types,
  // not while profiling) as parallel branches forked from and joined to s
  auto per_type = [&](auto&& fn) {
    const size_t nt = m->types.size();
    std::vector<DevType> views;
    std::vector<DevType*> ds;
    if (part == 0) {
      for (auto& D : m->types) ds.push_back(&D);
    } else {
      views.reserve(nt);
      for (size_t t = 0; t < nt; ++t) {
        const DevType& D = m->types[t];
        const long long ni = t < m->n_int.size() ? m->n_int[t] : D.ne;
        const long long e0 = part == 1 ? 0 : ni, n = part == 1 ? ni : D.ne - ni;
        if (n <= 0) continue;
        views.push_back(sub_view(m, D, e0, n));
      }
      for (auto& V : views) ds.push_back(&V);
    }
    if (!m->par_types || prof || ds.size() < 2 || m->par_st.size() < ds.size()) {
      for (DevType* D : ds) fn(*D, s);
      return;
    }
    cudaEventRecord(m->par_ev[0], s);
    for (size_t t = 0; t < ds.size(); ++t) {
      cudaStreamWaitEvent(m->par_st[t], m->par_ev[0], 0);
      fn(*ds[t], m->par_st[t]);
      cudaEventRecord(m->par_ev[1 + t], m->par_st[t]);
    }
    for (size_t t = 0; t < ds.size(); ++t) cudaStreamWaitEvent(s, m->par_ev[1 + t], 0);
  };
  // boundary points of this part: [b0, b0 + nbp)
  const long long b0 = part == 2 ? m->nb_x0 : 0;
  const long long nbp = part == 0 ? m->nb : (part == 1 ? m->nb_x0 : m->nb - m->nb_x0);
  const bool pairs = part != 2;
  const int nvg = sizeof(T) == 4 ? 5 : 15;
  const int32_t* bidx = m->bidx + b0;
  const int32_t* bbc = m->bbc + b0;
  const T* bnp = m->bn ? (const T*)m->bn + 4 * b0 : nullptr;
  const T* xup = m->xu ? (const T*)m->xu + 5 * b0 : nullptr;
  const T* xgp = m->xg ? (const T*)m->xg + nvg * b0 : nullptr;
  const T* xmp = m->xm ? (const T*)m->xm + b0 : nullptr;
  // stage input: the solution register X for a bare RHS and the first
  // stage, the stage register Y afterwards
  const bool from_x = (mode == 0 || stage == 0);
  const bool filt = m->filter_on && mode != 0;
  const bool last_stage = (mode == 1 && stage == 3) || (mode == 2 && stage == 4);
  if (filt && (phase & 1)) {
    PROF_BEGIN(FR_KC_FILTER);
    launch_entropy_min<T, TR>(m, s, from_x);
    PROF_END(FR_KC_FILTER);
  }
  if (ns && (phase & 1)) {
    if (m->np && pairs) {
      PROF_BEGIN(FR_KC_FACE_U);
      k_face_ucommon<T><<<nblk(m->np, tb), tb, 0, s>>>(
          m->np, m->pl, m->pr, (const T*)m->uf, (T*)m->du, m->tt, ph.beta);
      PROF_END(FR_KC_FACE_U);
    }
    if (nbp > 0) {
      PROF_BEGIN(FR_KC_BND_U);
      k_bnd_ucommon<T><<<nblk(nbp, tb), tb, 0, s>>>(
          int(nbp), bidx, bbc, (const T*)m->uf, (T*)m->du, m->tt, bc, xup, ph.beta);
      PROF_END(FR_KC_BND_U);
    }
    per_type([&](DevType& D, cudaStream_t s) {
      const T* du = (const T*)m->du + D.off_f;
      ViscArgs<T> va{(const T*)m->uf + D.off_f, (const T*)D.fnv, D.fbc,
                     (T*)m->gradf + D.off_f * (sizeof(T) == 4 ? 1 : 3)};
      va.fbi = D.fbi;
      va.xp = (const T*)m->xu;
      PROF_BEGIN(FR_KC_GRAD);
      if (use_hex(m, D) && sizeof(T) == 4 && D.verts &&
          m->active == FR_VARIANT_SUMFACT_VERTEX) {
        hex_dispatch(m->order, [&](auto n) {
          constexpr int N = decltype(n)::value;
          constexpr int E = hex_epb<N>();
          const int eb = D.tile_grad > 0 ? D.tile_grad : E;
          k_hex_grad_v<T, TR, N, E>
              <<<nblk(D.ne, eb), eb * N * N * N, hexv_grad_smem<T, N>() / E * eb, s>>>(
                  D.ne, from_x ? nullptr : (const T*)D.Y, (const TR*)D.X, du,
                  (const T*)D.verts, hexops<T>(D), va, bc, ph);
        });
      } else if (use_hex(m, D)) {
        hex_dispatch(m->order, [&](auto n) {
          constexpr int N = decltype(n)::value;
          constexpr int E = hex_epb<N>();
          const int eb = D.tile_grad > 0 ? D.tile_grad : E;
          k_hex_grad<T, TR, N, E, sizeof(T) == 4>
              <<<nblk(D.ne, eb), eb * N * N * N, hex_grad_smem<T, N>() / E * eb, s>>>(
                  D.ne, from_x ? nullptr : (const T*)D.Y, (const TR*)D.X, du,
                  (const T*)D.smat, (const T*)D.rcpdjac, hexops<T>(D),
                  (T*)D.grad, va, bc, ph);
        });
      } else if (use_tc_grad(m, D)) {
        launch_grad_tc<T, TR>(m, D, s, from_x, du, va, bc, ph);
      } else if (use_pri(m, D)) {
        dispatch(D.kind, m->order, [&](auto nu, auto nf) {
          constexpr int NU = decltype(nu)::value, NF = decltype(nf)::value;
          if constexpr (pri_order(NU, NF) > 0) {
            constexpr int E = dense_epb<NU>();
            const unsigned grid = unsigned(std::min<long long>(
                (D.ne + E - 1) / E,
                (long long)m->num_sms * (D.tile_grad > 0 ? D.tile_grad : D.pri_grad_ctas)));
            k_grad_pri<T, NU, NF, E, sizeof(T) == 4>
                <<<grid, E * NU, pri_grad_smem<T, NU, NF>(D), s>>>(
                    D.ne, from_x ? (const T*)D.X : (const T*)D.Y, du, (const T*)D.smat,
                    (const T*)D.rcpdjac, pri_ops_of<T>(m, D), (T*)D.grad, va, bc, ph);
          }
        });
      } else {
        dispatch(D.kind, m->order, [&](auto nu, auto nf) {
          constexpr int NU = decltype(nu)::value, NF = decltype(nf)::value;
          constexpr int E = dense_epb<NU>();
          const size_t sm = dense_grad_smem<T, NU, NF>();
          const unsigned grid = unsigned(std::min<long long>(
              (D.ne + E - 1) / E,
              (long long)m->num_sms * (D.tile_grad > 0 ? D.tile_grad : D.grad_ctas)));
          k_grad_dense<T, NU, NF, E, sizeof(T) == 4><<<grid, E * NU, sm, s>>>(
              D.ne, from_x ? (const T*)D.X : (const T*)D.Y, du,
              (const T*)D.smat, (const T*)D.rcpdjac, stage_ops_of<T>(m, D), (T*)D.grad,
              va, bc, ph);
        });
      }
      PROF_END(FR_KC_GRAD);
    });
  }
  if (!(phase & 2)) return;
  if (m->np && pairs) {
    PROF_BEGIN(FR_KC_FACE_F);
    if (ns && sizeof(T) == 4)
      k_face_flux_ns<T><<<nblk(m->np, tb), tb, 0, s>>>(
          m->np, m->pl, m->pr, (const T*)m->pn, (const T*)m->pmr,
          (const T*)m->uf, (const T*)m->gradf, (T*)m->fc, m->tt, ph);
    else if (ns)
      k_face_flux<T, true><<<nblk(m->np, tb), tb, 0, s>>>(
          m->np, m->pl, m->pr, (const T*)m->pn, (const T*)m->pmr,
          (const T*)m->uf, (const T*)m->gradf, (T*)m->fc, m->tt, ph);
    else
      k_face_flux<T, false><<<nblk(m->np, tb), tb, 0, s>>>(
          m->np, m->pl, m->pr, (const T*)m->pn, (const T*)m->pmr,
          (const T*)m->uf, nullptr, (T*)m->fc, m->tt, ph);
    PROF_END(FR_KC_FACE_F);
  }
  if (nbp > 0) {
    PROF_BEGIN(FR_KC_BND_F);
    if (ns && sizeof(T) == 4)
      k_bnd_flux_ns<T><<<nblk(nbp, tb), tb, 0, s>>>(
          int(nbp), bidx, bbc, bnp, (const T*)m->uf, (const T*)m->gradf, (T*)m->fc,
          m->tt, ph, bc, xup, xgp, xmp);
    else if (ns)
      k_bnd_flux<T, true><<<nblk(nbp, tb), tb, 0, s>>>(
          int(nbp), bidx, bbc, bnp, (const T*)m->uf, (const T*)m->gradf, (T*)m->fc,
          m->tt, ph, bc, xup, xgp);
    else
      k_bnd_flux<T, false><<<nblk(nbp, tb), tb, 0, s>>>(
          int(nbp), bidx, bbc, bnp, (const T*)m->uf, nullptr, (T*)m->fc, m->tt, ph,
          bc, xup);
    PROF_END(FR_KC_BND_F);
  }
  const bool aa = m->aa_qdeg > 0;
  per_type([&](DevType& D, cudaStream_t s) {
    T* uf_next = mode == 0 ? nullptr : (T*)m->uf + D.off_f;
    const T* fc = (const T*)m->fc + D.off_f;
    if (aa) {
      PROF_BEGIN(FR_KC_AAFLUX);
      launch_aa_flux<T, TR>(m, D, s, from_x, ns, ph);
      PROF_END(FR_KC_AAFLUX);
    }
    PROF_BEGIN(FR_KC_VOL);
    if (use_hex(m, D)) {
      HexStage<T, TR> sa{mode, stage, (TR*)D.X, (TR*)D.A, (T*)D.Y, (T*)D.R,
                         m->d_dt, m->d_flag, uf_next};
      sa.E = m->err_on ? (TR*)D.E : nullptr;
      hex_dispatch(m->order, [&](auto n) {
        constexpr int N = decltype(n)::value;
        constexpr int E = hex_epb<N>();
        const int eb = D.tile_vol > 0 ? D.tile_vol : E;
        const size_t sm = hex_vol_smem<T, TR, N>() / E * eb;
        const T* uin = from_x ? nullptr : (const T*)D.Y;
        if (sizeof(T) == 4 && D.verts && m->active == FR_VARIANT_SUMFACT_VERTEX) {
          const size_t smv = hexv_vol_smem<T, TR, N>() / E * eb;
          const T* dup = (const T*)m->du + D.off_f;
          if (ns)
            k_hex_vol_v<T, TR, N, E, true><<<nblk(D.ne, eb), eb * N * N * N, smv, s>>>(
                D.ne, uin, dup, fc, (const T*)D.verts, hexops<T>(D), ph, sa);
          else
            k_hex_vol_v<T, TR, N, E, false><<<nblk(D.ne, eb), eb * N * N * N, smv, s>>>(
                D.ne, uin, nullptr, fc, (const T*)D.verts, hexops<T>(D), ph, sa);
          return;
        }
        if (aa && ns)
          k_hex_vol<T, TR, N, E, true, true><<<nblk(D.ne, eb), eb * N * N * N, sm, s>>>(
              D.ne, uin, nullptr, fc, nullptr, (const T*)D.rcpdjac, hexops<T>(D),
              ph, sa, (const T*)D.tf);
        else if (aa)
          k_hex_vol<T, TR, N, E, false, true><<<nblk(D.ne, eb), eb * N * N * N, sm, s>>>(
              D.ne, uin, nullptr, fc, nullptr, (const T*)D.rcpdjac, hexops<T>(D),
              ph, sa, (const T*)D.tf);
        else if (ns)
          k_hex_vol<T, TR, N, E, true><<<nblk(D.ne, eb), eb * N * N * N, sm, s>>>(
              D.ne, uin, (const T*)D.grad, fc, (const T*)D.smat,
              (const T*)D.rcpdjac, hexops<T>(D), ph, sa);
        else
          k_hex_vol<T, TR, N, E, false><<<nblk(D.ne, eb), eb * N * N * N, sm, s>>>(
              D.ne, uin, nullptr, fc, (const T*)D.smat, (const T*)D.rcpdjac,
              hexops<T>(D), ph, sa);
      });
    } else if (use_tc_vol(m, D)) {
      HexStage<T, TR> sa{mode, stage, (TR*)D.X, (TR*)D.A, (T*)D.Y, (T*)D.R,
                         m->d_dt, m->d_flag, uf_next};
      sa.E = m->err_on ? (TR*)D.E : nullptr;
      launch_vol_tc<T, TR>(m, D, s, from_x, ns, fc, ph, sa);
    } else {
      StageArgs<T> sa;
      sa.mode = mode;
      sa.stage = stage;
      sa.X = (T*)D.X;
      sa.A = (T*)D.A;
      sa.Y = (T*)D.Y;
      sa.out = (T*)D.R;
      sa.dt = m->d_dt;
      sa.flag = m->d_flag;
      sa.uf_next = uf_next;
      sa.E = m->err_on ? (T*)D.E : nullptr;
      const T* uin = from_x ? (const T*)D.X : (const T*)D.Y;
      if (use_pri(m, D)) {
        dispatch(D.kind, m->order, [&](auto nu, auto nf) {
          constexpr int NU = decltype(nu)::value, NF = decltype(nf)::value;
          if constexpr (pri_order(NU, NF) > 0) {
            constexpr int E = dense_epb<NU>();
            const unsigned grid = unsigned(std::min<long long>(
                (D.ne + E - 1) / E,
                (long long)m->num_sms * (D.tile_vol > 0 ? D.tile_vol : D.pri_vol_ctas)));
            const size_t sm = pri_vol_smem<T, NU, NF>(D);
            if (ns)
              k_vol_pri<T, NU, NF, E, true><<<grid, E * NU, sm, s>>>(
                  D.ne, uin, (const T*)D.grad, fc, (const T*)D.smat, (const T*)D.rcpdjac,
                  pri_ops_of<T>(m, D), ph, sa);
            else
              k_vol_pri<T, NU, NF, E, false><<<grid, E * NU, sm, s>>>(
                  D.ne, uin, nullptr, fc, (const T*)D.smat, (const T*)D.rcpdjac,
                  pri_ops_of<T>(m, D), ph, sa);
          }
        });
      } else
      dispatch(D.kind, m->order, [&](auto nu, auto nf) {
        constexpr int NU = decltype(nu)::value, NF = decltype(nf)::value;
        constexpr int E = dense_epb<NU>();
        const size_t sm = dense_vol_smem<T, NU, NF>();
        const unsigned grid = unsigned(std::min<long long>(
            (D.ne + E - 1) / E,
            (long long)m->num_sms * (D.tile_vol > 0 ? D.tile_vol : D.vol_ctas)));
        if (aa)
          k_vol_dense<T, NU, NF, E, false, true><<<grid, E * NU, sm, s>>>(
              D.ne, uin, nullptr, fc, nullptr, (const T*)D.rcpdjac,
              stage_ops_of<T>(m, D), ph, sa, (const T*)D.tf);
        else if (ns)
          k_vol_dense<T, NU, NF, E, true><<<grid, E * NU, sm, s>>>(
              D.ne, uin, (const T*)D.grad, fc, (const T*)D.smat,
              (const T*)D.rcpdjac, stage_ops_of<T>(m, D), ph, sa);
        else
          k_vol_dense<T, NU, NF, E, false><<<grid, E * NU, sm, s>>>(
              D.ne, uin, nullptr, fc, (const T*)D.smat, (const T*)D.rcpdjac,
              stage_ops_of<T>(m, D), ph, sa);
      });
    }
    PROF_END(FR_KC_VOL);
    if (filt) {
      PROF_BEGIN(FR_KC_FILTER);
      launch_filter<T, TR>(m, s, D, last_stage);
      PROF_END(FR_KC_FILTER);
    }
  });
}

// layout conversion kernels: host layout [ne][nu][5] FP64 <-> [ne][5][nu] T
// host layout [ne][nu][5] of type S <-> register layout [ne][5][nu] of type T
template <typename S, typename T>
__global__ void k_layout_in(long long n, int nu, const S* __restrict__ src,
                            T* __restrict__ dst) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  long long e = i / (5 * nu);
  int r = int(i - e * 5 * nu);
  int k = r / nu, z = r - k * nu;
  dst[i] = T(src[(e * nu + z) * 5 + k]);
}

template <typename T, typename S>
__global__ void k_layout_out(long long n, int nu, const T* __restrict__ src,
                             S* __restrict__ dst) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  long long e = i / (5 * nu);
  int r = int(i - e * 5 * nu);
  int k = r / nu, z = r - k * nu;
  dst[(e * nu + z) * 5 + k] = S(src[i]);
}

DevType* type_ptr(fr_mesh* m, int etype) {
  if (m->host_only) return nullptr;
  if (etype < 0 || etype > 2 || m->type_of_kind[etype] < 0) return nullptr;
  return &m->types[m->type_of_kind[etype]];
}

const HostType* host_ptr(const fr_mesh* m, int etype) {
  if (etype < 0 || etype > 2 || m->type_of_kind[etype] < 0) return nullptr;
  return &m->host[m->type_of_kind[etype]];
}

template <typename TR, typename S = double>
int set_solution_dev(fr_mesh* m, DevType& D, const S* dsrc) {
  long long n = D.ne * 5 * D.nu;
  k_layout_in<S, TR><<<nblk(n, 256), 256, 0, m->stream>>>(n, D.nu, dsrc, (TR*)D.X);
  CK(cudaGetLastError());
  m->uf_valid = false;
  return FR_OK;
}

template <typename T, typename S = double>
int get_dev(fr_mesh* m, const DevType& D, const void* src, S* ddst) {
  long long n = D.ne * 5 * D.nu;
  k_layout_out<T, S><<<nblk(n, 256), 256, 0, m->stream>>>(n, D.nu, (const T*)src,
                                                          ddst);
  CK(cudaGetLastError());
  return FR_OK;
}

template <typename T, typename TR>
int ensure_uf(fr_mesh* m) {
  if (m->uf_valid) return FR_OK;
  launch_interp<T, TR>(m, m->stream);
  CK(cudaGetLastError());
  m->uf_valid = true;
  return FR_OK;
}

template <typename T, typename TR>
int resolve_variant(fr_mesh* m, int scheme, double dt);

template <typename T, typename TR>
int do_rhs(fr_mesh* m) {
  if (m->variant != FR_VARIANT_AUTO) {  // a fixed family; no tuning here
    int rv = resolve_variant<T, TR>(m, FR_RK4, 0.0);
    if (rv) return rv;
  }
  int rc = ensure_uf<T, TR>(m);
  if (rc) return rc;
  CK(cudaMemsetAsync(m->d_flag, 0, sizeof(int), m->stream));
  launch_stage<T, TR>(m, m->stream, 0, 0);
  CK(cudaGetLastError());
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, m->d_flag, sizeof(int), cudaMemcpyDeviceToHost,
                     m->stream));
  CK(cudaStreamSynchronize(m->stream));
  if (flag & 2) return fail(FR_ETIMEOUT, "a tensor-core wait timed out");
  if (flag) return fail(FR_ENONFINITE, "right-hand side is not finite");
  return FR_OK;
}

// ---------------------------------------------------------------- adaptive
constexpr int kAdaptive = 2;      // graph index of the adaptive RK45 step
constexpr int kErrBlocks = 256;   // partial sums per element type

// Sum of (e / (atol + rtol max(|x0|, |x1|)))^2 over n components, one
// partial sum per block (fixed grid and order: deterministic).  C is the
// arithmetic type of the scaled error (FP64 for FP64 values, else FP32).
template <typename TR, typename C>
__global__ void __launch_bounds__(256)
    k_err_partial(long long n, const TR* __restrict__ x0, const TR* __restrict__ x1,
                  const TR* __restrict__ e, const double* __restrict__ tol,
                  double* __restrict__ part) {
  __shared__ double red[8];
  const C atol = C(tol[0]), rtol = C(tol[1]);
  C acc = C(0);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const C sc = atol + rtol * fmax(fabs(C(x0[i])), fabs(C(x1[i])));
    const C q = C(e[i]) / sc;
    acc += q * q;
  }
  double v = double(acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

__global__ void k_err_final(int np, const double* __restrict__ part,
                            double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < np; ++i) t += part[i];
    out[0] = t;
  }
}

template <typename T, typename TR>
void launch_err_norm(fr_mesh* m, cudaStream_t s) {
  using C = typename std::conditional<sizeof(T) == 8, double, float>::type;
  int off = 0;
  for (auto& D : m->types) {
    const long long n = D.ne * 5 * D.nu;
    k_err_partial<TR, C><<<kErrBlocks, 256, 0, s>>>(n, (const TR*)D.Xs, (const TR*)D.X,
                                                    (const TR*)D.E, m->d_tol,
                                                    m->d_errpart + off);
    off += kErrBlocks;
  }
  k_err_final<<<1, 32, 0, s>>>(off, m->d_errpart, m->d_errsum);
}

template <typename T, typename TR>
int build_graph(fr_mesh* m, int scheme) {
  cudaStream_t s = m->stream;
  CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  if (scheme == kAdaptive) {
    // save u^n, five RK45 stages accumulating the embedded error, error norm
    for (auto& D : m->types)
      cudaMemcpyAsync(D.Xs, D.X, size_t(D.ne) * 5 * D.nu * sizeof(TR),
                      cudaMemcpyDeviceToDevice, s);
    m->err_on = true;
    for (int st = 0; st < 5; ++st) launch_stage<T, TR>(m, s, 2, st);
    m->err_on = false;
    launch_err_norm<T, TR>(m, s);
  } else {
    const int nst = scheme == FR_RK4 ? 4 : 5;
    for (int st = 0; st < nst; ++st)
      launch_stage<T, TR>(m, s, scheme == FR_RK4 ? 1 : 2, st);
  }
  cudaGraph_t g;
  cudaError_t e = cudaStreamEndCapture(s, &g);
  if (e != cudaSuccess)
    return fail(FR_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  if (m->graph[scheme]) cudaGraphExecDestroy(m->graph[scheme]);
  e = cudaGraphInstantiate(&m->graph[scheme], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess)
    return fail(FR_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  m->graph_stream[scheme] = s;
  m->graph_epoch[scheme] = m->epoch;
  return FR_OK;
}

// Kernel family for hexahedra: the requested one, or the autotuner's pick.
// The tuner runs one warm-up and one timed step of every applicable family
// from a saved copy of the solution registers, keeps the fastest and
// restores the registers (and the filter counters), so the caller's state is
// unchanged.
template <typename T, typename TR>
int resolve_variant(fr_mesh* m, int scheme, double dt) {
  bool has_hex = false, has_tc = false, curved = false, dense_aa_ok = true;
  for (auto& D : m->types) {
    has_hex |= D.kind == EK_HEX;
    has_tc |= D.tc_ok;
    curved |= D.curved;
    dense_aa_ok &= m->aa_qdeg == 0 || D.kind != EK_HEX || D.aa_dense;
  }
  // The vertex-metric family rebuilds trilinear metrics in the kernel: not
  // for curved (quadratic-map) hexahedra, whose metrics are the tables, nor
  // with anti-aliasing (the flux is then taken at the quadrature points).
  const bool vertex_ok = sizeof(T) == 4 && !curved && m->aa_qdeg == 0;
  if (m->variant != FR_VARIANT_AUTO) {
    int v = m->variant;
    if (v == FR_VARIANT_SUMFACT_VERTEX && !vertex_ok) v = FR_VARIANT_SUMFACT;
    if (v == FR_VARIANT_DENSE && !dense_aa_ok) v = FR_VARIANT_SUMFACT;
    if (v == FR_VARIANT_TENSOR && !has_tc) v = FR_VARIANT_SUMFACT;
    bool changed = v != m->active;
    for (auto& D : m->types) {  // a requested tensor family: every capable type
      changed |= !D.tc_grad_on || !D.tc_vol_on;
      D.tc_grad_on = D.tc_vol_on = true;
    }
    if (changed) {
      m->active = v;
      m->uf_valid = false;
      for (auto& D : m->types) D.tile_grad = D.tile_vol = 0;  // tiles of another family
      ++m->epoch;
    }
    return FR_OK;
  }
  if (m->tuned) return FR_OK;
  std::vector<int> cand = {FR_VARIANT_SUMFACT};
  if (has_hex && vertex_ok) cand.push_back(FR_VARIANT_SUMFACT_VERTEX);
  if (has_hex && m->precision != FR_MIXED && dense_aa_ok) cand.push_back(FR_VARIANT_DENSE);
  if (has_tc) cand.push_back(FR_VARIANT_TENSOR);
  std::vector<void*> saved;
  auto release = [&]() {
    for (void* p : saved)
      if (p) cudaFree(p);
  };
  for (auto& D : m->types) {
    void* p = nullptr;
    size_t bytes = size_t(D.ne) * 5 * D.nu * sizeof(TR);
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      release();
      return fail(FR_ENOMEM, "autotuner: no room for a state copy");
    }
    saved.push_back(p);
    cudaMemcpyAsync(p, D.X, bytes, cudaMemcpyDeviceToDevice, m->stream);
  }
  FilterStats st0{};
  if (m->d_fstats)
    cudaMemcpyAsync(&st0, m->d_fstats, sizeof(st0), cudaMemcpyDeviceToHost, m->stream);
  m->h_dt = dt;
  cudaMemcpyAsync(m->d_dt, &m->h_dt, sizeof(double), cudaMemcpyHostToDevice, m->stream);
  const int nst = scheme == FR_RK4 ? 4 : 5, mode = scheme == FR_RK4 ? 1 : 2;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const size_t nt = m->types.size();
  // per-type gradient and volume kernel times (ms) of one profiled step:
  // [2 t] gradient, [2 t + 1] volume
  std::vector<float> t_cc(2 * nt, 0.f), t_tc(2 * nt, 0.f);
  // One warm-up and one timed step of the active configuration from the
  // saved state; with `per_type`, a third step launched kernel by kernel
  // with events, its gradient and volume times summed per type.
  auto run = [&](std::vector<float>* per_type, float* ms) -> int {
    for (int rep = 0; rep < (per_type ? 3 : 2); ++rep) {
      for (size_t t = 0; t < nt; ++t)
        cudaMemcpyAsync(m->types[t].X, saved[t],
                        size_t(m->types[t].ne) * 5 * m->types[t].nu * sizeof(TR),
                        cudaMemcpyDeviceToDevice, m->stream);
      m->uf_valid = false;
      ensure_uf<T, TR>(m);
      Prof prof;
      if (rep == 1) cudaEventRecord(e0, m->stream);
      for (int s2 = 0; s2 < nst; ++s2)
        launch_stage<T, TR>(m, m->stream, mode, s2, rep == 2 ? &prof : nullptr);
      if (rep == 1) cudaEventRecord(e1, m->stream);
      cudaError_t err = cudaStreamSynchronize(m->stream);
      if (err != cudaSuccess)
        return fail(FR_ECUDA, std::string("autotuner: ") + cudaGetErrorString(err));
      if (rep == 1) cudaEventElapsedTime(ms, e0, e1);
      if (rep == 2) {
        // grad and volume launches come once per type per stage, in type order
        size_t ng = 0, nv = 0;
        for (size_t i = 0; i < prof.cls.size(); ++i) {
          float t = 0.f;
          cudaEventElapsedTime(&t, prof.ev[2 * i], prof.ev[2 * i + 1]);
          if (prof.cls[i] == FR_KC_GRAD) (*per_type)[2 * (ng++ % nt)] += t;
          if (prof.cls[i] == FR_KC_VOL) (*per_type)[2 * (nv++ % nt) + 1] += t;
        }
      }
      for (cudaEvent_t ev : prof.ev) cudaEventDestroy(ev);
    }
    return FR_OK;
  };
  float best = 1e30f;
  int pick = FR_VARIANT_SUMFACT;
  for (auto& D : m->types) D.tc_grad_on = D.tc_vol_on = true;
  for (int c : cand) {
    m->active = c;
    float ms = 0.f;
    std::vector<float>* pt = nullptr;
    if (has_tc && c == FR_VARIANT_SUMFACT) pt = &t_cc;
    if (c == FR_VARIANT_TENSOR) pt = &t_tc;
    if (int rr = run(pt, &ms)) {
      release();
      return rr;
    }
    m->tune_ms[c] = ms;
    if (ms < best) {
      best = ms;
      pick = c;
    }
  }
  if (has_tc) {
    // tensor cores only for the kernels (gradient, volume) of the types that
    // ran faster there; re-time the tensor family with that choice
    bool any = false, all = true;
    for (size_t t = 0; t < nt; ++t) {
      DevType& D = m->types[t];
      if (!D.tc_ok) continue;
      D.tc_grad_on = t_tc[2 * t] < t_cc[2 * t];
      D.tc_vol_on = t_tc[2 * t + 1] < t_cc[2 * t + 1];
      any |= D.tc_grad_on || D.tc_vol_on;
      all &= D.tc_grad_on && D.tc_vol_on;
    }
    if (!any) {
      if (pick == FR_VARIANT_TENSOR) {  // no type gains: best CUDA-core family
        best = 1e30f;
        for (int c : cand)
          if (c != FR_VARIANT_TENSOR && m->tune_ms[c] < best) {
            best = m->tune_ms[c];
            pick = c;
          }
      }
    } else if (!all) {
      m->active = FR_VARIANT_TENSOR;
      float ms = 0.f;
      if (int rr = run(nullptr, &ms)) {
        release();
        return rr;
      }
      m->tune_ms[FR_VARIANT_TENSOR] = ms;
      if (ms < best) {
        best = ms;
        pick = FR_VARIANT_TENSOR;
      }
    }
  }
  // Tiles and schedule of the picked family (Section 3.1, "Matrix
  // multiplications": kernel configurations benchmarked at run time, the
  // fastest kept): per type the elements per CTA of the hexahedron kernels
  // or the persistent CTAs per SM of the dense ones (timed per kernel from a
  // profiled step), then the interface kernels' block size and the parallel
  // per-type branches (timed per step).
  m->active = pick;
  {
    float ms = 0.f;
    if (int rr = run(nullptr, &ms)) {
      release();
      return rr;
    }
    m->sched_ms[0] = ms;
    std::vector<std::vector<int>> cg(nt), cv(nt);
    size_t nc = 1;
    for (size_t t = 0; t < nt; ++t) {
      DevType& D = m->types[t];
      const bool tcg = pick == FR_VARIANT_TENSOR && use_tc_grad(m, D);
      const bool tcv = pick == FR_VARIANT_TENSOR && use_tc_vol(m, D);
      cg[t] = tcg ? std::vector<int>{0} : tile_candidates(m, D, true);
      cv[t] = tcv ? std::vector<int>{0} : tile_candidates(m, D, false);
      nc = std::max({nc, cg[t].size(), cv[t].size()});
    }
    std::vector<float> bg(nt, 1e30f), bv(nt, 1e30f);
    std::vector<int> pg(nt, 0), pv(nt, 0);
    for (size_t i = 0; i < nc && nc > 1; ++i) {
      for (size_t t = 0; t < nt; ++t) {
        m->types[t].tile_grad = cg[t][std::min(i, cg[t].size() - 1)];
        m->types[t].tile_vol = cv[t][std::min(i, cv[t].size() - 1)];
      }
      std::vector<float> pt(2 * nt, 0.f);
      if (int rr = run(&pt, &ms)) {
        release();
        return rr;
      }
      for (size_t t = 0; t < nt; ++t) {
        if (pt[2 * t] < bg[t]) {
          bg[t] = pt[2 * t];
          pg[t] = m->types[t].tile_grad;
        }
        if (pt[2 * t + 1] < bv[t]) {
          bv[t] = pt[2 * t + 1];
          pv[t] = m->types[t].tile_vol;
        }
      }
    }
    for (size_t t = 0; t < nt; ++t) {
      m->types[t].tile_grad = nc > 1 ? pg[t] : 0;
      m->types[t].tile_vol = nc > 1 ? pv[t] : 0;
    }
    float bt = 1e30f;
    int btb = 256;
    for (int tb : {128, 256, 512}) {
      m->face_tb = tb;
      if (int rr = run(nullptr, &ms)) {
        release();
        return rr;
      }
      if (ms < bt) {
        bt = ms;
        btb = tb;
      }
    }
    m->face_tb = btb;
    if (nt > 1 && ensure_par(m) == FR_OK) {
      m->par_types = true;
      if (int rr = run(nullptr, &ms)) {
        release();
        return rr;
      }
      if (ms < bt)
        bt = ms;
      else
        m->par_types = false;
    }
    m->sched_ms[1] = bt;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (size_t t = 0; t < m->types.size(); ++t)
    cudaMemcpyAsync(m->types[t].X, saved[t],
                    size_t(m->types[t].ne) * 5 * m->types[t].nu * sizeof(TR),
                    cudaMemcpyDeviceToDevice, m->stream);
  if (m->d_fstats)
    cudaMemcpyAsync(m->d_fstats, &st0, sizeof(st0), cudaMemcpyHostToDevice, m->stream);
  CK(cudaStreamSynchronize(m->stream));
  release();
  m->active = pick;
  m->tuned = true;
  m->uf_valid = false;
  ++m->epoch;
  return FR_OK;
}

template <typename T, typename TR>
int do_rk(fr_mesh* m, int scheme, double dt, int nsteps) {
  int rc = resolve_variant<T, TR>(m, scheme, dt);
  if (rc) return rc;
  rc = ensure_uf<T, TR>(m);
  if (rc) return rc;
  if (!m->graph[scheme] || m->graph_stream[scheme] != m->stream ||
      m->graph_epoch[scheme] != m->epoch) {
    if ((rc = build_graph<T, TR>(m, scheme))) return rc;
  }
  m->h_dt = dt;
  CK(cudaMemcpyAsync(m->d_dt, &m->h_dt, sizeof(double), cudaMemcpyHostToDevice,
                     m->stream));
  CK(cudaMemsetAsync(m->d_flag, 0, sizeof(int), m->stream));
  for (int i = 0; i < nsteps; ++i) CK(cudaGraphLaunch(m->graph[scheme], m->stream));
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, m->d_flag, sizeof(int), cudaMemcpyDeviceToHost,
                     m->stream));
  CK(cudaStreamSynchronize(m->stream));
  if (flag & 2) return fail(FR_ETIMEOUT, "a tensor-core wait timed out");
  if (flag) return fail(FR_ENONFINITE, "a Runge-Kutta stage is not finite");
  return FR_OK;
}

// One attempted adaptive step (Section 3.5): the stages, the embedded error
// estimate and its norm run in kernels captured as one graph; acceptance,
// the restore of a rejected step and the PI step-size controller are host
// logic on the norm.
template <typename T, typename TR>
int do_rk_adaptive(fr_mesh* m, fr_adapt_t* ctl, double* dt, int* accepted, double* err) {
  if (m->filter_on)
    return fail(FR_EINVAL, "adaptive steps with the entropy filter are not supported");
  if (!(*dt > 0.0) || !(ctl->atol >= 0.0) || !(ctl->rtol >= 0.0) ||
      !(ctl->atol + ctl->rtol > 0.0) || !(ctl->err_prev > 0.0))
    return fail(FR_EINVAL, "adaptive step: dt, tolerances and err_prev must be positive");
  int rc = resolve_variant<T, TR>(m, FR_RK45, *dt);
  if (rc) return rc;
  if (!m->d_errsum) {
    for (auto& D : m->types) {
      const size_t bytes = size_t(D.ne) * 5 * D.nu * sizeof(TR);
      if ((rc = dev_zeros(m, bytes, &D.E))) return rc;
      if ((rc = dev_zeros(m, bytes, &D.Xs))) return rc;
    }
    m->n_errpart = kErrBlocks * int(m->types.size());
    void* p = nullptr;
    if ((rc = dev_zeros(m, size_t(m->n_errpart) * sizeof(double), &p))) return rc;
    m->d_errpart = (double*)p;
    if ((rc = dev_zeros(m, sizeof(double), &p))) return rc;
    m->d_errsum = (double*)p;
    if ((rc = dev_zeros(m, 2 * sizeof(double), &p))) return rc;
    m->d_tol = (double*)p;
  }
  rc = ensure_uf<T, TR>(m);
  if (rc) return rc;
  if (!m->graph[kAdaptive] || m->graph_stream[kAdaptive] != m->stream ||
      m->graph_epoch[kAdaptive] != m->epoch) {
    if ((rc = build_graph<T, TR>(m, kAdaptive))) return rc;
  }
  m->h_dt = *dt;
  m->h_tol[0] = ctl->atol;
  m->h_tol[1] = ctl->rtol;
  CK(cudaMemcpyAsync(m->d_dt, &m->h_dt, sizeof(double), cudaMemcpyHostToDevice, m->stream));
  CK(cudaMemcpyAsync(m->d_tol, m->h_tol, 2 * sizeof(double), cudaMemcpyHostToDevice,
                     m->stream));
  CK(cudaMemsetAsync(m->d_flag, 0, sizeof(int), m->stream));
  CK(cudaGraphLaunch(m->graph[kAdaptive], m->stream));
  int flag = 0;
  double sum = 0.0;
  CK(cudaMemcpyAsync(&flag, m->d_flag, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
  CK(cudaMemcpyAsync(&sum, m->d_errsum, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  CK(cudaStreamSynchronize(m->stream));
  if (flag & 2) return fail(FR_ETIMEOUT, "a tensor-core wait timed out");
  long long ncomp = 0;
  for (auto& D : m->types) ncomp += D.ne * 5 * D.nu;
  // a non-finite stage counts as a rejection
  const double e = flag ? INFINITY : std::sqrt(sum / double(ncomp));
  const bool ok = e <= 1.0;
  if (!ok) {  // restore u^n; its flux-point traces are recomputed on demand
    for (auto& D : m->types)
      CK(cudaMemcpyAsync(D.X, D.Xs, size_t(D.ne) * 5 * D.nu * sizeof(TR),
                         cudaMemcpyDeviceToDevice, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    m->uf_valid = false;
  }
  // PI controller: exponents 0.7/4 and 0.4/4 (the estimate is O(dt^4)),
  // safety 0.9, factors clipped to [0.2, 5], no growth right after a
  // rejection; a rejected step shrinks by max(0.2, 0.9 err^-1/4)
  double fac;
  if (ok) {
    fac = 0.9 * std::pow(std::max(e, 1e-10), -0.7 / 4.0) * std::pow(ctl->err_prev, 0.4 / 4.0);
    fac = std::min(std::max(fac, 0.2), 5.0);
    if (ctl->after_reject) fac = std::min(fac, 1.0);
    ctl->err_prev = std::max(e, 1e-4);
    ctl->after_reject = 0;
  } else {
    fac = std::max(0.2, 0.9 * std::pow(e, -0.25));
    ctl->after_reject = 1;
  }
  *dt *= fac;
  *accepted = ok ? 1 : 0;
  *err = e;
  return FR_OK;
}

template <typename T, typename TR>
int do_profile(fr_mesh* m, int scheme, double dt, double* ms, int* launches) {
  int rc = resolve_variant<T, TR>(m, scheme, dt);
  if (rc) return rc;
  rc = ensure_uf<T, TR>(m);
  if (rc) return rc;
  m->h_dt = dt;
  CK(cudaMemcpyAsync(m->d_dt, &m->h_dt, sizeof(double), cudaMemcpyHostToDevice,
                     m->stream));
  Prof prof;
  const int nst = scheme == FR_RK4 ? 4 : 5;
  for (int st = 0; st < nst; ++st)
    launch_stage<T, TR>(m, m->stream, scheme == FR_RK4 ? 1 : 2, st, &prof);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(m->stream));
  for (int k = 0; k < FR_KC_COUNT; ++k) {
    ms[k] = 0.0;
    launches[k] = 0;
  }
  for (size_t i = 0; i < prof.cls.size(); ++i) {
    float t = 0.f;
    cudaEventElapsedTime(&t, prof.ev[2 * i], prof.ev[2 * i + 1]);
    ms[prof.cls[i]] += t;
    launches[prof.cls[i]] += 1;
  }
  for (cudaEvent_t e : prof.ev) cudaEventDestroy(e);
  return FR_OK;
}

// Run fn<T, TR>(m) for the handle's precision.
// Device side of fr_set_antialias: release the previous buffers, then (for
// qdeg > 0) upload the transposed operators, the metric at the quadrature
// points and allocate the projected-flux buffer of every type.
void dev_release(fr_mesh* m, void** p) {
  if (!*p) return;
  cudaFree(*p);
  m->allocs.erase(std::remove(m->allocs.begin(), m->allocs.end(), *p), m->allocs.end());
  *p = nullptr;
}

template <typename T, typename TR>
int aa_setup(fr_mesh* m) {
  int rc;
  for (size_t t = 0; t < m->types.size(); ++t) {
    DevType& D = m->types[t];
    const HostType& H = m->host[t];
    for (void** p : {&D.aaBT, &D.aaPT, &D.aasmq, &D.tf}) dev_release(m, p);
    D.aa_nq = 0;
    if (m->aa_qdeg == 0) continue;
    const int nq = int(H.aa_w.size()), nu = D.nu;
    int smax = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    size_t need = 0;
    dispatch(D.kind, m->order, [&](auto nuc, auto) {
      need = aa_dense_smem<T, decltype(nuc)::value>(nq);
    });
    const int q1 = m->aa_qdeg / 2 + 1, n1 = m->order + 1;
    D.aa_hex = D.kind == EK_HEX && q1 <= kAaQMax && hex_aa_smem<T>(n1, q1) <= size_t(smax);
    D.aa_dense = need <= size_t(smax);
    if (need > size_t(smax) && !D.aa_hex) {
      m->aa_qdeg = 0;
      return fail(FR_EINVAL, "quadrature rule too large for the shared memory of a block");
    }
    if (D.aa_hex) {
      // 1D factors: Lagrange values of the solution points at the rule's
      // Gauss points, and the 1D least-squares projection back.
      std::vector<double> xg(q1), wg(q1);
      gauss_legendre(q1, xg.data(), wg.data());
      const std::vector<double>& xs = H.ref.x1;
      HexAaOps<double> o64{};
      HexAaOps<float> o32{};
      o64.q = o32.q = q1;
      for (int i = 0; i < q1; ++i)
        for (int a = 0; a < n1; ++a) {
          double l = 1.0;
          for (int k = 0; k < n1; ++k)
            if (k != a) l *= (xg[i] - xs[k]) / (xs[a] - xs[k]);
          double pr = 0.0;
          for (int mm = 0; mm < n1; ++mm)
            pr += jacobi_p(mm, 0.0, 0.0, xs[a]) * jacobi_p(mm, 0.0, 0.0, xg[i]);
          o64.b1[i][a] = l;
          o64.p1[a][i] = wg[i] * pr;
          o32.b1[i][a] = float(l);
          o32.p1[a][i] = float(wg[i] * pr);
        }
      D.hxaa64 = o64;
      D.hxaa32 = o32;
      hex_dispatch(m->order, [&](auto nc) {
        constexpr int N = decltype(nc)::value;
        const int sm = int(hex_aa_smem<T>(N, q1));
        // resident CTAs per SM of the variant that will run (rule size q1)
        int amin = 1 << 20;
        auto attr = [&](auto fn, bool used) {
          int a = 0;
          cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, fn, kAaThreads, sm);
          if (used) amin = std::min(amin, a);
        };
        const bool q_n1 = sizeof(T) == 4 && q1 == N + 1, q_n2 = sizeof(T) == 4 && q1 == N + 2;
        attr(k_hex_aa_flux<T, TR, N, 0, true>, !q_n1 && !q_n2);
        attr(k_hex_aa_flux<T, TR, N, 0, false>, !q_n1 && !q_n2);
        if constexpr (sizeof(T) == 4) {
          attr(k_hex_aa_flux<T, TR, N, N + 1, true>, q_n1);
          attr(k_hex_aa_flux<T, TR, N, N + 1, false>, q_n1);
          attr(k_hex_aa_flux<T, TR, N, N + 2, true>, q_n2);
          attr(k_hex_aa_flux<T, TR, N, N + 2, false>, q_n2);
        }
        D.aa_hex_ctas = amin > 0 && amin < (1 << 20) ? amin : 1;
      });
    }
    std::vector<double> bt(size_t(nu) * nq), pt(size_t(nq) * nu);
    for (int q = 0; q < nq; ++q)
      for (int z = 0; z < nu; ++z) {
        bt[size_t(z) * nq + q] = H.aa_B[size_t(q) * nu + z];
        pt[size_t(q) * nu + z] = H.aa_P[size_t(z) * nq + q];
      }
    std::vector<double> smq;
    metric_points(H, nq, H.aa_x.data(), smq);
    if ((rc = dev_upload<T>(m, bt, &D.aaBT))) return rc;
    if ((rc = dev_upload<T>(m, pt, &D.aaPT))) return rc;
    if ((rc = dev_upload<T>(m, smq, &D.aasmq))) return rc;
    if ((rc = dev_zeros(m, size_t(D.ne) * 15 * nu * sizeof(T), &D.tf))) return rc;
    D.aa_nq = nq;
    if (need <= size_t(smax)) dispatch(D.kind, m->order, [&](auto nuc, auto nfc) {
      constexpr int NU = decltype(nuc)::value;
      // vectorised form: several elements per pass (3 NU threads each in the
      // projection) while a block stays <= 110 KB (two or more per SM)
      int epb = std::max(1, std::min(8, (kAaVThreads + 3 * NU - 1) / (3 * NU)));
      while (epb > 1 && aa_dense_v_smem<T, NU>(nq, epb) > 110 * 1024) --epb;
      D.aa_epb = epb;
      D.aa_dv = aa_dense_v_smem<T, NU>(nq, epb) <= 110 * 1024;
      if (D.aa_dv) {
        const int smv = int(aa_dense_v_smem<T, NU>(nq, epb));
        int av = 1 << 20;
        for (auto fn : {k_aa_flux_dense_v<T, TR, NU, true>, k_aa_flux_dense_v<T, TR, NU, false>}) {
          int a1 = 0;
          cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smv);
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a1, fn, kAaVThreads, smv);
          av = std::min(av, a1);
        }
        D.aa_dv_ctas = av > 0 && av < (1 << 20) ? av : 1;
      }
      const int sm = int(aa_dense_smem<T, NU>(nq));
      int a = 0;
      for (auto fn : {k_aa_flux_dense<T, TR, NU, true>, k_aa_flux_dense<T, TR, NU, false>}) {
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, fn, kAaThreads, sm);
      }
      D.aa_ctas = a > 0 ? a : 1;
    });
  }
  CK(cudaGetLastError());
  return FR_OK;
}

}  // namespace

// ============================================================ partition groups
// Partitions of one mesh on one device, run together.  Every exchange point
// of a member is matched (by physical position, periodic translations
// included) with exactly one exchange point of another member; at each
// coupling point of a stage (solution traces before the common solution /
// fluxes; for NS also the gradient traces or the viscous normal fluxes
// before the common fluxes) every member pushes its traces into the
// partners' receive buffers, as a halo exchange between GPUs would.
struct fr_group {
  std::vector<fr_mesh*> m;
  struct Push {
    int32_t* code = nullptr;  // sender flux points
    int32_t* to = nullptr;    // receiving member
    int32_t* slot = nullptr;  // receiver's boundary-point index
    int n = 0;
  };
  std::vector<Push> push;
  void** d_xu = nullptr;  // members' xu pointers (device array)
  void** d_xg = nullptr;  // members' xg pointers
  std::vector<void*> allocs;
  // one captured step per scheme (RK4, RK45), valid for the members' epochs
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  std::vector<long long> graph_epoch[2];
  // one stream and event per member: the members' kernels of a phase are
  // captured as parallel branches between the exchange points
  std::vector<cudaStream_t> aux;
  std::vector<cudaEvent_t> ev;
  cudaEvent_t fork = nullptr;
  ~fr_group() {
    for (auto& ge : graph)
      if (ge) cudaGraphExecDestroy(ge);
    for (cudaStream_t st : aux)
      if (st) cudaStreamDestroy(st);
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
    if (fork) cudaEventDestroy(fork);
    for (void* p : allocs)
      if (p) cudaFree(p);
    for (fr_mesh* x : m) x->in_group = false;
  }
};

namespace {

struct CellHash {
  size_t operator()(const std::array<int64_t, 3>& k) const {
    uint64_t h = 1469598103934665603ull;
    for (int i = 0; i < 3; ++i) {
      h ^= uint64_t(k[i]);
      h *= 1099511628211ull;
    }
    return size_t(h);
  }
};

template <typename T, typename TR>
int group_run(fr_group* g, int mode, double dt, int nsteps) {
  fr_mesh* m0 = g->m[0];
  cudaStream_t s = m0->stream;
  for (fr_mesh* m : g->m) {
    CK(cudaStreamSynchronize(m->stream));
    if (m->variant != FR_VARIANT_AUTO) {
      int rv = resolve_variant<T, TR>(m, FR_RK4, 0.0);
      if (rv) return rv;
    } else {
      m->tuned = true;  // no tuning inside a group: the members' default family
    }
  }
  std::vector<cudaStream_t> own(g->m.size());
  for (size_t i = 0; i < g->m.size(); ++i) {
    own[i] = g->m[i]->stream;
    g->m[i]->stream = s;
  }
  auto restore = [&]() {
    for (size_t i = 0; i < g->m.size(); ++i) g->m[i]->stream = own[i];
  };
  const bool ns = m0->physics == FR_NAVIER_STOKES;
  const int nv2 = sizeof(T) == 4 ? 5 : 15;
  auto push = [&](int which) {
    for (size_t r = 0; r < g->m.size(); ++r) {
      const fr_group::Push& p = g->push[r];
      if (!p.n) continue;
      fr_mesh* m = g->m[r];
      k_exchange_push<T><<<nblk(p.n, 256), 256, 0, s>>>(
          p.n, p.code, p.to, p.slot, which == 0 ? (const T*)m->uf : (const T*)m->gradf,
          which == 0 ? 5 : nv2, reinterpret_cast<T* const*>(which == 0 ? g->d_xu : g->d_xg),
          m->tt);
    }
  };
  for (fr_mesh* m : g->m) {
    if (!m->uf_valid) {
      launch_interp<T, TR>(m, s);
      m->uf_valid = true;
    }
    m->h_dt = dt;
    cudaMemcpyAsync(m->d_dt, &m->h_dt, sizeof(double), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(m->d_flag, 0, sizeof(int), s);
  }
  const int nst = mode == 0 ? 1 : (mode == 1 ? 4 : 5);
  // members' launches of one phase on their own streams, joined back into s
  auto phase_all = [&](int st, int ph, bool par) {
    if (!par) {
      for (fr_mesh* m : g->m) launch_stage<T, TR>(m, s, mode, st, nullptr, ph);
      return;
    }
    cudaEventRecord(g->fork, s);
    for (size_t r = 0; r < g->m.size(); ++r) {
      cudaStreamWaitEvent(g->aux[r], g->fork, 0);
      launch_stage<T, TR>(g->m[r], g->aux[r], mode, st, nullptr, ph);
      cudaEventRecord(g->ev[r], g->aux[r]);
    }
    for (size_t r = 0; r < g->m.size(); ++r) cudaStreamWaitEvent(s, g->ev[r], 0);
  };
  auto one_step = [&](bool par) {
    for (int st = 0; st < nst; ++st) {
      push(0);
      if (ns) {
        phase_all(st, 1, par);
        push(1);
      }
      phase_all(st, 2, par);
    }
  };
  if (mode == 0) {
    one_step(false);
  } else {
    // RK steps replay one captured graph (rebuilt when a member's launch
    // configuration changed)
    const int gi = mode - 1;
    std::vector<long long> ep;
    for (fr_mesh* m : g->m) ep.push_back(m->epoch);
    if (!g->graph[gi] || g->graph_epoch[gi] != ep) {
      cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
      one_step(g->m.size() > 1);
      cudaGraph_t gr;
      cudaError_t ce = cudaStreamEndCapture(s, &gr);
      if (ce != cudaSuccess) {
        restore();
        return fail(FR_ECUDA, std::string("group graph capture: ") + cudaGetErrorString(ce));
      }
      if (g->graph[gi]) cudaGraphExecDestroy(g->graph[gi]);
      ce = cudaGraphInstantiate(&g->graph[gi], gr, 0);
      cudaGraphDestroy(gr);
      if (ce != cudaSuccess) {
        g->graph[gi] = nullptr;
        restore();
        return fail(FR_ECUDA, std::string("group graph instantiate: ") + cudaGetErrorString(ce));
      }
      g->graph_epoch[gi] = ep;
    }
    for (int it = 0; it < nsteps; ++it) cudaGraphLaunch(g->graph[gi], s);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    restore();
    return fail(FR_ECUDA, cudaGetErrorString(e));
  }
  int bad = 0;
  for (fr_mesh* m : g->m) {
    int flag = 0;
    cudaMemcpyAsync(&flag, m->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    bad |= flag;
  }
  restore();
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(FR_ECUDA, cudaGetErrorString(e));
  if (bad & 2) return fail(FR_ETIMEOUT, "a tensor-core wait timed out");
  if (bad) return fail(FR_ENONFINITE, "a partitioned stage is not finite");
  return FR_OK;
}

// ------------------------------------------------- exchange between processes
// One phase of one RK stage of a part whose partners live in other
// processes; the caller moves the traces between the phases
// (exchange_pack / exchange_unpack around its transport).  phase 1: NS
// common solution and gradients (nothing for Euler); phase 2: common
// fluxes, volume kernels and the stage's RK update.  part: 0 all, 1
// interior (no exchange point involved), 2 exchange-adjacent.
template <typename T, typename TR>
int do_stage(fr_mesh* m, int scheme, double dt, int stage, int phase, int part) {
  const int mode = scheme == FR_RK4 ? 1 : 2, nst = scheme == FR_RK4 ? 4 : 5;
  if (stage == 0 && phase == 1 && part <= 1) {
    if (m->variant != FR_VARIANT_AUTO) {
      int rv = resolve_variant<T, TR>(m, scheme, dt);
      if (rv) return rv;
    } else {
      m->tuned = true;  // no tuning of a part: every rank runs the default family
    }
    m->h_dt = dt;
    CK(cudaMemcpyAsync(m->d_dt, &m->h_dt, sizeof(double), cudaMemcpyHostToDevice, m->stream));
    CK(cudaMemsetAsync(m->d_flag, 0, sizeof(int), m->stream));
    int rc = ensure_uf<T, TR>(m);
    if (rc) return rc;
  }
  launch_stage<T, TR>(m, m->stream, mode, stage, nullptr, phase, part);
  CK(cudaGetLastError());
  if (stage == nst - 1 && phase == 2 && part != 1) {
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, m->d_flag, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    if (flag & 2) return fail(FR_ETIMEOUT, "a tensor-core wait timed out");
    if (flag) return fail(FR_ENONFINITE, "a stage of the part is not finite");
  }
  return FR_OK;
}

// what 0: solution traces (5 values per point); 1: gradient traces (15,
// FP64 values) or viscous normal fluxes (5, FP32 values).
template <typename T, typename TR>
int exchange_pack(fr_mesh* m, int what, void* buf) {
  if (what == 0) {
    int rc = ensure_uf<T, TR>(m);
    if (rc) return rc;
  }
  if (m->n_xlist == 0) return FR_OK;
  const int nv = what == 0 ? 5 : (sizeof(T) == 4 ? 5 : 15);
  k_exchange_gather<T><<<nblk(m->n_xlist, 256), 256, 0, m->stream>>>(
      int(m->n_xlist), m->x_list, m->bidx, what == 0 ? (const T*)m->uf : (const T*)m->gradf,
      nv, (T*)buf, m->tt);
  CK(cudaGetLastError());
  return FR_OK;
}

template <typename T, typename TR>
int exchange_unpack(fr_mesh* m, int what, const void* buf) {
  if (m->n_xlist == 0) return FR_OK;
  const int nv = what == 0 ? 5 : (sizeof(T) == 4 ? 5 : 15);
  k_exchange_scatter<T><<<nblk(m->n_xlist, 256), 256, 0, m->stream>>>(
      int(m->n_xlist), m->x_list, (const T*)buf, nv, what == 0 ? (T*)m->xu : (T*)m->xg);
  CK(cudaGetLastError());
  return FR_OK;
}

// Match every member's exchange points with their partners; fills the push
// lists and the partners' |S^T n~| (xm) of every member.
template <typename T, typename TR>
int group_setup(fr_group* g) {
  // Exchange points grouped by face: flux points on face edges of
  // simplices occur on two faces, so faces are matched first (by translated
  // centroid), then points within each matched face pair.
  struct XF {
    int r;
    std::vector<int> pt;  // boundary-point indices in member r
    double c[3];
  };
  std::vector<XF> fl;
  auto pos = [&](const fr_mesh* m, int i, double* x) {
    const int32_t code = m->conn.bidx[i];
    const HostType& H = m->host[code >> 29];
    const int64_t rem = code & ((int64_t(1) << 29) - 1);
    const int64_t e = rem / (5 * H.ref.nfpts);
    const int f = int(rem - e * 5 * H.ref.nfpts);
    for (int k = 0; k < 3; ++k) x[k] = H.fpts_x[(size_t(e) * H.ref.nfpts + f) * 3 + k];
    return std::array<int64_t, 3>{code >> 29, e, H.ref.fpts_face[f]};
  };
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (size_t r = 0; r < g->m.size(); ++r) {
    const fr_mesh* m = g->m[r];
    std::array<int64_t, 3> prev = {-1, -1, -1};
    for (size_t i = 0; i < m->conn.bidx.size(); ++i) {
      if (m->bc64.kind[m->conn.bbc[i]] != FR_BC_EXCHANGE) continue;
      double x[3];
      const std::array<int64_t, 3> face = pos(m, int(i), x);
      if (face != prev || fl.empty() || fl.back().r != int(r)) {
        fl.push_back(XF{int(r), {}, {0, 0, 0}});
        prev = face;
      }
      fl.back().pt.push_back(int(i));
      for (int k = 0; k < 3; ++k) {
        fl.back().c[k] += x[k];
        lo[k] = std::min(lo[k], x[k]);
        hi[k] = std::max(hi[k], x[k]);
      }
    }
  }
  for (XF& f : fl)
    for (int k = 0; k < 3; ++k) f.c[k] /= double(f.pt.size());
  double ext = 0.0;
  for (int k = 0; k < 3; ++k) ext = std::max(ext, hi[k] - lo[k]);
  const double tol = 1e-8 * std::max(ext, 1e-300), cell = 16.0 * tol;
  auto key = [&](const double* x, int dx, int dy, int dz) {
    return std::array<int64_t, 3>{int64_t(std::floor(x[0] / cell)) + dx,
                                  int64_t(std::floor(x[1] / cell)) + dy,
                                  int64_t(std::floor(x[2] / cell)) + dz};
  };
  std::unordered_multimap<std::array<int64_t, 3>, int, CellHash> grid;
  for (int j = 0; j < int(fl.size()); ++j) grid.emplace(key(fl[j].c, 0, 0, 0), j);
  // translations: sums of -1, 0 or +1 times each periodic vector
  const std::vector<double>& pv = g->m[0]->periodic;
  const int np = int(pv.size() / 3);
  std::vector<std::array<double, 3>> shifts;
  int ncomb = 1;
  for (int a = 0; a < np; ++a) ncomb *= 3;
  for (int c = 0; c < ncomb; ++c) {
    std::array<double, 3> sh = {0, 0, 0};
    int cc = c;
    for (int a = 0; a < np; ++a, cc /= 3)
      for (int k = 0; k < 3; ++k) sh[k] += double(cc % 3 - 1) * pv[3 * a + k];
    shifts.push_back(sh);
  }
  std::vector<std::vector<int32_t>> code(g->m.size()), to(g->m.size()), slot(g->m.size());
  std::vector<std::vector<double>> xm(g->m.size());
  for (size_t r = 0; r < g->m.size(); ++r) xm[r].assign(g->m[r]->conn.bidx.size(), 1.0);
  for (const XF& F : fl) {
    int found = -1, hits = 0;
    std::array<double, 3> fsh = {0, 0, 0};
    for (const auto& sh : shifts) {
      const double y[3] = {F.c[0] + sh[0], F.c[1] + sh[1], F.c[2] + sh[2]};
      for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dz = -1; dz <= 1; ++dz) {
            auto rng = grid.equal_range(key(y, dx, dy, dz));
            for (auto it = rng.first; it != rng.second; ++it) {
              const XF& G = fl[it->second];
              if (G.r == F.r || G.pt.size() != F.pt.size()) continue;
              double d2 = 0;
              for (int k = 0; k < 3; ++k) d2 += (G.c[k] - y[k]) * (G.c[k] - y[k]);
              if (d2 <= tol * tol) {
                found = it->second;
                fsh = sh;
                ++hits;
              }
            }
          }
    }
    if (hits != 1)
      return fail(FR_EMESH, hits ? "an exchange face matches several partners"
                                 : "an exchange face has no partner in the group");
    const XF& G = fl[found];
    const fr_mesh* ms = g->m[F.r];
    const fr_mesh* mr = g->m[G.r];
    std::vector<char> taken(G.pt.size(), 0);
    for (int i : F.pt) {
      double x[3], y[3];
      pos(ms, i, x);
      for (int k = 0; k < 3; ++k) x[k] += fsh[k];
      int best = -1;
      double bd = 1e300;
      for (size_t j = 0; j < G.pt.size(); ++j) {
        pos(mr, G.pt[j], y);
        double d2 = 0;
        for (int k = 0; k < 3; ++k) d2 += (x[k] - y[k]) * (x[k] - y[k]);
        if (d2 < bd) {
          bd = d2;
          best = int(j);
        }
      }
      if (best < 0 || bd > tol * tol || taken[best])
        return fail(FR_EMESH, "flux points do not conform across an exchange face");
      taken[best] = 1;
      const int q = G.pt[best];
      code[F.r].push_back(ms->conn.bidx[i]);  // F's point pushes to G's slot q
      to[F.r].push_back(G.r);
      slot[F.r].push_back(q);
      xm[G.r][q] = ms->conn.bn[4 * i + 3];    // q's partner magnitude
    }
  }
  g->push.resize(g->m.size());
  for (size_t r = 0; r < g->m.size(); ++r) {
    fr_mesh* m = g->m[r];
    fr_group::Push& p = g->push[r];
    p.n = int(code[r].size());
    if (p.n) {
      for (auto pr : {std::make_pair(&code[r], &p.code), std::make_pair(&to[r], &p.to),
                      std::make_pair(&slot[r], &p.slot)}) {
        CK(cudaMalloc((void**)pr.second, size_t(p.n) * sizeof(int32_t)));
        g->allocs.push_back(*pr.second);
        CK(cudaMemcpy(*pr.second, pr.first->data(), size_t(p.n) * sizeof(int32_t),
                      cudaMemcpyHostToDevice));
      }
    }
    if (m->xm) {
      std::vector<T> h(xm[r].begin(), xm[r].end());
      CK(cudaMemcpy(m->xm, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    }
  }
  std::vector<void*> xu(g->m.size()), xg(g->m.size());
  for (size_t r = 0; r < g->m.size(); ++r) {
    xu[r] = g->m[r]->xu;
    xg[r] = g->m[r]->xg;
  }
  for (auto pr : {std::make_pair(&xu, &g->d_xu), std::make_pair(&xg, &g->d_xg)}) {
    CK(cudaMalloc((void**)pr.second, g->m.size() * sizeof(void*)));
    g->allocs.push_back(*pr.second);
    CK(cudaMemcpy(*pr.second, pr.first->data(), g->m.size() * sizeof(void*),
                  cudaMemcpyHostToDevice));
  }
  return FR_OK;
}

}  // namespace
#include "fr_filter_impl.cuh"

namespace frgb {

// The precision-dependent entry points, one table per (T, TR): FP64
// (double, double), FP32 (float, float) and mixed (float values, double RK
// registers).  Each table is defined in its own translation unit
// (fr_prec_*.cu), so the three sets of kernels compile in parallel.
struct PrecTable {
  int (*setup_device)(fr_mesh*);
  int (*prepare_kernels)(fr_mesh*);
  int (*do_rhs)(fr_mesh*);
  int (*do_rk)(fr_mesh*, int, double, int);
  int (*do_rk_adaptive)(fr_mesh*, fr_adapt_t*, double*, int*, double*);
  int (*do_profile)(fr_mesh*, int, double, double*, int*);
  int (*aa_setup)(fr_mesh*);
  int (*group_setup)(fr_group*);
  int (*group_run)(fr_group*, int, double, int);
  int (*filter_solution)(fr_mesh*, const double*);
  int (*do_stage)(fr_mesh*, int, double, int, int, int);
  int (*exchange_pack)(fr_mesh*, int, void*);
  int (*exchange_unpack)(fr_mesh*, int, const void*);
};

extern const PrecTable kPrecF64, kPrecF32, kPrecMixed;

inline const PrecTable& prec_table(int precision) {
  return precision == FR_FP64 ? kPrecF64 : precision == FR_FP32 ? kPrecF32 : kPrecMixed;
}

}  // namespace frgb

#define FR_DEFINE_PREC_TABLE(name, T, TR)                                     \
  namespace frgb {                                                            \
  const PrecTable name = {&setup_device<T, TR>,   &prepare_kernels<T, TR>,    \
                          &do_rhs<T, TR>,         &do_rk<T, TR>,              \
                          &do_rk_adaptive<T, TR>, &do_profile<T, TR>,         \
                          &aa_setup<T, TR>,       &group_setup<T, TR>,        \
                          &group_run<T, TR>,      &filter_solution<T, TR>,    \
                          &do_stage<T, TR>,       &exchange_pack<T, TR>,      \
                          &exchange_unpack<T, TR>};                           \
  }


// C ABI of the FR library: argument checks, host set-up and the calls into
// the precision tables (fr_prec_*.cu).  See include/frgb.h.
#include "fr_impl.cuh"

#include <cmath>
#include <cstring>

using namespace frgb;

#define FR_PREC(m, fn, ...) (prec_table((m)->precision).fn(__VA_ARGS__))


// ===================================================================== ABI
extern "C" {

const char* fr_last_error(void) { return g_err.c_str(); }

int fr_mesh_create(const fr_mesh_desc* d, fr_mesh** out) {
  if (!d || !out) return fail(FR_EINVAL, "null argument");
  *out = nullptr;
  if (d->order < 1 || d->order > 4) return fail(FR_EINVAL, "order must be 1..4");
  if (d->physics != FR_EULER && d->physics != FR_NAVIER_STOKES)
    return fail(FR_EINVAL, "unknown physics");
  if (d->precision != FR_FP64 && d->precision != FR_FP32 &&
      d->precision != FR_MIXED)
    return fail(FR_EINVAL, "unknown precision");
  if (d->n_bcs < 0 || d->n_bcs > kMaxBC) return fail(FR_EINVAL, "too many boundary conditions");
  if (d->n_periodic < 0 || d->n_periodic > 3) return fail(FR_EINVAL, "n_periodic must be 0..3");
  if (d->n_nodes <= 0 || !d->nodes) return fail(FR_EINVAL, "no nodes");
  if (d->gamma <= 1.0) return fail(FR_EINVAL, "gamma must exceed 1");
  if (d->physics == FR_NAVIER_STOKES && (d->mu < 0 || d->prandtl <= 0))
    return fail(FR_EINVAL, "bad viscosity or Prandtl number");
  std::unique_ptr<fr_mesh> m(new fr_mesh());
  m->device = d->device;
  m->precision = d->precision;
  m->physics = d->physics;
  m->order = d->order;
  m->gamma = d->gamma;
  m->mu = d->mu;
  m->prandtl = d->prandtl > 0 ? d->prandtl : 0.72;
  m->wsize = d->precision == FR_FP64 ? 8 : 4;
  m->rsize = d->precision == FR_FP32 ? 4 : 8;
  MeshInput in;
  in.n_nodes = d->n_nodes;
  in.nodes = d->nodes;
  in.order = d->order;
  if (d->point_family != FR_POINTS_GL && d->point_family != FR_POINTS_GLL)
    return fail(FR_EINVAL, "unknown point family");
  in.family = d->point_family;
  bool seen[3] = {false, false, false};
  for (int i = 0; i < d->n_etypes; ++i) {
    const fr_etype_desc& t = d->etypes[i];
    if (t.etype < 0 || t.etype > 2 || seen[t.etype])
      return fail(FR_EINVAL, "bad or repeated element type");
    if (t.n_elem < 0 || (t.n_elem > 0 && !t.conn)) return fail(FR_EINVAL, "bad connectivity");
    if (t.map_order < 0 || t.map_order > 3)
      return fail(FR_EINVAL, "map order must be 0, 1, 2 or 3");
    if (t.map_order >= 2 && t.n_elem > 0 && !t.map_conn)
      return fail(FR_EINVAL, "curved maps need map_conn");
    seen[t.etype] = true;
    if (t.etype == FR_PRI6 && t.n_elem > 0 && d->point_family == FR_POINTS_GLL)
      return fail(FR_EINVAL, "Gauss-Lobatto hexahedra cannot meet prisms (their quad faces carry Gauss-Legendre points)");
  }
  for (int k = 0; k < 3; ++k)  // canonical type order: hex, prism, tet
    for (int i = 0; i < d->n_etypes; ++i)
      if (d->etypes[i].etype == k) {
        in.types.push_back({k, {d->etypes[i].n_elem, d->etypes[i].conn}});
        in.map_order.push_back(d->etypes[i].map_order >= 2 ? d->etypes[i].map_order : 1);
        in.map_conn.push_back(d->etypes[i].map_order >= 2 ? d->etypes[i].map_conn : nullptr);
      }
  for (int i = 0; i < d->n_periodic; ++i)
    in.periodic.push_back({d->periodic[i][0], d->periodic[i][1], d->periodic[i][2]});
  in.n_bfaces = d->n_bfaces;
  in.bface_nodes = d->bface_nodes;
  in.bface_tags = d->bface_tags;
  if (d->n_bfaces > 0 && (!d->bface_nodes || !d->bface_tags))
    return fail(FR_EINVAL, "boundary faces without nodes or tags");
  for (int i = 0; i < d->n_bcs; ++i) {
    const fr_bc_desc& b = d->bcs[i];
    if (b.kind != FR_BC_STATE && b.kind != FR_BC_EXTRAPOLATE && b.kind != FR_BC_EXCHANGE &&
        b.kind != FR_BC_PRESCRIBED)
      return fail(FR_EINVAL, "unknown boundary condition");
    m->has_presc |= b.kind == FR_BC_PRESCRIBED;
    in.bc_tags.push_back(b.tag);
    m->bc_tags.push_back(b.tag);
    double rho = b.state[0], u = b.state[1], v = b.state[2], w = b.state[3],
           p = b.state[4];
    double cons[5] = {rho, rho * u, rho * v, rho * w,
                      p / (d->gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)};
    m->bc64.kind[i] = b.kind;
    m->bc32.kind[i] = b.kind;
    for (int k = 0; k < 5; ++k) {
      m->bc64.state[i][k] = cons[k];
      m->bc32.state[i][k] = float(cons[k]);
    }
  }
  bool emesh = false;
  std::string err;
  try {
    err = build_mesh(in, m->host, m->conn, &emesh);
  } catch (const std::exception& ex) {
    return fail(FR_EINVAL, ex.what());
  }
  if (!err.empty()) return fail(emesh ? FR_EMESH : FR_EINVAL, err);
  for (auto& p : in.periodic) m->periodic.insert(m->periodic.end(), p.begin(), p.end());
  for (int32_t b : m->conn.bbc) m->has_exch |= m->bc64.kind[b] == FR_BC_EXCHANGE;
  {
    // exchange points last (a contiguous range the halo part of a stage
    // launches on its own), and per type the leading elements that own no
    // exchange point (the interior part of a stage)
    HostConn& C = m->conn;
    const size_t nb = C.bidx.size();
    std::vector<size_t> perm(nb);
    for (size_t i = 0; i < nb; ++i) perm[i] = i;
    std::stable_partition(perm.begin(), perm.end(), [&](size_t i) {
      return m->bc64.kind[C.bbc[i]] != FR_BC_EXCHANGE;
    });
    std::vector<int32_t> bi(nb), bb(nb);
    std::vector<double> bn(4 * nb);
    for (size_t k = 0; k < nb; ++k) {
      bi[k] = C.bidx[perm[k]];
      bb[k] = C.bbc[perm[k]];
      for (int c = 0; c < 4; ++c) bn[4 * k + c] = C.bn[4 * perm[k] + c];
    }
    C.bidx.swap(bi);
    C.bbc.swap(bb);
    C.bn.swap(bn);
    m->nb_x0 = 0;
    while (m->nb_x0 < (long long)nb && m->bc64.kind[C.bbc[m->nb_x0]] != FR_BC_EXCHANGE)
      ++m->nb_x0;
    m->n_int.assign(m->host.size(), 0);
    for (size_t t = 0; t < m->host.size(); ++t) m->n_int[t] = m->host[t].ne;
    for (long long i = m->nb_x0; i < (long long)nb; ++i) {
      const int32_t code = C.bidx[i];
      const int t = code >> 29;
      const long long e = (code & ((1 << 29) - 1)) / (5 * m->host[t].ref.nfpts);
      m->n_int[t] = std::min<long long>(m->n_int[t], e);
    }
  }
  if (d->device < 0) {  // host-only handle: geometry and operators, no GPU
    m->host_only = true;
    for (size_t t = 0; t < m->host.size(); ++t) m->type_of_kind[m->host[t].kind] = int(t);
    *out = m.release();
    return FR_OK;
  }
  CK(cudaSetDevice(d->device));
  CK(cudaStreamCreateWithFlags(&m->own_stream, cudaStreamNonBlocking));
  m->stream = m->own_stream;
  if (m->precision == FR_MIXED)
    for (auto& H : m->host)
      if (H.kind != EK_HEX)
        return fail(FR_EINVAL, "FR_MIXED supports hexahedral meshes only");
  int rc = FR_PREC(m, setup_device, m.get());
  if (rc) return rc;
  rc = FR_PREC(m, prepare_kernels, m.get());
  if (rc) return rc;
  if (m->has_exch || m->has_presc) {
    const size_t nb = m->conn.bidx.size();
    if ((rc = dev_zeros(m.get(), nb * 5 * m->wsize, &m->xu))) return rc;
  }
  if (m->has_exch) {
    const size_t nb = m->conn.bidx.size();
    if ((rc = dev_zeros(m.get(), nb * 15 * m->wsize, &m->xg))) return rc;
    if ((rc = dev_zeros(m.get(), nb * m->wsize, &m->xm))) return rc;
  }
  *out = m.release();
  return FR_OK;
}

int fr_mesh_destroy(fr_mesh* m) {
  if (!m) return FR_OK;
  if (m->in_group) return fail(FR_EINVAL, "the mesh belongs to a group: destroy the group first");
  if (!m->host_only) {
    cudaSetDevice(m->device);
    if (m->stream) cudaStreamSynchronize(m->stream);
  }
  delete m;
  return FR_OK;
}

int fr_get_info(const fr_mesh* m, int etype, int64_t* ne, int* nu, int* nf) {
  if (!m) return fail(FR_EINVAL, "null mesh");
  const HostType* H = host_ptr(m, etype);
  if (ne) *ne = H ? H->ne : 0;
  if (nu) *nu = H ? H->ref.nupts : 0;
  if (nf) *nf = H ? H->ref.nfpts : 0;
  return FR_OK;
}

int fr_get_points(const fr_mesh* m, int etype, double* xyz) {
  if (!m || !xyz) return fail(FR_EINVAL, "null argument");
  const HostType* H = host_ptr(m, etype);
  if (!H) return fail(FR_EINVAL, "mesh has no elements of this type");
  std::memcpy(xyz, H->upts_x.data(), H->upts_x.size() * sizeof(double));
  return FR_OK;
}

static int ensure_staging(fr_mesh* m, size_t bytes) {
  if (m->staging_bytes >= bytes) return FR_OK;
  if (m->d_staging) {
    cudaStreamSynchronize(m->stream);
    cudaFree(m->d_staging);
    m->d_staging = nullptr;
    m->staging_bytes = 0;
  }
  CK(cudaMalloc(&m->d_staging, bytes));
  m->staging_bytes = bytes;
  return FR_OK;
}

// Host solution in: one copy into a device staging buffer (host layout,
// FP64), then the layout kernel writes the element-major device register.
int fr_set_solution(fr_mesh* m, int etype, const double* u) {
  if (!m || !u) return fail(FR_EINVAL, "null argument");
  DevType* D = type_ptr(m, etype);
  if (!D) return fail(FR_EINVAL, "mesh has no elements of this type");
  CK(cudaSetDevice(m->device));
  size_t bytes = size_t(D->ne) * 5 * D->nu * sizeof(double);
  int rc = ensure_staging(m, bytes);
  if (rc) return rc;
  CK(cudaMemcpyAsync(m->d_staging, u, bytes, cudaMemcpyHostToDevice, m->stream));
  rc = m->rsize == 8
           ? set_solution_dev<double>(m, *D, (const double*)m->d_staging)
           : set_solution_dev<float>(m, *D, (const double*)m->d_staging);
  if (rc) return rc;
  CK(cudaStreamSynchronize(m->stream));
  return FR_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free solution upload.
//
// fr_set_solution stages the host array in a device buffer that it
// allocates with cudaMalloc on first use.  Some callers cannot allow that:
// an application whose device memory is reserved up front by its own pool
// allocator (a further cudaMalloc fails or escapes its accounting), or a
// time-stepping loop that must not pay the device-wide synchronisation that
// cudaMalloc / cudaFree can imply.  fr_set_solution_static runs the same
// copy and the same layout kernel, but stages through a fixed array that is
// part of the library image: kStaticStageDoubles FP64 values (16 MiB), held
// by every GPU that loads the library until the process exits.
constexpr size_t kStaticStageDoubles = size_t(1) << 21;
static __device__ __align__(256) double g_static_stage[kStaticStageDoubles];

// In host code `g_static_stage` names a host-side stand-in, not device
// memory; its device address is looked up once per device, with that device
// current, and cached here.
static double* g_static_stage_dev[64] = {nullptr};
static std::mutex g_static_stage_mu;

static int static_stage_address(int device, double** out) {
  if (device < 0 || device >= 64) return fail(FR_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_static_stage_mu);
  if (!g_static_stage_dev[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_stage);
    if (e != cudaSuccess || !p)
      return fail(FR_ECUDA, std::string("cudaGetSymbolAddress(static stage): ") +
                                cudaGetErrorString(e));
    g_static_stage_dev[device] = static_cast<double*>(p);
  }
  *out = g_static_stage_dev[device];
  return FR_OK;
}

int fr_set_solution_static(fr_mesh* m, int etype, const double* u) {
  if (!m || !u) return fail(FR_EINVAL, "null argument");
  DevType* D = type_ptr(m, etype);
  if (!D) return fail(FR_EINVAL, "mesh has no elements of this type");
  size_t n = size_t(D->ne) * 5 * D->nu;
  if (n > kStaticStageDoubles)
    return fail(FR_EINVAL, "solution of " + std::to_string(n) +
                               " values exceeds the static staging limit of " +
                               std::to_string(kStaticStageDoubles) +
                               " FP64 values; use fr_set_solution");
  CK(cudaSetDevice(m->device));
  double* stage = nullptr;
  int rc = static_stage_address(m->device, &stage);
  if (rc) return rc;
  CK(cudaMemcpyAsync(stage, u, n * sizeof(double), cudaMemcpyHostToDevice,
                     m->stream));
  rc = m->rsize == 8 ? set_solution_dev<double>(m, *D, stage)
                     : set_solution_dev<float>(m, *D, stage);
  if (rc) return rc;
  CK(cudaStreamSynchronize(m->stream));
  return FR_OK;
}

static int get_host(const fr_mesh* mc, int etype, double* out, bool rhs) {
  fr_mesh* m = const_cast<fr_mesh*>(mc);
  if (!m || !out) return fail(FR_EINVAL, "null argument");
  DevType* D = type_ptr(m, etype);
  if (!D) return fail(FR_EINVAL, "mesh has no elements of this type");
  CK(cudaSetDevice(m->device));
  size_t bytes = size_t(D->ne) * 5 * D->nu * sizeof(double);
  int rc = ensure_staging(m, bytes);
  if (rc) return rc;
  const void* src = rhs ? D->R : D->X;
  bool dbl = rhs ? m->wsize == 8 : m->rsize == 8;
  rc = dbl ? get_dev<double>(m, *D, src, (double*)m->d_staging)
           : get_dev<float>(m, *D, src, (double*)m->d_staging);
  if (rc) return rc;
  CK(cudaMemcpyAsync(out, m->d_staging, bytes, cudaMemcpyDeviceToHost, m->stream));
  CK(cudaStreamSynchronize(m->stream));
  return FR_OK;
}

int fr_get_solution(const fr_mesh* m, int etype, double* u) {
  return get_host(m, etype, u, false);
}

int fr_get_rhs(const fr_mesh* m, int etype, double* r) {
  return get_host(m, etype, r, true);
}

int fr_set_solution_device(fr_mesh* m, int etype, const void* dptr, int dtype) {
  if (!m || !dptr) return fail(FR_EINVAL, "null argument");
  if (dtype != FR_DTYPE_F64 && dtype != FR_DTYPE_F32) return fail(FR_EINVAL, "unknown dtype");
  DevType* D = type_ptr(m, etype);
  if (!D) return fail(FR_EINVAL, "mesh has no elements of this type");
  CK(cudaSetDevice(m->device));
  if (dtype == FR_DTYPE_F64)
    return m->rsize == 8 ? set_solution_dev<double>(m, *D, (const double*)dptr)
                         : set_solution_dev<float>(m, *D, (const double*)dptr);
  return m->rsize == 8 ? set_solution_dev<double, float>(m, *D, (const float*)dptr)
                       : set_solution_dev<float, float>(m, *D, (const float*)dptr);
}

int fr_get_solution_device(const fr_mesh* mc, int etype, void* dptr, int dtype) {
  fr_mesh* m = const_cast<fr_mesh*>(mc);
  if (!m || !dptr) return fail(FR_EINVAL, "null argument");
  if (dtype != FR_DTYPE_F64 && dtype != FR_DTYPE_F32) return fail(FR_EINVAL, "unknown dtype");
  DevType* D = type_ptr(m, etype);
  if (!D) return fail(FR_EINVAL, "mesh has no elements of this type");
  CK(cudaSetDevice(m->device));
  if (dtype == FR_DTYPE_F64)
    return m->rsize == 8 ? get_dev<double>(m, *D, D->X, (double*)dptr)
                         : get_dev<float>(m, *D, D->X, (double*)dptr);
  return m->rsize == 8 ? get_dev<double, float>(m, *D, D->X, (float*)dptr)
                       : get_dev<float, float>(m, *D, D->X, (float*)dptr);
}

}  // extern "C"

namespace {

// Device time of the timed calls: a pair of events around each, kept in a
// ring and folded into ms_device once the second event has completed (the
// oldest pair is waited for only when the ring is full).  Nothing is
// recorded on a stream that is being captured into a graph.
bool stats_capturing(fr_mesh* m) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(m->stream, &cs) != cudaSuccess ||
         cs != cudaStreamCaptureStatusNone;
}

int stats_harvest(fr_mesh* m, bool wait_all) {
  while (m->ev_count > 0) {
    int i = (m->ev_head - m->ev_count + fr_mesh::kEvRing) % fr_mesh::kEvRing;
    if (!wait_all && m->ev_count < fr_mesh::kEvRing) {
      cudaError_t q = cudaEventQuery(m->ev_b[i]);
      if (q == cudaErrorNotReady) break;
      CK(q);
    } else {
      CK(cudaEventSynchronize(m->ev_b[i]));
    }
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, m->ev_a[i], m->ev_b[i]));
    m->ms_device += ms;
    --m->ev_count;
  }
  return FR_OK;
}

// Records the opening event of a timed call; returns the ring slot or -1.
int stats_begin(fr_mesh* m) {
  if (stats_capturing(m)) return -1;
  if (stats_harvest(m, false)) return -1;
  if (m->ev_count == fr_mesh::kEvRing && stats_harvest(m, false)) return -1;
  int i = m->ev_head;
  if (!m->ev_a[i] && (cudaEventCreate(&m->ev_a[i]) != cudaSuccess ||
                      cudaEventCreate(&m->ev_b[i]) != cudaSuccess))
    return -1;
  if (cudaEventRecord(m->ev_a[i], m->stream) != cudaSuccess) return -1;
  return i;
}

void stats_end(fr_mesh* m, int slot) {
  if (slot < 0) return;
  if (cudaEventRecord(m->ev_b[slot], m->stream) != cudaSuccess) return;
  m->ev_head = (m->ev_head + 1) % fr_mesh::kEvRing;
  ++m->ev_count;
}

int stages_of(int scheme) { return scheme == FR_RK4 ? 4 : 5; }

// Every FR_BC_PRESCRIBED condition must have its states (fr_set_bc_state).
int bc_ready(const fr_mesh* m) {
  if (!m->has_presc) return FR_OK;
  for (size_t b = 0; b < m->bc_tags.size(); ++b)
    if (m->bc64.kind[b] == FR_BC_PRESCRIBED && (b >= m->presc_set.size() || !m->presc_set[b]))
      return fail(FR_EINVAL, "a prescribed boundary condition has no state: call fr_set_bc_state");
  return FR_OK;
}

}  // namespace

extern "C" {

int fr_rhs(fr_mesh* m, double t, double* rhs_host, void* rhs_dev) {
  if (!m) return fail(FR_EINVAL, "null mesh");
  if (int rb = bc_ready(m)) return rb;
  if (m->host_only) return fail(FR_EINVAL, "host-only handle (device < 0)");
  if (m->has_exch) return fail(FR_EINVAL, "mesh has exchange faces: run it in a group");
  if (!std::isfinite(t)) return fail(FR_EINVAL, "time is not finite");
  CK(cudaSetDevice(m->device));
  int slot = stats_begin(m);
  int rc = FR_PREC(m, do_rhs, m);
  stats_end(m, slot);
  if (rc) return rc;
  m->t_last = t;
  ++m->n_rhs;
  ++m->n_stages;
  if (!rhs_host && !rhs_dev) return FR_OK;
  size_t total = 0;
  for (auto& D : m->types) total += size_t(D.ne) * 5 * D.nu;
  // device output, then host output through the staging buffer; both in
  // the host layout, element types in mesh order
  double* outs[2] = {static_cast<double*>(rhs_dev), nullptr};
  if (rhs_host) {
    rc = ensure_staging(m, total * sizeof(double));
    if (rc) return rc;
    outs[1] = static_cast<double*>(m->d_staging);
  }
  for (double* base : outs) {
    if (!base) continue;
    size_t off = 0;
    for (auto& D : m->types) {
      rc = m->wsize == 8 ? get_dev<double>(m, D, D.R, base + off)
                         : get_dev<float>(m, D, D.R, base + off);
      if (rc) return rc;
      off += size_t(D.ne) * 5 * D.nu;
    }
  }
  if (rhs_host) {
    CK(cudaMemcpyAsync(rhs_host, m->d_staging, total * sizeof(double),
                       cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
  }
  return FR_OK;
}

int fr_rk_step(fr_mesh* m, int scheme, double dt, int nsteps) {
  if (!m) return fail(FR_EINVAL, "null mesh");
  if (int rb = bc_ready(m)) return rb;
  if (m->host_only) return fail(FR_EINVAL, "host-only handle (device < 0)");
  if (scheme != FR_RK4 && scheme != FR_RK45) return fail(FR_EINVAL, "unknown scheme");
  if (nsteps < 0) return fail(FR_EINVAL, "negative step count");
  if (m->has_exch) return fail(FR_EINVAL, "mesh has exchange faces: run it in a group");
  if (nsteps == 0) return FR_OK;
  CK(cudaSetDevice(m->device));
  int slot = stats_begin(m);
  int rc = FR_PREC(m, do_rk, m, scheme, dt, nsteps);
  stats_end(m, slot);
  if (rc) return rc;
  m->n_steps += (unsigned long long)nsteps;
  m->n_stages += (unsigned long long)nsteps * stages_of(scheme);
  return FR_OK;
}

int fr_rk_adaptive_step(fr_mesh* m, fr_adapt_t* ctl, double* dt, int* accepted,
                        double* err) {
  if (!m || !ctl || !dt || !accepted || !err) return fail(FR_EINVAL, "null argument");
  if (int rb = bc_ready(m)) return rb;
  if (m->host_only) return fail(FR_EINVAL, "host-only handle (device < 0)");
  if (m->has_exch) return fail(FR_EINVAL, "mesh has exchange faces: run it in a group");
  CK(cudaSetDevice(m->device));
  int slot = stats_begin(m);
  int rc = FR_PREC(m, do_rk_adaptive, m, ctl, dt, accepted, err);
  stats_end(m, slot);
  if (rc) return rc;
  ++m->n_attempts;
  m->n_rejected += *accepted ? 0 : 1;
  m->n_stages += 5;
  return FR_OK;
}

int fr_profile_step(fr_mesh* m, int scheme, double dt, double* ms,
                    int* launches) {
  if (!m || !ms || !launches) return fail(FR_EINVAL, "null argument");
  if (int rb = bc_ready(m)) return rb;
  if (m->host_only) return fail(FR_EINVAL, "host-only handle (device < 0)");
  if (m->has_exch) return fail(FR_EINVAL, "mesh has exchange faces: run it in a group");
  if (scheme != FR_RK4 && scheme != FR_RK45) return fail(FR_EINVAL, "unknown scheme");
  CK(cudaSetDevice(m->device));
  int rc = FR_PREC(m, do_profile, m, scheme, dt, ms, launches);
  if (rc) return rc;
  for (int k = 0; k < FR_KC_COUNT; ++k) {
    m->prof_ms[k] = ms[k];
    m->prof_launches[k] = launches[k];
  }
  m->n_steps += 1;
  m->n_stages += stages_of(scheme);
  return FR_OK;
}

int fr_stats(fr_mesh* m, fr_stats_t* out, int reset) {
  if (!m || !out) return fail(FR_EINVAL, "null argument");
  std::memset(out, 0, sizeof(*out));
  if (!m->host_only) {
    CK(cudaSetDevice(m->device));
    int rc = stats_harvest(m, true);
    if (rc) return rc;
    if (m->d_fstats) {
      FilterStats st;
      CK(cudaMemcpyAsync(&st, m->d_fstats, sizeof(st), cudaMemcpyDeviceToHost, m->stream));
      CK(cudaStreamSynchronize(m->stream));
      out->filtered = st.filtered;
      out->filter_evals = st.evals;
      out->filter_fallbacks = st.fallbacks;
      out->predictor_used = st.guessed;
      if (reset) {
        CK(cudaMemsetAsync(m->d_fstats, 0, sizeof(FilterStats), m->stream));
        CK(cudaStreamSynchronize(m->stream));
      }
    }
  }
  out->rhs_calls = m->n_rhs;
  out->rk_steps = m->n_steps;
  out->rk_attempts = m->n_attempts;
  out->rk_rejected = m->n_rejected;
  out->stages = m->n_stages;
  out->ms_device = m->ms_device;
  for (int k = 0; k < FR_KC_COUNT; ++k) {
    out->ms_kernel[k] = m->prof_ms[k];
    out->launches[k] = m->prof_launches[k];
  }
  out->kernel_family = m->active;
  out->t_last = m->t_last;
  if (reset) {
    m->n_rhs = m->n_steps = m->n_attempts = m->n_rejected = m->n_stages = 0;
    m->ms_device = 0.0;
  }
  return FR_OK;
}

int fr_set_kernel_variant(fr_mesh* m, int variant) {
  if (!m) return fail(FR_EINVAL, "null mesh");
  if (variant != FR_VARIANT_AUTO && variant != FR_VARIANT_DENSE &&
      variant != FR_VARIANT_SUMFACT && variant != FR_VARIANT_SUMFACT_VERTEX &&
      variant != FR_VARIANT_TENSOR)
    return fail(FR_EINVAL, "unknown kernel variant");
  if (variant == FR_VARIANT_DENSE && m->precision == FR_MIXED)
    return fail(FR_EINVAL, "FR_MIXED runs the sum-factorised kernels only");
  m->variant = variant;
  m->tuned = false;
  ++m->epoch;
  return FR_OK;
}

int fr_get_tuning(const fr_mesh* m, int* active, float* ms) {
  if (!m) return fail(FR_EINVAL, "null mesh");
  if (active) *active = m->active;
  if (ms)
    for (int i = 0; i < 5; ++i) ms[i] = m->tune_ms[i];
  return FR_OK;
}

}  // extern "C"

namespace {

// Exchange faces of a part in boundary-point order: consecutive exchange
// points of one (type, element, face) form a face.
struct XFace {
  std::vector<int32_t> pt;  // own boundary-point indices
  double c[3] = {0, 0, 0};  // centroid of the face's points
};

std::vector<XFace> exchange_faces_of(const fr_mesh* m) {
  std::vector<XFace> fl;
  std::array<int64_t, 3> prev = {-1, -1, -1};
  for (long long i = m->nb_x0; i < (long long)m->conn.bidx.size(); ++i) {
    const int32_t code = m->conn.bidx[i];
    const HostType& H = m->host[code >> 29];
    const int64_t rem = code & ((int64_t(1) << 29) - 1);
    const int64_t e = rem / (5 * H.ref.nfpts);
    const int f = int(rem - e * 5 * H.ref.nfpts);
    const std::array<int64_t, 3> key = {code >> 29, e, H.ref.fpts_face[f]};
    if (key != prev || fl.empty()) {
      fl.push_back(XFace{});
      prev = key;
    }
    fl.back().pt.push_back(int32_t(i));
    for (int k = 0; k < 3; ++k)
      fl.back().c[k] += H.fpts_x[(size_t(e) * H.ref.nfpts + f) * 3 + k];
  }
  for (XFace& F : fl)
    for (int k = 0; k < 3; ++k) F.c[k] /= double(F.pt.size());
  return fl;
}

const double* bpt_x(const fr_mesh* m, int32_t i) {
  const int32_t code = m->conn.bidx[i];
  const HostType& H = m->host[code >> 29];
  const int64_t rem = code & ((int64_t(1) << 29) - 1);
  const int64_t e = rem / (5 * H.ref.nfpts);
  const int f = int(rem - e * 5 * H.ref.nfpts);
  return &H.fpts_x[(size_t(e) * H.ref.nfpts + f) * 3];
}

}  // namespace

extern "C" {

int fr_set_bc_state(fr_mesh* m, int tag, fr_bc_fn fn, double t, void* ctx) {
  if (!m || !fn) return fail(FR_EINVAL, "null argument");
  if (m->host_only) return fail(FR_EINVAL, "host-only handle (device < 0)");
  int b = -1;
  for (size_t i = 0; i < m->bc_tags.size(); ++i)
    if (m->bc_tags[i] == tag) b = int(i);
  if (b < 0 || m->bc64.kind[b] != FR_BC_PRESCRIBED)
    return fail(FR_EINVAL, "no prescribed boundary condition with this tag");
  std::vector<int32_t> slot;
  std::vector<double> x;
  for (size_t i = 0; i < m->conn.bidx.size(); ++i) {
    if (m->conn.bbc[i] != b) continue;
    slot.push_back(int32_t(i));
    const double* p = bpt_x(m, int32_t(i));
    x.insert(x.end(), p, p + 3);
  }
  const size_t n = slot.size();
  std::vector<double> prim(5 * n, 0.0), cons(5 * n);
  if (n) fn(int64_t(n), x.data(), t, prim.data(), ctx);
  for (size_t q = 0; q < n; ++q) {
    const double* w = &prim[5 * q];
    if (!(w[0] > 0.0) || !(w[4] > 0.0) || !std::isfinite(w[1]) || !std::isfinite(w[2]) ||
        !std::isfinite(w[3]))
      return fail(FR_EINVAL, "prescribed state with non-positive density or pressure");
    cons[5 * q] = w[0];
    for (int k = 0; k < 3; ++k) cons[5 * q + 1 + k] = w[0] * w[1 + k];
    cons[5 * q + 4] = w[4] / (m->gamma - 1.0) +
                      0.5 * w[0] * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]);
  }
  CK(cudaSetDevice(m->device));
  if (n) {
    void *dv = nullptr, *ds = nullptr;
    CK(cudaMalloc(&dv, 5 * n * m->wsize));
    cudaError_t e = cudaMalloc(&ds, n * sizeof(int32_t));
    if (e == cudaSuccess) {
      if (m->wsize == 8) {
        e = cudaMemcpy(dv, cons.data(), 5 * n * 8, cudaMemcpyHostToDevice);
      } else {
        std::vector<float> c32(cons.begin(), cons.end());
        e = cudaMemcpy(dv, c32.data(), 5 * n * 4, cudaMemcpyHostToDevice);
      }
    }
    if (e == cudaSuccess) e = cudaMemcpy(ds, slot.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
      CK(cudaStreamSynchronize(m->stream));
      if (m->wsize == 8)
        k_exchange_scatter<double><<<nblk((long long)n, 256), 256, 0, m->stream>>>(
            int(n), (const int32_t*)ds, (const double*)dv, 5, (double*)m->xu);
      else
        k_exchange_scatter<float><<<nblk((long long)n, 256), 256, 0, m->stream>>>(
            int(n), (const int32_t*)ds, (const float*)dv, 5, (float*)m->xu);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    }
    cudaFree(dv);
    cudaFree(ds);
    if (e != cudaSuccess) return fail(FR_ECUDA, std::string("fr_set_bc_state: ") + cudaGetErrorString(e));
  }
  if (m->presc_set.size() < m->bc_tags.size()) m->presc_set.resize(m->bc_tags.size(), 0);
  m->presc_set[b] = 1;
  return FR_OK;
}

int fr_exchange_faces(const fr_mesh* m, int64_t* n_faces, int64_t* n_points,
                      int32_t* face_npts, double* centroids, double* pt_x,
                      double* pt_mag) {
  if (!m || !n_faces || !n_points) return fail(FR_EINVAL, "null argument");
  const std::vector<XFace> fl = exchange_faces_of(m);
  *n_faces = int64_t(fl.size());
  int64_t np = 0;
  for (const XFace& F : fl) np += int64_t(F.pt.size());
  *n_points = np;
  int64_t q = 0;
  for (size_t j = 0; j < fl.size(); ++j) {
    if (face_npts) face_npts[j] = int32_t(fl[j].pt.size());
    if (centroids)
      for (int k = 0; k < 3; ++k) centroids[3 * j + k] = fl[j].c[k];
    for (int32_t i : fl[j].pt) {
      const double* x = bpt_x(m, i);
      if (pt_x)
        for (int k = 0; k < 3; ++k) pt_x[3 * q + k] = x[k];
      if (pt_mag) pt_mag[q] = m->conn.bn[4 * size_t(i) + 3];
      ++q;
    }
  }
  return FR_OK;
}

int fr_exchange_setup(fr_mesh* m, int rank, int nranks, const int64_t* faces_per_rank,
                      const int64_t* points_per_rank, const int32_t* face_npts,
                      const double* centroids, const double* pt_x,
                      const double* pt_mag, int64_t* counts) {
  if (!m || !faces_per_rank || !points_per_rank || !counts)
    return fail(FR_EINVAL, "null argument");
  if (nranks < 1 || rank < 0 || rank >= nranks) return fail(FR_EINVAL, "bad rank");
  if (m->in_group) return fail(FR_EINVAL, "the mesh belongs to a group");
  // other ranks' faces: (rank, first point, point count, centroid)
  struct RF {
    int r;
    int64_t p0, np;
    const double* c;
  };
  std::vector<RF> rf;
  std::vector<int64_t> pbase(nranks + 1, 0);
  int64_t fo = 0;
  for (int r = 0; r < nranks; ++r) {
    if (faces_per_rank[r] < 0 || points_per_rank[r] < 0) return fail(FR_EINVAL, "negative count");
    pbase[r + 1] = pbase[r] + points_per_rank[r];
    int64_t po = pbase[r];
    for (int64_t j = 0; j < faces_per_rank[r]; ++j, ++fo) {
      if (r != rank) rf.push_back(RF{r, po, face_npts[fo], centroids + 3 * fo});
      po += face_npts[fo];
    }
    if (po != pbase[r + 1]) return fail(FR_EINVAL, "face point counts do not add up");
  }
  const std::vector<XFace> own = exchange_faces_of(m);
  {
    int64_t np = 0;
    for (const XFace& F : own) np += int64_t(F.pt.size());
    if (faces_per_rank[rank] != int64_t(own.size()) || points_per_rank[rank] != np)
      return fail(FR_EINVAL, "this rank's entries differ from fr_exchange_faces");
  }
  // grid of the other ranks' face centroids
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t q = 0; q < pbase[nranks]; ++q)
    for (int k = 0; k < 3; ++k) {
      lo[k] = std::min(lo[k], pt_x[3 * q + k]);
      hi[k] = std::max(hi[k], pt_x[3 * q + k]);
    }
  double ext = 0.0;
  for (int k = 0; k < 3; ++k) ext = std::max(ext, hi[k] - lo[k]);
  const double tol = 1e-8 * std::max(ext, 1e-300), cell = 16.0 * tol;
  auto key = [&](const double* x, int dx, int dy, int dz) {
    return std::array<int64_t, 3>{int64_t(std::floor(x[0] / cell)) + dx,
                                  int64_t(std::floor(x[1] / cell)) + dy,
                                  int64_t(std::floor(x[2] / cell)) + dz};
  };
  std::unordered_multimap<std::array<int64_t, 3>, int, CellHash> grid;
  for (int j = 0; j < int(rf.size()); ++j) grid.emplace(key(rf[j].c, 0, 0, 0), j);
  const int np = int(m->periodic.size() / 3);
  std::vector<std::array<double, 3>> shifts;
  int ncomb = 1;
  for (int a = 0; a < np; ++a) ncomb *= 3;
  for (int c = 0; c < ncomb; ++c) {
    std::array<double, 3> sh = {0, 0, 0};
    int cc = c;
    for (int a = 0; a < np; ++a, cc /= 3)
      for (int k = 0; k < 3; ++k) sh[k] += double(cc % 3 - 1) * m->periodic[3 * a + k];
    shifts.push_back(sh);
  }
  // pairs: (partner rank, canonical key, own boundary point, partner |S^T n~|)
  struct PairX {
    int r;
    int64_t key;
    int32_t own;
    double mag;
  };
  std::vector<PairX> pairs;
  int64_t own_idx = 0;  // own exchange index (position in fr_exchange_faces order)
  for (const XFace& F : own) {
    int found = -1, hits = 0;
    std::array<double, 3> fsh = {0, 0, 0};
    for (const auto& sh : shifts) {
      const double y[3] = {F.c[0] + sh[0], F.c[1] + sh[1], F.c[2] + sh[2]};
      for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dz = -1; dz <= 1; ++dz) {
            auto rg = grid.equal_range(key(y, dx, dy, dz));
            for (auto it = rg.first; it != rg.second; ++it) {
              const RF& G = rf[it->second];
              if (G.np != int64_t(F.pt.size())) continue;
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
                                 : "an exchange face has no partner among the ranks");
    const RF& G = rf[found];
    std::vector<char> taken(size_t(G.np), 0);
    for (size_t a = 0; a < F.pt.size(); ++a, ++own_idx) {
      const double* x0 = bpt_x(m, F.pt[a]);
      const double x[3] = {x0[0] + fsh[0], x0[1] + fsh[1], x0[2] + fsh[2]};
      int64_t best = -1;
      double bd = 1e300;
      for (int64_t j = 0; j < G.np; ++j) {
        const double* y = pt_x + 3 * (G.p0 + j);
        double d2 = 0;
        for (int k = 0; k < 3; ++k) d2 += (x[k] - y[k]) * (x[k] - y[k]);
        if (d2 < bd) {
          bd = d2;
          best = j;
        }
      }
      if (best < 0 || bd > tol * tol || taken[best])
        return fail(FR_EMESH, "flux points do not conform across an exchange face");
      taken[best] = 1;
      const int64_t partner_idx = G.p0 + best - pbase[G.r];  // index in that rank's list
      // both sides order a rank pair's points by the lower rank's index
      pairs.push_back(PairX{G.r, rank < G.r ? own_idx : partner_idx, F.pt[a],
                            pt_mag[G.p0 + best]});
    }
  }
  std::stable_sort(pairs.begin(), pairs.end(), [](const PairX& x, const PairX& y) {
    return x.r != y.r ? x.r < y.r : x.key < y.key;
  });
  std::vector<int32_t> list(pairs.size());
  m->x_counts.assign(nranks, 0);
  std::vector<double> xm(m->conn.bidx.size(), 1.0);
  for (size_t k = 0; k < pairs.size(); ++k) {
    list[k] = pairs[k].own;
    ++m->x_counts[pairs[k].r];
    xm[pairs[k].own] = pairs[k].mag;
  }
  for (int r = 0; r < nranks; ++r) counts[r] = m->x_counts[r];
  m->n_xlist = (long long)list.size();
  m->x_list_host = list;
  if (m->host_only) return FR_OK;
  CK(cudaSetDevice(m->device));
  CK(cudaStreamSynchronize(m->stream));
  if (m->x_list) {
    cudaFree(m->x_list);
    m->x_list = nullptr;
  }
  if (!list.empty()) {
    CK(cudaMalloc((void**)&m->x_list, list.size() * sizeof(int32_t)));
    CK(cudaMemcpy(m->x_list, list.data(), list.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  }
  if (m->xm) {
    if (m->wsize == 8) {
      CK(cudaMemcpy(m->xm, xm.data(), xm.size() * sizeof(double), cudaMemcpyHostToDevice));
    } else {
      std::vector<float> h(xm.begin(), xm.end());
      CK(cudaMemcpy(m->xm, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
  }
  return FR_OK;
}

int fr_exchange_list(const fr_mesh* m, int32_t* points, int64_t* n) {
  if (!m || !n) return fail(FR_EINVAL, "null argument");
  *n = int64_t(m->x_list_host.size());
  if (points) std::copy(m->x_list_host.begin(), m->x_list_host.end(), points);
  return FR_OK;
}

int fr_exchange_pack(fr_mesh* m, int what, void* dev_buf) {
  if (!m || (!dev_buf && m && m->n_xlist)) return fail(FR_EINVAL, "null argument");
  if (m->host_only) return fail(FR_EINVAL, "host-only handle (device < 0)");
  if (what != FR_XCH_SOLUTION && what != FR_XCH_GRADIENT) return fail(FR_EINVAL, "bad trace kind");
  CK(cudaSetDevice(m->device));
  return FR_PREC(m, exchange_pack, m, what, dev_buf);
}

int fr_exchange_unpack(fr_mesh* m, int what, const void* dev_buf) {
  if (!m || (!dev_buf && m && m->n_xlist)) return fail(FR_EINVAL, "null argument");
  if (m->host_only) return fail(FR_EINVAL, "host-only handle (device < 0)");
  if (what != FR_XCH_SOLUTION && what != FR_XCH_GRADIENT) return fail(FR_EINVAL, "bad trace kind");
  CK(cudaSetDevice(m->device));
  return FR_PREC(m, exchange_unpack, m, what, dev_buf);
}

int fr_rk_stage(fr_mesh* m, int scheme, double dt, int stage, int phase, int part) {
  if (!m) return fail(FR_EINVAL, "null mesh");
  if (int rb = bc_ready(m)) return rb;
  if (m->host_only) return fail(FR_EINVAL, "host-only handle (device < 0)");
  if (m->in_group) return fail(FR_EINVAL, "the mesh belongs to a group");
  if (m->filter_on) return fail(FR_EINVAL, "not with the entropy filter");
  if (scheme != FR_RK4 && scheme != FR_RK45) return fail(FR_EINVAL, "unknown scheme");
  const int nst = scheme == FR_RK4 ? 4 : 5;
  if (stage < 0 || stage >= nst || (phase != 1 && phase != 2) || part < 0 || part > 2)
    return fail(FR_EINVAL, "bad stage, phase or part");
  if (m->has_exch && m->n_xlist == 0 && m->nb > m->nb_x0)
    return fail(FR_EINVAL, "exchange points without fr_exchange_setup");
  CK(cudaSetDevice(m->device));
  int rc = FR_PREC(m, do_stage, m, scheme, dt, stage, phase, part);
  if (rc) return rc;
  if (phase == 2 && part != 1) ++m->n_stages;
  if (stage == nst - 1 && phase == 2 && part != 1) ++m->n_steps;
  return FR_OK;
}

int fr_get_schedule(const fr_mesh* m, fr_schedule_t* out) {
  if (!m || !out) return fail(FR_EINVAL, "null argument");
  std::memset(out, 0, sizeof(*out));
  for (int k = 0; k < 3; ++k) {
    out->tile_grad[k] = out->tile_vol[k] = -1;
    const int t = m->type_of_kind[k];
    if (t < 0 || m->host_only) continue;
    const DevType& D = m->types[t];
    out->tile_grad[k] = D.tile_grad;
    out->tile_vol[k] = D.tile_vol;
    out->tensor_grad[k] = use_tc_grad(m, D) ? 1 : 0;
    out->tensor_vol[k] = use_tc_vol(m, D) ? 1 : 0;
    out->structured[k] = use_hex(m, D) || use_pri(m, D) || use_m0s(m, D) ? 1 : 0;
  }
  out->face_block = m->face_tb;
  out->parallel_types = m->par_types ? 1 : 0;
  out->ms_default = m->sched_ms[0];
  out->ms_tuned = m->sched_ms[1];
  return FR_OK;
}

int fr_set_schedule(fr_mesh* m, const fr_schedule_t* in) {
  if (!m || !in) return fail(FR_EINVAL, "null argument");
  if (m->host_only) return fail(FR_EINVAL, "host-only handle (device < 0)");
  if (in->face_block < 32 || in->face_block > 1024 || in->face_block % 32)
    return fail(FR_EINVAL, "face_block must be a multiple of 32 in 32..1024");
  for (int k = 0; k < 3; ++k) {
    const int t = m->type_of_kind[k];
    if (t < 0) continue;
    const DevType& D = m->types[t];
    const bool hexk = D.kind == EK_HEX && m->active != FR_VARIANT_DENSE;
    const bool prik = use_pri(m, D);
    const int mg = hexk ? hex_tile_max(m->order) : prik ? D.pri_grad_ctas : D.grad_ctas;
    const int mv = hexk ? hex_tile_max(m->order) : prik ? D.pri_vol_ctas : D.vol_ctas;
    if (in->tile_grad[k] < 0 || in->tile_grad[k] > mg || in->tile_vol[k] < 0 ||
        in->tile_vol[k] > mv)
      return fail(FR_EINVAL, "tile out of range for this kernel");
  }
  CK(cudaSetDevice(m->device));
  if (in->parallel_types) {
    int rc = ensure_par(m);
    if (rc) return rc;
  }
  CK(cudaStreamSynchronize(m->stream));
  for (int k = 0; k < 3; ++k) {
    const int t = m->type_of_kind[k];
    if (t < 0) continue;
    m->types[t].tile_grad = in->tile_grad[k];
    m->types[t].tile_vol = in->tile_vol[k];
  }
  m->face_tb = in->face_block;
  m->par_types = in->parallel_types != 0;
  ++m->epoch;
  return FR_OK;
}

int fr_set_stream(fr_mesh* m, void* s) {
  if (!m) return fail(FR_EINVAL, "null mesh");
  if (m->host_only) return fail(FR_EINVAL, "host-only handle (device < 0)");
  CK(cudaSetDevice(m->device));
  CK(cudaStreamSynchronize(m->stream));
  m->stream = s ? (cudaStream_t)s : m->own_stream;
  return FR_OK;
}

int fr_sync(fr_mesh* m) {
  if (!m) return fail(FR_EINVAL, "null mesh");
  if (m->host_only) return fail(FR_EINVAL, "host-only handle (device < 0)");
  CK(cudaSetDevice(m->device));
  CK(cudaStreamSynchronize(m->stream));
  return FR_OK;
}

int fr_get_operator(const fr_mesh* m, int etype, int which, double* out) {
  if (!m || !out) return fail(FR_EINVAL, "null argument");
  const HostType* H = host_ptr(m, etype);
  if (!H) return fail(FR_EINVAL, "mesh has no elements of this type");
  const RefElement& R = H->ref;
  const std::vector<double>* v = nullptr;
  switch (which) {
    case FR_OP_M0: v = &R.M0; break;
    case FR_OP_D: v = &R.D; break;
    case FR_OP_LIFT: v = &R.LIFT; break;
    case FR_OP_WEIGHTS: v = &R.W; break;
    case FR_OP_UPTS: v = &R.upts; break;
    case FR_OP_FPTS: v = &R.fpts; break;
    case FR_OP_AA_QPTS: v = &H->aa_x; break;
    case FR_OP_AA_QWTS: v = &H->aa_w; break;
    case FR_OP_AA_B: v = &H->aa_B; break;
    case FR_OP_AA_P: v = &H->aa_P; break;
    default: return fail(FR_EINVAL, "unknown operator");
  }
  if (v->empty()) return fail(FR_EINVAL, "anti-aliasing is off (fr_set_antialias)");
  std::memcpy(out, v->data(), v->size() * sizeof(double));
  return FR_OK;
}

int fr_get_metrics(const fr_mesh* m, int etype, double* smat, double* rcpdjac) {
  if (!m) return fail(FR_EINVAL, "null argument");
  const HostType* H = host_ptr(m, etype);
  if (!H) return fail(FR_EINVAL, "mesh has no elements of this type");
  if (smat) std::memcpy(smat, H->smat.data(), H->smat.size() * sizeof(double));
  if (rcpdjac) std::memcpy(rcpdjac, H->rcpdjac.data(), H->rcpdjac.size() * sizeof(double));
  return FR_OK;
}

int fr_set_viscous_scheme(fr_mesh* m, double beta, double tau) {
  if (!m) return fail(FR_EINVAL, "null argument");
  if (m->physics != FR_NAVIER_STOKES) return fail(FR_EINVAL, "viscous scheme of a Navier-Stokes mesh only");
  if (!(beta >= -0.5 && beta <= 0.5) || !(tau >= 0.0) || !std::isfinite(tau))
    return fail(FR_EINVAL, "beta must lie in [-1/2, 1/2] and tau be finite and >= 0");
  if (m->in_group && beta != 0.0)
    return fail(FR_EINVAL, "an LDG bias needs one interface orientation: not across parts");
  m->ldg_beta = beta;
  m->ldg_tau = tau;
  ++m->epoch;  // the constants are kernel arguments captured in the graphs
  return FR_OK;
}

int fr_set_antialias(fr_mesh* m, int qdeg) {
  if (!m) return fail(FR_EINVAL, "null argument");
  if (qdeg < 0 || qdeg > 24) return fail(FR_EINVAL, "quadrature degree must be 0..24");
  for (auto& H : m->host) {
    H.aa_qdeg = qdeg;
    H.aa_x.clear();
    H.aa_w.clear();
    H.aa_B.clear();
    H.aa_P.clear();
    if (qdeg == 0) continue;
    aa_rule(H.kind, qdeg, H.aa_x, H.aa_w);
    aa_operators(H.ref, H.aa_x, H.aa_w, H.aa_B, H.aa_P);
  }
  m->aa_qdeg = qdeg;
  if (m->host_only) return FR_OK;
  CK(cudaSetDevice(m->device));
  CK(cudaStreamSynchronize(m->stream));
  int rc = FR_PREC(m, aa_setup, m);
  if (rc) return rc;
  ++m->epoch;            // graphs hold the old launch sequence
  if (m->variant == FR_VARIANT_AUTO) m->tuned = false;
  return FR_OK;
}

int fr_get_boundary_points(const fr_mesh* m, double* x, int* kind) {
  if (!m) return fail(FR_EINVAL, "null argument");
  for (size_t i = 0; i < m->conn.bidx.size(); ++i) {
    const int32_t code = m->conn.bidx[i];
    const HostType& H = m->host[code >> 29];
    const int64_t rem = code & ((int64_t(1) << 29) - 1);
    const int64_t e = rem / (5 * H.ref.nfpts);
    const int f = int(rem - e * 5 * H.ref.nfpts);
    if (x)
      for (int k = 0; k < 3; ++k) x[3 * i + k] = H.fpts_x[(size_t(e) * H.ref.nfpts + f) * 3 + k];
    if (kind) kind[i] = m->bc64.kind[m->conn.bbc[i]];
  }
  return FR_OK;
}

int fr_get_interfaces(const fr_mesh* m, int64_t* left, int64_t* right) {
  if (!m) return fail(FR_EINVAL, "null argument");
  std::vector<int64_t> eoff(m->host.size(), 0);
  for (size_t t = 1; t < m->host.size(); ++t) eoff[t] = eoff[t - 1] + m->host[t - 1].ne;
  auto elem = [&](int32_t code) {
    const int t = code >> 29;
    const int64_t rem = code & ((int64_t(1) << 29) - 1);
    return eoff[t] + rem / (5 * m->host[t].ref.nfpts);
  };
  for (size_t i = 0; i < m->conn.pl.size(); ++i) {
    if (left) left[i] = elem(m->conn.pl[i]);
    if (right) right[i] = elem(m->conn.pr[i]);
  }
  return FR_OK;
}

int fr_get_adjacency(const fr_mesh* m, int etype, int64_t* nbr) {
  if (!m || !nbr) return fail(FR_EINVAL, "null argument");
  const HostType* H = host_ptr(m, etype);
  if (!H) return fail(FR_EINVAL, "mesh has no elements of this type");
  std::memcpy(nbr, H->nbr.data(), H->nbr.size() * sizeof(int64_t));
  return FR_OK;
}

int fr_partition(const fr_mesh* m, int nparts, int mode, const double* weights,
                 int32_t* part) {
  if (!m || !part) return fail(FR_EINVAL, "null argument");
  const double ones[3] = {1.0, 1.0, 1.0};
  std::vector<int32_t> p;
  std::string err = partition_elements(m->host, nparts, mode, weights ? weights : ones, p);
  if (!err.empty()) return fail(FR_EINVAL, err);
  std::memcpy(part, p.data(), p.size() * sizeof(int32_t));
  return FR_OK;
}

int fr_partition_faces(const fr_mesh* m, const int32_t* part, int rank,
                       int64_t* faces, int64_t* count) {
  if (!m || !part || !count) return fail(FR_EINVAL, "null argument");
  int64_t n = 0, off = 0;
  for (const HostType& H : m->host) {
    const int nf = H.ref.nfaces, nv = H.ref.nverts;
    for (int64_t e = 0; e < H.ne; ++e) {
      if (part[off + e] != rank) continue;
      for (int f = 0; f < nf; ++f) {
        const int64_t nb = H.nbr[size_t(e) * nf + f];
        if (nb < 0 || part[nb] == rank) continue;
        if (faces) {
          const RefFace& F = H.ref.faces[f];
          for (int i = 0; i < 4; ++i)
            faces[4 * n + i] = i < F.nv ? H.conn[size_t(e) * nv + F.verts[i]] : -1;
        }
        ++n;
      }
    }
    off += H.ne;
  }
  *count = n;
  return FR_OK;
}

int fr_get_pairs(const fr_mesh* m, int64_t* n_interior, int64_t* n_boundary) {
  if (!m) return fail(FR_EINVAL, "null argument");
  if (n_interior) *n_interior = int64_t(m->conn.pl.size());
  if (n_boundary) *n_boundary = int64_t(m->conn.bidx.size());
  return FR_OK;
}

int fr_group_create(fr_mesh* const* meshes, int n, fr_group** out) {
  if (!meshes || !out || n < 1) return fail(FR_EINVAL, "null argument or empty group");
  *out = nullptr;
  const fr_mesh* a = meshes[0];
  for (int i = 0; i < n; ++i) {
    const fr_mesh* m = meshes[i];
    if (!m) return fail(FR_EINVAL, "null member");
    if (m->host_only) return fail(FR_EINVAL, "host-only member");
    if (m->in_group) return fail(FR_EINVAL, "mesh already belongs to a group");
    if (m->device != a->device || m->precision != a->precision || m->physics != a->physics ||
        m->order != a->order || m->gamma != a->gamma || m->mu != a->mu ||
        m->prandtl != a->prandtl || m->periodic != a->periodic)
      return fail(FR_EINVAL, "members differ in device, precision, physics, order or constants");
    if (m->filter_on) return fail(FR_EINVAL, "the entropy filter is not supported in a group");
    if (m->ldg_beta != 0.0)
      return fail(FR_EINVAL, "an LDG bias needs one interface orientation: not across parts");
    for (int j = 0; j < i; ++j)
      if (meshes[j] == m) return fail(FR_EINVAL, "a mesh appears twice in the group");
  }
  CK(cudaSetDevice(a->device));
  auto g = std::make_unique<fr_group>();
  g->m.assign(meshes, meshes + n);
  int rc = FR_PREC(a, group_setup, g.get());
  if (rc) return rc;
  g->aux.assign(n, nullptr);
  g->ev.assign(n, nullptr);
  for (int i = 0; i < n; ++i) {
    CK(cudaStreamCreateWithFlags(&g->aux[i], cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&g->ev[i], cudaEventDisableTiming));
  }
  CK(cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming));
  for (fr_mesh* m : g->m) m->in_group = true;
  *out = g.release();
  return FR_OK;
}

int fr_group_destroy(fr_group* g) {
  if (!g) return FR_OK;
  cudaSetDevice(g->m[0]->device);
  cudaStreamSynchronize(g->m[0]->stream);
  delete g;
  return FR_OK;
}

int fr_group_rhs(fr_group* g) {
  if (!g) return fail(FR_EINVAL, "null group");
  CK(cudaSetDevice(g->m[0]->device));
  return FR_PREC(g->m[0], group_run, g, 0, 0.0, 1);
}

int fr_group_rk_step(fr_group* g, int scheme, double dt, int nsteps) {
  if (!g) return fail(FR_EINVAL, "null group");
  if (scheme != FR_RK4 && scheme != FR_RK45) return fail(FR_EINVAL, "unknown scheme");
  if (nsteps < 0) return fail(FR_EINVAL, "negative step count");
  if (nsteps == 0) return FR_OK;
  CK(cudaSetDevice(g->m[0]->device));
  return FR_PREC(g->m[0], group_run, g, scheme == FR_RK4 ? 1 : 2, dt, nsteps);
}

}  // extern "C"

#include "fr_api_filter.inc"


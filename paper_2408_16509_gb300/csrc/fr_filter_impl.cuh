// Entropy filter and filter-strength predictor: device set-up and the
// per-stage launches (templated; included by fr_impl.cuh).
#pragma once

namespace {

template <typename T>
int setup_filter(fr_mesh* m) {
  int rc;
  for (size_t t = 0; t < m->types.size(); ++t) {
    DevType& D = m->types[t];
    if (D.fVT) continue;
    const RefElement& R = m->host[t].ref;
    const int nu = D.nu, nf = D.nf, np = nu + nf;
    std::vector<double> vinvt(size_t(nu) * nu), vt(size_t(nu) * np), deg(nu);
    for (int k = 0; k < nu; ++k)
      for (int z = 0; z < nu; ++z) vinvt[size_t(z) * nu + k] = R.vdm_inv[size_t(k) * nu + z];
    std::vector<double> bu(size_t(nu) * nu), bf(size_t(nf) * nu);
    R.basis(nu, R.upts.data(), bu.data());
    R.basis(nf, R.fpts.data(), bf.data());
    for (int k = 0; k < nu; ++k) {
      for (int i = 0; i < nu; ++i) vt[size_t(k) * np + i] = bu[size_t(i) * nu + k];
      for (int f = 0; f < nf; ++f) vt[size_t(k) * np + nu + f] = bf[size_t(f) * nu + k];
      deg[k] = double(R.mdeg[k]) / R.p;
    }
    if ((rc = dev_upload<T>(m, vinvt, &D.fVinvT))) return rc;
    if ((rc = dev_upload<T>(m, vt, &D.fVT))) return rc;
    if ((rc = dev_upload<T>(m, deg, &D.fdeg))) return rc;
    if ((rc = dev_upload<T>(m, R.W, &D.fW))) return rc;
    if ((rc = dev_zeros(m, size_t(D.ne) * sizeof(double), (void**)&D.smin))) return rc;
    if ((rc = dev_zeros(m, size_t(D.ne) * sizeof(float), (void**)&D.zeta_last))) return rc;
    if ((rc = dev_zeros(m, size_t(D.ne) * sizeof(int), (void**)&D.evals_last))) return rc;
    if ((rc = dev_zeros(m, size_t(D.ne) * sizeof(int32_t), (void**)&D.flist))) return rc;
    if ((rc = dev_zeros(m, sizeof(int), (void**)&D.fcount))) return rc;
  }
  // partner flux point of every element flux point (-1 on boundaries)
  for (size_t t = 0; t < m->types.size(); ++t) {
    DevType& D = m->types[t];
    if (D.fpartner) continue;
    std::vector<int32_t> part(size_t(D.ne) * D.nf, -1);
    auto local = [&](int32_t code, int* tt, long long* e, int* f) {
      *tt = code >> 29;
      long long l = code & ((1 << 29) - 1);
      int nfx = m->types[*tt].nf;
      *e = l / (5 * nfx);
      *f = int(l - *e * 5 * nfx);
    };
    for (size_t i = 0; i < m->conn.pl.size(); ++i) {
      int ta, tb, fa, fb;
      long long ea, eb;
      local(m->conn.pl[i], &ta, &ea, &fa);
      local(m->conn.pr[i], &tb, &eb, &fb);
      if (ta == int(t)) part[size_t(ea) * D.nf + fa] = m->conn.pr[i];
      if (tb == int(t)) part[size_t(eb) * D.nf + fb] = m->conn.pl[i];
    }
    if ((rc = dev_upload_i32(m, part, &D.fpartner))) return rc;
  }
  if (!m->d_fstats) {
    if ((rc = dev_zeros(m, sizeof(FilterStats), (void**)&m->d_fstats))) return rc;
  }
  return FR_OK;
}

// Launched at the start of every filtered stage: s_min from the stage input.
template <typename T, typename TR>
void launch_entropy_min(fr_mesh* m, cudaStream_t s, bool from_x) {
  for (size_t t = 0; t < m->types.size(); ++t) {
    DevType& D = m->types[t];
    dispatch(D.kind, m->order, [&](auto nu, auto nf) {
      constexpr int NU = decltype(nu)::value, NF = decltype(nf)::value;
      long long threads = D.ne * 32;
      k_entropy_min<T, TR, NU, NF><<<nblk(threads, 256), 256, 0, s>>>(
          D.ne, from_x ? nullptr : (const T*)D.Y, (const TR*)D.X,
          (const T*)m->uf, m->tt, int(t), D.fpartner, m->gamma, D.smin);
    });
  }
}

// Launched after a type's volume kernel wrote the stage value and u_f.
template <typename T, typename TR>
void launch_filter(fr_mesh* m, cudaStream_t s, DevType& D, bool last_stage) {
  FilterOps<T> op{(const T*)D.fVinvT, (const T*)D.fVT, (const T*)D.fdeg,
                  (const T*)D.fW, D.fpartner};
  FilterArgs fa;
  fa.gamma = m->gamma;
  fa.tau = m->wsize == 8 ? 1e-8 : 1.0 / 1048576.0;
  fa.ratio = m->mlp_ratio;
  fa.zeta_last = D.zeta_last;
  fa.evals_last = D.evals_last;
  fa.smin = D.smin;
  fa.stats = m->d_fstats;
  fa.samples = m->d_samples;
  fa.cap = m->sample_cap;
  fa.mlp = m->mlp_on ? m->d_mlp : nullptr;
  fa.mlp_norm = m->d_mlp_norm;
  T* uf = (T*)m->uf + D.off_f;
  T* reg = last_stage ? nullptr : (T*)D.Y;
  TR* regR = last_stage ? (TR*)D.X : nullptr;
  // the zeta = 0 test of every element (a warp each), then k_filter on the
  // elements it lists (one CTA per element; CTAs past the count return)
  cudaMemsetAsync(D.fcount, 0, sizeof(int), s);
  dispatch(D.kind, m->order, [&](auto nu, auto nf) {
    constexpr int NU = decltype(nu)::value, NF = decltype(nf)::value;
    k_filter_check<T, TR, NU, NF><<<nblk(D.ne * 32, 256), 256, 0, s>>>(
        D.ne, reg, regR, uf, fa, D.flist, D.fcount);
    k_filter<T, TR, NU, NF><<<unsigned(D.ne), kFilterThreads, 0, s>>>(
        D.ne, reg, regR, uf, op, fa, D.flist, D.fcount);
  });
}

// Filter the current solution register in place.  s_min comes from the
// caller (host, per element, types in mesh order) or, when smin_host is
// null, from the solution itself; the flux-point traces follow.
template <typename T, typename TR>
int filter_solution(fr_mesh* m, const double* smin_host) {
  int rc = ensure_uf<T, TR>(m);
  if (rc) return rc;
  if (smin_host) {
    size_t off = 0;
    for (auto& D : m->types) {
      CK(cudaMemcpyAsync(D.smin, smin_host + off, size_t(D.ne) * sizeof(double),
                         cudaMemcpyHostToDevice, m->stream));
      off += size_t(D.ne);
    }
  } else {
    launch_entropy_min<T, TR>(m, m->stream, true);
  }
  for (auto& D : m->types) launch_filter<T, TR>(m, m->stream, D, true);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(m->stream));
  return FR_OK;
}

}  // namespace

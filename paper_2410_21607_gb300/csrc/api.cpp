// C ABI entry points (include/sem.h), device tables and the reference state.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "sem_internal.h"

namespace sem {

static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }
int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

static long long g_serial = 0;

template <typename T>
static int upload(T*& dst, const std::vector<T>& src) {
  size_t n = src.size() ? src.size() : 1;
  SEM_CUDA_TRY(cudaMalloc((void**)&dst, n * sizeof(T)));
  if (!src.empty()) SEM_CUDA_TRY(cudaMemcpy(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
  return SEM_OK;
}

void free_device(Mesh& m) {
  if (!m.dev) return;
  int cur = -1;
  cudaGetDevice(&cur);
  if (m.dev_id >= 0 && cur != m.dev_id) cudaSetDevice(m.dev_id);
  DeviceTables& D = *m.dev;
  void* ptrs[] = {D.hmap, D.hang_h, D.hang_w, D.qt_ptr, D.qt_src, D.qt_w, D.Minv_h, D.Minv_z,
                  D.Mh, D.Mz, D.Minv_h32, D.Minv_z32, D.qt_w32, D.qt_rec_src, D.qt_rec_w, D.qt_rec_unit, D.hang_w32, D.mirror, D.spg, D.spg32, D.ref, D.ref32, D.col_level, D.col_x0, D.col_y0, D.xh, D.yh, D.zk, D.hzk, D.hzk32, D.scratch,
                  D.status, D.org, D.elem_cmax, D.elem_flags, D.diag_buf,
                  D.tr_comp_ptr, D.tr_nodes, D.tr_A_ptr, D.tr_A_col, D.tr_A_val, D.tr_coupled,
                  D.zG, D.zH, D.metric, D.metric32, D.Minv_g, D.Minv_g32, D.refG, D.refH, D.refG32, D.refH32,
                  D.ref4G, D.ref4H};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete m.dev;
  m.dev = nullptr;
  if (m.dev_id >= 0 && cur >= 0 && cur != m.dev_id) cudaSetDevice(cur);
  m.dev_id = -1;
}

int ensure_device(Mesh& m) {
  int cur = 0;
  SEM_CUDA_TRY(cudaGetDevice(&cur));
  if (m.dev) {
    if (m.dev_id != cur) return fail(SEM_ERR_ARG, "mesh tables live on another device");
    return SEM_OK;
  }
  m.dev = new (std::nothrow) DeviceTables();
  if (!m.dev) return fail(SEM_ERR_ARG, "out of host memory");
  m.dev_id = cur;
  DeviceTables& D = *m.dev;
  int rc;
  std::vector<double> minvh(m.NH), minvz(m.NZ);
  for (long long h = 0; h < m.NH; ++h) minvh[h] = 1.0 / m.Mh[h];
  for (int k = 0; k < m.NZ; ++k) minvz[k] = 1.0 / m.Mz[k];
  std::vector<float> minvh32(m.NH), minvz32(m.NZ), qtw32(m.qt_w.size()), hw32(m.hang_w.size());
  for (long long h = 0; h < m.NH; ++h) minvh32[h] = (float)minvh[h];
  for (int k = 0; k < m.NZ; ++k) minvz32[k] = (float)minvz[k];
  for (size_t k = 0; k < qtw32.size(); ++k) qtw32[k] = (float)m.qt_w[k];
  for (size_t k = 0; k < hw32.size(); ++k) hw32[k] = (float)m.hang_w[k];
  // compact Q_h^T records: the up to 4 sources of a horizontal node and their
  // weights side by side (one 16-byte load each), in the CSR order
  std::vector<int> rsrc((size_t)m.NH * 4, -1), runit((size_t)m.NH * 4, -1);
  std::vector<float> rw((size_t)m.NH * 4, 0.f);
  for (long long h = 0; h < m.NH; ++h) {
    const int beg = m.qt_ptr[h], cnt = m.qt_ptr[h + 1] - beg;
    bool unit = cnt <= 4;
    for (int e = 0; e < cnt && unit; ++e) unit = m.qt_w[beg + e] == 1.0;
    if (unit) {
      for (int e = 0; e < cnt; ++e) runit[(size_t)h * 4 + e] = m.qt_src[beg + e];
    } else {
      runit[(size_t)h * 4] = -2;
    }
    if (cnt > 4) {
      rsrc[(size_t)h * 4] = -2;
      continue;
    }
    for (int e = 0; e < cnt; ++e) {
      rsrc[(size_t)h * 4 + e] = m.qt_src[beg + e];
      rw[(size_t)h * 4 + e] = qtw32[beg + e];
    }
  }
  std::vector<double> hzk(m.nz);
  std::vector<float> hzk32(m.nz);
  for (int k = 0; k < m.nz; ++k) {
    hzk[k] = m.hz(k);
    hzk32[k] = (float)hzk[k];
  }
  std::vector<int> lev(m.Ncol());
  std::vector<double> cx0(m.Ncol()), cy0(m.Ncol());
  for (long long c = 0; c < m.Ncol(); ++c) {
    const Leaf& L = m.leaves[c];
    lev[c] = L.l;
    cx0[c] = -0.5 * m.Lx + L.i * m.hx(L.l);
    cy0[c] = -0.5 * m.Ly + L.j * m.hy(L.l);
  }
  if ((rc = upload(D.hmap, m.hmap)) || (rc = upload(D.hang_h, m.hang_h)) ||
      (rc = upload(D.hang_w, m.hang_w)) || (rc = upload(D.qt_ptr, m.qt_ptr)) ||
      (rc = upload(D.qt_src, m.qt_src)) || (rc = upload(D.qt_w, m.qt_w)) ||
      (rc = upload(D.Minv_h, minvh)) || (rc = upload(D.Minv_z, minvz)) ||
      (rc = upload(D.Mh, m.Mh)) || (rc = upload(D.Mz, m.Mz)) || (rc = upload(D.col_level, lev)) ||
      (rc = upload(D.xh, m.xh)) || (rc = upload(D.yh, m.yh)) || (rc = upload(D.zk, m.zk)) ||
      (rc = upload(D.hzk, hzk)) || (rc = upload(D.hzk32, hzk32)) ||
      (rc = upload(D.Minv_h32, minvh32)) || (rc = upload(D.Minv_z32, minvz32)) ||
      (rc = upload(D.qt_w32, qtw32)) || (rc = upload(D.hang_w32, hw32)) ||
      (rc = upload(D.qt_rec_src, rsrc)) || (rc = upload(D.qt_rec_w, rw)) || (rc = upload(D.qt_rec_unit, runit)) ||
      (rc = upload(D.col_x0, cx0)) || (rc = upload(D.col_y0, cy0))) {
    free_device(m);
    return rc;
  }
  // column residual scratch: [Ncol][Nq][5][NZr], float64 (also holds float32)
  D.scratch_bytes = (size_t)m.Ncol() * m.Nq * kFields * m.NZr() * sizeof(double);
  cudaError_t e = cudaMalloc(&D.scratch, D.scratch_bytes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&D.status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(D.status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&D.ref, (size_t)m.NZ * kRef * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&D.ref32, (size_t)m.NZ * (kRef + 4) * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&D.elem_cmax, (size_t)m.Ne() * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&D.elem_flags, (size_t)m.Ne());
  if (e == cudaSuccess) e = cudaMalloc((void**)&D.diag_buf, (size_t)m.NZ * 4 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&D.mirror, (size_t)m.NG * kFields * sizeof(float));
  if (e != cudaSuccess) {
    free_device(m);
    return fail(SEM_ERR_CUDA, std::string("device allocation: ") + cudaGetErrorString(e));
  }
  if (m.warped()) {
    std::vector<float> met32(m.metric.size()), mg32(m.Mg.size());
    std::vector<double> minvg(m.Mg.size());
    for (size_t k = 0; k < m.metric.size(); ++k) met32[k] = (float)m.metric[k];
    for (size_t k = 0; k < m.Mg.size(); ++k) {
      minvg[k] = 1.0 / m.Mg[k];
      mg32[k] = (float)minvg[k];
    }
    const size_t nh = m.zH.size() ? m.zH.size() : 1;
    cudaError_t e2 = cudaSuccess;
    if ((rc = upload(D.zG, m.zG)) || (rc = upload(D.zH, m.zH)) || (rc = upload(D.metric, m.metric)) ||
        (rc = upload(D.metric32, met32)) ||
        (rc = upload(D.Minv_g, minvg)) || (rc = upload(D.Minv_g32, mg32))) {
      free_device(m);
      return rc;
    }
    e2 = cudaMalloc((void**)&D.refG, (size_t)m.NG * kRef * sizeof(double));
    if (e2 == cudaSuccess) e2 = cudaMalloc((void**)&D.refH, nh * kRef * sizeof(double));
    if (e2 == cudaSuccess) e2 = cudaMalloc((void**)&D.refG32, (size_t)m.NG * kRef * sizeof(float));
    if (e2 == cudaSuccess) e2 = cudaMalloc((void**)&D.refH32, nh * kRef * sizeof(float));
    if (e2 == cudaSuccess) e2 = cudaMalloc((void**)&D.ref4G, (size_t)m.NG * 4 * sizeof(float));
    if (e2 == cudaSuccess) e2 = cudaMalloc((void**)&D.ref4H, nh * 4 * sizeof(float));
    if (e2 != cudaSuccess) {
      free_device(m);
      return fail(SEM_ERR_CUDA, std::string("device allocation: ") + cudaGetErrorString(e2));
    }
  }
  if (!m.origin.empty()) {
    std::vector<int> org((size_t)m.Ncol() * 6);
    for (long long c = 0; c < m.Ncol(); ++c) {
      const Origin& o = m.origin[c];
      org[c * 6 + 0] = o.kind;
      for (int q = 0; q < 4; ++q) org[c * 6 + 1 + q] = o.src[q];
      org[c * 6 + 5] = o.a + 2 * o.b;
    }
    if ((rc = upload(D.org, org))) {
      free_device(m);
      return rc;
    }
  }
  return SEM_OK;
}

// Hydrostatic reference state at every vertical level (Eqs. rho_split ..
// hydro_bal): the constant buoyancy-frequency atmosphere
//   theta0 = theta_s exp(N^2 z / g),
//   pi0 = 1 + g^2/(c_p theta_s N^2) (exp(-N^2 z/g) - 1),
//   p0 = p00 pi0^(c_p/R_d),  rho0 = p00 pi0^(c_v/R_d) / (R_d theta0),
// which satisfies dp0/dz = -rho0 g and p0 = p00 (R_d rho0 theta0 / p00)^gamma.
bool reference_stale(const Mesh& m, const sem_params& p) {
  if (!m.dev) return true;
  const double key[8] = {p.g, p.R_d, p.c_p, p.p00, p.theta_s, p.N_bv, 0, 0};
  return !(m.dev->ref_valid && std::memcmp(key, m.dev->ref_key, sizeof(key)) == 0);
}

int ensure_reference(Mesh& m, const sem_params& p) {
  DeviceTables& D = *m.dev;
  double key[8] = {p.g, p.R_d, p.c_p, p.p00, p.theta_s, p.N_bv, 0, 0};
  if (!reference_stale(m, p)) return SEM_OK;
  if (!(p.N_bv > 0) || !(p.g > 0) || !(p.c_p > p.R_d) || !(p.R_d > 0))
    return fail(SEM_ERR_ARG, "reference state needs g > 0, N_bv > 0, c_p > R_d > 0");
  const double c_v = p.c_p - p.R_d, N2 = p.N_bv * p.N_bv;
  // one row: theta0, pi0, p0, rho0, (rho theta)0, dtheta0/dz, 1/(rho theta)0, z
  auto row = [&](double z, double* r) {
    const double th0 = p.theta_s * std::exp(N2 * z / p.g);
    const double pi0 = 1.0 + p.g * p.g / (p.c_p * p.theta_s * N2) * (std::exp(-N2 * z / p.g) - 1.0);
    if (!(pi0 > 0)) return false;
    const double p0 = p.p00 * std::pow(pi0, p.c_p / p.R_d);
    const double rho0 = p.p00 * std::pow(pi0, c_v / p.R_d) / (p.R_d * th0);
    const double v[kRef] = {th0, pi0, p0, rho0, rho0 * th0, th0 * N2 / p.g, 1.0 / (rho0 * th0), z};
    for (int q = 0; q < kRef; ++q) r[q] = v[q];
    return true;
  };
  // a table of rows at heights z[0..n): float64, float32 and packed float32
  // rows (p0, rho0, (rho theta)0, 1/(rho theta)0)
  auto table = [&](const std::vector<double>& z, std::vector<double>& t64, std::vector<float>& t32,
                   std::vector<float>& t4) {
    const size_t n = z.size();
    t64.assign(n * kRef, 0.0);
    t32.assign(n * kRef, 0.f);
    t4.assign(n * 4, 0.f);
    for (size_t k = 0; k < n; ++k) {
      double* r = &t64[k * kRef];
      if (!row(z[k], r)) return false;
      for (int q = 0; q < kRef; ++q) t32[k * kRef + q] = (float)r[q];
      t4[k * 4 + 0] = (float)r[2];
      t4[k * 4 + 1] = (float)r[3];
      t4[k * 4 + 2] = (float)r[4];
      t4[k * 4 + 3] = (float)r[6];
    }
    return true;
  };
  std::vector<double> ref;
  std::vector<float> ref32, r4;
  if (!table(m.zk, ref, ref32, r4)) return fail(SEM_ERR_ARG, "reference state: Exner pressure <= 0 below the lid");
  ref32.insert(ref32.end(), r4.begin(), r4.end());   // packed rows after the table
  SEM_CUDA_TRY(cudaMemcpy(D.ref, ref.data(), ref.size() * sizeof(double), cudaMemcpyHostToDevice));
  SEM_CUDA_TRY(cudaMemcpy(D.ref32, ref32.data(), ref32.size() * sizeof(float), cudaMemcpyHostToDevice));
  if (m.warped()) {
    // warped layers: the reference state at every node's own height
    std::vector<double> g64, h64;
    std::vector<float> g32, h32, g4, h4;
    if (!table(m.zG, g64, g32, g4) || !table(m.zH, h64, h32, h4))
      return fail(SEM_ERR_ARG, "reference state: Exner pressure <= 0 below the lid");
    SEM_CUDA_TRY(cudaMemcpy(D.refG, g64.data(), g64.size() * sizeof(double), cudaMemcpyHostToDevice));
    SEM_CUDA_TRY(cudaMemcpy(D.refG32, g32.data(), g32.size() * sizeof(float), cudaMemcpyHostToDevice));
    SEM_CUDA_TRY(cudaMemcpy(D.ref4G, g4.data(), g4.size() * sizeof(float), cudaMemcpyHostToDevice));
    if (!h64.empty()) {
      SEM_CUDA_TRY(cudaMemcpy(D.refH, h64.data(), h64.size() * sizeof(double), cudaMemcpyHostToDevice));
      SEM_CUDA_TRY(cudaMemcpy(D.refH32, h32.data(), h32.size() * sizeof(float), cudaMemcpyHostToDevice));
      SEM_CUDA_TRY(cudaMemcpy(D.ref4H, h4.data(), h4.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
  }
  std::memcpy(D.ref_key, key, sizeof(key));
  D.ref_valid = true;
  return SEM_OK;
}

int check_params(const sem_params* p) {
  if (!p) return fail(SEM_ERR_ARG, "params is NULL");
  if (p->eqset != SEM_EQ_CONSERVATIVE && p->eqset != SEM_EQ_NONCONSERVATIVE)
    return fail(SEM_ERR_ARG, "unknown equation set");
  if (p->precision != SEM_PREC_FP64 && p->precision != SEM_PREC_MIXED)
    return fail(SEM_ERR_ARG, "unknown precision");
  if (p->n_thresholds < 0 || p->n_thresholds > SEM_MAX_THRESHOLDS)
    return fail(SEM_ERR_ARG, "n_thresholds out of range");
  if (!(p->smag_cs >= 0.0) || !(p->sponge_gamma >= 0.0) || (p->sponge_gamma > 0.0 && !(p->sponge_depth > 0.0)))
    return fail(SEM_ERR_ARG, "smag_cs and sponge_gamma must be >= 0, sponge_depth > 0");
  for (int k = 0; k < SEM_MAX_THRESHOLDS; ++k)
    if (p->criterion[k] < SEM_CRIT_SPEED || p->criterion[k] > SEM_CRIT_PV)
      return fail(SEM_ERR_ARG, "unknown criterion variable");
  if (!(p->heat_q0 >= 0.0) || (p->heat_q0 > 0.0 && !(p->heat_width > 0.0 && p->heat_ramp > 0.0 &&
                                                       p->heat_ztop > 0.0 && p->heat_rmax >= 0.0)) ||
      !std::isfinite(p->time))
    return fail(SEM_ERR_ARG, "heating needs heat_q0 >= 0, heat_width, heat_ramp, heat_ztop > 0; finite time");
  return SEM_OK;
}

static int prepare(sem_mesh* mh, const sem_params* p) {
  if (!mh) return fail(SEM_ERR_ARG, "mesh is NULL");
  int rc = check_params(p);
  if (rc) return rc;
  if ((rc = ensure_device(mh->m))) return rc;
  return ensure_reference(mh->m, *p);
}

}  // namespace sem

using namespace sem;

extern "C" {

const char* sem_last_error(void) { return g_err.c_str(); }

int sem_params_default(sem_params* p) {
  if (!p) return fail(SEM_ERR_ARG, "params is NULL");
  std::memset(p, 0, sizeof(*p));
  p->g = 9.81;
  p->f = 5.0e-5;
  p->R_d = 287.0;
  p->c_p = 1004.0;
  p->p00 = 1.0e5;
  p->theta_s = 300.0;
  p->N_bv = 0.01;
  p->eqset = SEM_EQ_CONSERVATIVE;
  p->precision = SEM_PREC_FP64;
  p->n_thresholds = 3;
  p->lvl_max = 3;
  p->thresholds[0] = 7.5;
  p->thresholds[1] = 15.0;
  p->thresholds[2] = 22.5;
  p->smag_cs = 0.0;
  p->sponge_gamma = 0.0;
  p->sponge_depth = 4000.0;
  p->heat_q0 = 0.0;
  p->heat_r0 = 27.5e3;
  p->heat_width = 10.0e3;
  p->heat_rmax = 60.0e3;
  p->heat_ztop = 15.0e3;
  p->heat_ramp = 600.0;
  p->time = 0.0;
  return SEM_OK;
}

int sem_mesh_create(const sem_mesh_desc* d, sem_mesh** out) {
  if (!d || !out) return fail(SEM_ERR_ARG, "NULL argument");
  *out = nullptr;
  if (d->nx <= 0 || d->ny <= 0 || d->nz <= 0 || !(d->Lx > 0) || !(d->Ly > 0) || !(d->Lz > 0))
    return fail(SEM_ERR_ARG, "sizes must be positive");
  if (d->N < 2 || d->N > kMaxN) return fail(SEM_ERR_UNSUPPORTED, "order N must be in 2..6");
  if (d->n_leaves < 0 || (d->n_leaves > 0 && !d->leaves)) return fail(SEM_ERR_ARG, "bad leaf list");
  if (d->lvl_max < 0 || d->lvl_max > 12) return fail(SEM_ERR_ARG, "lvl_max out of range");
  sem_mesh* mh = new (std::nothrow) sem_mesh();
  if (!mh) return fail(SEM_ERR_ARG, "out of host memory");
  Mesh& m = mh->m;
  m.Lx = d->Lx; m.Ly = d->Ly; m.Lz = d->Lz;
  m.nx = d->nx; m.ny = d->ny; m.nz = d->nz; m.N = d->N;
  m.px = d->periodic_x != 0; m.py = d->periodic_y != 0;
  m.lvl_max = d->lvl_max;
  m.zf.resize(m.nz + 1);
  if (d->z_faces) {
    for (int k = 0; k <= m.nz; ++k) m.zf[k] = d->z_faces[k];
    bool ok = m.zf[0] == 0.0 && m.zf[m.nz] == m.Lz;
    for (int k = 0; k < m.nz; ++k) ok = ok && m.zf[k + 1] > m.zf[k];
    if (!ok) {
      delete mh;
      return fail(SEM_ERR_ARG, "z_faces must rise strictly from 0 to Lz");
    }
  } else {
    for (int k = 0; k < m.nz; ++k) m.zf[k] = k * (m.Lz / m.nz);
    m.zf[m.nz] = m.Lz;
  }
  if (!std::isfinite(d->warp_amplitude) || (d->warp_amplitude != 0.0 && (d->warp_kx < 0 || d->warp_ky < 0))) {
    delete mh;
    return fail(SEM_ERR_ARG, "warp: finite amplitude and non-negative wave numbers");
  }
  m.warp_A = d->warp_amplitude;
  m.warp_kx = d->warp_kx;
  m.warp_ky = d->warp_ky;
  if (d->n_leaves == 0) {
    for (int j = 0; j < d->ny; ++j)
      for (int i = 0; i < d->nx; ++i) m.leaves.push_back({0, i, j});
  } else {
    for (int k = 0; k < d->n_leaves; ++k)
      m.leaves.push_back({d->leaves[3 * k], d->leaves[3 * k + 1], d->leaves[3 * k + 2]});
  }
  int rc = build_mesh(m);
  if (rc) {
    delete mh;
    return rc;
  }
  m.serial = ++g_serial;
  *out = mh;
  return SEM_OK;
}

void sem_mesh_destroy(sem_mesh* mh) {
  if (!mh) return;
  free_device(mh->m);
  delete mh;
}

int sem_mesh_get_info(const sem_mesh* mh, sem_mesh_info* o) {
  if (!mh || !o) return fail(SEM_ERR_ARG, "NULL argument");
  const Mesh& m = mh->m;
  std::memset(o, 0, sizeof(*o));
  o->Ne = m.Ne();
  o->NL = m.Ne() * m.P;
  o->NG = m.NG;
  o->NH = m.NH;
  o->NZ = m.NZ;
  o->Ncol = m.Ncol();
  o->n_hanging_h = (long long)m.hang_h.size() / (m.N + 1);
  o->n_nonconforming_faces = m.n_nonconf_sides;
  o->N = m.N;
  o->nz = m.nz;
  o->max_level = m.Lf;
  for (auto& f : m.leaves)
    if (f.l < 16) o->level_hist[f.l]++;
  return SEM_OK;
}

int sem_mesh_coords_host(const sem_mesh* mh, double* xyz) {
  if (!mh || !xyz) return fail(SEM_ERR_ARG, "NULL argument");
  const Mesh& m = mh->m;
  for (long long h = 0; h < m.NH; ++h)
    for (int k = 0; k < m.NZ; ++k) {
      long long g = h * m.NZ + k;
      xyz[g] = m.xh[h];
      xyz[m.NG + g] = m.yh[h];
      xyz[2 * m.NG + g] = m.warped() ? m.zG[g] : m.zk[k];
    }
  return SEM_OK;
}

int sem_mesh_leaves_host(const sem_mesh* mh, int* out) {
  if (!mh || !out) return fail(SEM_ERR_ARG, "NULL argument");
  const Mesh& m = mh->m;
  for (long long c = 0; c < m.Ncol(); ++c) {
    out[3 * c] = m.leaves[c].l;
    out[3 * c + 1] = m.leaves[c].i;
    out[3 * c + 2] = m.leaves[c].j;
  }
  return SEM_OK;
}

int sem_mesh_hmap_host(const sem_mesh* mh, int* hmap, int* hh, double* hw) {
  if (!mh) return fail(SEM_ERR_ARG, "NULL argument");
  const Mesh& m = mh->m;
  if (hmap) std::memcpy(hmap, m.hmap.data(), m.hmap.size() * sizeof(int));
  if (hh) std::memcpy(hh, m.hang_h.data(), m.hang_h.size() * sizeof(int));
  if (hw) std::memcpy(hw, m.hang_w.data(), m.hang_w.size() * sizeof(double));
  return SEM_OK;
}

int sem_mesh_mass_host(const sem_mesh* mh, double* M) {
  if (!mh || !M) return fail(SEM_ERR_ARG, "NULL argument");
  const Mesh& m = mh->m;
  for (long long h = 0; h < m.NH; ++h)
    for (int k = 0; k < m.NZ; ++k) M[h * m.NZ + k] = m.warped() ? m.Mg[h * m.NZ + k] : m.Mh[h] * m.Mz[k];
  return SEM_OK;
}

int sem_mesh_coords(sem_mesh* mh, double* xyz, cudaStream_t st) {
  if (!mh || !xyz) return fail(SEM_ERR_ARG, "NULL argument");
  int rc = ensure_device(mh->m);
  if (rc) return rc;
  return launch_coords(mh->m, xyz, st);
}

int sem_rhs(sem_mesh* mh, const sem_params* p, const double* q, double* rhs, cudaStream_t st) {
  int rc = prepare(mh, p);
  if (rc) return rc;
  if (!q || !rhs || q == rhs) return fail(SEM_ERR_ARG, "q and rhs must be distinct device arrays");
  StageArgs s{nullptr, q, rhs, nullptr, nullptr, 0.0, 0.0, 1.0, 1, nullptr};
  s.time = p->time;
  return launch_rhs_stage(mh->m, *p, s, st);
}

static const double kA[3] = {0.0, 0.75, 1.0 / 3.0};
static const double kB[3] = {1.0, 0.25, 2.0 / 3.0};
static const double kC[3] = {1.0, 0.25, 2.0 / 3.0};
static const double kT[3] = {0.0, 1.0, 0.5};   // stage times in units of dt

int sem_rk_stage(sem_mesh* mh, const sem_params* p, int stage, const double* qn,
                 const double* qs, double* qout, double dt, cudaStream_t st) {
  int rc = prepare(mh, p);
  if (rc) return rc;
  if (stage < 0 || stage > 2) return fail(SEM_ERR_ARG, "stage must be 0, 1 or 2");
  if (!qn || !qs || !qout || qout == qn || qout == qs)
    return fail(SEM_ERR_ARG, "qout must not alias qn or qs");
  StageArgs s{qn, qs, qout, nullptr, nullptr, kA[stage], kB[stage], kC[stage] * dt, 0, nullptr};
  s.time = p->time + kT[stage] * dt;
  return launch_rhs_stage(mh->m, *p, s, st);
}

int sem_rk_stage_mixed(sem_mesh* mh, const sem_params* p, int stage, const double* qn,
                       const double* qs, const float* qs32, double* qout, float* qout32,
                       double dt, cudaStream_t st) {
  int rc = prepare(mh, p);
  if (rc) return rc;
  if (p->precision != SEM_PREC_MIXED) return fail(SEM_ERR_ARG, "sem_rk_stage_mixed needs SEM_PREC_MIXED");
  if (stage < 0 || stage > 2) return fail(SEM_ERR_ARG, "stage must be 0, 1 or 2");
  if (!qn || !qs || !qs32 || !qout || !qout32 || qout == qn || qout == qs ||
      (const void*)qout32 == (const void*)qs32)
    return fail(SEM_ERR_ARG, "outputs must not alias inputs");
  StageArgs s{qn, qs, qout, qs32, qout32, kA[stage], kB[stage], kC[stage] * dt, 0, nullptr};
  s.time = p->time + kT[stage] * dt;
  return launch_rhs_stage(mh->m, *p, s, st);
}

int sem_step_mixed(sem_mesh* mh, const sem_params* p, double* q, float* q32, float* work32,
                   double dt, cudaStream_t st) {
  int rc = prepare(mh, p);
  if (rc) return rc;
  if (p->precision != SEM_PREC_MIXED) return fail(SEM_ERR_ARG, "sem_step_mixed needs SEM_PREC_MIXED");
  if (!q || !q32 || !work32) return fail(SEM_ERR_ARG, "NULL argument");
  if (mh->m.NG * kFields >= (1ll << 31)) return fail(SEM_ERR_ARG, "mesh too large for 32-bit indexing");
  return launch_step_mixed(mh->m, *p, q, q32, work32, dt, st);
}

int sem_autotune(sem_mesh* mh, const sem_params* p, const float* q32, int reps, sem_tune_out* out,
                 cudaStream_t st) {
  int rc = prepare(mh, p);
  if (rc) return rc;
  if (!q32 || !out || reps < 1) return fail(SEM_ERR_ARG, "bad argument");
  std::memset(out, 0, sizeof(*out));
  return autotune_pencil(mh->m, *p, q32, reps, out, st);
}

int sem_autotune_select(sem_mesh* mh, int eqset, int row) {
  if (!mh) return fail(SEM_ERR_ARG, "bad argument");
  if (eqset != SEM_EQ_CONSERVATIVE && eqset != SEM_EQ_NONCONSERVATIVE) return fail(SEM_ERR_ARG, "unknown equation set");
  return select_pencil(mh->m, eqset, row);
}

int sem_batch_create(sem_mesh* const* meshes, int n, sem_batch** out) {
  if (!meshes || !out || n <= 0) return fail(SEM_ERR_ARG, "bad argument");
  *out = nullptr;
  std::vector<Mesh*> ms(n);
  for (int k = 0; k < n; ++k) {
    if (!meshes[k]) return fail(SEM_ERR_ARG, "NULL mesh");
    ms[k] = &meshes[k]->m;
  }
  sem_batch* b = new (std::nothrow) sem_batch();
  if (!b) return fail(SEM_ERR_ARG, "out of host memory");
  int rc = batch_create(ms.data(), n, &b->impl);
  if (rc) {
    delete b;
    return rc;
  }
  b->n = n;
  cudaGetDevice(&b->dev);
  *out = b;
  return SEM_OK;
}

void sem_batch_destroy(sem_batch* b) {
  if (!b) return;
  batch_destroy(b->impl);
  delete b;
}

int sem_batch_step_mixed(sem_batch* b, const sem_params* p, double* const* q, float* const* q32,
                         float* const* work32, const double* dt, int use_graph, cudaStream_t st) {
  if (!b || !p || !q || !q32 || !work32 || !dt) return fail(SEM_ERR_ARG, "NULL argument");
  int rc = check_params(p);
  if (rc) return rc;
  if (p->precision != SEM_PREC_MIXED) return fail(SEM_ERR_ARG, "batched steps need SEM_PREC_MIXED");
  for (int k = 0; k < b->n; ++k)
    if (!q[k] || !q32[k] || !work32[k]) return fail(SEM_ERR_ARG, "NULL array");
  return batch_step_mixed(b->impl, *p, q, q32, work32, dt, use_graph, st);
}

int sem_batch_status(sem_batch* b, int* status, cudaStream_t st) {
  if (!b || !status) return fail(SEM_ERR_ARG, "NULL argument");
  return batch_status(b->impl, status, st);
}

int sem_mlp_create(unsigned long long seed, int max_rows, sem_mlp** out) {
  if (!out || max_rows <= 0) return fail(SEM_ERR_ARG, "bad argument");
  *out = nullptr;
  sem_mlp* m = new (std::nothrow) sem_mlp();
  if (!m) return fail(SEM_ERR_ARG, "out of host memory");
  int rc = mlp_create(seed, max_rows, &m->impl);
  if (rc) {
    delete m;
    return rc;
  }
  m->max_rows = max_rows;
  *out = m;
  return SEM_OK;
}

void sem_mlp_destroy(sem_mlp* m) {
  if (!m) return;
  mlp_destroy(m->impl);
  delete m;
}

int sem_mlp_param_count(void) { return mlp_param_count(); }

int sem_mlp_get_params(sem_mlp* m, float* host) {
  if (!m || !host) return fail(SEM_ERR_ARG, "NULL argument");
  return mlp_params(m->impl, host, 0, 0);
}

int sem_mlp_set_params(sem_mlp* m, const float* host) {
  if (!m || !host) return fail(SEM_ERR_ARG, "NULL argument");
  return mlp_params(m->impl, const_cast<float*>(host), 1, 0);
}

int sem_mlp_get_grads(sem_mlp* m, float* host) {
  if (!m || !host) return fail(SEM_ERR_ARG, "NULL argument");
  return mlp_params(m->impl, host, 0, 1);
}

int sem_mlp_features(sem_mesh* mh, const double* q, const float* scales, float* feats,
                     cudaStream_t st) {
  if (!mh || !q || !scales || !feats) return fail(SEM_ERR_ARG, "NULL argument");
  for (int f = 0; f < kFields; ++f)
    if (!(scales[f] != 0.0f)) return fail(SEM_ERR_ARG, "feature scales must be non-zero");
  int rc = ensure_device(mh->m);
  if (rc) return rc;
  return mlp_features_api(mh->m, q, scales, feats, st);
}

int sem_mlp_forward(sem_mlp* m, const float* feats, int n, float* prob, cudaStream_t st) {
  if (!m || !feats || !prob || n < 0) return fail(SEM_ERR_ARG, "bad argument");
  return mlp_forward_api(m->impl, feats, n, prob, nullptr, st);
}

int sem_mlp_predict_flags(sem_mlp* m, const float* feats, int n, int8_t* flags, cudaStream_t st) {
  if (!m || !feats || !flags || n < 0) return fail(SEM_ERR_ARG, "bad argument");
  return mlp_forward_api(m->impl, feats, n, nullptr, flags, st);
}

int sem_mlp_backward(sem_mlp* m, const float* feats, const int8_t* labels, const float* class_w,
                     int n, double* loss_host, cudaStream_t st) {
  if (!m || !feats || !labels || !class_w) return fail(SEM_ERR_ARG, "NULL argument");
  return mlp_backward_api(m->impl, feats, labels, class_w, n, loss_host, st);
}

int sem_mlp_adam(sem_mlp* m, float lr, cudaStream_t st) {
  if (!m || !(lr > 0)) return fail(SEM_ERR_ARG, "bad argument");
  return mlp_adam_api(m->impl, lr, st);
}

int sem_mlp_select_forward(sem_mlp* m, int tc) {
  if (!m) return fail(SEM_ERR_ARG, "NULL argument");
  return mlp_select_forward(m->impl, tc);
}

int sem_mlp_status(sem_mlp* m, int* status, cudaStream_t st) {
  if (!m || !status) return fail(SEM_ERR_ARG, "NULL argument");
  return mlp_status(m->impl, status, st);
}

// ---------------------------------------------------------------------------
// checkpoints: header, leaves, float64 state, FNV-1a checksum of everything
namespace {
const char kMagic[8] = {'S', 'E', 'M', 'C', 'K', 'P', 'T', '3'};
const char kMagicV2[8] = {'S', 'E', 'M', 'C', 'K', 'P', 'T', '2'};   // before warped layers
struct CkptHead {
  char magic[8];
  double Lx, Ly, Lz, time;
  int nx, ny, nz, N, px, py, lvl_max, pad;
  long long ncol, NG, step;
  double warp_A;              // warped layers (0: box elements)
  int warp_kx, warp_ky;
};
uint64_t fnv1a(const void* p, size_t n, uint64_t h = 1469598103934665603ull) {
  const unsigned char* c = (const unsigned char*)p;
  for (size_t i = 0; i < n; ++i) {
    h ^= c[i];
    h *= 1099511628211ull;
  }
  return h;
}
int read_ckpt(const char* path, CkptHead& H, std::vector<int>& leaves, std::vector<double>& zf,
              std::vector<double>* state) {
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(SEM_ERR_IO, std::string("cannot open ") + path);
  auto bad = [&](const char* why) {
    std::fclose(f);
    return fail(SEM_ERR_IO, std::string("checkpoint ") + path + ": " + why);
  };
  if (std::fread(&H, sizeof(H), 1, f) != 1) return bad("truncated header");
  if (std::memcmp(H.magic, kMagicV2, 8) == 0) return bad("written by an earlier version of the format");
  if (std::memcmp(H.magic, kMagic, 8) != 0) return bad("not a checkpoint");
  if (H.ncol <= 0 || H.ncol > (1ll << 30) || H.NG <= 0 || H.NG > (1ll << 36)) return bad("bad sizes");
  leaves.resize((size_t)H.ncol * 3);
  if (std::fread(leaves.data(), sizeof(int), leaves.size(), f) != leaves.size()) return bad("truncated leaves");
  if (H.nz <= 0 || H.nz > (1 << 20)) return bad("bad sizes");
  zf.resize((size_t)H.nz + 1);
  if (std::fread(zf.data(), sizeof(double), zf.size(), f) != zf.size()) return bad("truncated layer faces");
  uint64_t h = fnv1a(&H, sizeof(H));
  h = fnv1a(leaves.data(), leaves.size() * sizeof(int), h);
  h = fnv1a(zf.data(), zf.size() * sizeof(double), h);
  std::vector<double> tmp;
  std::vector<double>& q = state ? *state : tmp;
  q.resize((size_t)H.NG * kFields);
  if (std::fread(q.data(), sizeof(double), q.size(), f) != q.size()) return bad("truncated state");
  h = fnv1a(q.data(), q.size() * sizeof(double), h);
  uint64_t stored = 0;
  if (std::fread(&stored, sizeof(stored), 1, f) != 1) return bad("missing checksum");
  std::fclose(f);
  if (stored != h) return fail(SEM_ERR_IO, std::string("checkpoint ") + path + ": checksum mismatch");
  return SEM_OK;
}
}  // namespace

int sem_checkpoint_write(sem_mesh* mh, const double* q, double time, long long step, const char* path,
                         cudaStream_t st) {
  if (!mh || !q || !path) return fail(SEM_ERR_ARG, "NULL argument");
  const Mesh& m = mh->m;
  CkptHead H;
  std::memset(&H, 0, sizeof(H));
  std::memcpy(H.magic, kMagic, 8);
  H.Lx = m.Lx; H.Ly = m.Ly; H.Lz = m.Lz; H.time = time;
  H.nx = m.nx; H.ny = m.ny; H.nz = m.nz; H.N = m.N; H.px = m.px; H.py = m.py; H.lvl_max = m.lvl_max;
  H.ncol = m.Ncol(); H.NG = m.NG; H.step = step;
  H.warp_A = m.warp_A; H.warp_kx = m.warp_kx; H.warp_ky = m.warp_ky;
  std::vector<int> leaves((size_t)m.Ncol() * 3);
  for (long long c = 0; c < m.Ncol(); ++c) {
    leaves[3 * c] = m.leaves[c].l;
    leaves[3 * c + 1] = m.leaves[c].i;
    leaves[3 * c + 2] = m.leaves[c].j;
  }
  std::vector<double> host((size_t)m.NG * kFields);
  SEM_CUDA_TRY(cudaMemcpyAsync(host.data(), q, host.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  SEM_CUDA_TRY(cudaStreamSynchronize(st));
  uint64_t h = fnv1a(&H, sizeof(H));
  h = fnv1a(leaves.data(), leaves.size() * sizeof(int), h);
  h = fnv1a(m.zf.data(), m.zf.size() * sizeof(double), h);
  h = fnv1a(host.data(), host.size() * sizeof(double), h);
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return fail(SEM_ERR_IO, "cannot create " + tmp);
  bool ok = std::fwrite(&H, sizeof(H), 1, f) == 1 &&
            std::fwrite(leaves.data(), sizeof(int), leaves.size(), f) == leaves.size() &&
            std::fwrite(m.zf.data(), sizeof(double), m.zf.size(), f) == m.zf.size() &&
            std::fwrite(host.data(), sizeof(double), host.size(), f) == host.size() &&
            std::fwrite(&h, sizeof(h), 1, f) == 1;
  ok = (std::fclose(f) == 0) && ok;
  if (!ok || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return fail(SEM_ERR_IO, std::string("cannot write ") + path);
  }
  return SEM_OK;
}

int sem_checkpoint_read_mesh(const char* path, sem_mesh** out, double* time, long long* step) {
  if (!path || !out) return fail(SEM_ERR_ARG, "NULL argument");
  *out = nullptr;
  CkptHead H;
  std::vector<int> leaves;
  std::vector<double> zf;
  int rc = read_ckpt(path, H, leaves, zf, nullptr);
  if (rc) return rc;
  sem_mesh_desc d;
  std::memset(&d, 0, sizeof(d));
  d.Lx = H.Lx; d.Ly = H.Ly; d.Lz = H.Lz; d.nx = H.nx; d.ny = H.ny; d.nz = H.nz; d.N = H.N;
  d.periodic_x = H.px; d.periodic_y = H.py; d.lvl_max = H.lvl_max;
  d.n_leaves = (int)H.ncol;
  d.leaves = leaves.data();
  d.z_faces = zf.data();
  d.warp_amplitude = H.warp_A;
  d.warp_kx = H.warp_kx;
  d.warp_ky = H.warp_ky;
  if ((rc = sem_mesh_create(&d, out))) return rc;
  if ((*out)->m.NG != H.NG) {
    sem_mesh_destroy(*out);
    *out = nullptr;
    return fail(SEM_ERR_IO, "checkpoint node count does not match its mesh");
  }
  if (time) *time = H.time;
  if (step) *step = H.step;
  return SEM_OK;
}

int sem_checkpoint_read_state(const char* path, sem_mesh* mh, double* q, cudaStream_t st) {
  if (!path || !mh || !q) return fail(SEM_ERR_ARG, "NULL argument");
  CkptHead H;
  std::vector<int> leaves;
  std::vector<double> host, zf;
  int rc = read_ckpt(path, H, leaves, zf, &host);
  if (rc) return rc;
  const Mesh& m = mh->m;
  bool same = H.NG == m.NG && H.ncol == m.Ncol() && zf == m.zf && H.warp_A == m.warp_A &&
              (m.warp_A == 0.0 || (H.warp_kx == m.warp_kx && H.warp_ky == m.warp_ky));
  for (long long c = 0; same && c < m.Ncol(); ++c)
    same = leaves[3 * c] == m.leaves[c].l && leaves[3 * c + 1] == m.leaves[c].i &&
           leaves[3 * c + 2] == m.leaves[c].j;
  if (!same) return fail(SEM_ERR_ARG, "checkpoint was written for another mesh");
  SEM_CUDA_TRY(cudaMemcpyAsync(q, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  SEM_CUDA_TRY(cudaStreamSynchronize(st));
  return SEM_OK;
}

int sem_mirror(sem_mesh* mh, const double* q, float* q32, cudaStream_t st) {
  if (!mh || !q || !q32) return fail(SEM_ERR_ARG, "NULL argument");
  int rc = ensure_device(mh->m);
  if (rc) return rc;
  return launch_mirror(q, q32, (long long)kFields * mh->m.NG, st);
}

int sem_step(sem_mesh* mh, const sem_params* p, double* q, double* w1, double* w2, double dt,
             cudaStream_t st) {
  if (!q || !w1 || !w2 || q == w1 || q == w2 || w1 == w2)
    return fail(SEM_ERR_ARG, "q, w1, w2 must be distinct");
  int rc;
  if ((rc = sem_rk_stage(mh, p, 0, q, q, w1, dt, st))) return rc;
  if ((rc = sem_rk_stage(mh, p, 1, q, w1, w2, dt, st))) return rc;
  // the last stage writes w1 and copies it back into q
  if ((rc = sem_rk_stage(mh, p, 2, q, w2, w1, dt, st))) return rc;
  SEM_CUDA_TRY(cudaMemcpyAsync(q, w1, (size_t)mh->m.NG * kFields * sizeof(double),
                               cudaMemcpyDeviceToDevice, st));
  return SEM_OK;
}

int sem_adapt_flags(sem_mesh* mh, const sem_params* p, const double* q, int8_t* flags,
                    double* cmax, cudaStream_t st) {
  int rc = prepare(mh, p);
  if (rc) return rc;
  if (!q || !flags) return fail(SEM_ERR_ARG, "NULL argument");
  if (p->lvl_max > p->n_thresholds) return fail(SEM_ERR_ARG, "need one threshold per level");
  return launch_adapt(mh->m, *p, q, flags, cmax, st);
}

int sem_adapt_flags_levels(sem_mesh* mh, const sem_params* p, const double* q, const int8_t* level,
                           int level_all, int8_t* flags, double* cmax, cudaStream_t st) {
  int rc = prepare(mh, p);
  if (rc) return rc;
  if (!q || !flags) return fail(SEM_ERR_ARG, "NULL argument");
  if (p->lvl_max > p->n_thresholds) return fail(SEM_ERR_ARG, "need one threshold per level");
  if (!level && (level_all < 0 || level_all > p->lvl_max))
    return fail(SEM_ERR_ARG, "level_all must be in 0..lvl_max when no level array is given");
  return launch_adapt(mh->m, *p, q, flags, cmax, st, level, level ? -1 : level_all);
}

int sem_merge_flags(const int8_t* crit, const int8_t* pred, const int8_t* level, int lvl_max, long long n,
                    int8_t* out, cudaStream_t st) {
  if (n < 0 || (n > 0 && (!crit || !pred || !level || !out))) return fail(SEM_ERR_ARG, "NULL argument");
  if (lvl_max < 0) return fail(SEM_ERR_ARG, "lvl_max must be >= 0");
  if (n == 0) return SEM_OK;
  return launch_merge_flags(crit, pred, level, lvl_max, n, out, st);
}

int sem_adapt_flags_host(sem_mesh* mh, const sem_params* p, const double* q, int8_t* flags_host,
                         cudaStream_t st) {
  int rc = prepare(mh, p);
  if (rc) return rc;
  if (!flags_host) return fail(SEM_ERR_ARG, "NULL argument");
  int8_t* dflags = mh->m.dev->elem_flags;
  rc = sem_adapt_flags(mh, p, q, dflags, nullptr, st);
  if (rc) return rc;
  SEM_CUDA_TRY(cudaMemcpyAsync(flags_host, dflags, (size_t)mh->m.Ne(), cudaMemcpyDeviceToHost, st));
  SEM_CUDA_TRY(cudaStreamSynchronize(st));
  return SEM_OK;
}

int sem_transfer_plan(const sem_mesh* oldh, const int8_t* flags, sem_mesh** out) {
  if (!oldh || !flags || !out) return fail(SEM_ERR_ARG, "NULL argument");
  *out = nullptr;
  const Mesh& o = oldh->m;
  if (o.warped()) return fail(SEM_ERR_UNSUPPORTED, "adaptation of warped meshes is not built");
  std::vector<Leaf> nl;
  std::vector<Origin> org;
  int rc = adapt_leaves(o, flags, nl, org);
  if (rc) return rc;
  sem_mesh* nh = new (std::nothrow) sem_mesh();
  if (!nh) return fail(SEM_ERR_ARG, "out of host memory");
  Mesh& m = nh->m;
  m.Lx = o.Lx; m.Ly = o.Ly; m.Lz = o.Lz;
  m.nx = o.nx; m.ny = o.ny; m.nz = o.nz; m.N = o.N;
  m.px = o.px; m.py = o.py; m.lvl_max = o.lvl_max;
  m.zf = o.zf;
  m.leaves = nl;
  rc = build_mesh(m);   // sorts the leaves into Morton order
  if (rc) {
    delete nh;
    return rc;
  }
  // carry the provenance over to the sorted order
  m.origin.resize(m.leaves.size());
  {
    std::vector<std::pair<long long, int>> idx;
    auto key = [](const Leaf& f) { return ((long long)f.l << 50) | ((long long)f.i << 25) | f.j; };
    std::vector<std::pair<long long, int>> a;
    for (size_t k = 0; k < nl.size(); ++k) a.push_back({key(nl[k]), (int)k});
    std::sort(a.begin(), a.end());
    for (size_t c = 0; c < m.leaves.size(); ++c) {
      auto it = std::lower_bound(a.begin(), a.end(), std::make_pair(key(m.leaves[c]), -1));
      m.origin[c] = org[it->second];
    }
  }
  m.parent_serial = o.serial;
  m.serial = ++g_serial;
  *out = nh;
  return SEM_OK;
}

int sem_transfer(sem_mesh* oldh, sem_mesh* newh, const double* qold, double* qnew, cudaStream_t st) {
  if (!oldh || !newh || !qold || !qnew) return fail(SEM_ERR_ARG, "NULL argument");
  if (newh->m.parent_serial != oldh->m.serial || newh->m.origin.empty())
    return fail(SEM_ERR_ARG, "new mesh was not planned from this old mesh");
  int rc;
  if ((rc = ensure_device(oldh->m)) || (rc = ensure_device(newh->m))) return rc;
  return launch_transfer(oldh->m, newh->m, qold, qnew, st);
}

int sem_diag(sem_mesh* mh, const sem_params* p, const double* q, double half_width,
             sem_diag_out* out, cudaStream_t st) {
  int rc = prepare(mh, p);
  if (rc) return rc;
  if (!q || !out) return fail(SEM_ERR_ARG, "NULL argument");
  return launch_diag(mh->m, *p, q, half_width, out, st);
}

int sem_status(sem_mesh* mh, int* status, cudaStream_t st) {
  if (!mh || !status) return fail(SEM_ERR_ARG, "NULL argument");
  int rc = ensure_device(mh->m);
  if (rc) return rc;
  int v = 0;
  SEM_CUDA_TRY(cudaMemcpyAsync(&v, mh->m.dev->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  SEM_CUDA_TRY(cudaMemsetAsync(mh->m.dev->status, 0, sizeof(int), st));
  SEM_CUDA_TRY(cudaStreamSynchronize(st));
  *status = (v & 4) ? SEM_ERR_TIMEOUT : (v ? SEM_ERR_NUMERIC : SEM_OK);
  return SEM_OK;
}

}  // extern "C"

extern "C" int sem_selftest_device_once(int n_devices, int n_threads, int* calls) {
  if (n_devices < 1 || n_devices > kMaxDevices || n_threads < 1 || n_threads > 64 || !calls)
    return fail(SEM_ERR_ARG, "n_devices and n_threads must be in 1..64, calls non-NULL");
  DeviceOnce once;
  std::vector<std::atomic<int>> cnt(n_devices);
  for (auto& c : cnt) c.store(0);
  std::atomic<int> bad{0};
  std::vector<std::thread> th;
  for (int t = 0; t < n_threads; ++t)
    th.emplace_back([&, t] {
      for (int rep = 0; rep < 3; ++rep)
        for (int k = 0; k < n_devices; ++k) {
          const int d = (k + t * 7 + rep) % n_devices;
          const int rc = device_once_on(once, d, [&] {
            cnt[d].fetch_add(1);
            std::this_thread::yield();
            return (int)SEM_OK;
          });
          if (rc != SEM_OK) bad.fetch_add(1);
        }
    });
  for (auto& x : th) x.join();
  for (int d = 0; d < n_devices; ++d) calls[d] = cnt[d].load();
  // ordinals beyond the table are refused, and a failed set-up runs again
  int ran = 0;
  if (device_once_on(once, kMaxDevices, [&] { ++ran; return (int)SEM_OK; }) != SEM_ERR_ARG || ran)
    return fail(SEM_ERR_ARG, "device_once accepted an ordinal outside the table");
  DeviceOnce again;
  device_once_on(again, 0, [] { return (int)SEM_ERR_CUDA; });
  if (device_once_on(again, 0, [&] { ++ran; return (int)SEM_OK; }) != SEM_OK || ran != 1)
    return fail(SEM_ERR_ARG, "device_once did not retry a failed set-up");
  if (bad.load()) return fail(SEM_ERR_ARG, "device_once failed on a valid ordinal");
  return SEM_OK;
}

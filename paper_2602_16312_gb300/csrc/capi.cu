// C ABI of libaggmg (declared in include/aggmg.h): argument checking, the
// host set-up calls and dispatch to the per-block-size device engines.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <string>

#include "../../include/aggmg.h"
#include "cg_kernels.cuh"
#include "engine.h"
#include "handles.h"
#include "setup.h"

namespace aggmg {
EngineBase* make_engine_b4(int);
EngineBase* make_engine_b8(int);
EngineBase* make_engine_b9(int);
EngineBase* make_engine_b16(int);
EngineBase* make_engine_b27_f64();
EngineBase* make_engine_b27_f32();
EngineBase* make_engine_b27_bf16();
EngineBase* make_engine_b64_f64();
EngineBase* make_engine_b64_f32();
EngineBase* make_engine_b64_bf16();

static EngineBase* make_engine_b27(int precision) {
  switch (precision) {
    case AGG_F64: return make_engine_b27_f64();
    case AGG_F32: return make_engine_b27_f32();
    case AGG_F32_BF16SMOOTH: return make_engine_b27_bf16();
    default: return nullptr;
  }
}

static EngineBase* make_engine_b64(int precision) {
  switch (precision) {
    case AGG_F64: return make_engine_b64_f64();
    case AGG_F32: return make_engine_b64_f32();
    case AGG_F32_BF16SMOOTH: return make_engine_b64_bf16();
    default: return nullptr;
  }
}

EngineBase* make_engine(int B, int precision) {
  switch (B) {
    case 4: return make_engine_b4(precision);
    case 8: return make_engine_b8(precision);
    case 9: return make_engine_b9(precision);
    case 16: return make_engine_b16(precision);
    case 27: return make_engine_b27(precision);
    case 64: return make_engine_b64(precision);
    default: return nullptr;
  }
}
}  // namespace aggmg

using namespace aggmg;



struct agg_sim {
  agg_hier* h = nullptr;
  int64_t clock = 0;
};

namespace {
thread_local std::string g_err;

agg_status fail(agg_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

}  // namespace

namespace aggmg {
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace aggmg

namespace {
agg_status check_device(const agg_hier* h) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(AGG_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev != h->device) return fail(AGG_EINVAL, "current device differs from the hierarchy's device");
  return AGG_OK;
}
}  // namespace

extern "C" {

const char* agg_last_error(void) { return g_err.c_str(); }

const char* agg_status_string(int s) {
  switch (s) {
    case AGG_OK: return "ok";
    case AGG_EINVAL: return "invalid argument";
    case AGG_ENOMEM: return "out of memory";
    case AGG_ECUDA: return "CUDA error";
    case AGG_ENOTSPD: return "matrix not symmetric positive definite";
    case AGG_ENOTCONV: return "PCG did not converge within max_it";
    case AGG_ENAN: return "NaN or Inf in the residual";
    case AGG_EUNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
  }
}

agg_status agg_dg_mesh_create(const agg_mesh_desc* d, agg_mesh_t* out) {
  if (!d || !out) return fail(AGG_EINVAL, "NULL argument");
  if (!d->vertices || !d->elements || !d->conductivity) return fail(AGG_EINVAL, "NULL mesh array");
  if (d->n_vertices <= 0 || d->n_elements <= 0) return fail(AGG_EINVAL, "empty mesh");
  if (d->dim != 2 && d->dim != 3) return fail(AGG_EINVAL, "dim must be 2 or 3");
  if (d->penalty_mode != 0 && d->penalty_mode != 1) return fail(AGG_EINVAL, "penalty_mode must be 0 or 1");
  std::unique_ptr<agg_mesh> mh;
  try {
    mh.reset(new agg_mesh());
    Mesh& m = mh->m;
    m.dim = d->dim;
    m.p = d->degree;
    m.nv = d->n_vertices;
    m.ne = d->n_elements;
    const int V = 1 << d->dim;
    m.X.assign(d->vertices, d->vertices + d->n_vertices * d->dim);
    m.cells.assign(d->elements, d->elements + d->n_elements * V);
    m.D.assign(d->conductivity, d->conductivity + d->n_elements * d->dim * d->dim);
    if (d->theta || d->theta_map || d->n_theta) {
      if (!d->theta || !d->theta_map || d->n_theta <= 0) return fail(AGG_EINVAL, "theta needs theta, theta_map and n_theta > 0");
      m.theta.assign(d->theta, d->theta + d->n_theta);
      m.theta_map.assign(d->theta_map, d->theta_map + d->n_elements);
      for (double t : m.theta)
        if (!(t > 0.0) || !std::isfinite(t)) return fail(AGG_EINVAL, "theta must be finite and > 0");
      const int dd = d->dim * d->dim;
      for (int64_t e = 0; e < d->n_elements; ++e) {
        const int32_t k = m.theta_map[e];
        if (k < 0 || k >= d->n_theta) return fail(AGG_EINVAL, "theta_map entry out of range");
        for (int i = 0; i < dd; ++i) m.D[(size_t)e * dd + i] *= m.theta[k];
      }
    }
    m.penalty_mode = d->penalty_mode;
    m.penalty_coeff = d->penalty_coeff;
    m.quad_extra = d->quad_extra;
    m.adjoint_data = d->adjoint_data != 0;
    std::string err;
    int s = mesh_build(m, err);
    if (s) return fail((agg_status)s, err);
  } catch (const std::bad_alloc&) {
    return fail(AGG_ENOMEM, "host allocation failed");
  }
  *out = mh.release();
  return AGG_OK;
}

agg_status agg_dg_mesh_destroy(agg_mesh_t m) {
  delete m;
  return AGG_OK;
}

agg_status agg_dg_mesh_info(agg_mesh_t m, int64_t* n_dofs, int64_t* n_faces) {
  if (!m) return fail(AGG_EINVAL, "NULL mesh");
  if (n_dofs) *n_dofs = m->m.ne * m->m.B;
  if (n_faces) *n_faces = m->m.n_faces;
  return AGG_OK;
}

agg_status agg_dg_mesh_locate(agg_mesh_t mh, int64_t n, const double* pts, int64_t* elem, double* weights) {
  if (!mh || n < 0 || (n > 0 && (!pts || !elem || !weights))) return fail(AGG_EINVAL, "bad argument");
  std::string err;
  int rc = mesh_locate(mh->m, n, pts, elem, weights, err);
  if (rc) return fail((agg_status)rc, err);
  return AGG_OK;
}

agg_status agg_rtree_agglomerate(agg_mesh_t mh, int max_entries, int n_maps, int32_t* const* maps,
                                 int64_t* n_units, int* tree_levels) {
  if (!mh || n_maps < 0) return fail(AGG_EINVAL, "bad argument");
  std::string err;
  int rc = rtree_agglomerate(mh->m, max_entries, n_maps, maps, n_units, tree_levels, err);
  if (rc) return fail((agg_status)rc, err);
  return AGG_OK;
}

agg_status agg_dg_mesh_nnzb(agg_mesh_t m, int64_t* nnzb) {
  if (!m || !nnzb) return fail(AGG_EINVAL, "NULL argument");
  *nnzb = m->m.A.nnzb();
  return AGG_OK;
}

agg_status agg_dg_mesh_copy(agg_mesh_t mh, int what, void* dst) {
  if (!mh || !dst) return fail(AGG_EINVAL, "NULL argument");
  const Mesh& m = mh->m;
  switch (what) {
    case 0: std::memcpy(dst, m.A.rowptr.data(), sizeof(int64_t) * m.A.rowptr.size()); break;
    case 1: std::memcpy(dst, m.A.col.data(), sizeof(int32_t) * m.A.col.size()); break;
    case 2: std::memcpy(dst, m.A.val.data(), sizeof(double) * m.A.val.size()); break;
    case 3: std::memcpy(dst, m.Me.data(), sizeof(double) * m.Me.size()); break;
    case 4: std::memcpy(dst, m.vol.data(), sizeof(double) * m.vol.size()); break;
    case 5:
    case 6:
      if (!m.adjoint_data) return fail(AGG_EINVAL, "mesh has no adjoint data");
      if (what == 5) std::memcpy(dst, m.Ke.data(), sizeof(double) * m.Ke.size());
      else adjoint_face_parts_full(m, static_cast<double*>(dst));
      break;
    default: return fail(AGG_EINVAL, "what");
  }
  return AGG_OK;
}

void agg_mg_opts_default(agg_mg_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->n_levels = 1;
  o->smoother_degree = 3;
  o->block_jacobi = 1;
  o->lanczos_steps = 12;
  o->cheb_upper_safety = 1.2;
  o->cheb_range = 20.0;
  o->vcycle_precision = AGG_F64;
  o->fine_operator = 0;
  o->coarse_persistent = 0;
  o->coarse_cluster = 0;
  o->coarse_operator = 0;
}

static agg_status check_mg_opts(const agg_mg_opts* o, double mass_coeff);
static HierOptions host_options(const agg_mg_opts* o);

agg_status agg_mg_hierarchy_setup(agg_mesh_t mesh, double mass_coeff, const agg_mg_opts* o, void* stream,
                                  agg_hier_t* out) {
  if (!mesh || !out) return fail(AGG_EINVAL, "NULL argument");
  agg_status chk = check_mg_opts(o, mass_coeff);
  if (chk) return chk;
  const Mesh& m = mesh->m;
  std::unique_ptr<agg_hier> h(new agg_hier());
  h->mesh = mesh;
  cudaError_t ce = cudaGetDevice(&h->device);
  if (ce != cudaSuccess) return fail(AGG_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(ce));
  h->L = o->n_levels;
  h->B = m.B;
  h->precision = o->vcycle_precision;
  h->mass_coeff = mass_coeff;
  std::unique_ptr<EngineBase> eng(make_engine(m.B, o->vcycle_precision));
  if (!eng) return fail(AGG_EUNSUPPORTED, "no engine for this element block size (B = " + std::to_string(m.B) + ")");
  std::string err;
  try {
    HostHierarchy hh;
    int s = hierarchy_build(m, mass_coeff, host_options(o), hh, err);
    if (s) return fail((agg_status)s, err);
    for (int l = 0; l < hh.L; ++l) {
      h->units.push_back(hh.lev[l].n);
      h->nnzb.push_back(hh.lev[l].A.nnzb());
      h->lam_max.push_back(hh.lev[l].lam_max);
    }
    h->perm0 = hh.lev[0].perm;
    s = eng->init(hh, m, o->vcycle_precision, o->fine_operator, o->coarse_persistent, o->coarse_cluster,
                  (cudaStream_t)stream, err);
    if (s) return fail((agg_status)s, err);
  } catch (const std::bad_alloc&) {
    return fail(AGG_ENOMEM, "host allocation failed");
  }
  h->eng = eng.release();
  *out = h.release();
  return AGG_OK;
}

agg_status agg_mg_hierarchy_destroy(agg_hier_t h) {
  if (!h) return AGG_OK;
  for (void* p : {(void*)h->d_tptr, (void*)h->d_tmem, (void*)h->d_theta})
    if (p) cudaFree(p);
  delete h->eng;
  delete h;
  return AGG_OK;
}

agg_status agg_hier_stats(agg_hier_t h, int* n_levels, int64_t* units, int64_t* nnzb, double* lambda_max,
                          double* op_complexity) {
  if (!h) return fail(AGG_EINVAL, "NULL hierarchy");
  if (n_levels) *n_levels = h->L;
  double tot = 0;
  for (int l = 0; l < h->L; ++l) {
    if (units) units[l] = h->units[l];
    if (nnzb) nnzb[l] = h->nnzb[l];
    if (lambda_max && l + 1 < h->L) lambda_max[l] = h->lam_max[l];
    tot += (double)h->nnzb[l];
  }
  if (op_complexity) *op_complexity = tot / (double)h->nnzb[0];
  return AGG_OK;
}

struct agg_host_hier {
  HostHierarchy h;
};

static agg_status check_mg_opts(const agg_mg_opts* o, double mass_coeff) {
  if (!o) return fail(AGG_EINVAL, "NULL options");
  if (o->n_levels < 1) return fail(AGG_EINVAL, "n_levels must be >= 1");
  if (o->n_levels > 1 && !o->agg_maps) return fail(AGG_EINVAL, "agg_maps is NULL");
  if (o->smoother_degree != 3) return fail(AGG_EUNSUPPORTED, "smoother_degree must be 3");
  if (o->vcycle_precision < AGG_F64 || o->vcycle_precision > AGG_F32_BF16SMOOTH)
    return fail(AGG_EINVAL, "vcycle_precision");
  if (!(o->cheb_upper_safety > 0) || !(o->cheb_range > 1) || o->lanczos_steps < 1)
    return fail(AGG_EINVAL, "Chebyshev options");
  if (!(mass_coeff >= 0) || !std::isfinite(mass_coeff)) return fail(AGG_EINVAL, "mass_coeff");
  if (o->fine_operator != 0 && o->fine_operator != 1) return fail(AGG_EINVAL, "fine_operator");
  if (o->coarse_persistent != 0 && o->coarse_persistent != 1) return fail(AGG_EINVAL, "coarse_persistent");
  if (o->coarse_cluster != 0 && o->coarse_cluster != 1) return fail(AGG_EINVAL, "coarse_cluster");
  if (o->coarse_operator != 0 && o->coarse_operator != 1) return fail(AGG_EINVAL, "coarse_operator");
  return AGG_OK;
}

static HierOptions host_options(const agg_mg_opts* o) {
  HierOptions ho;
  ho.L = o->n_levels;
  ho.maps = o->agg_maps;
  ho.degree = o->smoother_degree;
  ho.block_jacobi = o->block_jacobi != 0;
  ho.lanczos_steps = o->lanczos_steps;
  ho.safety = o->cheb_upper_safety;
  ho.range = o->cheb_range;
  ho.direct = o->coarse_operator == 1;
  return ho;
}

agg_status agg_host_hierarchy_build(agg_mesh_t mesh, double mass_coeff, const agg_mg_opts* o, agg_host_hier_t* out) {
  if (!mesh || !out) return fail(AGG_EINVAL, "NULL argument");
  agg_status s = check_mg_opts(o, mass_coeff);
  if (s) return s;
  std::unique_ptr<agg_host_hier> hh;
  try {
    hh.reset(new agg_host_hier());
    std::string err;
    int rc = hierarchy_build(mesh->m, mass_coeff, host_options(o), hh->h, err);
    if (rc) return fail((agg_status)rc, err);
  } catch (const std::bad_alloc&) {
    return fail(AGG_ENOMEM, "host allocation failed");
  }
  *out = hh.release();
  return AGG_OK;
}

agg_status agg_host_hierarchy_destroy(agg_host_hier_t hh) {
  delete hh;
  return AGG_OK;
}

agg_status agg_host_hierarchy_level(agg_host_hier_t hh, int l, int64_t* n, int64_t* nnzb, double* lam) {
  if (!hh || l < 0 || l >= hh->h.L) return fail(AGG_EINVAL, "level");
  const HostLevel& v = hh->h.lev[l];
  if (n) *n = v.n;
  if (nnzb) *nnzb = v.A.nnzb();
  if (lam) *lam = v.lam_max;
  return AGG_OK;
}

agg_status agg_host_hierarchy_copy(agg_host_hier_t hh, int l, int what, void* dst) {
  if (!hh || !dst || l < 0 || l >= hh->h.L) return fail(AGG_EINVAL, "bad argument");
  const HostLevel& v = hh->h.lev[l];
  switch (what) {
    case 0: std::memcpy(dst, v.perm.data(), sizeof(int64_t) * v.perm.size()); break;
    case 1: std::memcpy(dst, v.A.rowptr.data(), sizeof(int64_t) * v.A.rowptr.size()); break;
    case 2: std::memcpy(dst, v.A.col.data(), sizeof(int32_t) * v.A.col.size()); break;
    case 3: std::memcpy(dst, v.A.val.data(), sizeof(double) * v.A.val.size()); break;
    case 4:
      if (v.Dinv.empty()) return fail(AGG_EINVAL, "no smoother on the coarsest level");
      std::memcpy(dst, v.Dinv.data(), sizeof(double) * v.Dinv.size());
      break;
    case 5:
      if (v.P.empty()) return fail(AGG_EINVAL, "no prolongation from the coarsest level");
      std::memcpy(dst, v.P.data(), sizeof(double) * v.P.size());
      break;
    case 6:
      if (v.parent.empty()) return fail(AGG_EINVAL, "no parent on the coarsest level");
      std::memcpy(dst, v.parent.data(), sizeof(int32_t) * v.parent.size());
      break;
    default: return fail(AGG_EINVAL, "what");
  }
  return AGG_OK;
}

static agg_status check_pcg_opts(const agg_pcg_opts* o) {
  if (!o) return fail(AGG_EINVAL, "NULL pcg options");
  if (!(o->rtol >= 0) || !(o->atol >= 0) || o->max_it < 1) return fail(AGG_EINVAL, "pcg options");
  return AGG_OK;
}

agg_status agg_pcg_solve(agg_hier_t h, const double* b, double* x, const agg_pcg_opts* o, agg_pcg_result* res,
                         void* stream) {
  if (!h || !b || !x) return fail(AGG_EINVAL, "NULL argument");
  agg_status s = check_pcg_opts(o);
  if (s) return s;
  if ((s = check_device(h))) return s;
  SolveOpts so;
  so.rtol = o->rtol;
  so.atol = o->atol;
  so.max_it = o->max_it;
  so.flexible = o->flexible;
  SolveResult r;
  std::string err;
  int rc = h->eng->pcg_solve(b, x, so, r, (cudaStream_t)stream, err);
  if (rc) return fail((agg_status)rc, err);
  if (res) {
    res->iterations = r.iterations;
    res->r0_norm = r.r0;
    res->r_norm = r.rn;
    res->status = r.status;
  }
  if (r.status) return fail((agg_status)r.status, agg_status_string(r.status));
  return AGG_OK;
}

agg_status agg_operator_apply(agg_hier_t h, int level, const double* x, double* y, void* stream) {
  if (!h || !x || !y) return fail(AGG_EINVAL, "NULL argument");
  agg_status s = check_device(h);
  if (s) return s;
  std::string err;
  int rc = h->eng->apply_level(level, x, y, (cudaStream_t)stream, err);
  if (rc) return fail((agg_status)rc, err);
  return AGG_OK;
}

agg_status agg_vcycle_apply(agg_hier_t h, const double* r, double* z, void* stream) {
  if (!h || !r || !z) return fail(AGG_EINVAL, "NULL argument");
  agg_status s = check_device(h);
  if (s) return s;
  std::string err;
  int rc = h->eng->vcycle_apply(r, z, (cudaStream_t)stream, err);
  if (rc) return fail((agg_status)rc, err);
  return AGG_OK;
}

agg_status agg_ionic_update(const agg_ionic_params* p, double dt, int64_t n, const double* u, double* w,
                            void* stream) {
  if (!p || (n > 0 && (!u || !w))) return fail(AGG_EINVAL, "NULL argument");
  if (n < 0) return fail(AGG_EINVAL, "n < 0");
  if (p->model < AGG_FHN || p->model > AGG_BUENO_OROVIO) return fail(AGG_EINVAL, "ionic model");
  if (n == 0) return AGG_OK;
  IonicParams ip{p->model, p->k, p->a, p->eps, p->gamma, p->mu1, p->mu2, p->bo};
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 16);
  k_ionic_update<<<blocks, 256, 0, (cudaStream_t)stream>>>(ip, dt, n, u, w);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(AGG_ECUDA, cudaGetErrorString(e));
  return AGG_OK;
}

agg_status agg_monodomain_create(agg_hier_t h, const agg_sim_opts* o, agg_sim_t* out) {
  if (!h || !o || !out) return fail(AGG_EINVAL, "NULL argument");
  if (h->sim_active) return fail(AGG_EINVAL, "the hierarchy already drives a simulation");
  agg_status s = check_pcg_opts(&o->pcg);
  if (s) return s;
  if ((s = check_device(h))) return s;
  if (!(o->dt > 0) || !(o->chi_m > 0) || !(o->c_m > 0)) return fail(AGG_EINVAL, "dt, chi_m, c_m must be > 0");
  if (o->scheme != 0 && o->scheme != 1) return fail(AGG_EINVAL, "scheme must be 0 or 1");
  const double c = (o->scheme == 1 ? 1.5 : 1.0) * o->chi_m * o->c_m / o->dt;
  if (std::fabs(c - h->mass_coeff) > 1e-12 * std::fabs(c))
    return fail(AGG_EINVAL, o->scheme == 1 ? "hierarchy mass_coeff differs from 3 chi_m c_m / (2 dt)"
                                           : "hierarchy mass_coeff differs from chi_m c_m / dt");
  if (o->ionic.model < AGG_FHN || o->ionic.model > AGG_BUENO_OROVIO) return fail(AGG_EINVAL, "ionic model");
  SimParams sp;
  sp.model = o->ionic.model;
  sp.k = o->ionic.k;
  sp.a = o->ionic.a;
  sp.eps = o->ionic.eps;
  sp.gamma = o->ionic.gamma;
  sp.mu1 = o->ionic.mu1;
  sp.mu2 = o->ionic.mu2;
  sp.bo = o->ionic.bo;
  sp.dt = o->dt;
  sp.chi = o->chi_m;
  sp.cm = o->c_m;
  sp.iapp_value = o->iapp_mask_dev ? o->iapp_value : 0.0;
  sp.iapp_steps = o->iapp_steps;
  sp.scheme = o->scheme;
  sp.pcg.rtol = o->pcg.rtol;
  sp.pcg.atol = o->pcg.atol;
  sp.pcg.max_it = o->pcg.max_it;
  sp.pcg.flexible = o->pcg.flexible;
  std::string err;
  int rc = h->eng->sim_create(sp, o->iapp_mask_dev, nullptr, err);
  if (rc) return fail((agg_status)rc, err);
  agg_sim* sim = new (std::nothrow) agg_sim();
  if (!sim) return fail(AGG_ENOMEM, "host allocation failed");
  sim->h = h;
  h->sim_active = true;
  *out = sim;
  return AGG_OK;
}

agg_status agg_monodomain_step(agg_sim_t sim, int n_steps, double* u, double* w, int* iters, void* stream) {
  if (!sim || !u || !w) return fail(AGG_EINVAL, "NULL argument");
  if (n_steps < 0) return fail(AGG_EINVAL, "n_steps < 0");
  agg_status s = check_device(sim->h);
  if (s) return s;
  if (n_steps == 0) return AGG_OK;
  std::string err;
  int rc = sim->h->eng->sim_step(n_steps, u, w, iters, sim->clock, (cudaStream_t)stream, err);
  if (rc) return fail((agg_status)rc, err.empty() ? agg_status_string(rc) : err);
  return AGG_OK;
}

agg_status agg_profile_kernel(agg_hier_t h, int kernel, int reps, void* stream) {
  if (!h || reps < 0) return fail(AGG_EINVAL, "bad argument");
  agg_status s = check_device(h);
  if (s) return s;
  std::string err;
  int rc = h->eng->kernel_loop(kernel, reps, (cudaStream_t)stream, err);
  if (rc) return fail((agg_status)rc, err);
  return AGG_OK;
}

agg_status agg_kernel_cost(agg_hier_t h, int kernel, double* bytes, double* flops) {
  if (!h || !bytes || !flops) return fail(AGG_EINVAL, "NULL argument");
  const int rc = h->eng->kernel_cost(kernel, *bytes, *flops);
  if (rc == AGG_EUNSUPPORTED)
    return fail(AGG_EUNSUPPORTED, kernel == 5 ? "kernel 5 is built by its first agg_profile_kernel or "
                                                "agg_operator_apply(level -2) call"
                                              : "kernels 1-3 need n_levels >= 2");
  if (rc) return fail(AGG_EINVAL, "unknown kernel id");
  return AGG_OK;
}

agg_status agg_hier_launches(agg_hier_t h, int* per_vcycle, int* per_iteration, int* per_setup, int* persistent,
                             int* cluster_level, int* cluster_ctas) {
  if (!h || !per_vcycle || !per_iteration || !per_setup || !persistent) return fail(AGG_EINVAL, "NULL argument");
  int cl = -1, cc = 0;
  h->eng->launch_counts(*per_vcycle, *per_iteration, *per_setup, *persistent, cl, cc);
  if (cluster_level) *cluster_level = cl;
  if (cluster_ctas) *cluster_ctas = cc;
  return AGG_OK;
}

agg_status agg_monodomain_adjoint_step(agg_sim_t sim, const double* u_n, const double* w_n, const double* u_np1,
                                       double* ubar, double* wbar, double* grad, void* stream) {
  if (!sim || !u_n || !w_n || !u_np1 || !ubar || !wbar || !grad) return fail(AGG_EINVAL, "NULL argument");
  agg_status s = check_device(sim->h);
  if (s) return s;
  std::string err;
  SolveResult r;
  int rc = sim->h->eng->adjoint_step(u_n, w_n, u_np1, ubar, wbar, grad, r, (cudaStream_t)stream, err);
  if (rc) return fail((agg_status)rc, err);
  if (r.status) return fail((agg_status)r.status, std::string("adjoint solve: ") + agg_status_string(r.status));
  return AGG_OK;
}

agg_status agg_monodomain_set_clock(agg_sim_t sim, int64_t step) {
  if (!sim || step < 0) return fail(AGG_EINVAL, "bad argument");
  sim->clock = step;
  sim->h->eng->sim_invalidate_history();
  return AGG_OK;
}

agg_status agg_monodomain_destroy(agg_sim_t sim) {
  if (!sim) return AGG_OK;
  sim->h->eng->sim_destroy();
  sim->h->sim_active = false;
  delete sim;
  return AGG_OK;
}

}  // extern "C"

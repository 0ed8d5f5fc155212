// C ABI of libgrmhd: argument validation and orchestration of the kernels.
#include <cmath>
#include <cstdint>

#include "internal.h"

namespace grmhd {

DevGrid make_grid(const grmhd_grid& g) {
  DevGrid d;
  for (int i = 0; i < 3; ++i) {
    d.n[i] = g.n[i];
    d.N[i] = g.n[i] + 2 * g.ng;
    d.dx[i] = g.dx[i];
    d.idx[i] = 1.0 / g.dx[i];
    d.idxf[i] = (float)d.idx[i];
  }
  d.ng = g.ng;
  d.sy = d.N[0];
  d.sz = (long long)d.N[0] * d.N[1];
  d.ncell = d.sz * d.N[2];
  return d;
}

DevParams make_params(const grmhd_params& p) {
  DevParams d;
  d.gamma = p.gamma;
  d.gfac = p.gamma / (p.gamma - 1.0);
  d.gm1g = (p.gamma - 1.0) / p.gamma;
  d.rho_atm = p.rho_atm;
  d.p_atm = p.p_atm;
  d.nr_tol = p.nr_tol;
  d.weno_eps = p.weno_eps;
  d.nr_maxit = p.nr_maxit;
  d.recon = p.recon;
  d.bc = p.bc;
  d.precision = p.precision;
  d.tile = p.tile;
  d.flags = p.flags;
  d.eos = p.eos;
  d.poly_K = p.poly_K;
  d.poly_g2 = p.gamma == 2.0;
  d.gammaf = (float)d.gamma;
  d.gfacf = (float)d.gfac;
  d.weno_epsf = (float)d.weno_eps;
  d.eps13f = (float)(d.weno_eps * (12.0 / 13.0));
  d.gm1gf = (float)d.gm1g;
  d.rho_atmf = (float)d.rho_atm;
  // the polytrope's atmosphere pressure
  if (p.eos == GRMHD_EOS_POLYTROPE) d.p_atm = p.poly_K * std::pow(p.rho_atm, p.gamma);
  d.p_atmf = (float)d.p_atm;
  return d;
}

}  // namespace grmhd

using namespace grmhd;

namespace {

cudaError_t launch_rhs(const DevGrid& g, const DevParams& p, const double* prim, const double* metric,
                       const double* kij, const StageEpilogue& ep, cudaStream_t s) {
  if (p.precision == GRMHD_MIXED) return launch_rhs_mixed(g, p, prim, metric, kij, ep, s);
  return launch_rhs_fp64(g, p, prim, metric, kij, ep, s);
}

// Bytes of the cached-path scratch: geometry cache, FP32 primitives, inverse-
// metric cache, and the multi-pass FP64 RHS buffers: face fluxes (24 doubles
// per point) followed by the WENO5 face states (48 doubles per point).
constexpr int kFaceBufComps = 24, kStateBufComps = 48;
size_t cache_bytes(const DevGrid& g) {
  return round256((size_t)kGeomCacheComps * g.ncell * sizeof(double)) + round256((size_t)8 * g.ncell * sizeof(float)) +
         round256((size_t)kMetricCacheComps * g.ncell * sizeof(double)) +
         round256((size_t)(kFaceBufComps + kStateBufComps) * g.ncell * sizeof(double));
}

}  // namespace

extern "C" {

int grmhd_version(void) { return 100; }

const char* grmhd_error_string(int code) {
  switch (code) {
    case GRMHD_OK: return "ok";
    case GRMHD_ERR_ARG: return "invalid argument";
    case GRMHD_ERR_CUDA: return "CUDA error";
    case GRMHD_ERR_TIMEOUT: return "device wait timed out";
    case GRMHD_ERR_SIZE: return "workspace too small";
    default: return "unknown error";
  }
}

int grmhd_prim2con(const grmhd_grid* grid, const grmhd_params* params, const double* prim, const double* metric,
                   double* cons, void* stream) {
  int e = check_params(params);
  if (e) return e;
  if ((e = check_grid(grid, 0))) return e;
  if (!prim || !cons || !aligned8(prim) || !aligned8(cons) || (metric && !aligned8(metric)))
    return GRMHD_ERR_ARG;
  return cuda_status(launch_prim2con(make_grid(*grid), make_params(*params), prim, metric, cons,
                                     (cudaStream_t)stream));
}

int grmhd_con2prim(const grmhd_grid* grid, const grmhd_params* params, const double* cons, const double* metric,
                   double* prim, int8_t* status, int32_t* nfail, void* stream) {
  int e = check_params(params);
  if (e) return e;
  if ((e = check_grid(grid, 0))) return e;
  if (!prim || !cons || !aligned8(prim) || !aligned8(cons) || (metric && !aligned8(metric))) return GRMHD_ERR_ARG;
  if (nfail && (reinterpret_cast<uintptr_t>(nfail) & 3u)) return GRMHD_ERR_ARG;
  return cuda_status(launch_con2prim(make_grid(*grid), make_params(*params), cons, metric, prim, status, nfail,
                                     (cudaStream_t)stream));
}

int grmhd_fill_ghosts(const grmhd_grid* grid, int32_t bc, int32_t nvar, double* field, void* stream) {
  int e = check_grid(grid, 0);
  if (e) return e;
  if (bc != GRMHD_BC_PERIODIC && bc != GRMHD_BC_COPY) return GRMHD_ERR_ARG;
  if (nvar < 1 || nvar > 64 || !field || !aligned8(field)) return GRMHD_ERR_ARG;
  return cuda_status(launch_fill_ghosts(make_grid(*grid), bc, nvar, field, (cudaStream_t)stream));
}

int grmhd_rhs(const grmhd_grid* grid, const grmhd_params* params, const double* prim, const double* metric,
              const double* kij, double* rhs, void* stream) {
  int e = check_params(params);
  if (e) return e;
  if ((e = check_grid(grid, min_ghosts(params, metric)))) return e;
  if (!prim || !rhs || !aligned8(prim) || !aligned8(rhs)) return GRMHD_ERR_ARG;
  if ((metric && !aligned8(metric)) || (kij && !aligned8(kij))) return GRMHD_ERR_ARG;
  if (kij && !metric) return GRMHD_ERR_ARG;
  StageEpilogue ep = no_epilogue();
  ep.rhs = rhs;
  return cuda_status(launch_rhs(make_grid(*grid), make_params(*params), prim, metric, kij, ep,
                                (cudaStream_t)stream));
}

size_t grmhd_rhs_workspace_bytes(const grmhd_grid* grid) {
  if (check_grid(grid, 0)) return 0;
  return cache_bytes(make_grid(*grid));
}

int grmhd_rhs_cached(const grmhd_grid* grid, const grmhd_params* params, const double* prim, const double* metric,
                     const double* kij, double* rhs, void* ws, size_t ws_bytes, void* stream) {
  int e = check_params(params);
  if (e) return e;
  if ((e = check_grid(grid, min_ghosts(params, metric)))) return e;
  if (!prim || !rhs || !ws || !aligned8(prim) || !aligned8(rhs)) return GRMHD_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(ws) & 255u) != 0) return GRMHD_ERR_ARG;
  if ((metric && !aligned8(metric)) || (kij && !aligned8(kij)) || (kij && !metric)) return GRMHD_ERR_ARG;
  if (ws_bytes < grmhd_rhs_workspace_bytes(grid)) return GRMHD_ERR_SIZE;
  const DevGrid g = make_grid(*grid);
  const DevParams p = make_params(*params);
  cudaStream_t s = (cudaStream_t)stream;
  StageEpilogue ep = no_epilogue();
  ep.rhs = rhs;
  char* base = static_cast<char*>(ws);
  void* geom = base;
  float* prim32 = reinterpret_cast<float*>(base + round256((size_t)kGeomCacheComps * g.ncell * sizeof(double)));
  double* mcache = reinterpret_cast<double*>(reinterpret_cast<char*>(prim32) +
                                             round256((size_t)8 * g.ncell * sizeof(float)));
  double* faces = reinterpret_cast<double*>(reinterpret_cast<char*>(mcache) +
                                            round256((size_t)kMetricCacheComps * g.ncell * sizeof(double)));
  const bool mixed = p.precision == GRMHD_MIXED;
  const bool reuse = (p.flags & GRMHD_REUSE_GEOMETRY) != 0;
  if (metric && !reuse && launch_geom_cache(g, metric, geom, !mixed, mcache, s) != cudaSuccess) return GRMHD_ERR_CUDA;
  if (mixed) {
    if (launch_prim_to_f32_pairs(g.ncell, prim, prim32, s) != cudaSuccess) return GRMHD_ERR_CUDA;
    return cuda_status(launch_rhs_mixed_cached(g, p, prim32, static_cast<const float*>(geom), kij, metric != nullptr,
                                               ep, s));
  }
  if (!metric) return cuda_status(launch_rhs(g, p, prim, metric, kij, ep, s));
  if (!(p.flags & GRMHD_SINGLE_PASS)) {
    ep.faces = faces;
    ep.states = faces + (size_t)kFaceBufComps * g.ncell;
  }
  return cuda_status(launch_rhs_fp64_cached(g, p, prim, static_cast<const double*>(geom), kij, ep, s));
}

size_t grmhd_rk_workspace_bytes(const grmhd_grid* grid, int32_t scheme) {
  if (check_grid(grid, 0)) return 0;
  if (scheme != GRMHD_RK2 && scheme != GRMHD_RK3 && scheme != GRMHD_RK4) return 0;
  const DevGrid g = make_grid(*grid);
  const size_t field = round256((size_t)8 * g.ncell * sizeof(double));
  return scheme == GRMHD_RK4 ? 2 * field : field;
}

size_t grmhd_rk_workspace_bytes_cached(const grmhd_grid* grid, int32_t scheme) {
  const size_t base = grmhd_rk_workspace_bytes(grid, scheme);
  if (base == 0) return 0;
  return base + cache_bytes(make_grid(*grid));
}

}  // extern "C"

namespace {

// One step; with record != NULL the FP64 primitives after every stage are
// also copied to record + k * 8 * ncell (k = 0 .. stages-1).
int rk_step_impl(const grmhd_grid* grid, const grmhd_params* params, int32_t scheme, double dt, double* cons,
                 double* prim, const double* metric, const double* kij, void* ws, size_t ws_bytes, int32_t* nfail,
                 void* stream, double* record, const CtStep* ct = nullptr) {
  int e = check_params(params);
  if (e) return e;
  if ((e = check_grid(grid, min_ghosts(params, metric)))) return e;
  if (scheme != GRMHD_RK2 && scheme != GRMHD_RK3 && scheme != GRMHD_RK4) return GRMHD_ERR_ARG;
  if (!(dt > 0.0) || !std::isfinite(dt)) return GRMHD_ERR_ARG;
  if (!cons || !prim || !ws || !aligned8(cons) || !aligned8(prim)) return GRMHD_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(ws) & 255u) != 0) return GRMHD_ERR_ARG;
  if ((metric && !aligned8(metric)) || (kij && !aligned8(kij)) || (kij && !metric)) return GRMHD_ERR_ARG;
  if (nfail && (reinterpret_cast<uintptr_t>(nfail) & 3u)) return GRMHD_ERR_ARG;
  if (ws_bytes < grmhd_rk_workspace_bytes(grid, scheme)) return GRMHD_ERR_SIZE;

  const DevGrid g = make_grid(*grid);
  const DevParams p = make_params(*params);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t field = round256((size_t)8 * g.ncell * sizeof(double));
  double* u0 = static_cast<double*>(ws);
  double* acc = scheme == GRMHD_RK4 ? reinterpret_cast<double*>(static_cast<char*>(ws) + field) : nullptr;

  cudaError_t ce = cudaMemcpyAsync(u0, cons, (size_t)8 * g.ncell * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (ce != cudaSuccess) return GRMHD_ERR_CUDA;
  // Mixed precision with room for the caches: FP32 primitive copy + geometry
  // cache (rebuilt here, once per step) feed the RHS; otherwise the RHS reads
  // the FP64 inputs directly.
  // Cached paths (workspace >= grmhd_rk_workspace_bytes_cached):
  //  mixed: FP32 primitive copy + FP32 geometry cache + FP64 inverse-metric cache;
  //  FP64 on a metric: FP64 geometry cache + FP64 inverse-metric cache.
  // The caches are rebuilt once per call unless GRMHD_REUSE_GEOMETRY is set.
  const bool cached = ws_bytes >= grmhd_rk_workspace_bytes_cached(grid, scheme);
  const bool fast_mixed = p.precision == GRMHD_MIXED && cached;
  const bool fast_fp64 = p.precision == GRMHD_FP64 && cached && metric != nullptr;
  float* prim32 = nullptr;
  void* geom = nullptr;
  double* mcache = nullptr;
  double* faces = nullptr;
  if (fast_mixed || fast_fp64) {
    char* after = static_cast<char*>(ws) + grmhd_rk_workspace_bytes(grid, scheme);
    geom = after;
    after += round256((size_t)kGeomCacheComps * g.ncell * sizeof(double));
    prim32 = reinterpret_cast<float*>(after);
    after += round256((size_t)8 * g.ncell * sizeof(float));
    mcache = reinterpret_cast<double*>(after);
    after += round256((size_t)kMetricCacheComps * g.ncell * sizeof(double));
    if (fast_fp64 && !(p.flags & GRMHD_SINGLE_PASS)) faces = reinterpret_cast<double*>(after);
    const bool reuse = (p.flags & GRMHD_REUSE_GEOMETRY) != 0;
    if (metric && !reuse && launch_geom_cache(g, metric, geom, fast_fp64, mcache, s) != cudaSuccess)
      return GRMHD_ERR_CUDA;
    if (fast_mixed && launch_prim_to_f32_pairs(g.ncell, prim, prim32, s) != cudaSuccess) return GRMHD_ERR_CUDA;
  }

  RkStage st[4];
  const int ns = rk_stages(scheme, dt, st);
  for (int k = 0; k < ns; ++k) {
    StageEpilogue ep = no_epilogue();
    ep.u = cons;
    ep.u0 = u0;
    ep.acc_in = st[k].acc_in ? acc : nullptr;
    ep.acc_out = st[k].acc_out ? acc : nullptr;
    ep.c0 = st[k].c0;
    ep.c1 = st[k].c1;
    ep.cr = st[k].cr;
    ep.ca = st[k].ca;
    ep.wa = st[k].wa;
    ep.wr = st[k].wr;
    ep.fb = ct ? ct->fb : nullptr;
    ep.faces = faces;
    ep.states = faces ? faces + (size_t)kFaceBufComps * g.ncell : nullptr;
    if (fast_fp64) {
      if (launch_rhs_fp64_cached(g, p, prim, static_cast<const double*>(geom), kij, ep, s) != cudaSuccess)
        return GRMHD_ERR_CUDA;
    } else if (fast_mixed) {
      if (launch_rhs_mixed_cached(g, p, prim32, static_cast<const float*>(geom), kij, metric != nullptr, ep, s) !=
          cudaSuccess)
        return GRMHD_ERR_CUDA;
    } else if (launch_rhs(g, p, prim, metric, kij, ep, s) != cudaSuccess) {
      return GRMHD_ERR_CUDA;
    }
    // constrained transport: the face update by the curl of the edge field,
    // and the cell field as the mean of the faces (replacing the cell-centred
    // field update of the epilogue) before the recovery
    if (ct) {
      if (launch_ct_faces(g, ct->fb, ct->E, nullptr, ct->b, ct->b0, st[k].acc_in ? ct->acc : nullptr,
                          st[k].acc_out ? ct->acc : nullptr, st[k].c0, st[k].c1, st[k].cr, st[k].ca, st[k].wa,
                          st[k].wr, s) != cudaSuccess)
        return GRMHD_ERR_CUDA;
      if (launch_ct_face_to_cell(g, ct->b, cons, s) != cudaSuccess) return GRMHD_ERR_CUDA;
    }
    if (fast_fp64) {
      if (launch_con2prim_cached(g, p, cons, metric, mcache, prim, nfail, s) != cudaSuccess) return GRMHD_ERR_CUDA;
      if (launch_fill_ghosts(g, p.bc, 8, prim, s) != cudaSuccess) return GRMHD_ERR_CUDA;
    } else if (fast_mixed) {
      // the FP64 primitives are needed after the last stage (and when recording)
      const bool result64 = k == ns - 1 || record;
      if (launch_con2prim_mixed(g, p, cons, metric, prim, prim32, metric ? mcache : nullptr,
                                metric ? static_cast<const float*>(geom) : nullptr, result64, nfail, s) != cudaSuccess)
        return GRMHD_ERR_CUDA;
      if (launch_fill_ghosts_f32(g, p.bc, 8, prim32, s) != cudaSuccess) return GRMHD_ERR_CUDA;
      if (result64 && launch_fill_ghosts(g, p.bc, 8, prim, s) != cudaSuccess) return GRMHD_ERR_CUDA;
    } else {
      if ((ce = launch_con2prim(g, p, cons, metric, prim, nullptr, nfail, s)) != cudaSuccess) return GRMHD_ERR_CUDA;
      if ((ce = launch_fill_ghosts(g, p.bc, 8, prim, s)) != cudaSuccess) return GRMHD_ERR_CUDA;
    }
    if (record && cudaMemcpyAsync(record + (size_t)k * 8 * g.ncell, prim, (size_t)8 * g.ncell * sizeof(double),
                                  cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return GRMHD_ERR_CUDA;
  }
  return GRMHD_OK;
}

}  // namespace

extern "C" {

int grmhd_rk_step(const grmhd_grid* grid, const grmhd_params* params, int32_t scheme, double dt, double* cons,
                  double* prim, const double* metric, const double* kij, void* ws, size_t ws_bytes,
                  int32_t* nfail, void* stream) {
  return rk_step_impl(grid, params, scheme, dt, cons, prim, metric, kij, ws, ws_bytes, nfail, stream, nullptr);
}

int grmhd_rk_step_record(const grmhd_grid* grid, const grmhd_params* params, int32_t scheme, double dt,
                         double* cons, double* prim, const double* metric, const double* kij, void* ws,
                         size_t ws_bytes, double* stage_prims, int32_t* nfail, void* stream) {
  if (!stage_prims || !aligned8(stage_prims)) return GRMHD_ERR_ARG;
  return rk_step_impl(grid, params, scheme, dt, cons, prim, metric, kij, ws, ws_bytes, nfail, stream, stage_prims);
}

}  // extern "C"

// ------------------------------------------------ constrained transport --

namespace {

// Field-flux register plus the edge fields.
size_t ct_flux_bytes(const DevGrid& g) {
  return round256((size_t)9 * g.ncell * sizeof(double)) + round256((size_t)3 * g.ncell * sizeof(double));
}

// Bytes of the CT part of the step workspace: field fluxes, edge fields, the
// step-start face field and (RK4) the face-rate accumulator.
size_t ct_part_bytes(const DevGrid& g, int32_t scheme) {
  const size_t face = round256((size_t)3 * g.ncell * sizeof(double));
  return ct_flux_bytes(g) + face + (scheme == GRMHD_RK4 ? face : 0);
}

double* ct_edges_of(const DevGrid& g, void* ws) {
  return reinterpret_cast<double*>(static_cast<char*>(ws) + round256((size_t)9 * g.ncell * sizeof(double)));
}

}  // namespace

extern "C" {

size_t grmhd_ct_flux_bytes(const grmhd_grid* grid) {
  if (check_grid(grid, 0)) return 0;
  return ct_flux_bytes(make_grid(*grid));
}

size_t grmhd_ct_workspace_bytes(const grmhd_grid* grid, int32_t scheme) {
  const size_t rk = grmhd_rk_workspace_bytes(grid, scheme);
  return rk ? ct_part_bytes(make_grid(*grid), scheme) + rk : 0;
}

size_t grmhd_ct_workspace_bytes_cached(const grmhd_grid* grid, int32_t scheme) {
  const size_t rk = grmhd_rk_workspace_bytes_cached(grid, scheme);
  return rk ? ct_part_bytes(make_grid(*grid), scheme) + rk : 0;
}

int grmhd_ct_rate(const grmhd_grid* grid, const grmhd_params* params, const double* prim, const double* metric,
                  const double* kij, double* rate, void* ws, size_t ws_bytes, void* stream) {
  int e = check_params(params);
  if (e) return e;
  if ((e = check_grid(grid, min_ghosts(params, metric)))) return e;
  if (!prim || !rate || !ws || !aligned8(prim) || !aligned8(rate)) return GRMHD_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(ws) & 255u) != 0) return GRMHD_ERR_ARG;
  if ((metric && !aligned8(metric)) || (kij && !aligned8(kij)) || (kij && !metric)) return GRMHD_ERR_ARG;
  if (ws_bytes < grmhd_ct_flux_bytes(grid)) return GRMHD_ERR_SIZE;
  const DevGrid g = make_grid(*grid);
  const DevParams p = make_params(*params);
  cudaStream_t s = (cudaStream_t)stream;
  double* fb = static_cast<double*>(ws);
  StageEpilogue ep = no_epilogue();
  ep.fb = fb;
  if (launch_rhs(g, p, prim, metric, kij, ep, s) != cudaSuccess) return GRMHD_ERR_CUDA;
  if (cudaMemsetAsync(rate, 0, (size_t)3 * g.ncell * sizeof(double), s) != cudaSuccess) return GRMHD_ERR_CUDA;
  return cuda_status(
      launch_ct_faces(g, fb, ct_edges_of(g, ws), rate, nullptr, nullptr, nullptr, nullptr, 0, 0, 0, 0, 0, 0, s));
}

int grmhd_ct_rk_step(const grmhd_grid* grid, const grmhd_params* params, int32_t scheme, double dt, double* cons,
                     double* prim, double* bface, const double* metric, const double* kij, void* ws,
                     size_t ws_bytes, int32_t* nfail, void* stream) {
  int e = check_params(params);
  if (e) return e;
  if ((e = check_grid(grid, min_ghosts(params, metric)))) return e;
  if (scheme != GRMHD_RK2 && scheme != GRMHD_RK3 && scheme != GRMHD_RK4) return GRMHD_ERR_ARG;
  if (!(dt > 0.0) || !std::isfinite(dt)) return GRMHD_ERR_ARG;
  if (!cons || !prim || !bface || !aligned8(cons) || !aligned8(prim) || !aligned8(bface)) return GRMHD_ERR_ARG;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0) return GRMHD_ERR_ARG;
  if ((metric && !aligned8(metric)) || (kij && !aligned8(kij)) || (kij && !metric)) return GRMHD_ERR_ARG;
  if (nfail && (reinterpret_cast<uintptr_t>(nfail) & 3u)) return GRMHD_ERR_ARG;
  if (ws_bytes < grmhd_ct_workspace_bytes(grid, scheme)) return GRMHD_ERR_SIZE;
  const DevGrid g = make_grid(*grid);
  const size_t part = ct_part_bytes(g, scheme);
  char* base = static_cast<char*>(ws);
  CtStep ct;
  ct.fb = reinterpret_cast<double*>(base);
  ct.E = ct_edges_of(g, ws);
  ct.b = bface;
  double* b0 = reinterpret_cast<double*>(base + ct_flux_bytes(g));
  ct.b0 = b0;
  ct.acc = scheme == GRMHD_RK4 ? reinterpret_cast<double*>(base + ct_flux_bytes(g) +
                                                           round256((size_t)3 * g.ncell * sizeof(double)))
                               : nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(b0, bface, (size_t)3 * g.ncell * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return GRMHD_ERR_CUDA;
  return rk_step_impl(grid, params, scheme, dt, cons, prim, metric, kij, base + part, ws_bytes - part, nfail, stream,
                      nullptr, &ct);
}

int grmhd_ct_cell_field(const grmhd_grid* grid, const double* bface, const double* metric, double* prim,
                        void* stream) {
  const int e = check_grid(grid, 1);
  if (e) return e;
  if (!bface || !prim || !aligned8(bface) || !aligned8(prim) || (metric && !aligned8(metric))) return GRMHD_ERR_ARG;
  return cuda_status(launch_ct_cell_field(make_grid(*grid), bface, metric, prim, (cudaStream_t)stream));
}

int grmhd_ct_divergence(const grmhd_grid* grid, const double* bface, double* div, double* maxabs, void* stream) {
  const int e = check_grid(grid, 1);
  if (e) return e;
  if (!bface || !aligned8(bface) || (div && !aligned8(div)) || (maxabs && !aligned8(maxabs)) || (!div && !maxabs))
    return GRMHD_ERR_ARG;
  return cuda_status(launch_ct_divergence(make_grid(*grid), bface, div, maxabs, (cudaStream_t)stream));
}

}  // extern "C"

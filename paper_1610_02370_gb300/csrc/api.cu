// The C ABI of libddtm (include/ddtm.h): argument checking, host<->device
// marshalling and the translation of internal errors into status codes.
#include <string.h>

#include <chrono>
#include <cmath>

#include "common.cuh"
#include "ddtm_internal.h"
#include "coarse.h"
#include "solver.h"
#include "timer.h"

using namespace ddtm;

#define API_BEGIN(ctx)                                   \
  if (!(ctx)) return DDTM_ERR_ARG;                       \
  (ctx)->err.clear();                                    \
  try {
#define API_END(ctx)                                     \
  }                                                      \
  catch (const ddtm::Error& e) {                         \
    (ctx)->err = e.what();                               \
    return e.code;                                       \
  }                                                      \
  catch (const std::exception& e) {                      \
    (ctx)->err = e.what();                               \
    return DDTM_ERR_CUDA;                                \
  }                                                      \
  return DDTM_OK;

namespace ddtm {

size_t store2_bytes(int prec) { return prec == PREC_F64 ? 16 : (prec == PREC_F32 ? 8 : 4); }

void check_prec(int prec) {
  if (prec != PREC_F64 && prec != PREC_F32 && prec != PREC_F16) throw Error(DDTM_ERR_ARG, "invalid precision");
}
void check_loc(int loc) {
  if (loc != DDTM_LOC_HOST && loc != DDTM_LOC_DEVICE) throw Error(DDTM_ERR_ARG, "invalid location");
}

void require_gauge(ddtm_ctx* c) {
  if (!c->gauge) throw Error(DDTM_ERR_STATE, "no gauge field loaded (call ddtm_load_gauge first)");
}

// links/clover in precision prec, converted lazily from the FP64 copies
void ensure_fine_prec(ddtm_ctx* c, int prec) {
  require_gauge(c);
  if (prec == PREC_F64) return;
  size_t nl = (size_t)c->g.V * 36, nc = (size_t)c->g.V * 36;
  if (!c->links[prec].p) {
    c->links[prec].ensure(nl * store2_bytes(prec));
    launch_convert_complex(c->links[0].as<double>(), prec, c->links[prec].p, nl, c->stream);
  }
  if (!c->clover[prec].p) {
    c->clover[prec].ensure(nc * store2_bytes(prec));
    launch_convert_complex(c->clover[0].as<double>(), prec, c->clover[prec].p, nc, c->stream);
  }
}

// even-site inverses of (site term + i mu gamma5) in precision prec for this mu
void ensure_site_inverse(ddtm_ctx* c, int prec, double mu) {
  require_gauge(c);
  if (c->sinv_ok[prec] && c->sinv_mu[prec] == mu) return;
  c->sinv[prec].ensure((size_t)c->g.V / 2 * 72 * store2_bytes(prec));
  launch_site_inverse(c->g, prec, c->sinv[prec].p, c->clover[0].as<double>(), mu, c->stream);
  c->sinv_mu[prec] = mu;
  c->sinv_ok[prec] = true;
}

// device view of nrhs canonical fine spinors: either the caller's device
// pointer or a staged copy of host memory
const double* stage_in(ddtm_ctx* c, const char* name, const double* x, size_t ncomplex, int loc) {
  if (loc == DDTM_LOC_DEVICE) return x;
  double* d = (double*)c->scratch.get(name, ncomplex * 16);
  CK(cudaMemcpyAsync(d, x, ncomplex * 16, cudaMemcpyHostToDevice, c->stream));
  return d;
}
double* stage_out(ddtm_ctx* c, const char* name, double* y, size_t ncomplex, int loc) {
  if (loc == DDTM_LOC_DEVICE) return y;
  return (double*)c->scratch.get(name, ncomplex * 16);
}
void unstage_out(ddtm_ctx* c, double* y, const double* d, size_t ncomplex, int loc) {
  if (loc == DDTM_LOC_DEVICE) return;
  CK(cudaMemcpyAsync(y, d, ncomplex * 16, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
}

void field_alloc(ddtm_field* f) {
  size_t V = f->ctx->g.V;
  f->stride = V * 12;
  f->data.ensure(f->stride * f->nrhs * store2_bytes(f->prec));
  if (f->prec == PREC_F16) f->nrm.ensure(V * f->nrhs * sizeof(float));
}

void* field_ptr(const ddtm_field* f, int r) {
  return (char*)f->data.p + (size_t)r * f->stride * store2_bytes(f->prec);
}
float* field_nrm(const ddtm_field* f, int r) {
  return f->prec == PREC_F16 ? f->nrm.as<float>() + (size_t)r * f->ctx->g.V : nullptr;
}

void dslash_field(ddtm_ctx* c, ddtm_field* y, const ddtm_field* x, double mu) {
  ensure_fine_prec(c, x->prec);
  launch_dslash_multi(c->g, x->prec, field_ptr(y, 0), field_nrm(y, 0), field_ptr(x, 0), field_nrm(x, 0),
                      c->links[x->prec].p, c->clover[x->prec].p, mu, x->nrhs, c->stream);
}

}  // namespace ddtm

void* ddtm_ctx::scratch_host(const std::string& name, size_t bytes) {
  auto it = host_bufs.find(name);
  if (it != host_bufs.end() && it->second.second >= bytes) return it->second.first;
  if (it != host_bufs.end()) cudaFreeHost(it->second.first);
  void* p = nullptr;
  CK(cudaMallocHost(&p, bytes));
  host_bufs[name] = std::make_pair(p, bytes);
  return p;
}

void ddtm_ctx::events(const std::string& name, cudaEvent_t ev[2]) {
  auto it = event_pairs.find(name);
  if (it == event_pairs.end()) {
    cudaEvent_t a, b;
    CK(cudaEventCreateWithFlags(&a, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&b, cudaEventDisableTiming));
    it = event_pairs.emplace(name, std::make_pair(a, b)).first;
  }
  ev[0] = it->second.first;
  ev[1] = it->second.second;
}

ddtm_ctx::~ddtm_ctx() {
  for (auto& kv : graphs)
    if (kv.second.first) cudaGraphExecDestroy(kv.second.first);
  if (capture_stream) cudaStreamDestroy(capture_stream);
  for (auto& kv : host_bufs) cudaFreeHost(kv.second.first);
  for (auto& kv : event_pairs) {
    cudaEventDestroy(kv.second.first);
    cudaEventDestroy(kv.second.second);
  }
}

extern "C" {

int ddtm_default_params(ddtm_params* p) {
  if (!p) return DDTM_ERR_ARG;
  memset(p, 0, sizeof(*p));
  p->n_levels = 2;
  p->n_setup = 5;
  p->nv[0] = 28;
  p->nv[1] = 28;
  for (int m = 0; m < 4; m++) {
    p->block[0][m] = 4;
    p->block[1][m] = 2;
  }
  p->post_smooth = 4;
  p->nmr = 3;
  p->kcycle_restart = 5;
  p->kcycle_max_restarts = 2;
  p->kcycle_tol = 1e-1;
  p->coarse_restart = 100;
  p->coarse_max_restarts = 5;
  p->coarse_tol = 1e-1;
  p->delta = 5.2;
  p->outer_restart = 30;
  p->outer_max_iters = 1000;
  p->outer_tol = 1e-10;
  p->restart_tol = 1e-6;
  p->smoother_prec = DDTM_PREC_F16;
  p->coarse_prec = DDTM_PREC_F32;
  return DDTM_OK;
}

int ddtm_create(ddtm_ctx** out, const int dims[4], const int block[4], int bc_t) {
  if (!out || !dims) return DDTM_ERR_ARG;
  *out = nullptr;
  int b[4] = {4, 4, 4, 4};
  if (block)
    for (int m = 0; m < 4; m++) b[m] = block[m];
  if (bc_t != 0 && bc_t != 1) return DDTM_ERR_ARG;
  for (int m = 0; m < 4; m++) {
    if (dims[m] <= 0 || b[m] <= 0 || b[m] % 2 || dims[m] % b[m]) return DDTM_ERR_ARG;
    int nb = dims[m] / b[m];
    if (nb < 2 || nb % 2) return DDTM_ERR_ARG;
  }
  if ((long)b[0] * b[1] * b[2] * b[3] > 65536) return DDTM_ERR_ARG;
  ddtm_ctx* c = new ddtm_ctx();
  ddtm_default_params(&c->p);
  try {
    for (int m = 0; m < 4; m++) {
      c->g.L[m] = dims[m];
      c->g.b[m] = b[m];
      c->g.NB[m] = dims[m] / b[m];
      c->p.block[0][m] = b[m];
    }
    c->g.bc_t = bc_t;
    build_geometry(c->g);
  } catch (const Error& e) {
    delete c;
    return e.code;
  }
  *out = c;
  return DDTM_OK;
}

int ddtm_destroy(ddtm_ctx* ctx) {
  if (!ctx) return DDTM_ERR_ARG;
  cudaStreamSynchronize(ctx->stream);
  delete ctx;
  return DDTM_OK;
}

const char* ddtm_last_error(ddtm_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int ddtm_set_stream(ddtm_ctx* ctx, void* stream) {
  API_BEGIN(ctx)
  ctx->stream = (cudaStream_t)stream;
  API_END(ctx)
}

int ddtm_get_params(ddtm_ctx* ctx, ddtm_params* p) {
  API_BEGIN(ctx)
  if (!p) throw Error(DDTM_ERR_ARG, "null params");
  *p = ctx->p;
  API_END(ctx)
}

int ddtm_set_params(ddtm_ctx* ctx, const ddtm_params* p) {
  API_BEGIN(ctx)
  if (!p) throw Error(DDTM_ERR_ARG, "null params");
  validate_params(ctx, *p);
  bool hierarchy_changed = p->n_levels != ctx->p.n_levels || p->nv[0] != ctx->p.nv[0] || p->nv[1] != ctx->p.nv[1] ||
                           memcmp(p->block, ctx->p.block, sizeof(p->block)) != 0 || p->coarse_prec != ctx->p.coarse_prec;
  const bool block1_changed = memcmp(p->block[1], ctx->p.block[1], sizeof(p->block[1])) != 0;
  ctx->p = *p;
  if (hierarchy_changed) invalidate_setup(ctx);
  if (block1_changed) {  // the level-1 aggregates and the level-2 lattice follow block[1]
    ctx->a1.geom = false;
    ctx->c2_geom = false;
  }
  API_END(ctx)
}

int ddtm_load_gauge(ddtm_ctx* ctx, const double* U, int loc, double kappa, double c_sw) {
  API_BEGIN(ctx)
  check_loc(loc);
  if (!U) throw Error(DDTM_ERR_ARG, "null gauge field");
  if (!(kappa > 0) || !std::isfinite(kappa) || !std::isfinite(c_sw)) throw Error(DDTM_ERR_ARG, "invalid kappa or c_sw");
  size_t n = (size_t)ctx->g.V * 36;  // complex entries
  const double* dU = stage_in(ctx, "gauge_canon", U, n, loc);
  int* cnt = (int*)ctx->scratch.get("nan_count", 4);
  CK(cudaMemsetAsync(cnt, 0, 4, ctx->stream));
  launch_count_nonfinite(dU, n * 2, cnt, ctx->stream);
  int h = 0;
  CK(cudaMemcpyAsync(&h, cnt, 4, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (h) throw Error(DDTM_ERR_NAN, "gauge field holds " + std::to_string(h) + " non-finite values");
  for (int p = 0; p < 3; p++) {
    ctx->links[p].release();
    ctx->clover[p].release();
    ctx->sinv_ok[p] = false;
  }
  ctx->links[0].ensure(n * 16);
  ctx->clover[0].ensure((size_t)ctx->g.V * 36 * 16);
  launch_links_from_canon(ctx->g, ctx->links[0].as<double>(), dU, ctx->stream);
  ctx->kappa = kappa;
  ctx->csw = c_sw;
  double m = 1.0 / (2.0 * kappa) - 4.0;
  launch_clover_build(ctx->g, ctx->clover[0].as<double>(), dU, m + 4.0, c_sw, ctx->stream);
  if (ctx->theta[0] != 0 || ctx->theta[1] != 0 || ctx->theta[2] != 0 || ctx->theta[3] != 0)
    launch_link_phases(ctx->g, ctx->links[0].as<double>(), ctx->theta, ctx->stream);  // after the clover term
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->gauge = true;
  invalidate_setup(ctx);
  API_END(ctx)
}

int ddtm_set_boundary_phases(ddtm_ctx* ctx, const double theta[4]) {
  API_BEGIN(ctx)
  if (!theta) throw Error(DDTM_ERR_ARG, "null theta");
  for (int m = 0; m < 4; m++)
    if (!std::isfinite(theta[m])) throw Error(DDTM_ERR_ARG, "non-finite boundary phase");
  if (ctx->gauge) {
    // change the phases of the loaded links by the difference, drop the lower-precision copies
    // (converted again on first use) and the setup (the operator changed)
    double d[4];
    for (int m = 0; m < 4; m++) d[m] = theta[m] - ctx->theta[m];
    launch_link_phases(ctx->g, ctx->links[0].as<double>(), d, ctx->stream);
    ctx->links[1].release();
    ctx->links[2].release();
    CK(cudaStreamSynchronize(ctx->stream));
    invalidate_setup(ctx);
  }
  for (int m = 0; m < 4; m++) ctx->theta[m] = theta[m];
  API_END(ctx)
}

int ddtm_apply_D(ddtm_ctx* ctx, double* y, const double* x, int nrhs, double mu, int prec, int loc) {
  API_BEGIN(ctx)
  check_prec(prec);
  check_loc(loc);
  if (!x || !y || nrhs < 0) throw Error(DDTM_ERR_ARG, "invalid arguments");
  if (nrhs == 0) return DDTM_OK;
  ensure_fine_prec(ctx, prec);
  size_t nsp = (size_t)ctx->g.V * 12;
  ddtm_field fx{ctx, prec, 1}, fy{ctx, prec, 1};
  field_alloc(&fx);
  field_alloc(&fy);
  for (int r = 0; r < nrhs; r++) {
    const double* din = stage_in(ctx, "canon_in", x + 2 * nsp * r, nsp, loc);
    double* dout = stage_out(ctx, "canon_out", y + 2 * nsp * r, nsp, loc);
    launch_spinor_from_canon(ctx->g, prec, fx.data.p, fx.nrm.as<float>(), din, ctx->stream);
    dslash_field(ctx, &fy, &fx, mu);
    launch_spinor_to_canon(ctx->g, prec, fy.data.p, fy.nrm.as<float>(), dout, ctx->stream);
    unstage_out(ctx, y + 2 * nsp * r, dout, nsp, loc);
  }
  CK(cudaStreamSynchronize(ctx->stream));
  API_END(ctx)
}

int ddtm_field_create(ddtm_ctx* ctx, int prec, int nrhs, ddtm_field** out) {
  API_BEGIN(ctx)
  check_prec(prec);
  if (!out || nrhs <= 0) throw Error(DDTM_ERR_ARG, "invalid arguments");
  *out = nullptr;
  ddtm_field* f = new ddtm_field{ctx, prec, nrhs};
  try {
    field_alloc(f);
  } catch (...) {
    delete f;
    throw;
  }
  *out = f;
  API_END(ctx)
}

int ddtm_field_destroy(ddtm_field* f) {
  if (!f) return DDTM_ERR_ARG;
  cudaStreamSynchronize(f->ctx->stream);
  delete f;
  return DDTM_OK;
}

int ddtm_field_import(ddtm_ctx* ctx, ddtm_field* f, const double* x, int loc) {
  API_BEGIN(ctx)
  check_loc(loc);
  if (!f || !x || f->ctx != ctx) throw Error(DDTM_ERR_ARG, "invalid arguments");
  size_t nsp = (size_t)ctx->g.V * 12;
  for (int r = 0; r < f->nrhs; r++) {
    const double* din = stage_in(ctx, "canon_in", x + 2 * nsp * r, nsp, loc);
    launch_spinor_from_canon(ctx->g, f->prec, field_ptr(f, r), field_nrm(f, r), din, ctx->stream);
  }
  if (loc == DDTM_LOC_HOST) CK(cudaStreamSynchronize(ctx->stream));
  API_END(ctx)
}

int ddtm_field_export(ddtm_ctx* ctx, const ddtm_field* f, double* x, int loc) {
  API_BEGIN(ctx)
  check_loc(loc);
  if (!f || !x || f->ctx != ctx) throw Error(DDTM_ERR_ARG, "invalid arguments");
  size_t nsp = (size_t)ctx->g.V * 12;
  for (int r = 0; r < f->nrhs; r++) {
    double* dout = stage_out(ctx, "canon_out", x + 2 * nsp * r, nsp, loc);
    launch_spinor_to_canon(ctx->g, f->prec, field_ptr(f, r), field_nrm(f, r), dout, ctx->stream);
    unstage_out(ctx, x + 2 * nsp * r, dout, nsp, loc);
  }
  API_END(ctx)
}

int ddtm_apply_D_field(ddtm_ctx* ctx, ddtm_field* y, const ddtm_field* x, double mu) {
  API_BEGIN(ctx)
  if (!x || !y || x->ctx != ctx || y->ctx != ctx || x->prec != y->prec || x->nrhs != y->nrhs || x == y)
    throw Error(DDTM_ERR_ARG, "fields must differ and share context, precision and nrhs");
  dslash_field(ctx, y, x, mu);
  API_END(ctx)
}

int ddtm_set_option(ddtm_ctx* ctx, const char* name, int value) {
  API_BEGIN(ctx)
  if (!name) throw Error(DDTM_ERR_ARG, "null option name");
  const std::string n(name);
  if (n == "graphs") {
    ctx->use_graphs = value != 0;
  } else if (n == "autotune") {
    tc_autotune_enable(value != 0);
  } else if (n == "tc_forced_timeout_us") {
    if (value < 0 || value > 1000000) throw Error(DDTM_ERR_ARG, "tc_forced_timeout_us must lie in [0, 1000000]");
    tc_set_forced_wait_ns((uint64_t)value * 1000ull);
  } else {
    throw Error(DDTM_ERR_ARG, "unknown option " + n);
  }
  API_END(ctx)
}

int ddtm_get_option(ddtm_ctx* ctx, const char* name, int* value) {
  API_BEGIN(ctx)
  if (!name || !value) throw Error(DDTM_ERR_ARG, "null argument");
  const std::string n(name);
  if (n == "graphs") *value = ctx->use_graphs ? 1 : 0;
  else if (n == "graphs_cached") *value = (int)ctx->graphs.size();
  else if (n == "tc_forced_timeout_us") *value = (int)(tc_forced_wait_ns() / 1000ull);
  else throw Error(DDTM_ERR_ARG, "unknown option " + n);
  API_END(ctx)
}

int ddtm_autotune_report(char* buf, int len) {
  if (!buf || len <= 0) return DDTM_ERR_ARG;
  try {
    const std::string s = tc_autotune_report();
    const size_t n = s.size() < (size_t)len - 1 ? s.size() : (size_t)len - 1;
    memcpy(buf, s.data(), n);
    buf[n] = 0;
  } catch (const std::exception&) {
    return DDTM_ERR_CUDA;
  }
  return DDTM_OK;
}

int ddtm_release_workspace(ddtm_ctx* ctx) {
  API_BEGIN(ctx)
  CK(cudaStreamSynchronize(ctx->stream));
  for (auto& kv : ctx->graphs)  // captured graphs refer to the workspace
    if (kv.second.first) CK(cudaGraphExecDestroy(kv.second.first));
  ctx->graphs.clear();
  ctx->scratch.clear();
  API_END(ctx)
}

int ddtm_set_memory_limit(size_t bytes) {
  set_device_memory_limit(bytes);
  return DDTM_OK;
}

int ddtm_memory_in_use(size_t* bytes) {
  if (!bytes) return DDTM_ERR_ARG;
  *bytes = device_bytes_in_use();
  return DDTM_OK;
}

int ddtm_timer_enable(ddtm_ctx* ctx, int on) {
  API_BEGIN(ctx)
  timer_enable(on != 0);
  API_END(ctx)
}

int ddtm_timer_reset(ddtm_ctx* ctx) {
  API_BEGIN(ctx)
  timer_reset();
  API_END(ctx)
}

int ddtm_timer_report(ddtm_ctx* ctx, char* buf, int len) {
  API_BEGIN(ctx)
  if (!buf || len <= 0) throw Error(DDTM_ERR_ARG, "invalid buffer");
  std::string r = timer_report_json();
  snprintf(buf, (size_t)len, "%s", r.c_str());
  API_END(ctx)
}

}  // extern "C"

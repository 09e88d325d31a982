// Multigrid setup, smoother and solver entry points of the C ABI.
#include "common.cuh"
#include "ddtm_internal.h"
#include "solver.h"

using namespace ddtm;

namespace ddtm {

void validate_params(ddtm_ctx* c, const ddtm_params& p) {
  if (p.n_levels != 2) throw Error(DDTM_ERR_ARG, "n_levels must be 2");
  for (int m = 0; m < 4; m++)
    if (p.block[0][m] != c->g.b[m]) throw Error(DDTM_ERR_ARG, "block[0] is fixed at ddtm_create");
  if (p.nv[0] < 1 || p.nv[0] > 64) throw Error(DDTM_ERR_ARG, "nv[0] must be in 1..64");
  if (p.n_setup < 1 || p.post_smooth < 0 || p.nmr < 1) throw Error(DDTM_ERR_ARG, "invalid smoother/setup counts");
  if (p.coarse_restart < 1 || p.coarse_max_restarts < 0 || p.outer_restart < 1 || p.outer_max_iters < 1)
    throw Error(DDTM_ERR_ARG, "invalid Krylov parameters");
  if (!(p.outer_tol > 0) || !(p.coarse_tol > 0) || !(p.delta > 0)) throw Error(DDTM_ERR_ARG, "invalid tolerances");
  if (p.smoother_prec != DDTM_PREC_F32 && p.smoother_prec != DDTM_PREC_F16)
    throw Error(DDTM_ERR_ARG, "smoother_prec must be F32 or F16");
  if (p.coarse_prec != DDTM_PREC_F32 && p.coarse_prec != DDTM_PREC_F16)
    throw Error(DDTM_ERR_ARG, "coarse_prec must be F32 or F16");
}

void sap_run(ddtm_ctx* c, int prec, void* x, float* xn, const void* b, const float* bn, double mu, int ncycles,
             int nmr) {
  ensure_fine_prec(c, prec);
  ensure_site_inverse(c, prec, mu);
  const FineGeom& g = c->g;
  int half = g.Nb / 2;
  const int* red = g.colour_blocks.as<int>();
  const int* black = red + half;
  if (ncycles <= 0) {
    size_t n = (size_t)g.V * 12 * store2_bytes(prec);
    CK(cudaMemsetAsync(x, 0, n, c->stream));
    if (xn) CK(cudaMemsetAsync(xn, 0, (size_t)g.V * sizeof(float), c->stream));
    return;
  }
  for (int cyc = 0; cyc < ncycles; cyc++) {
    launch_sap_half(g, prec, x, xn, b, bn, c->links[prec].p, c->clover[prec].p, c->sinv[prec].p, red, black, half,
                    cyc == 0, nmr, mu, c->stream);
    launch_sap_half(g, prec, x, xn, b, bn, c->links[prec].p, c->clover[prec].p, c->sinv[prec].p, black, red, half,
                    0, nmr, mu, c->stream);
  }
}

void invalidate_setup(ddtm_ctx* c) {
  c->setup_done = false;
  c->have_P = false;
  c->c1.built = false;
  c->c1.inv_valid = false;
}

}  // namespace ddtm

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

extern "C" {

int ddtm_sap(ddtm_ctx* ctx, double* x, const double* b, int nrhs, double mu, int ncycles, int nmr, int prec, int loc) {
  API_BEGIN(ctx)
  check_prec(prec);
  check_loc(loc);
  if (!x || !b || nrhs < 0 || ncycles < 0 || nmr < 0) throw Error(DDTM_ERR_ARG, "invalid arguments");
  if (nrhs == 0) return DDTM_OK;
  ensure_fine_prec(ctx, prec);
  size_t nsp = (size_t)ctx->g.V * 12;
  ddtm_field fx{ctx, prec, 1}, fb{ctx, prec, 1};
  field_alloc(&fx);
  field_alloc(&fb);
  for (int r = 0; r < nrhs; r++) {
    const double* din = stage_in(ctx, "canon_in", b + 2 * nsp * r, nsp, loc);
    double* dout = stage_out(ctx, "canon_out", x + 2 * nsp * r, nsp, loc);
    launch_spinor_from_canon(ctx->g, prec, fb.data.p, fb.nrm.as<float>(), din, ctx->stream);
    sap_run(ctx, prec, fx.data.p, fx.nrm.as<float>(), fb.data.p, fb.nrm.as<float>(), mu, ncycles, nmr);
    launch_spinor_to_canon(ctx->g, prec, fx.data.p, fx.nrm.as<float>(), dout, ctx->stream);
    unstage_out(ctx, x + 2 * nsp * r, dout, nsp, loc);
  }
  CK(cudaStreamSynchronize(ctx->stream));
  API_END(ctx)
}

int ddtm_sap_field(ddtm_ctx* ctx, ddtm_field* x, const ddtm_field* b, double mu, int ncycles, int nmr) {
  API_BEGIN(ctx)
  if (!x || !b || x == b || x->ctx != ctx || b->ctx != ctx || x->prec != b->prec || x->nrhs != b->nrhs)
    throw Error(DDTM_ERR_ARG, "fields must differ and share context, precision and nrhs");
  if (ncycles < 0 || nmr < 0) throw Error(DDTM_ERR_ARG, "invalid cycle counts");
  for (int r = 0; r < x->nrhs; r++)
    sap_run(ctx, x->prec, field_ptr(x, r), field_nrm(x, r), field_ptr(b, r), field_nrm(b, r), mu, ncycles, nmr);
  API_END(ctx)
}

}  // extern "C"

#define NOT_YET(name)                                                   \
  if (!ctx) return DDTM_ERR_ARG;                                        \
  ctx->err = std::string(name) + ": not available in this build";        \
  return DDTM_ERR_STATE;

extern "C" {
int ddtm_setup(ddtm_ctx* ctx, double, uint64_t) { NOT_YET("ddtm_setup") }
int ddtm_set_test_vectors(ddtm_ctx* ctx, int, const double*, int, int) { NOT_YET("ddtm_set_test_vectors") }
int ddtm_build_coarse(ddtm_ctx* ctx) { NOT_YET("ddtm_build_coarse") }
int ddtm_get_prolongator(ddtm_ctx* ctx, int, double*, int) { NOT_YET("ddtm_get_prolongator") }
int ddtm_restrict(ddtm_ctx* ctx, int, double*, const double*, int, int) { NOT_YET("ddtm_restrict") }
int ddtm_prolong(ddtm_ctx* ctx, int, double*, const double*, int, int) { NOT_YET("ddtm_prolong") }
int ddtm_apply_Dc(ddtm_ctx* ctx, int, double*, const double*, int, double, int) { NOT_YET("ddtm_apply_Dc") }
int ddtm_coarse_solve(ddtm_ctx* ctx, double*, const double*, double, int, int*) { NOT_YET("ddtm_coarse_solve") }
int ddtm_solve(ddtm_ctx* ctx, double*, const double*, int, double, int, ddtm_solve_info*) { NOT_YET("ddtm_solve") }
int ddtm_save_setup(ddtm_ctx* ctx, const char*) { NOT_YET("ddtm_save_setup") }
int ddtm_load_setup(ddtm_ctx* ctx, const char*) { NOT_YET("ddtm_load_setup") }
}

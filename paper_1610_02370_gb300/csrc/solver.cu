// Multigrid setup, smoother driver, coarsest-level even-odd GMRES, K-cycle
// preconditioner and the outer flexible GMRES (Sec. 2.2 - 2.6), plus the C-ABI
// entry points that reach them.  Host code orchestrates; every vector
// operation runs in the kernels of blas.cu, coarse.cu, transfer.cu, sap.cu and
// dirac.cu.  Krylov scalars (Hessenberg column, Givens rotations) live on the
// host in FP64.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <complex>
#include <functional>

#include "blas.h"
#include "coarse.h"
#include "common.cuh"
#include "ddtm_internal.h"
#include "solver.h"

using namespace ddtm;
typedef std::complex<double> zc;

namespace ddtm {

void validate_params(ddtm_ctx* c, const ddtm_params& p) {
  if (p.n_levels != 2) throw Error(DDTM_ERR_ARG, "n_levels must be 2");
  for (int m = 0; m < 4; m++)
    if (p.block[0][m] != c->g.b[m]) throw Error(DDTM_ERR_ARG, "block[0] is fixed at ddtm_create");
  if (p.nv[0] < 1 || p.nv[0] > 64) throw Error(DDTM_ERR_ARG, "nv[0] must be in 1..64");
  if (p.n_setup < 1 || p.post_smooth < 0 || p.nmr < 1) throw Error(DDTM_ERR_ARG, "invalid smoother/setup counts");
  if (p.coarse_restart < 1 || p.coarse_restart > 250 || p.coarse_max_restarts < 0 || p.outer_restart < 1 ||
      p.outer_restart > 250 || p.outer_max_iters < 1)
    throw Error(DDTM_ERR_ARG, "invalid Krylov parameters");
  if (!(p.outer_tol > 0) || !(p.coarse_tol > 0) || !(p.delta > 0) || !(p.restart_tol > 0))
    throw Error(DDTM_ERR_ARG, "invalid tolerances");
  if (p.smoother_prec != DDTM_PREC_F32 && p.smoother_prec != DDTM_PREC_F16)
    throw Error(DDTM_ERR_ARG, "smoother_prec must be F32 or F16");
  if (p.coarse_prec != DDTM_PREC_F32 && p.coarse_prec != DDTM_PREC_F16)
    throw Error(DDTM_ERR_ARG, "coarse_prec must be F32 or F16");
}

void invalidate_setup(ddtm_ctx* c) {
  c->setup_done = false;
  c->have_P = false;
  c->c1.built = false;
  c->c1.inv_valid = false;
}

void sap_run(ddtm_ctx* c, int prec, void* x, float* xn, const void* b, const float* bn, double mu, int ncycles, int nmr,
             bool from_zero) {
  ensure_fine_prec(c, prec);
  ensure_site_inverse(c, prec, mu);
  const FineGeom& g = c->g;
  int half = g.Nb / 2;
  const int* red = g.colour_blocks.as<int>();
  const int* black = red + half;
  if (ncycles <= 0) {
    if (from_zero) {
      CK(cudaMemsetAsync(x, 0, (size_t)g.V * 12 * store2_bytes(prec), c->stream));
      if (xn) CK(cudaMemsetAsync(xn, 0, (size_t)g.V * sizeof(float), c->stream));
    }
    return;
  }
  for (int cyc = 0; cyc < ncycles; cyc++) {
    launch_sap_half(g, prec, x, xn, b, bn, c->links[prec].p, c->clover[prec].p, c->sinv[prec].p, red, black, half,
                    from_zero && cyc == 0, nmr, mu, c->stream);
    launch_sap_half(g, prec, x, xn, b, bn, c->links[prec].p, c->clover[prec].p, c->sinv[prec].p, black, red, half, 0,
                    nmr, mu, c->stream);
  }
}

// ---- hierarchy -----------------------------------------------------------------------
static size_t fine_field_bytes(const FineGeom& g, int prec) { return (size_t)g.V * 12 * store2_bytes(prec); }

// P from the current test vectors, then the Galerkin coarse operator
void build_hierarchy(ddtm_ctx* c) {
  const FineGeom& g = c->g;
  int nv = c->nv0;
  ensure_fine_prec(c, PREC_F32);
  if (!c->faces_ready) {
    build_faces(g, c->faces);
    c->faces_ready = true;
  }
  size_t pelems = (size_t)g.V * 12 * nv;  // complex entries of P
  c->P0.ensure(pelems * sizeof(float2));
  launch_build_P(g, c->P0.as<float2>(), c->tv0.as<float2>(), nv, c->stream);
  if (c->p.smoother_prec == PREC_F16) {
    c->P0h.ensure(pelems * sizeof(__half2));
    launch_P_to_half(c->P0.as<float2>(), c->P0h.as<__half2>(), pelems, c->stream);
  }
  CoarseLevel& L = c->c1;
  if (!c->c1_geom) {
    build_coarse_geometry(g, L);
    c->c1_geom = true;
  }
  L.nv = nv;
  L.n = 2 * nv;
  L.prec = c->p.coarse_prec;
  L.Dc.ensure((size_t)L.Nc * 9 * L.n * L.n * (L.prec == PREC_F16 ? 4 : 8));
  launch_galerkin(g, c->faces, L.prec, L.Dc.p, c->P0.as<float2>(), c->links[PREC_F32].p, c->clover[PREC_F32].p, nv,
                  c->stream);
  L.inv_valid = false;
  L.built = true;
  c->have_P = true;
}

void require_hierarchy(ddtm_ctx* c) {
  require_gauge(c);
  if (!c->have_P || !c->c1.built) throw Error(DDTM_ERR_STATE, "no aggregation / coarse operator (call ddtm_setup)");
}

// P in the storage used by the transfer kernels of precision prec
static const void* P_for(ddtm_ctx* c, int prec, int* pprec) {
  if (prec == PREC_F16 && c->P0h.p) {
    *pprec = PREC_F16;
    return c->P0h.p;
  }
  *pprec = PREC_F32;
  return c->P0.p;
}

// ---- GMRES on FP32 vectors ---------------------------------------------------------------
typedef std::function<void(cplx<float>*, const cplx<float>*)> OpF32;

// GMRES(m) with restarts for A x = b (complex FP32 vectors of length L, FP64
// inner products): classical Gram-Schmidt with one reorthogonalisation,
// Givens rotations on the host.  x is overwritten (zero start).  Returns the
// iteration count; *relres the last residual estimate relative to ||b||.
static int gmres_f32(ddtm_ctx* c, const OpF32& A, cplx<float>* x, const cplx<float>* b, size_t L, int m, int max_restarts,
                     double tol, double* relres, const char* tag) {
  Blas B(c->stream, &c->scratch);
  std::string t(tag);
  cplx<float>* V = (cplx<float>*)c->scratch.get(t + "_V", (size_t)(m + 1) * L * sizeof(float2));
  cplx<float>* w = (cplx<float>*)c->scratch.get(t + "_w", L * sizeof(float2));
  CK(cudaMemsetAsync(x, 0, L * sizeof(float2), c->stream));
  double bn = sqrt(B.norm2(b, 1, L));
  *relres = 0;
  if (bn == 0) return 0;
  std::vector<zc> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1);
  std::vector<double2> h(m + 1), h2(m + 1);
  int iters = 0;
  double est = 1;
  for (int cyc = 0; cyc <= max_restarts; cyc++) {
    // r = b - A x into V_0
    if (cyc == 0) {
      CK(cudaMemcpyAsync(V, b, L * sizeof(float2), cudaMemcpyDeviceToDevice, c->stream));
    } else {
      A(w, x);
      CK(cudaMemcpyAsync(V, b, L * sizeof(float2), cudaMemcpyDeviceToDevice, c->stream));
      B.axpby(make_double2(-1, 0), w, 1, make_double2(1, 0), V, 1, L);
    }
    double beta = sqrt(B.norm2(V, 1, L));
    est = beta / bn;
    if (est <= tol || beta == 0) break;
    B.axpby(make_double2(0, 0), V, 1, make_double2(1.0 / beta, 0), V, 1, L);
    std::fill(g.begin(), g.end(), zc(0));
    g[0] = beta;
    int k = 0;
    for (int j = 0; j < m; j++) {
      A(w, V + (size_t)j * L);
      B.dots(V, 1, L, j + 1, w, 1, L, h.data());
      B.multi_axpy(w, 1, V, 1, L, j + 1, h.data(), L, -1.0);
      B.dots(V, 1, L, j + 1, w, 1, L, h2.data());
      B.multi_axpy(w, 1, V, 1, L, j + 1, h2.data(), L, -1.0);
      for (int i = 0; i <= j; i++) H[(size_t)i * m + j] = zc(h[i].x + h2[i].x, h[i].y + h2[i].y);
      double hn = sqrt(B.norm2(w, 1, L));
      H[(size_t)(j + 1) * m + j] = hn;
      for (int i = 0; i < j; i++) {
        zc a = H[(size_t)i * m + j], bb = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = std::conj(cs[i]) * a + std::conj(sn[i]) * bb;
        H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
      }
      zc a = H[(size_t)j * m + j];
      double rho = sqrt(std::norm(a) + hn * hn);
      cs[j] = rho > 0 ? a / rho : zc(1);
      sn[j] = rho > 0 ? zc(hn / rho) : zc(0);
      H[(size_t)j * m + j] = rho;
      H[(size_t)(j + 1) * m + j] = 0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = std::conj(cs[j]) * g[j];
      k = j + 1;
      iters++;
      est = std::abs(g[j + 1]) / bn;
      if (est <= tol || hn == 0 || !std::isfinite(est)) break;
      B.axpby(make_double2(1.0 / hn, 0), w, 1, make_double2(0, 0), V + (size_t)(j + 1) * L, 1, L);  // V_{j+1} = w / hn
    }
    if (!std::isfinite(est)) throw Error(DDTM_ERR_NAN, "non-finite residual in GMRES (" + t + ")");
    std::vector<zc> y(k);
    for (int i = k - 1; i >= 0; i--) {
      zc s = g[i];
      for (int l = i + 1; l < k; l++) s -= H[(size_t)i * m + l] * y[l];
      y[i] = s / H[(size_t)i * m + i];
    }
    std::vector<double2> yd(k);
    for (int i = 0; i < k; i++) yd[i] = make_double2(y[i].real(), y[i].imag());
    B.multi_axpy(x, 1, V, 1, L, k, yd.data(), L, +1.0);
    if (est <= tol) break;
  }
  *relres = est;
  return iters;
}

// ---- coarsest level: even-odd GMRES (Sec. 2.5) ------------------------------------------
// D_c(mu_c) phi = eta:  rhat = eta_o - D_oe D_ee^-1 eta_e;  GMRES on
// D_hat = D_oo - D_oe D_ee^-1 D_eo;  phi_e = D_ee^-1 (eta_e - D_eo phi_o).
int coarse_eo_solve(ddtm_ctx* c, cplx<float>* x_full, const cplx<float>* b_full, double mu_c, int restart,
                    int max_restarts, double tol, double* relres) {
  CoarseLevel& L = c->c1;
  if (!L.inv_valid || L.inv_mu != mu_c) launch_self_inverse(L, mu_c, c->stream);
  size_t ne = L.h_even.size(), no = L.h_odd.size(), n = L.n;
  cplx<float>* be = (cplx<float>*)c->scratch.get("ceo_be", ne * n * 8);
  cplx<float>* bo = (cplx<float>*)c->scratch.get("ceo_bo", no * n * 8);
  cplx<float>* te = (cplx<float>*)c->scratch.get("ceo_te", ne * n * 8);
  cplx<float>* xo = (cplx<float>*)c->scratch.get("ceo_xo", no * n * 8);
  launch_parity_copy(L, 0, be, (cplx<float>*)b_full, 0, c->stream);
  launch_parity_copy(L, 1, bo, (cplx<float>*)b_full, 0, c->stream);
  launch_coarse_even(L, te, be, nullptr, 1.f, 0.f, c->stream);                   // te = D_ee^-1 eta_e
  launch_coarse_apply_odd(L, bo, nullptr, te, mu_c, 2, -1.f, 1.f, c->stream);     // rhat = eta_o - D_oe te
  cplx<float>* tA = (cplx<float>*)c->scratch.get("ceo_tA", ne * n * 8);
  OpF32 Dhat = [&](cplx<float>* out, const cplx<float>* in) {
    launch_coarse_even(L, tA, nullptr, in, 0.f, 1.f, c->stream);                 // tA = D_ee^-1 D_eo in
    launch_coarse_apply_odd(L, out, in, nullptr, mu_c, 1, 1.f, 0.f, c->stream);  // out = D_oo in
    launch_coarse_apply_odd(L, out, nullptr, tA, mu_c, 2, -1.f, 1.f, c->stream); // out -= D_oe tA
  };
  int it = gmres_f32(c, Dhat, xo, bo, no * n, restart, max_restarts, tol, relres, "cgm");
  launch_coarse_even(L, te, be, xo, 1.f, -1.f, c->stream);  // phi_e = D_ee^-1 (eta_e - D_eo phi_o)
  launch_parity_copy(L, 0, te, x_full, 1, c->stream);
  launch_parity_copy(L, 1, xo, x_full, 1, c->stream);
  c->coarse_iters += it;
  return it;
}

// ---- K-cycle preconditioner (Sec. 2.2): z = P D_c^-1 R v, then post-smoothing ----------
void mg_precondition(ddtm_ctx* c, int prec, void* z, float* zn, const void* v, const float* vn, double mu) {
  const FineGeom& g = c->g;
  CoarseLevel& L = c->c1;
  size_t nc = (size_t)L.Nc * L.n;
  cplx<float>* cv = (cplx<float>*)c->scratch.get("mg_c", nc * 8);
  cplx<float>* ev = (cplx<float>*)c->scratch.get("mg_e", nc * 8);
  int pprec;
  const void* P = P_for(c, prec, &pprec);
  launch_restrict(g, prec, cv, v, vn, P, pprec, L.nv, c->stream);
  double rr;
  coarse_eo_solve(c, ev, cv, c->p.delta * mu, c->p.coarse_restart, c->p.coarse_max_restarts, c->p.coarse_tol, &rr);
  launch_prolong(g, prec, z, zn, ev, P, pprec, L.nv, 0, c->stream);
  sap_run(c, prec, z, zn, v, vn, mu, c->p.post_smooth, c->p.nmr, false);
}

// ---- outer flexible GMRES in FP64 (Sec. 2.5) --------------------------------------------
// Arnoldi basis V and all orthogonalisation in FP64; Z_j = M v_j stored in the
// smoother precision (a flexible method takes Z_j as it is: w = D Z_j is
// applied to exactly the stored Z_j, and x is updated with the same Z_j).  A
// cycle ends at the restart length or when its residual estimate drops below
// restart_tol times the cycle's starting residual (Table 1: mixed-precision
// restart criterion) or below the target; every cycle starts from the true
// FP64 residual b - D x.
struct OuterResult {
  int iters = 0, restarts = 0;
  double relres = 1;
  bool converged = false;
};

OuterResult outer_fgmres(ddtm_ctx* c, double* x, const double* b, double mu) {
  const FineGeom& g = c->g;
  const ddtm_params& p = c->p;
  Blas B(c->stream, &c->scratch);
  int sp = p.smoother_prec, m = p.outer_restart;
  size_t n = (size_t)g.V * 12;  // complex entries of a fine field
  double* V = (double*)c->scratch.get("out_V", (m + 1) * n * 16);
  char* Z = (char*)c->scratch.get("out_Z", (size_t)m * fine_field_bytes(g, sp));
  float* Zn = (float*)c->scratch.get("out_Zn", (size_t)m * g.V * sizeof(float));
  double* w = (double*)c->scratch.get("out_w", n * 16);
  double* t64 = (double*)c->scratch.get("out_t64", n * 16);
  void* vs = c->scratch.get("out_vs", fine_field_bytes(g, sp));
  float* vsn = (float*)c->scratch.get("out_vsn", (size_t)g.V * sizeof(float));
  auto Zj = [&](int j) { return (void*)(Z + (size_t)j * fine_field_bytes(g, sp)); };
  auto Zjn = [&](int j) { return sp == PREC_F16 ? Zn + (size_t)j * g.V : (float*)nullptr; };
  auto D64 = [&](double* out, const double* in) {
    launch_dslash(g, PREC_F64, out, nullptr, in, nullptr, c->links[0].p, c->clover[0].p, mu, c->stream);
  };
  OuterResult res;
  double bn = sqrt(B.norm2(b, 0, n));
  CK(cudaMemsetAsync(x, 0, n * 16, c->stream));
  if (bn == 0) {
    res.relres = 0;
    res.converged = true;
    return res;
  }
  std::vector<zc> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1);
  std::vector<double2> h(m + 1), h2(m + 1);
  bool first = true;
  while (true) {
    // true residual r = b - D x into V_0
    if (first) {
      CK(cudaMemcpyAsync(V, b, n * 16, cudaMemcpyDeviceToDevice, c->stream));
    } else {
      D64(w, x);
      CK(cudaMemcpyAsync(V, b, n * 16, cudaMemcpyDeviceToDevice, c->stream));
      B.axpby(make_double2(-1, 0), w, 0, make_double2(1, 0), V, 0, n);
      res.restarts++;
    }
    first = false;
    double beta = sqrt(B.norm2(V, 0, n));
    res.relres = beta / bn;
    if (!std::isfinite(res.relres)) throw Error(DDTM_ERR_NAN, "non-finite outer residual");
    if (res.relres <= p.outer_tol) {
      res.converged = true;
      break;
    }
    if (res.iters >= p.outer_max_iters) break;
    B.axpby(make_double2(0, 0), V, 0, make_double2(1.0 / beta, 0), V, 0, n);
    std::fill(gv.begin(), gv.end(), zc(0));
    gv[0] = beta;
    int k = 0;
    for (int j = 0; j < m; j++) {
      launch_field_convert(g, PREC_F64, V + 2 * (size_t)j * n, nullptr, sp, vs, vsn, c->stream);
      mg_precondition(c, sp, Zj(j), Zjn(j), vs, vsn, mu);
      launch_field_convert(g, sp, Zj(j), Zjn(j), PREC_F64, t64, nullptr, c->stream);
      D64(w, t64);
      B.dots(V, 0, n, j + 1, w, 0, n, h.data());
      B.multi_axpy(w, 0, V, 0, n, j + 1, h.data(), n, -1.0);
      B.dots(V, 0, n, j + 1, w, 0, n, h2.data());
      B.multi_axpy(w, 0, V, 0, n, j + 1, h2.data(), n, -1.0);
      for (int i = 0; i <= j; i++) H[(size_t)i * m + j] = zc(h[i].x + h2[i].x, h[i].y + h2[i].y);
      double hn = sqrt(B.norm2(w, 0, n));
      H[(size_t)(j + 1) * m + j] = hn;
      for (int i = 0; i < j; i++) {
        zc a = H[(size_t)i * m + j], bb = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = std::conj(cs[i]) * a + std::conj(sn[i]) * bb;
        H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
      }
      zc a = H[(size_t)j * m + j];
      double rho = sqrt(std::norm(a) + hn * hn);
      cs[j] = rho > 0 ? a / rho : zc(1);
      sn[j] = rho > 0 ? zc(hn / rho) : zc(0);
      H[(size_t)j * m + j] = rho;
      H[(size_t)(j + 1) * m + j] = 0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = std::conj(cs[j]) * gv[j];
      k = j + 1;
      res.iters++;
      double est = std::abs(gv[j + 1]);
      if (!std::isfinite(est)) throw Error(DDTM_ERR_NAN, "non-finite outer residual estimate");
      if (est <= p.outer_tol * bn || est <= p.restart_tol * beta || hn == 0 || res.iters >= p.outer_max_iters) break;
      B.axpby(make_double2(1.0 / hn, 0), w, 0, make_double2(0, 0), V + 2 * (size_t)(j + 1) * n, 0, n);  // V_{j+1} = w / hn
    }
    std::vector<zc> y(k);
    for (int i = k - 1; i >= 0; i--) {
      zc s = gv[i];
      for (int l = i + 1; l < k; l++) s -= H[(size_t)i * m + l] * y[l];
      y[i] = s / H[(size_t)i * m + i];
    }
    for (int j = 0; j < k; j++) {
      launch_field_convert(g, sp, Zj(j), Zjn(j), PREC_F64, t64, nullptr, c->stream);
      B.axpby(make_double2(y[j].real(), y[j].imag()), t64, 0, make_double2(1, 0), x, 0, n);
    }
  }
  return res;
}

// ---- adaptive setup (Sec. 2.6) -----------------------------------------------------------------
static void normalise_fields(ddtm_ctx* c, float2* tv, int nv) {
  Blas B(c->stream, &c->scratch);
  size_t n = (size_t)c->g.V * 12;
  for (int i = 0; i < nv; i++) {
    double nn = sqrt(B.norm2(tv + (size_t)i * n, 1, n));
    if (!(nn > 0) || !std::isfinite(nn)) throw Error(DDTM_ERR_NAN, "test vector vanished or became non-finite in setup");
    B.axpby(make_double2(0, 0), tv + (size_t)i * n, 1, make_double2(1.0 / nn, 0), tv + (size_t)i * n, 1, n);
  }
}

void run_setup(ddtm_ctx* c, double mu, uint64_t seed) {
  const FineGeom& g = c->g;
  const ddtm_params& p = c->p;
  int nv = p.nv[0];
  c->nv0 = nv;
  size_t n = (size_t)g.V * 12;
  c->tv0.ensure((size_t)nv * n * sizeof(float2));
  float2* tv = c->tv0.as<float2>();
  for (int i = 0; i < nv; i++) launch_gaussian(tv + (size_t)i * n, n, seed * 0x100000001b3ull + (uint64_t)i * (n * 2 + 17), c->stream);
  int sp = p.smoother_prec;
  void* bs = c->scratch.get("setup_b", fine_field_bytes(g, sp));
  float* bsn = (float*)c->scratch.get("setup_bn", (size_t)g.V * 4);
  void* xs = c->scratch.get("setup_x", fine_field_bytes(g, sp));
  float* xsn = (float*)c->scratch.get("setup_xn", (size_t)g.V * 4);
  // k = 1: SAP on each random vector
  for (int i = 0; i < nv; i++) {
    launch_field_convert(g, PREC_F32, tv + (size_t)i * n, nullptr, sp, bs, bsn, c->stream);
    sap_run(c, sp, xs, xsn, bs, bsn, mu, p.post_smooth, p.nmr, true);
    launch_field_convert(g, sp, xs, xsn, PREC_F32, tv + (size_t)i * n, nullptr, c->stream);
  }
  normalise_fields(c, tv, nv);
  build_hierarchy(c);
  // k >= 2: one multigrid iteration per test vector
  for (int k = 2; k <= p.n_setup; k++) {
    for (int i = 0; i < nv; i++) {
      launch_field_convert(g, PREC_F32, tv + (size_t)i * n, nullptr, sp, bs, bsn, c->stream);
      mg_precondition(c, sp, xs, xsn, bs, bsn, mu);
      launch_field_convert(g, sp, xs, xsn, PREC_F32, tv + (size_t)i * n, nullptr, c->stream);
    }
    normalise_fields(c, tv, nv);
    build_hierarchy(c);
  }
  CK(cudaStreamSynchronize(c->stream));
}

}  // namespace ddtm

// ---- C ABI ----------------------------------------------------------------------------------
#define API_BEGIN(ctx)             \
  if (!(ctx)) return DDTM_ERR_ARG; \
  (ctx)->err.clear();              \
  try {
#define API_END(ctx)                \
  }                                 \
  catch (const ddtm::Error& e) {    \
    (ctx)->err = e.what();          \
    return e.code;                  \
  }                                 \
  catch (const std::exception& e) { \
    (ctx)->err = e.what();          \
    return DDTM_ERR_CUDA;           \
  }                                 \
  return DDTM_OK;

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static void check_level(ddtm_ctx* c, int level, int lo) {
  if (level < lo || level > 1) throw Error(DDTM_ERR_ARG, "level out of range for a two-level hierarchy");
  (void)c;
}

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
    sap_run(ctx, prec, fx.data.p, fx.nrm.as<float>(), fb.data.p, fb.nrm.as<float>(), mu, ncycles, nmr, true);
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
    sap_run(ctx, x->prec, field_ptr(x, r), field_nrm(x, r), field_ptr(b, r), field_nrm(b, r), mu, ncycles, nmr, true);
  API_END(ctx)
}

int ddtm_setup(ddtm_ctx* ctx, double mu, uint64_t seed) {
  API_BEGIN(ctx)
  require_gauge(ctx);
  if (!std::isfinite(mu)) throw Error(DDTM_ERR_ARG, "invalid mu");
  invalidate_setup(ctx);
  double t0 = now_s();
  run_setup(ctx, mu, seed);
  ctx->setup_s = now_s() - t0;
  ctx->setup_done = true;
  ctx->setup_mu = mu;
  API_END(ctx)
}

int ddtm_set_test_vectors(ddtm_ctx* ctx, int level, const double* v, int nv, int loc) {
  API_BEGIN(ctx)
  require_gauge(ctx);
  check_loc(loc);
  if (level != 0) throw Error(DDTM_ERR_ARG, "test vectors can be set for level 0 only");
  if (!v || nv != ctx->p.nv[0]) throw Error(DDTM_ERR_ARG, "nv must equal params.nv[0]");
  size_t nsp = (size_t)ctx->g.V * 12;
  ctx->nv0 = nv;
  ctx->tv0.ensure((size_t)nv * nsp * sizeof(float2));
  for (int i = 0; i < nv; i++) {
    const double* din = stage_in(ctx, "canon_in", v + 2 * nsp * i, nsp, loc);
    launch_spinor_from_canon(ctx->g, PREC_F32, ctx->tv0.as<float2>() + (size_t)i * nsp, nullptr, din, ctx->stream);
  }
  build_hierarchy(ctx);
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->setup_done = true;
  API_END(ctx)
}

int ddtm_build_coarse(ddtm_ctx* ctx) {
  API_BEGIN(ctx)
  require_gauge(ctx);
  if (!ctx->tv0.p || ctx->nv0 <= 0) throw Error(DDTM_ERR_STATE, "no test vectors (call ddtm_setup)");
  build_hierarchy(ctx);
  CK(cudaStreamSynchronize(ctx->stream));
  API_END(ctx)
}

int ddtm_get_prolongator(ddtm_ctx* ctx, int level, double* W, int loc) {
  API_BEGIN(ctx)
  check_loc(loc);
  check_level(ctx, level, 0);
  if (level != 0 || !W) throw Error(DDTM_ERR_ARG, "invalid arguments");
  require_hierarchy(ctx);
  size_t n = (size_t)ctx->g.V * 12 * 2 * ctx->nv0;
  double* d = stage_out(ctx, "canon_P", W, n, loc);
  launch_P_to_canon(ctx->g, d, ctx->P0.as<float2>(), ctx->nv0, ctx->stream);
  unstage_out(ctx, W, d, n, loc);
  CK(cudaStreamSynchronize(ctx->stream));
  API_END(ctx)
}

int ddtm_restrict(ddtm_ctx* ctx, int level, double* cout, const double* x, int nrhs, int loc) {
  API_BEGIN(ctx)
  check_loc(loc);
  if (level != 0 || !cout || !x || nrhs < 0) throw Error(DDTM_ERR_ARG, "invalid arguments");
  require_hierarchy(ctx);
  Blas B(ctx->stream, &ctx->scratch);
  const FineGeom& g = ctx->g;
  CoarseLevel& L = ctx->c1;
  size_t nsp = (size_t)g.V * 12, nc = (size_t)L.Nc * L.n;
  float2* f = (float2*)ctx->scratch.get("abi_f32", nsp * 8);
  cplx<float>* cv = (cplx<float>*)ctx->scratch.get("abi_c32", nc * 8);
  for (int r = 0; r < nrhs; r++) {
    const double* din = stage_in(ctx, "canon_in", x + 2 * nsp * r, nsp, loc);
    double* dout = stage_out(ctx, "canon_cout", cout + 2 * nc * r, nc, loc);
    launch_spinor_from_canon(g, PREC_F32, f, nullptr, din, ctx->stream);
    launch_restrict(g, PREC_F32, cv, f, nullptr, ctx->P0.p, PREC_F32, L.nv, ctx->stream);
    B.axpby(make_double2(1, 0), cv, 1, make_double2(0, 0), dout, 0, nc);
    unstage_out(ctx, cout + 2 * nc * r, dout, nc, loc);
  }
  CK(cudaStreamSynchronize(ctx->stream));
  API_END(ctx)
}

int ddtm_prolong(ddtm_ctx* ctx, int level, double* x, const double* cin, int nrhs, int loc) {
  API_BEGIN(ctx)
  check_loc(loc);
  if (level != 0 || !cin || !x || nrhs < 0) throw Error(DDTM_ERR_ARG, "invalid arguments");
  require_hierarchy(ctx);
  Blas B(ctx->stream, &ctx->scratch);
  const FineGeom& g = ctx->g;
  CoarseLevel& L = ctx->c1;
  size_t nsp = (size_t)g.V * 12, nc = (size_t)L.Nc * L.n;
  float2* f = (float2*)ctx->scratch.get("abi_f32", nsp * 8);
  cplx<float>* cv = (cplx<float>*)ctx->scratch.get("abi_c32", nc * 8);
  for (int r = 0; r < nrhs; r++) {
    const double* din = stage_in(ctx, "canon_cin", cin + 2 * nc * r, nc, loc);
    double* dout = stage_out(ctx, "canon_out", x + 2 * nsp * r, nsp, loc);
    B.axpby(make_double2(1, 0), din, 0, make_double2(0, 0), cv, 1, nc);
    launch_prolong(g, PREC_F32, f, nullptr, cv, ctx->P0.p, PREC_F32, L.nv, 0, ctx->stream);
    launch_spinor_to_canon(g, PREC_F32, f, nullptr, dout, ctx->stream);
    unstage_out(ctx, x + 2 * nsp * r, dout, nsp, loc);
  }
  CK(cudaStreamSynchronize(ctx->stream));
  API_END(ctx)
}

int ddtm_apply_Dc(ddtm_ctx* ctx, int level, double* y, const double* x, int nrhs, double mu, int loc) {
  API_BEGIN(ctx)
  check_loc(loc);
  if (level != 1 || !x || !y || nrhs < 0) throw Error(DDTM_ERR_ARG, "invalid arguments (coarse level is 1)");
  require_hierarchy(ctx);
  Blas B(ctx->stream, &ctx->scratch);
  CoarseLevel& L = ctx->c1;
  size_t nc = (size_t)L.Nc * L.n;
  cplx<float>* xv = (cplx<float>*)ctx->scratch.get("abi_c32", nc * 8);
  cplx<float>* yv = (cplx<float>*)ctx->scratch.get("abi_c32b", nc * 8);
  for (int r = 0; r < nrhs; r++) {
    const double* din = stage_in(ctx, "canon_cin", x + 2 * nc * r, nc, loc);
    double* dout = stage_out(ctx, "canon_cout", y + 2 * nc * r, nc, loc);
    B.axpby(make_double2(1, 0), din, 0, make_double2(0, 0), xv, 1, nc);
    launch_coarse_apply_full(L, yv, xv, mu, 3, 1.f, 0.f, ctx->stream);
    B.axpby(make_double2(1, 0), yv, 1, make_double2(0, 0), dout, 0, nc);
    unstage_out(ctx, y + 2 * nc * r, dout, nc, loc);
  }
  CK(cudaStreamSynchronize(ctx->stream));
  API_END(ctx)
}

int ddtm_coarse_solve(ddtm_ctx* ctx, double* x, const double* b, double mu_c, int loc, int* iters) {
  API_BEGIN(ctx)
  check_loc(loc);
  if (!x || !b) throw Error(DDTM_ERR_ARG, "invalid arguments");
  require_hierarchy(ctx);
  Blas B(ctx->stream, &ctx->scratch);
  CoarseLevel& L = ctx->c1;
  size_t nc = (size_t)L.Nc * L.n;
  cplx<float>* bv = (cplx<float>*)ctx->scratch.get("abi_c32", nc * 8);
  cplx<float>* xv = (cplx<float>*)ctx->scratch.get("abi_c32b", nc * 8);
  const double* din = stage_in(ctx, "canon_cin", b, nc, loc);
  double* dout = stage_out(ctx, "canon_cout", x, nc, loc);
  B.axpby(make_double2(1, 0), din, 0, make_double2(0, 0), bv, 1, nc);
  double rr;
  int it = coarse_eo_solve(ctx, xv, bv, mu_c, ctx->p.coarse_restart, ctx->p.coarse_max_restarts, ctx->p.coarse_tol, &rr);
  B.axpby(make_double2(1, 0), xv, 1, make_double2(0, 0), dout, 0, nc);
  unstage_out(ctx, x, dout, nc, loc);
  CK(cudaStreamSynchronize(ctx->stream));
  if (iters) *iters = it;
  if (rr > ctx->p.coarse_tol) {
    ctx->err = "coarse solve stopped at relative residual " + std::to_string(rr);
    return DDTM_ERR_NOCONV;
  }
  API_END(ctx)
}

int ddtm_solve(ddtm_ctx* ctx, double* x, const double* b, int nrhs, double mu, int loc, ddtm_solve_info* info) {
  API_BEGIN(ctx)
  check_loc(loc);
  if (!x || !b || nrhs < 0 || !std::isfinite(mu)) throw Error(DDTM_ERR_ARG, "invalid arguments");
  if (!ctx->setup_done) throw Error(DDTM_ERR_STATE, "no setup (call ddtm_setup first)");
  require_hierarchy(ctx);
  double t0 = now_s();
  const FineGeom& g = ctx->g;
  size_t nsp = (size_t)g.V * 12;
  double* bf = (double*)ctx->scratch.get("solve_b", nsp * 16);
  double* xf = (double*)ctx->scratch.get("solve_x", nsp * 16);
  ddtm_solve_info acc;
  memset(&acc, 0, sizeof(acc));
  ctx->coarse_iters = 0;
  bool all_conv = true;
  for (int r = 0; r < nrhs; r++) {
    const double* din = stage_in(ctx, "canon_in", b + 2 * nsp * r, nsp, loc);
    double* dout = stage_out(ctx, "canon_out", x + 2 * nsp * r, nsp, loc);
    launch_spinor_from_canon(g, PREC_F64, bf, nullptr, din, ctx->stream);
    OuterResult o = outer_fgmres(ctx, xf, bf, mu);
    launch_spinor_to_canon(g, PREC_F64, xf, nullptr, dout, ctx->stream);
    unstage_out(ctx, x + 2 * nsp * r, dout, nsp, loc);
    acc.iters = o.iters > acc.iters ? o.iters : acc.iters;
    acc.restarts = o.restarts > acc.restarts ? o.restarts : acc.restarts;
    acc.max_relres = o.relres > acc.max_relres ? o.relres : acc.max_relres;
    all_conv = all_conv && o.converged;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  acc.coarse_iters = ctx->coarse_iters;
  acc.solve_s = now_s() - t0;
  acc.setup_s = ctx->setup_s;
  if (info) *info = acc;
  if (!all_conv) {
    ctx->err = "outer solver stopped at relative residual " + std::to_string(acc.max_relres);
    return DDTM_ERR_NOCONV;
  }
  API_END(ctx)
}

// Setup file: magic, dims, block, nv, then the nv test vectors (FP32 fields
// in the internal layout of this block size).
static const char MAGIC[8] = {'D', 'D', 'T', 'M', 'S', 'U', '0', '1'};

int ddtm_save_setup(ddtm_ctx* ctx, const char* path) {
  API_BEGIN(ctx)
  if (!path) throw Error(DDTM_ERR_ARG, "null path");
  if (!ctx->tv0.p || !ctx->setup_done) throw Error(DDTM_ERR_STATE, "no setup to save");
  size_t bytes = (size_t)ctx->nv0 * ctx->g.V * 12 * sizeof(float2);
  std::vector<char> host(bytes);
  CK(cudaMemcpyAsync(host.data(), ctx->tv0.p, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  FILE* f = fopen(path, "wb");
  if (!f) throw Error(DDTM_ERR_ARG, std::string("cannot open ") + path);
  int hdr[9] = {ctx->g.L[0], ctx->g.L[1], ctx->g.L[2], ctx->g.L[3], ctx->g.b[0], ctx->g.b[1], ctx->g.b[2], ctx->g.b[3],
                ctx->nv0};
  bool ok = fwrite(MAGIC, 1, 8, f) == 8 && fwrite(hdr, sizeof(int), 9, f) == 9 &&
            fwrite(&ctx->setup_mu, sizeof(double), 1, f) == 1 && fwrite(host.data(), 1, bytes, f) == bytes;
  fclose(f);
  if (!ok) throw Error(DDTM_ERR_ARG, std::string("short write to ") + path);
  API_END(ctx)
}

int ddtm_load_setup(ddtm_ctx* ctx, const char* path) {
  API_BEGIN(ctx)
  if (!path) throw Error(DDTM_ERR_ARG, "null path");
  require_gauge(ctx);
  FILE* f = fopen(path, "rb");
  if (!f) throw Error(DDTM_ERR_ARG, std::string("cannot open ") + path);
  char magic[8];
  int hdr[9];
  double mu;
  bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, MAGIC, 8) == 0 && fread(hdr, sizeof(int), 9, f) == 9 &&
            fread(&mu, sizeof(double), 1, f) == 1;
  if (ok)
    for (int m = 0; m < 4; m++) ok = ok && hdr[m] == ctx->g.L[m] && hdr[4 + m] == ctx->g.b[m];
  ok = ok && hdr[8] == ctx->p.nv[0];
  if (!ok) {
    fclose(f);
    throw Error(DDTM_ERR_ARG, "setup file does not match this lattice, block size or nv");
  }
  size_t bytes = (size_t)hdr[8] * ctx->g.V * 12 * sizeof(float2);
  std::vector<char> host(bytes);
  ok = fread(host.data(), 1, bytes, f) == bytes;
  fclose(f);
  if (!ok) throw Error(DDTM_ERR_ARG, "truncated setup file");
  ctx->nv0 = hdr[8];
  ctx->tv0.ensure(bytes);
  CK(cudaMemcpyAsync(ctx->tv0.p, host.data(), bytes, cudaMemcpyHostToDevice, ctx->stream));
  build_hierarchy(ctx);
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->setup_mu = mu;
  ctx->setup_done = true;
  API_END(ctx)
}

}  // extern "C"

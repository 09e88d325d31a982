// Even-odd preconditioned conjugate gradient on the normal equations of the
// Schur complement, the standard solver the paper compares DD-alpha-AMG with
// (Sec. 3.1.2: CG on the even-odd reduced operator).  FP64 throughout.
//
// With A = D_ee, D_oo the site-local blocks (clover + i mu Gamma5) and H the
// hopping term of D(mu) (Sec. 2.1), on odd sites
//   D_hat v = A_oo v - H_oe A_ee^-1 H_eo v,
//   rhat    = b_o - H_oe A_ee^-1 b_e,
// CG runs on D_hat^+ D_hat x_o = D_hat^+ rhat, with D_hat^+ = Gamma5 D_hat(-mu)
// Gamma5 (Gamma5-hermiticity of every piece), and the even sites follow as
//   x_e = A_ee^-1 (b_e - H_eo x_o).
// Half-lattice vectors are parity-compact per block: element (blk, c, i) at
// (blk * 12 + c) * Vh + i for the site of local index parity * Vh + i.
#include <math.h>

#include <chrono>
#include <vector>

#include "blas.h"
#include "common.cuh"
#include "ddtm_internal.h"
#include "solver.h"
#include "timer.h"

namespace ddtm {

typedef cplx<double> zd;

__device__ __forceinline__ void half_load(const double2* v, int blk, int i, int Vh, bool g5, zd p[12]) {
  const double2* q = v + (size_t)blk * 12 * Vh + i;
#pragma unroll
  for (int c = 0; c < 12; c++) {
    double2 a = __ldg(q + (size_t)c * Vh);
    p[c] = (g5 && c >= 6) ? zd(-a.x, -a.y) : zd(a.x, a.y);
  }
}
__device__ __forceinline__ void half_store(double2* v, int blk, int i, int Vh, bool g5, const zd p[12]) {
  double2* q = v + (size_t)blk * 12 * Vh + i;
#pragma unroll
  for (int c = 0; c < 12; c++) q[(size_t)c * Vh] = (g5 && c >= 6) ? make_double2(-p[c].re, -p[c].im)
                                                                   : make_double2(p[c].re, p[c].im);
}

// acc = sum over the 8 hops of site (blk, loc) of the hop term with the
// neighbour read from the half-lattice vector v of the other parity (Gamma5
// applied to it when g5); the hopping term of D is -1/2 acc.
__device__ __forceinline__ void hop_half(const double2* v, bool g5, const Links<PREC_F64>& U, const Geo& g, int blk,
                                         int loc, zd acc[12]) {
  const int Vh = g.Vb / 2;
#pragma unroll
  for (int c = 0; c < 12; c++) acc[c] = zd(0, 0);
#pragma unroll 2
  for (int k = 0; k < 8; k++) {
    const int mu = k >> 1;
    const bool fwd = (k & 1) == 0;
    Nbr n = neighbour(g, blk, loc, k);
    zd h[6], w[6], u[9];
    {
      zd p[12];
      half_load(v, n.blk, n.loc >= Vh ? n.loc - Vh : n.loc, Vh, g5, p);
      project<double>(mu, fwd, p, h);
    }
    if (fwd) {
      U.load(blk, loc, mu, u);
      mul_U<double>(u, h, w);
    } else {
      U.load(n.blk, n.loc, mu, u);
      mul_Udag<double>(u, h, w);
    }
    if (n.flip)
#pragma unroll
      for (int q = 0; q < 6; q++) w[q] = -w[q];
    reconstruct<double>(mu, fwd, w, acc);
  }
}

// even sites: t_e = A_ee^-1 (b_e + sh * H_eo (G v_o)), G = Gamma5 if g5; v or b may be null
__global__ void k_eo_even(double2* __restrict__ te, const double2* __restrict__ v, const double2* __restrict__ b,
                          double sh, int g5, Links<PREC_F64> U, SiteInv<PREC_F64> Ainv, Geo g) {
  const int Vh = g.Vb / 2;
  const long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= (long)g.Nb * Vh) return;
  const int blk = (int)(s / Vh), i = (int)(s - (long)blk * Vh);
  zd h[12], t[12];
  if (v) {
    hop_half(v, g5 != 0, U, g, blk, i, h);
#pragma unroll
    for (int c = 0; c < 12; c++) h[c] = (-0.5 * sh) * h[c];
  } else {
#pragma unroll
    for (int c = 0; c < 12; c++) h[c] = zd(0, 0);
  }
  if (b) {
    zd bb[12];
    half_load(b, blk, i, Vh, false, bb);
#pragma unroll
    for (int c = 0; c < 12; c++) h[c] = h[c] + bb[c];
  }
  Ainv.apply(blk, i, h, t);
  half_store(te, blk, i, Vh, false, t);
}

// odd sites: out = G [ A_oo(mu) (G s_o) (self = 1) or s_o (self = 2) or 0 (self = 0)
//                      - H_oe t_e ],  G = Gamma5 if g5
__global__ void k_eo_odd(double2* __restrict__ out, const double2* __restrict__ so, int self,
                         const double2* __restrict__ te, double mu, int g5, Links<PREC_F64> U, Clover<PREC_F64> C,
                         Geo g) {
  const int Vh = g.Vb / 2;
  const long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= (long)g.Nb * Vh) return;
  const int blk = (int)(s / Vh), i = (int)(s - (long)blk * Vh), lo = Vh + i;
  zd acc[12], o[12];
  hop_half(te, false, U, g, blk, lo, acc);
#pragma unroll
  for (int c = 0; c < 12; c++) o[c] = 0.5 * acc[c];  // - H_oe t_e = + 1/2 acc
  if (self) {
    zd x[12], y[12];
    half_load(so, blk, i, Vh, self == 1 && g5, x);
    if (self == 1) {
      C.apply(blk, lo, x, y);
#pragma unroll
      for (int c = 0; c < 12; c++) y[c] = y[c] + (c < 6 ? mu : -mu) * times_i(x[c]);
    } else {
#pragma unroll
      for (int c = 0; c < 12; c++) y[c] = x[c];
    }
#pragma unroll
    for (int c = 0; c < 12; c++) o[c] = o[c] + y[c];
  }
  half_store(out, blk, i, Vh, g5 != 0, o);
}

// full internal FP64 field <-> its two parity-compact halves
__global__ void k_eo_split(const double2* __restrict__ full, double2* __restrict__ ev, double2* __restrict__ od, int Vb,
                           long n, int dir) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;  // over Nb * 12 * Vb
  if (t >= n) return;
  const int Vh = Vb / 2;
  const long bc = t / Vb;
  const int loc = (int)(t - bc * Vb);
  double2* h = loc < Vh ? ev : od;
  const long hi = bc * Vh + (loc < Vh ? loc : loc - Vh);
  if (dir == 0) h[hi] = full[t];
  else const_cast<double2*>(full)[t] = h[hi];
}

static Geo eo_geo(const FineGeom& g) { return Geo{g.Vb, g.Nb, g.loc_nbr.as<uint32_t>(), g.blk_nbr.as<int>()}; }

struct EoOps {
  const FineGeom& g;
  cudaStream_t st;
  Links<PREC_F64> U;
  Clover<PREC_F64> C;
  SiteInv<PREC_F64> Ap, Am;  // A_ee^-1 for +mu and -mu
  double mu;
  double2* t;                // even-site work vector
  unsigned grid;
  void even(double2* te, const double2* v, const double2* b, double sh, bool g5, bool minus) const {
    k_eo_even<<<grid, 128, 0, st>>>(te, v, b, sh, g5, U, minus ? Am : Ap, eo_geo(g));
    CKL("eo_even");
  }
  void odd(double2* out, const double2* so, int self, const double2* te, bool g5, bool minus) const {
    k_eo_odd<<<grid, 128, 0, st>>>(out, so, self, te, minus ? -mu : mu, g5, U, C, eo_geo(g));
    CKL("eo_odd");
  }
  void dhat(double2* out, const double2* v) const {  // D_hat(mu) v
    ScopedTimer timer_("eo_dhat_f64", st);
    even(t, v, nullptr, 1.0, false, false);
    odd(out, v, 1, t, false, false);
  }
  void dhat_dag(double2* out, const double2* v) const {  // Gamma5 D_hat(-mu) Gamma5 v
    ScopedTimer timer_("eo_dhat_f64", st);
    even(t, v, nullptr, 1.0, true, true);
    odd(out, v, 1, t, true, true);
  }
};

// One right-hand side (internal full FP64 field b -> x) to the true relative
// residual ||b - D x|| / ||b|| <= tol.  CG stops first when the residual of the
// normal equations has dropped by tol (||r_k|| <= tol ||D_hat^+ rhat||), then
// the solution is retrieved and its true residual computed; while that is above
// tol, CG continues (same Krylov sequence) with the normal-equations threshold
// lowered by the missing factor.  Returns the CG iterations; *relres the final
// true residual, *conv whether it reached tol within max_iter.
static int eo_cg_one(ddtm_ctx* c, double* x, const double* b, double* rfull, double mu, double tol, int max_iter,
                     double* relres, bool* conv) {
  const FineGeom& g = c->g;
  const size_t nh = (size_t)g.Nb * 12 * (g.Vb / 2);  // complex entries of a half field
  const size_t hb = nh * sizeof(double2);
  const size_t nsp = (size_t)g.V * 12;
  double2* be = (double2*)c->scratch.get("eocg_be", hb);
  double2* bo = (double2*)c->scratch.get("eocg_bo", hb);
  double2* xo = (double2*)c->scratch.get("eocg_xo", hb);
  double2* r = (double2*)c->scratch.get("eocg_r", hb);
  double2* p = (double2*)c->scratch.get("eocg_p", hb);
  double2* q = (double2*)c->scratch.get("eocg_q", hb);
  double2* w = (double2*)c->scratch.get("eocg_w", hb);
  double2* te = (double2*)c->scratch.get("eocg_t", hb);
  double2* xe = (double2*)c->scratch.get("eocg_xe", hb);
  ensure_site_inverse(c, PREC_F64, mu);
  void* sinv_m = c->scratch.get("eocg_sinv_m", (size_t)g.Nb * 72 * (g.Vb / 2) * sizeof(double2));
  launch_site_inverse(g, PREC_F64, sinv_m, (const double*)c->clover[0].p, -mu, c->stream);
  const unsigned grid = (unsigned)(((size_t)g.Nb * (g.Vb / 2) + 127) / 128);
  EoOps op{g, c->stream, Links<PREC_F64>{(const double2*)c->links[0].p, g.Vb},
           Clover<PREC_F64>{(const double2*)c->clover[0].p, g.Vb},
           SiteInv<PREC_F64>{(const double2*)c->sinv[0].p, g.Vb / 2}, SiteInv<PREC_F64>{(const double2*)sinv_m, g.Vb / 2},
           mu, te, grid};
  const long nfull = (long)g.Nb * 12 * g.Vb;
  const unsigned gs = (unsigned)((nfull + 255) / 256);
  k_eo_split<<<gs, 256, 0, c->stream>>>((const double2*)b, be, bo, g.Vb, nfull, 0);
  CKL("eo_split");
  Blas B(c->stream, &c->scratch);
  const double bn2 = B.norm2(b, 0, nsp);
  if (!std::isfinite(bn2)) throw Error(DDTM_ERR_NAN, "non-finite right-hand side in even-odd CG");
  // rhat = b_o - H_oe A_ee^-1 b_e (in w), right-hand side of the normal equations D_hat^+ rhat (in r)
  op.even(te, nullptr, be, 0.0, false, false);
  op.odd(w, bo, 2, te, false, false);
  op.dhat_dag(r, w);
  CK(cudaMemsetAsync(xo, 0, hb, c->stream));
  CK(cudaMemcpyAsync(p, r, hb, cudaMemcpyDeviceToDevice, c->stream));
  double rr = B.norm2(r, 0, nh);
  double stop = tol * sqrt(rr);
  int it = 0;
  *relres = bn2 > 0 ? 1.0 : 0.0;
  *conv = bn2 == 0;
  while (!*conv) {
    while (sqrt(rr) > stop && it < max_iter) {
      op.dhat(w, p);
      op.dhat_dag(q, w);
      double2 pq;
      VSet vp{p, 0, nh, 1, false}, vq{q, 0, nh, 1, false};
      B.dots(vp, 0, 1, vq, &pq);
      if (!(pq.x > 0)) throw Error(DDTM_ERR_NAN, "even-odd CG: <p, D_hat^+ D_hat p> not positive");
      const double alpha = rr / pq.x;
      B.axpby(make_double2(alpha, 0), p, 0, make_double2(1, 0), xo, 0, nh);
      B.axpby(make_double2(-alpha, 0), q, 0, make_double2(1, 0), r, 0, nh);
      const double rr_new = B.norm2(r, 0, nh);
      if (!std::isfinite(rr_new)) throw Error(DDTM_ERR_NAN, "non-finite residual in even-odd CG");
      B.axpby(make_double2(1, 0), r, 0, make_double2(rr_new / rr, 0), p, 0, nh);
      rr = rr_new;
      it++;
    }
    // x_e = A_ee^-1 (b_e - H_eo x_o); true residual of the full system
    op.even(xe, xo, be, -1.0, false, false);
    k_eo_split<<<gs, 256, 0, c->stream>>>((const double2*)x, xe, xo, g.Vb, nfull, 1);
    CKL("eo_split");
    launch_dslash(g, PREC_F64, rfull, nullptr, x, nullptr, c->links[0].p, c->clover[0].p, mu, c->stream);
    B.axpby(make_double2(1, 0), b, 0, make_double2(-1, 0), rfull, 0, nsp);
    *relres = sqrt(B.norm2(rfull, 0, nsp) / bn2);
    *conv = *relres <= tol;
    if (*conv || it >= max_iter) break;
    stop = stop * 0.5 * tol / *relres;  // continue with a lower threshold on the normal equations
  }
  return it;
}

}  // namespace ddtm

using namespace ddtm;

static double eo_now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

extern "C" int ddtm_eo_cg(ddtm_ctx* ctx, double* x, const double* b, int nrhs, double mu, double tol, int max_iter,
                          int loc, ddtm_solve_info* info) {
  if (!ctx) return DDTM_ERR_ARG;
  ctx->err.clear();
  try {
    check_loc(loc);
    if (!x || !b || nrhs < 0 || !std::isfinite(mu) || !(tol > 0) || max_iter < 0)
      throw Error(DDTM_ERR_ARG, "invalid arguments");
    require_gauge(ctx);
    ensure_fine_prec(ctx, PREC_F64);
    const double t0 = eo_now_s();
    const FineGeom& g = ctx->g;
    const size_t nsp = (size_t)g.V * 12;
    double* bf = (double*)ctx->scratch.get("eocg_bfull", nsp * 16);
    double* xf = (double*)ctx->scratch.get("eocg_xfull", nsp * 16);
    double* rf = (double*)ctx->scratch.get("eocg_rfull", nsp * 16);
    ddtm_solve_info acc;
    memset(&acc, 0, sizeof(acc));
    bool all = true;
    for (int r = 0; r < nrhs; r++) {
      const double* din = stage_in(ctx, "canon_in", b + 2 * nsp * r, nsp, loc);
      launch_spinor_from_canon(g, PREC_F64, bf, nullptr, din, ctx->stream);
      bool conv = false;
      double rel = 0;
      const int it = eo_cg_one(ctx, xf, bf, rf, mu, tol, max_iter, &rel, &conv);
      double* dout = stage_out(ctx, "canon_out", x + 2 * nsp * r, nsp, loc);
      launch_spinor_to_canon(g, PREC_F64, xf, nullptr, dout, ctx->stream);
      unstage_out(ctx, x + 2 * nsp * r, dout, nsp, loc);
      acc.iters = it > acc.iters ? it : acc.iters;
      acc.max_relres = rel > acc.max_relres ? rel : acc.max_relres;
      all = all && conv;
    }
    CK(cudaStreamSynchronize(ctx->stream));
    acc.solve_s = eo_now_s() - t0;
    if (info) *info = acc;
    if (!all) {
      ctx->err = "even-odd CG stopped after " + std::to_string(acc.iters) + " iterations at relative residual " +
                 std::to_string(acc.max_relres);
      return DDTM_ERR_NOCONV;
    }
  } catch (const Error& e) {
    ctx->err = e.what();
    return e.code;
  } catch (const std::exception& e) {
    ctx->err = e.what();
    return DDTM_ERR_CUDA;
  }
  return DDTM_OK;
}
